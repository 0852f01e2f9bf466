"""The design study's swimmers on the GPU (the full study is a longer run
of the same path: python -m paper_1108_0786_gb300.design_study).

Three of the seventeen designs (three spheres; a parallel capsule in the
middle; three perpendicular capsules), at full size in the 100 x 100 x 200
channel, 2000 steps as one ensemble with the averaged load (the plain
explicit coupling is unstable at the paper's masses): no error, the bodies
move along the swimming axis only (the drive axes map to z, the set-up is symmetric about
it), and the FP32 ensemble matches FP64 runs of the same designs.
"""
import numpy as np
import pytest

from paper_1108_0786_gb300 import design_study as ds, lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1108_0786_gb300 import _build
    _build.build()
    return torch


def test_designs_move_along_the_swimming_axis(gpu):
    labels = ("a", "c", "k")
    scs = [ds.design(lab)[0] for lab in labels]
    start = [np.array([b.pos for b in sc.bodies]) for sc in scs]
    finals = {}
    for precision in ("f32", "f64"):
        lats = [lbm.from_scenario(sc, precision=precision, options=lbm.OPT_AVERAGE_FORCE) for sc in scs]
        ens = lbm.Ensemble(lats)
        ens.step(2000)
        ens.sync()
        finals[precision] = [lat.bodies() for lat in lats]
        ens.close()
        for lat in lats:
            lat.close()
    for lab, x0, f32, f64 in zip(labels, start, finals["f32"], finals["f64"]):
        dz = f64[:, 2] - x0[:, 2]
        assert np.abs(dz).max() > 0.1, lab                         # the drive moved the bodies
        assert np.abs(f64[:, 0:2] - x0[:, 0:2]).max() < 1e-6, lab   # along z only
        np.testing.assert_allclose(f32[:, 2], f64[:, 2], rtol=0, atol=1e-3 * np.abs(dz).max())
