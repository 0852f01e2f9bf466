"""Ensembles (lbm_ensemble_*): many independent lattices advanced by one graph.

Stepping members together must give, bit for bit, what stepping each alone
gives (the members share nothing); uneven step counts must be honoured; a
member's device error must surface at lbm_ensemble_sync; and members of the
seeded 96-box workload must match the FP64 oracle (parity for FP64 storage,
the FP32 tolerance for FP32 storage).
"""
import numpy as np
import pytest

import oracle
from paper_1108_0786_gb300 import lbm, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1108_0786_gb300 import _build
    _build.build()
    return torch


def members(count, edge_max=64):
    """The first `count` members of the seeded workload whose edge is at most edge_max."""
    return [sc for sc in wl.ensemble_members() if sc.nx <= edge_max][:count]


@pytest.mark.parametrize("precision,mode", [("f64", lbm.ENSEMBLE_BATCHED), ("f32", lbm.ENSEMBLE_BATCHED),
                                            ("f32", lbm.ENSEMBLE_BRANCHES)])
def test_ensemble_equals_members_stepped_alone(gpu, precision, mode):
    scs = members(5)
    steps = [48, 16, 33, 0, 70]
    alone = []
    for sc, n in zip(scs, steps):
        lat = lbm.from_scenario(sc, precision=precision)
        lat.step(n)
        alone.append((lat.bodies(), lat.pop(), lat.steps_done))
        lat.close()
    lats = [lbm.from_scenario(sc, precision=precision) for sc in scs]
    ens = lbm.Ensemble(lats)
    ens.set_mode(mode)
    ens.step(steps)
    ens.sync()
    for lat, (b, p, n) in zip(lats, alone):
        assert lat.steps_done == n
        assert np.array_equal(lat.bodies(), b)
        assert np.array_equal(lat.pop(), p)
    # a second call continues from where the members are (odd step counts included)
    ens.step([17, 16, 0, 32, 1])
    ens.sync()
    assert [lat.steps_done for lat in lats] == [65, 32, 33, 32, 71]
    ens.close()
    for lat in lats:
        lat.close()


def test_ensemble_members_match_the_oracle(gpu):
    """Two 48^3 members, 240 steps: FP64 storage to the parity bar, FP32
    within the displacement tolerance."""
    scs = [sc for sc in wl.ensemble_members() if sc.nx == 48][:2]
    n = 240
    refs = []
    for sc in scs:
        o = oracle.from_scenario(sc)
        x0 = o.bodies()[:, 0:3].copy()
        o.step(n)
        refs.append((o.bodies(), o.pop(), x0))
    for precision in ("f64", "f32"):
        lats = [lbm.from_scenario(sc, precision=precision) for sc in scs]
        ens = lbm.Ensemble(lats)
        ens.step(n)
        ens.sync()
        for lat, (b, p, x0) in zip(lats, refs):
            got = lat.bodies()
            if precision == "f64":
                np.testing.assert_allclose(got, b, rtol=1e-10, atol=1e-12)
                assert np.abs(lat.pop() - p).max() <= 1e-12
            else:
                disp_ref = np.linalg.norm(b[:, 0:3] - x0, axis=1)
                disp = np.linalg.norm(got[:, 0:3] - x0, axis=1)
                assert np.abs(disp - disp_ref).max() <= 1e-3 * disp_ref.max()
        ens.close()
        for lat in lats:
            lat.close()


def test_member_error_surfaces_at_sync(gpu):
    """One member's bodies overlap: its status word reports it at sync."""
    good = members(1)[0]
    bad = wl.Scenario("overlapping bodies", 48, 48, 48, 1.0)
    bad.bodies.append(wl.Body(wl.SPHERE, 4.0, 0.0, 500.0, (20.0, 24.0, 24.0)))
    bad.bodies.append(wl.Body(wl.SPHERE, 4.0, 0.0, 500.0, (26.0, 24.0, 24.0)))
    lats = [lbm.from_scenario(good, precision="f32"), lbm.from_scenario(bad, precision="f32")]
    ens = lbm.Ensemble(lats)
    ens.step(16)
    with pytest.raises(lbm.LbmError) as e:
        ens.sync()
    assert e.value.code == lbm.E_OVERLAP
    ens.close()
    for lat in lats:
        lat.close()


def mixed_members():
    """Members the batched launches must tell apart: storage precisions
    (one group each), walls, a box without bodies, odd and even extents."""
    out = []
    a = members(2)
    out.append((a[0], "f32"))
    out.append((a[1], "f64"))
    ch = wl.Scenario("walled channel", 40, 36, 44, 0.8, bc=wl.PERIODIC_Z, g=(0.0, 0.0, 2e-6))
    wl.add_swimmer(ch, (19.6, 17.8, 21.3), (0.7071, 0.0, -0.7071, 0.0), (wl.SPHERE, wl.CAPSULE, wl.SPHERE),
                   3.0, 4.0, 12.0, 0.02, 0.01, 2e-3, 64.0, density=2.0)
    out.append((ch, "f32"))
    fluid = wl.Scenario("no bodies", 33, 20, 24, 0.9, bc=wl.PERIODIC_X | wl.PERIODIC_Z, g=(1e-5, 0.0, 0.0))
    out.append((fluid, "bf16"))
    out.append((a[0], "bf16"))
    out.append((a[1], "f16"))
    return out


def test_batched_ensemble_of_mixed_members_equals_them_stepped_alone(gpu):
    mix = mixed_members()
    steps = [64, 48, 37, 80, 33, 50]
    alone = []
    for (sc, prec), n in zip(mix, steps):
        lat = lbm.from_scenario(sc, precision=prec)
        lat.step(n)
        alone.append((lat.bodies(), lat.pop()))
        lat.close()
    lats = [lbm.from_scenario(sc, precision=prec) for sc, prec in mix]
    ens = lbm.Ensemble(lats)
    ens.step(steps)
    ens.sync()
    for lat, (b, p) in zip(lats, alone):
        assert np.array_equal(lat.bodies(), b)
        assert np.array_equal(lat.pop(), p)
    ens.close()
    for lat in lats:
        lat.close()


def test_ensemble_autotune_keeps_the_bits(gpu):
    scs = members(4)
    alone = []
    for sc in scs:
        lat = lbm.from_scenario(sc, precision="f32")
        lat.step(64)
        alone.append(lat.pop())
        lat.close()
    lats = [lbm.from_scenario(sc, precision="f32") for sc in scs]
    ens = lbm.Ensemble(lats)
    ens.step(16)
    vec = ens.autotune(2)
    assert vec in (1, 2, 4)
    ens.step(48)
    ens.sync()
    for lat, p in zip(lats, alone):
        assert np.array_equal(lat.pop(), p)
    ens.close()
    for lat in lats:
        lat.close()
