"""The device-side running velocity average (lbm_average_*; Sec. 6, the
flow fields around one and three swimmers averaged over swimming cycles)
against the oracle's average on a reduced copy of the Sec. 6 channel: the
design (a) swimmer, alone and three side by side, in a 48 x 48 x 80 channel
(walls in x and y, periodic in z) with the study's parameters and a period
of 400 steps.  FP64 storage within the parity bar, FP32 storage within its
velocity bar; a member averaged inside an ensemble gives the bits of the
same run stepped alone."""
import numpy as np
import pytest

import oracle
from paper_1108_0786_gb300 import design_study as ds, lbm

pytestmark = pytest.mark.gpu

DOMAIN, PERIOD, WARM, STEPS = (48, 48, 80), 400, 48, 224


@pytest.fixture(scope="module", autouse=True)
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1108_0786_gb300 import _build
    _build.build()


_REF = {}


def reference(swimmers):
    if swimmers not in _REF:
        sc = ds.flow_field_scenario(swimmers, DOMAIN, PERIOD)
        o = oracle.from_scenario(sc, oracle.OPT_AVERAGE_FORCE)
        o.step(WARM)
        o.average_begin()
        o.step(STEPS)
        _REF[swimmers] = (sc, *o.average())
    return _REF[swimmers]


def gpu_average(sc, precision):
    lat = lbm.from_scenario(sc, precision=precision, options=lbm.OPT_AVERAGE_FORCE)
    lat.step(WARM)
    lat.average_begin()
    lat.step(STEPS)
    out = lat.average()
    lat.close()
    return out


@pytest.mark.parametrize("swimmers", [1, 3])
def test_fp64_average_matches_the_oracle(swimmers):
    sc, want, n_want = reference(swimmers)
    got, n = gpu_average(sc, "f64")
    assert n == n_want == STEPS
    assert np.abs(want).max() > 1e-7
    assert np.abs(got - want).max() <= 1e-12 + 1e-10 * np.abs(want).max()


@pytest.mark.parametrize("swimmers", [1, 3])
def test_fp32_average_within_the_velocity_bar(swimmers):
    sc, want, _ = reference(swimmers)
    got, _ = gpu_average(sc, "f32")
    assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)


def test_average_inside_an_ensemble_equals_the_solo_run():
    sc = ds.flow_field_scenario(1, DOMAIN, PERIOD)
    solo, n_solo = gpu_average(sc, "f32")
    lats = [lbm.from_scenario(sc, precision="f32", options=lbm.OPT_AVERAGE_FORCE) for _ in range(2)]
    ens = lbm.Ensemble(lats)
    ens.step([WARM, WARM])
    lats[0].average_begin()                  # only the first member averages
    ens.step([STEPS, STEPS])
    ens.sync()
    got, n = lats[0].average()
    assert n == n_solo == STEPS
    assert np.array_equal(got, solo)
    with pytest.raises(lbm.LbmError) as ei:
        lats[1].average()
    assert ei.value.code == lbm.E_STATE
    ens.close()
    for lat in lats:
        lat.close()
