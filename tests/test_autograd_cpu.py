"""Host-side parts of the autograd binding (no GPU): the library's body
properties (lbm_body_properties, the values lbm_add_body uses) agree with
the oracle's, their derivatives with respect to mass and capsule length agree
with central differences of the oracle's body properties, and the binding's
mass / length chain rule agrees with differences of a function of the
oracle's properties."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1108_0786_gb300 import _build, autograd as ag, lbm, workloads as wl

CASES = [(wl.SPHERE, 3.0, 0.0, 150.0), (wl.CAPSULE, 3.0, 4.0, 226.2), (wl.CAPSULE, 1.8, 2.0, 70.0),
         (wl.CAPSULE, 4.0, 8.0, 670.2)]


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


def oracle_props(shape, r, l, m):
    """(V, I1, I2, I3) from the oracle."""
    o = oracle.Oracle(32, 32, 32, 1.0)
    o.add_body(shape, r, l, m, (16.0, 16.0, 16.0))
    return o.body_props(0)


@pytest.mark.parametrize("shape,r,l,m", CASES)
def test_body_properties_match_the_oracle(shape, r, l, m):
    q, _, _ = lbm.body_properties(shape, r, l, m)
    np.testing.assert_allclose(q, oracle_props(shape, r, l, m), rtol=1e-14)


@pytest.mark.parametrize("shape,r,l,m", CASES)
def test_body_property_derivatives_against_differences(shape, r, l, m):
    _, d_m, d_l = lbm.body_properties(shape, r, l, m)
    h = 1e-4 * m
    fd_m = (oracle_props(shape, r, l, m + h) - oracle_props(shape, r, l, m - h)) / (2 * h)
    np.testing.assert_allclose(d_m, fd_m, rtol=1e-8, atol=1e-12)
    if shape == wl.CAPSULE:
        hl = 1e-4
        fd_l = (oracle_props(shape, r, l + hl, m) - oracle_props(shape, r, l - hl, m)) / (2 * hl)
        np.testing.assert_allclose(d_l, fd_l, rtol=1e-7)
    else:
        assert not d_l.any()


def test_body_properties_reject_bad_dimensions():
    for args in ((wl.SPHERE, 3.0, 1.0, 10.0), (wl.CAPSULE, -1.0, 2.0, 10.0), (7, 1.0, 0.0, 1.0)):
        with pytest.raises(lbm.LbmError):
            lbm.body_properties(*args)


def test_mass_length_chain_against_differences():
    body = wl.Body(wl.CAPSULE, 3.0, 4.0, 226.2, (8.0, 8.0, 8.0))
    gbody = np.array([0.3, -0.002, 0.01, 0.007, 0.05])       # dJ/d(m, I1, I2, I3, V)

    def J(m, l):
        vi = oracle_props(body.shape, body.radius, l, m)
        return float((gbody * np.concatenate(([m], vi[1:], vi[:1]))).sum())
    dm, dl = ag._mass_length_chain(body, body.mass, body.length, gbody)
    h = 1e-4
    assert abs(dm - (J(body.mass + h, body.length) - J(body.mass - h, body.length)) / (2 * h)) < 1e-8
    assert abs(dl - (J(body.mass, body.length + h) - J(body.mass, body.length - h)) / (2 * h)) < 1e-7
