"""Host-side parts of the autograd binding (no GPU): the body-property
formulas it differentiates agree with the oracle's, and its mass / length
chain rule agrees with differences of the oracle's body properties."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1108_0786_gb300 import autograd as ag, workloads as wl


@pytest.mark.parametrize("shape,r,l,m", [(wl.SPHERE, 3.0, 0.0, 150.0), (wl.CAPSULE, 3.0, 4.0, 226.2),
                                         (wl.CAPSULE, 1.8, 2.0, 70.0)])
def test_body_properties_match_the_oracle(shape, r, l, m):
    o = oracle.Oracle(16, 16, 16, 1.0)
    o.add_body(shape, r, l, m, (8.0, 8.0, 8.0))
    vol_inertia = o.body_props(0)
    inertia, vol = ag.body_properties(shape, r, torch.tensor(l, dtype=torch.float64),
                                      torch.tensor(m, dtype=torch.float64))
    np.testing.assert_allclose(inertia.numpy(), vol_inertia[1:], rtol=1e-14)
    assert abs(float(vol) - vol_inertia[0]) <= 1e-13 * vol_inertia[0]


def test_mass_length_chain_against_differences():
    body = wl.Body(wl.CAPSULE, 3.0, 4.0, 226.2, (8.0, 8.0, 8.0))
    gbody = np.array([0.3, -0.002, 0.01, 0.007, 0.05])       # dJ/d(m, I1, I2, I3, V)

    def J(m, l):
        o = oracle.Oracle(16, 16, 16, 1.0)
        o.add_body(body.shape, body.radius, l, m, body.pos)
        vi = o.body_props(0)
        return float((gbody * np.concatenate(([m], vi[1:], vi[:1]))).sum())
    dm, dl = ag._mass_length_chain(body, body.mass, body.length, gbody)
    h = 1e-4
    assert abs(dm - (J(body.mass + h, body.length) - J(body.mass - h, body.length)) / (2 * h)) < 1e-8
    assert abs(dl - (J(body.mass, body.length + h) - J(body.mass, body.length - h)) / (2 * h)) < 1e-7
