"""Pins of the oracle's D3Q19 lattice and equilibrium (Sec. 2.1).

The paper names the D3Q19 set of Qian, d'Humieres and Lallemand and the LBGK
collision but prints neither the weights nor f_eq.  These tests pin the
oracle's table and equilibrium to the closed-form lattice moments that define
them, so a wrong weight, a transposed velocity or a dropped term fails.
"""
import itertools

import numpy as np
import pytest

import oracle

# the population order documented in the headers
DOC_ORDER = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
             (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1),
             (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]


def test_velocity_set_is_documented_d3q19():
    e, w = oracle.lattice()
    assert [tuple(v) for v in e] == DOC_ORDER
    # D3Q19: the rest vector, the 6 face neighbours and the 12 edge neighbours
    norms = sorted(int(v @ v) for v in e)
    assert norms == [0] + [1] * 6 + [2] * 12


def test_weight_moments_are_isotropic():
    """sum w = 1, sum w e_i e_j = d_ij / 3, sum w e_i e_j e_k e_l = (dd+dd+dd)/9."""
    e, w = oracle.lattice()
    assert abs(w.sum() - 1.0) < 1e-15
    for i in range(3):
        assert abs((w * e[:, i]).sum()) < 1e-16
        for j in range(3):
            assert abs((w * e[:, i] * e[:, j]).sum() - (i == j) / 3.0) < 1e-15
            for k in range(3):
                assert abs((w * e[:, i] * e[:, j] * e[:, k]).sum()) < 1e-16
    d = np.eye(3)
    for i, j, k, l in itertools.product(range(3), repeat=4):
        m4 = (w * e[:, i] * e[:, j] * e[:, k] * e[:, l]).sum()
        iso = (d[i, j] * d[k, l] + d[i, k] * d[j, l] + d[i, l] * d[j, k]) / 9.0
        assert abs(m4 - iso) < 1e-15, (i, j, k, l)


@pytest.mark.parametrize("rho,u", [(1.0, (0.0, 0.0, 0.0)), (1.03, (0.02, -0.01, 0.005)),
                                   (0.97, (-0.04, 0.03, 0.01))])
def test_equilibrium_moments(rho, u):
    """f_eq reproduces rho, rho u and the momentum flux rho (u u + I / 3) exactly."""
    e, _ = oracle.lattice()
    f = oracle.equilibrium(rho, u)
    u = np.array(u)
    assert abs(f.sum() - rho) < 1e-14
    assert np.allclose(e.T @ f, rho * u, atol=1e-15, rtol=0)
    flux = np.einsum("a,ai,aj->ij", f, e, e)
    assert np.allclose(flux, rho * (np.outer(u, u) + np.eye(3) / 3.0), atol=1e-14, rtol=0)


def test_equilibrium_at_rest_is_the_weights():
    _, w = oracle.lattice()
    assert np.array_equal(oracle.equilibrium(1.0, (0.0, 0.0, 0.0)), w)
