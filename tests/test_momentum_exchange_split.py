"""The split of the momentum-exchange sums (Eq. hydroF) that the GPU force
kernel uses for 32/16-bit storage, checked against the direct sums.

Per link (x_f, a) with x_f fluid and x_f + e_a solid:
    F_link = e_a [2 f~_a + 6 w_a rho e_-a . u_w],   T_link = (x_f + e_a/2 - X) x F_link,
f~_a = w_a + delta_a.  With x_f - X = i - c (i the integer offset from the
centre's cell, c the centre's position within it) and v = 2 delta_a +
6 w_a rho e_-a . u_w the kernel forms
    F = S1 / 36 + Fv,   T = (S2 - c x S1) / 36 + Tv - c x Fv,
    S1 = sum 72 w_a e_a,  S2 = sum i x 72 w_a e_a          (integers),
    Fv = sum v e_a,  Tv = sum v (i x e_a)   (v in FP32, each term rounded to
                                             2^-40 and summed as int64).
A dropped term, a wrong sign or a transposed cross product fails the
comparison below by orders of magnitude more than the FP32 rounding of v.
"""
import numpy as np
import pytest

E = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
              [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1],
              [1, 0, -1], [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]])
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
FIX_BITS = 40


def to_fixed(v):
    """round(v 2^40) to the nearest integer, ties away from zero (as the kernel)."""
    s = np.asarray(v, dtype=np.float64) * 2.0 ** FIX_BITS
    return (np.sign(s) * np.floor(np.abs(s) + 0.5)).astype(np.int64)


def links(rng, n=3000):
    X = rng.uniform(0, 64, 3)
    i = rng.integers(-9, 10, size=(n, 3))              # integer offsets from the centre's cell
    a = rng.integers(1, 19, size=n)
    delta = rng.normal(0, 3e-3, n) * W[a]
    rho = 1.0 + rng.normal(0, 1e-3, n)
    V, Om = rng.normal(0, 1e-3, 3), rng.normal(0, 1e-4, 3)
    return X, i, a, delta, rho, V, Om


def direct(X, i, a, delta, rho, V, Om):
    c = X - np.floor(X)
    o = i - c                                           # x_f - X
    e = E[a]
    uw = V + np.cross(Om, o + e)                        # wall velocity at x_f + e_a
    eu = -(e * uw).sum(1)                               # e_-a . u_w
    mag = 2 * (W[a] + delta) + 6 * W[a] * rho * eu
    F = (e * mag[:, None]).sum(0)
    T = np.cross(o + 0.5 * e, e * mag[:, None]).sum(0)
    return F, T


def split(X, i, a, delta, rho, V, Om, mistake=None):
    c = X - np.floor(X)
    e = E[a]
    K = np.where(a < 7, 4, 2)                           # 72 w_a
    S1 = (K[:, None] * e).sum(0)
    ie = np.cross(i, e)                                 # integer i x e_a
    S2 = (K[:, None] * ie).sum(0)
    # the FP32 variable part (offsets, wall velocity and v in FP32)
    f32 = np.float32
    o32 = i.astype(f32) - c.astype(f32)
    uw = V.astype(f32) + np.cross(Om.astype(f32), (o32 + e).astype(f32)).astype(f32)
    eu = -(e.astype(f32) * uw).sum(1, dtype=f32)
    w6 = np.where(a < 7, f32(1 / 3), f32(1 / 6)).astype(f32)
    v = (f32(2) * delta.astype(f32) + w6 * rho.astype(f32) * eu).astype(f32)
    Fv = (e * to_fixed(v)[:, None]).sum(0) / 2.0 ** FIX_BITS
    Tv = to_fixed(ie.astype(f32) * v[:, None]).sum(0) / 2.0 ** FIX_BITS
    if mistake == "flip_s2":
        S2 = -S2
    F = S1 / 36.0 + Fv
    T = (S2 - np.cross(c, S1)) / 36.0 + Tv - (0.0 if mistake == "drop_c_fv" else np.cross(c, Fv))
    return F, T


def variable_scale(X, i, a, delta, rho, V, Om):
    """sum |v e_a| and sum |v (i x e_a)| per axis: a few FP32 roundings of
    each v bound the split's error (the constant part has none)."""
    c = X - np.floor(X)
    e = E[a]
    uw = V + np.cross(Om, i - c + e)
    v = 2 * delta + 6 * W[a] * rho * (-(e * uw).sum(1))
    return (np.abs(e * v[:, None])).sum(0), (np.abs(np.cross(i, e) * v[:, None])).sum(0)


@pytest.mark.parametrize("seed", range(5))
def test_split_sums_equal_the_direct_sums(seed):
    rng = np.random.default_rng(seed)
    args = links(rng)
    Fd, Td = direct(*args)
    Fs, Ts = split(*args)
    sf, st = variable_scale(*args)
    u = 2.0 ** -24                                      # FP32 unit roundoff
    c = args[0] - np.floor(args[0])
    bound_f = 8 * u * sf + 1e-12
    bound_t = 8 * u * (st + np.abs(c).max() * sf.sum()) + 1e-12     # T also carries c x (error of Fv)
    assert np.all(np.abs(Fs - Fd) <= bound_f), (Fs - Fd, bound_f)
    assert np.all(np.abs(Ts - Td) <= bound_t), (Ts - Td, bound_t)
    # the bound has teeth: mistakes planted in the split exceed it by far
    for mistake in ("drop_c_fv", "flip_s2"):
        _, Tw = split(*args, mistake=mistake)
        assert np.abs(Tw - Td).max() > 100 * bound_t.max(), mistake


def test_a_transposed_cross_product_is_caught():
    rng = np.random.default_rng(11)
    X, i, a, delta, rho, V, Om = links(rng)
    _, Td = direct(X, i, a, delta, rho, V, Om)
    c = X - np.floor(X)
    e = E[a]
    K = np.where(a < 7, 4, 2)
    S1 = (K[:, None] * e).sum(0)
    S2 = (K[:, None] * np.cross(i, e)).sum(0)
    wrong = (S2 - np.cross(S1, c)) / 36.0              # c x S1 transposed
    right = (S2 - np.cross(c, S1)) / 36.0
    assert np.abs(right - wrong).max() > 1e3 * 1e-8


def test_to_fixed_rounds_to_nearest_ties_away():
    q = 2.0 ** -FIX_BITS
    assert list(to_fixed(np.array([0.5 * q, -0.5 * q, 1.49 * q, -2.5 * q]))) == [1, -1, 1, -3]
