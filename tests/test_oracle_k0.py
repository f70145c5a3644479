"""Pins of the higher-order weight of the singular point (Sec. 2.1: the one-point correction
of the trapezoidal rule is O(h^4 log(1/h)) accurate): the discrete convolution of a smooth
Gaussian field, evaluated at its centre, converges to the exact integral (a radial
quadrature) with order about 4 with k0_corrected and about 2 with the ball-integral weight;
the corrected weight does not depend on the width of the fitting Gaussian beyond that order.
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_1408_4495_gb300 import workloads as W


def _exact_centre_value(d, omega, w):
    """int G(y) exp(-|y|^2 / (2 w^2)) dy by the test's own radial quadrature (scipy's Hankel
    function in 2D, the exponential in 3D), on a fine fixed-order Gauss-Legendre grid."""
    import scipy.special as sp
    xs, ws = np.polynomial.legendre.leggauss(400)
    R = 12 * w
    edges = np.linspace(0, R, 41)
    val = 0j
    for a, b in zip(edges, edges[1:]):
        r = 0.5 * (b - a) * xs + 0.5 * (a + b)
        if d == 2:
            g = 0.25j * sp.hankel1(0, omega * r) * 2 * math.pi * r
        else:
            g = np.exp(1j * omega * r) * r  # 4 pi r^2 / (4 pi r)
        val += 0.5 * (b - a) * np.sum(ws * g * np.exp(-r * r / (2 * w * w)))
    return val


def _centre_error(d, omega, n, k0, w=0.08):
    h = O.grid_h(n)
    idx = np.stack(np.meshgrid(*([np.arange(n)] * d), indexing="ij"), -1).reshape(-1, d)
    ic = np.full(d, (n - 1) // 2)
    x = (idx + 1) * h
    v = np.exp(-np.sum((x - 0.5) ** 2, axis=1) / (2 * w * w))
    k = O.kernel_value(d, omega, h, idx - ic, k0)
    exact = _exact_centre_value(d, omega, w)
    return abs(np.sum(k * v) - exact) / abs(exact)


@pytest.mark.parametrize("d,omega,ns", [(2, 2 * math.pi * 2, (15, 31, 63, 127)),
                                        (3, 2 * math.pi * 1, (15, 31, 63)),
                                        (3, 0.0, (15, 31, 63))])
def test_corrected_weight_converges_at_fourth_order(d, omega, ns):
    eb, ec = [], []
    for n in ns:
        h = O.grid_h(n)  # n odd: the centre 1/2 is a grid point
        eb.append(_centre_error(d, omega, n, None))
        ec.append(_centre_error(d, omega, n, O.k0_corrected(d, omega, h)))
    ob = [math.log2(a / b) for a, b in zip(eb, eb[1:])]
    oc = [math.log2(a / b) for a, b in zip(ec, ec[1:])]
    assert all(1.7 < o < 2.3 for o in ob), ob
    assert all(o > 3.5 for o in oc), oc
    assert all(c < b for b, c in zip(eb, ec))


def test_corrected_weight_does_not_depend_on_the_fitting_width():
    h = 1 / 64
    a = O.k0_corrected(2, 2 * math.pi * 2, h, width=6.0)
    b = O.k0_corrected(2, 2 * math.pi * 2, h, width=10.0)
    assert abs(a - b) < 2e-3 * abs(a)


# ---- the weight as a setup option: it reaches C, the operator and the right-hand side ----

def _dense_system(d, n, omega, k0):
    """K(i, j) = G(h |i - j|) h^d off the diagonal, k0 on it, straight from the Green's
    function (scipy's Hankel function / the exponential), independent of the oracle's table."""
    import scipy.special as sp
    h = 1.0 / (n + 1)
    idx = np.stack(np.meshgrid(*([np.arange(n)] * d), indexing="ij"), -1).reshape(-1, d)
    r = h * np.linalg.norm(idx[:, None, :] - idx[None, :, :], axis=-1)
    rs = np.where(r > 0, r, 1.0)
    if d == 2:
        G = 0.25j * sp.hankel1(0, omega * rs)
    else:
        G = np.exp(1j * omega * rs) / (4 * math.pi * rs)
    K = np.where(r > 0, G * h**d, k0)
    x = (idx + 1.0) * h
    return K, x


@pytest.mark.parametrize("d,n,omega", [(2, 16, 2 * math.pi * 2), (3, 8, 2 * math.pi * 1), (3, 8, 0.0)])
def test_weight_enters_C_through_the_diagonal_only(d, n, omega):
    # C = alpha K(mu, mu) and K(mu, mu) holds k_0 on its diagonal alone, so moving k_0 by
    # delta moves C by delta * alpha; alpha itself is unchanged (the far sets exclude mu)
    h = O.grid_h(n)
    kb, kc = O.k0_weight(d, omega, h), O.k0_corrected(d, omega, h)
    assert abs(kc - kb) > 1e-3 * abs(kb)
    sb, (mu, cb) = O.all_stencils(n, d, omega, 2)
    sc, (mu2, cc) = O.all_stencils(n, d, omega, 2, k0=kc)
    assert mu == mu2
    for cls in sb:
        assert np.array_equal(sb[cls][1], sc[cls][1])
    a0 = sb[(0,) * d][1]
    assert np.max(np.abs((cc - cb) - (kc - kb) * a0)) < 1e-13 * np.max(np.abs(cb))


@pytest.mark.parametrize("d,n,freq", [(2, 20, 3.0), (3, 8, 1.0)])
def test_solve_with_the_corrected_weight_matches_the_dense_system(d, n, freq):
    omega = 2 * math.pi * freq
    k0 = O.k0_corrected(d, omega, 1.0 / (n + 1))
    m = W.enforce_buffer(W.bumps(n, d, [-0.2], [0.1], [(0.5,) * d]), 2)
    dr = np.array([1.0, 0.0]) if d == 2 else np.array([0.0, 0.6, 0.8])
    res = O.solve(n, d, omega, m, [tuple(dr)], tol=1e-12, k0=k0)
    K, x = _dense_system(d, n, omega, k0)
    w2m = omega**2 * m.reshape(-1)
    g = -K @ (w2m * np.exp(1j * omega * (x @ dr)))
    u = np.linalg.solve(np.eye(n**d) + K * w2m[None, :], g)
    assert np.linalg.norm(res["g"][0] - g) < 1e-12 * np.linalg.norm(g)
    assert np.linalg.norm(res["u"][0] - u) < 1e-9 * np.linalg.norm(u)


def test_laplace_solve_with_the_corrected_weight_matches_the_dense_system():
    n = 8
    k0 = O.k0_corrected(3, 0.0, 1.0 / (n + 1))
    w = W.laplace_3d(n, 1, seed=5)
    V = W.enforce_buffer(w.V, 2)
    res = O.laplace_solve(n, V, w.points, tol=1e-12, k0=k0)
    K, _ = _dense_system(3, n, 0.0, k0)
    f = np.zeros(n**3)
    f[np.ravel_multi_index(tuple(w.points[0]), (n,) * 3)] = (n + 1) ** 3
    g = K @ f
    u = np.linalg.solve(np.eye(n**3) + K * V.reshape(-1)[None, :], g)
    assert np.linalg.norm(res["g"][0] - g) < 1e-12 * np.linalg.norm(g)
    assert np.linalg.norm(res["u"][0] - u) < 1e-9 * np.linalg.norm(u)


def test_solution_converges_at_fourth_order_with_the_corrected_weight():
    """Sec. 2.1: for a smooth medium the corrected trapezoid rule makes the discrete solution
    O(h^4 log(1/h)) accurate; the ball weight leaves it O(h^2).  Nested grids h = 1/16,
    1/32, 1/64 against h = 1/128 (corrected weight) on the shared points, for a C-infinity
    bump of compact support; the observed orders (about 2 and 4-5) are checked with margin."""
    omega = 2 * math.pi * 2.0

    def medium(n):
        x = (np.arange(n) + 1.0) / (n + 1)
        X, Y = np.meshgrid(x, x, indexing="ij")
        s = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2) / 0.3
        m = np.zeros_like(s)
        inside = s < 1
        m[inside] = -0.3 * np.exp(1 - 1 / (1 - s[inside] ** 2))
        return m

    def solve(n, corrected):
        k0 = O.k0_corrected(2, omega, 1.0 / (n + 1)) if corrected else None
        r = O.solve(n, 2, omega, medium(n), [(1.0, 0.0)], tol=1e-12, k0=k0)
        return r["u"][0].reshape(n, n)

    ref = solve(127, True)
    err = {}
    for corrected in (False, True):
        for n in (15, 31, 63):
            s = 128 // (n + 1)
            f = ref[s - 1::s, s - 1::s]
            err[corrected, n] = np.linalg.norm(solve(n, corrected) - f) / np.linalg.norm(f)
    for n0, n1 in ((15, 31), (31, 63)):
        ball = math.log2(err[False, n0] / err[False, n1])
        corr = math.log2(err[True, n0] / err[True, n1])
        assert 1.6 < ball < 2.6, (n0, ball)
        assert corr > 3.5, (n0, corr)
    assert err[True, 63] < err[False, 63] / 50
