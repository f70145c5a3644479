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
