"""Pins of the oracle's Green's function, Nystrom weights and kernel table (Sec. 1, Sec. 2.1).

Each check is a property fixed by the mathematics, not a re-call of the oracle's own
library routine: the PDE the Green's function solves, its singularity (scale and sign),
the outgoing radiation condition (which Hankel kind), and a numerical quadrature of the
disk / ball integral that defines the k_0 reading.
"""

import math

import numpy as np
import pytest
import scipy.integrate as si

import oracle as O


@pytest.mark.parametrize("d", [2, 3])
def test_green_solves_helmholtz_away_from_origin(d):
    # 4th-order central Laplacian of G at points away from 0: (Delta + omega^2) G = 0
    omega = 7.3
    dl = 2e-3
    rng = np.random.default_rng(0)
    for _ in range(5):
        x = rng.uniform(0.2, 0.8, d) * rng.choice([-1, 1], d)
        lap = 0.0
        for a in range(d):
            e = np.zeros(d)
            e[a] = dl
            f = lambda y: O.green(d, omega, np.linalg.norm(y))
            lap += (-f(x + 2 * e) + 16 * f(x + e) - 30 * f(x) + 16 * f(x - e) - f(x - 2 * e)) / (12 * dl * dl)
        g = O.green(d, omega, np.linalg.norm(x))
        assert abs(lap + omega**2 * g) < 1e-6 * omega**2 * abs(g)


def test_green_singularity_scale_and_sign():
    # fundamental solution of -Delta: 2D -(1/2pi) log r, 3D 1/(4 pi r)
    omega = 5.0
    r = 1e-7
    g2 = O.green(2, omega, r) - O.green(2, omega, 2 * r)
    assert abs(g2 - math.log(2.0) / (2 * math.pi)) < 1e-9
    g3 = O.green(3, omega, r) * 4 * math.pi * r
    assert abs(g3 - 1.0) < 1e-6


@pytest.mark.parametrize("d", [2, 3])
def test_green_is_outgoing(d):
    # Sommerfeld: r^{(d-1)/2} (dG/dr - i omega G) -> 0; the incoming kind would give -2i omega
    omega = 3.0
    for r in (200.0, 800.0):
        dr = 1e-4
        dG = (O.green(d, omega, r + dr) - O.green(d, omega, r - dr)) / (2 * dr)
        val = r ** ((d - 1) / 2) * (dG - 1j * omega * O.green(d, omega, r))
        scale = r ** ((d - 1) / 2) * omega * abs(O.green(d, omega, r))
        assert abs(val) < 5e-3 * scale


@pytest.mark.parametrize("omega,h", [(25.0, 1 / 33), (200.0, 1 / 257), (1.0, 0.1)])
def test_k0_equals_quadrature_over_equal_area_disk(omega, h):
    import scipy.special as sp
    a = h / math.sqrt(math.pi)
    # (i/4) * 2 pi * int_0^a r H0(omega r) dr, by adaptive quadrature of J0 and Y0 separately
    re = si.quad(lambda r: r * sp.j0(omega * r), 0, a, epsabs=0, epsrel=1e-13, limit=200)[0]
    im = si.quad(lambda r: r * sp.y0(omega * r), 0, a, epsabs=0, epsrel=1e-13, limit=200)[0]
    ref = 0.25j * 2 * math.pi * (re + 1j * im)
    assert abs(O.k0_weight(2, omega, h) - ref) < 1e-10 * abs(ref)


@pytest.mark.parametrize("omega,h", [(50.0, 1 / 65), (5.0, 0.1)])
def test_k0_equals_quadrature_over_equal_volume_ball(omega, h):
    a = h * (3 / (4 * math.pi)) ** (1 / 3)
    re = si.quad(lambda r: r * math.cos(omega * r), 0, a, epsabs=0, epsrel=1e-13)[0]
    im = si.quad(lambda r: r * math.sin(omega * r), 0, a, epsabs=0, epsrel=1e-13)[0]
    ref = re + 1j * im  # int over ball of e^{i w r}/(4 pi r) = int_0^a r e^{i w r} dr
    assert abs(O.k0_weight(3, omega, h) - ref) < 1e-11 * abs(ref)


def test_k0_laplace_limit_3d():
    # omega -> 0: int over ball of e^{i w r}/(4 pi r) = a^2/2 + i w a^3/3 + O(w^2 a^4)
    h = 0.05
    w = 1e-2
    a = h * (3 / (4 * math.pi)) ** (1 / 3)
    assert abs(O.k0_weight(3, w, h) - (a * a / 2 + 1j * w * a**3 / 3)) < 1e-10


@pytest.mark.parametrize("d,n", [(2, 7), (3, 4)])
def test_kernel_table_layout_and_symmetry(d, n):
    omega = 9.0
    h = O.grid_h(n)
    kt = O.kernel_table(n, d, omega)
    assert kt.shape == (2 * n - 1,) * d
    rng = np.random.default_rng(1)
    for _ in range(10):
        t = rng.integers(-(n - 1), n, d)
        v = kt[tuple(t + n - 1)]
        r = h * np.linalg.norm(t)
        ref = O.k0_weight(d, omega, h) if r == 0 else O.green(d, omega, r) * h**d
        assert v == ref
        assert kt[tuple(-t + n - 1)] == v                       # even
        assert kt[tuple(t[::-1] + n - 1)] == v                  # coordinate permutation
