"""Pins of the oracle's far-field pattern (exterior evaluation after the solve).

The scattered field outside the domain is u_s = -K(omega^2 m u) evaluated at exterior points;
its far-field pattern follows from the asymptotics of the Green's function.  Pins: the
pattern times e^{i omega r} r^{-(d-1)/2} equals the exterior field computed by the direct sum
of the Green's function at a distant point (which fixes the constant and the sign), the
pattern vanishes for m = 0, and reciprocity u_inf(theta; d) = u_inf(-d; -theta), which holds
exactly for the discrete system because K is symmetric (K(i, j) = k_{i-j} = k_{j-i}):
W (I + K W)^{-1} = (I + W K)^{-1} W is then symmetric.  Physics: for a constant-contrast
disk the pattern of the discrete solution converges to the Mie series' far field.
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_1408_4495_gb300 import workloads as W


def _solve_total(n, d, omega, m, dirs, tol):
    r = O.solve(n, d, omega, m, dirs, tol=tol)
    uI = np.array([O.plane_wave(n, d, omega, dr).reshape(-1) for dr in dirs])
    return r, uI + r["u"]


@pytest.mark.parametrize("d,n,freq", [(2, 32, 2.0), (3, 10, 1.0)])
def test_far_field_matches_the_exterior_field_at_a_distant_point(d, n, freq):
    omega = 2 * math.pi * freq
    rng = np.random.default_rng(2)
    m = W.enforce_buffer(W.bumps(n, d, [-0.2, 0.15], [0.1, 0.08], rng.uniform(0.35, 0.65, (2, d))), 2)
    dirs = np.eye(d)[:1]
    _, ut = _solve_total(n, d, omega, m, dirs, 1e-10)
    h = O.grid_h(n)
    X = np.stack([x.reshape(-1) for x in O.grid_coords(n, d)], -1)
    v = (omega**2 * m.reshape(-1) * ut[0])
    for th in (np.eye(d)[0], np.ones(d) / math.sqrt(d)):
        R = 1e6
        x = 0.5 + R * th  # far point in direction th from the domain centre
        rr = np.linalg.norm(x[None, :] - X, axis=1)
        us = -np.sum(O.green(d, omega, rr) * v) * h**d
        centre = 0.5 * np.ones(d)
        # u_inf is referred to the origin; shift the phase to the centre-based radius
        uinf = O.far_field(n, d, omega, m, ut[0].reshape((n,) * d), th[None, :])[0]
        r0 = np.linalg.norm(x)
        asym = np.exp(1j * omega * r0) * r0 ** (-(d - 1) / 2) * uinf
        assert abs(us - asym) < 1e-4 * abs(asym)


def test_far_field_of_zero_medium_is_zero():
    n, d = 16, 2
    u = np.ones((n, n), complex)
    assert np.all(O.far_field(n, d, 10.0, np.zeros((n, n)), u, np.array([[1.0, 0.0]])) == 0)


@pytest.mark.parametrize("d,n,freq,k", [(2, 32, 2.0, 8), (3, 10, 1.0, 6)])
def test_far_field_reciprocity_of_the_discrete_solution(d, n, freq, k):
    omega = 2 * math.pi * freq
    rng = np.random.default_rng(4)
    m = W.enforce_buffer(W.bumps(n, d, [-0.25, 0.2], [0.1, 0.07], rng.uniform(0.35, 0.65, (2, d))), 2)
    if d == 2:
        dirs = W.directions_circle(k)  # closed under negation for even k
    else:
        e = np.eye(3)
        dirs = np.concatenate([e, -e])
    neg = [int(np.argmin(np.linalg.norm(dirs + dr, axis=1))) for dr in dirs]
    assert all(np.allclose(dirs[neg[i]], -dirs[i]) for i in range(len(dirs)))
    _, ut = _solve_total(n, d, omega, m, dirs, 1e-12)
    F = np.array([O.far_field(n, d, omega, m, ut[i].reshape((n,) * d), dirs) for i in range(len(dirs))])
    # F[i, j] = u_inf(theta_j; d_i);  reciprocity: u_inf(theta_j; d_i) = u_inf(-d_i; -theta_j)
    G = np.array([[F[neg[j], neg[i]] for j in range(len(dirs))] for i in range(len(dirs))])
    assert np.max(np.abs(F - G)) < 1e-9 * np.max(np.abs(F))
    assert np.max(np.abs(F)) > 1e-3


def test_far_field_converges_to_the_mie_far_field():
    # discontinuous medium: no fixed order; measured 3.3e-2, 1.1e-2, 3.1e-3 at n = 32, 64, 128
    from oracle.mie import mie_disk_far_field
    omega = 2 * math.pi * 2
    th = np.linspace(0, 2 * math.pi, 16, endpoint=False)
    obs = np.stack([np.cos(th), np.sin(th)], axis=1)
    ref = mie_disk_far_field(th, omega, -0.3, 0.25)
    errs = []
    for n in (32, 64):
        X = O.grid_coords(n, 2)
        m = np.where(np.hypot(X[0] - 0.5, X[1] - 0.5) < 0.25, -0.3, 0.0)
        _, ut = _solve_total(n, 2, omega, m, [(1.0, 0.0)], 1e-10)
        F = O.far_field(n, 2, omega, m, ut[0].reshape(n, n), obs)
        errs.append(np.linalg.norm(F - ref) / np.linalg.norm(ref))
    assert errs[0] < 0.05
    assert errs[1] < 0.5 * errs[0]


def test_mie_far_field_is_the_limit_of_the_mie_field():
    # the pattern of the series equals u_s(x) e^{-i omega |x|} |x|^{1/2} at a distant x
    from oracle.mie import mie_disk_far_field, mie_disk_scattered
    omega = 2 * math.pi * 2
    th = np.array([0.0, 0.7, 2.0, 3.5, 5.1])
    rad = 1e6
    X1, X2 = rad * np.cos(th), rad * np.sin(th)
    us = mie_disk_scattered(X1, X2, omega, -0.3, 0.25)
    F = mie_disk_far_field(th, omega, -0.3, 0.25)
    lim = us * np.exp(-1j * omega * rad) * math.sqrt(rad)
    assert np.max(np.abs(lim - F)) < 1e-3 * np.max(np.abs(F))
