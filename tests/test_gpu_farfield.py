"""Far-field pattern (exterior evaluation) through the C-ABI, against the oracle.

ls_far_field is a plain FP64 sum, so it matches the oracle's sum to rounding (relative
<= 1e-12).  On solutions it must satisfy reciprocity u_inf(theta; d) = u_inf(-d; -theta),
which holds exactly for the discrete system (K symmetric), to the accuracy of the solve:
<= 1e-8 for FP64 solves to 1e-10, <= 1e-4 for mixed solves to 1e-6.
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_1408_4495_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def LS():
    from paper_1408_4495_gb300 import build, ls
    build.build()
    return ls


def medium(d, n, seed=0):
    rng = np.random.default_rng(seed)
    return W.enforce_buffer(W.bumps(n, d, rng.uniform(-0.25, 0.25, 3), rng.uniform(0.06, 0.12, 3),
                                    rng.uniform(0.3, 0.7, (3, d))), 2)


def obs_dirs(d, k, seed=3):
    if d == 2:
        return W.directions_circle(k)
    return W.directions_sphere(k, seed)


@pytest.mark.parametrize("d,n,freq", [(2, 32, 4.0), (2, 64, 6.0), (3, 16, 2.0)])
def test_far_field_matches_oracle(LS, d, n, freq):
    omega = 2 * math.pi * freq
    m = medium(d, n)
    dirs = obs_dirs(d, 3, 9)
    obs = obs_dirs(d, 7, 5)
    rng = np.random.default_rng(1)
    us = rng.standard_normal((3,) + (n,) * d) + 1j * rng.standard_normal((3,) + (n,) * d)
    with LS.Solver(m, omega, mixed=True) as s:
        F = s.far_field(dirs, us, obs)
    for r in range(3):
        ut = O.plane_wave(n, d, omega, dirs[r]) + us[r]
        ref = O.far_field(n, d, omega, m, ut, obs)
        assert np.max(np.abs(F[r] - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("mixed,tol,bound", [(False, 1e-10, 1e-8), (True, 1e-6, 1e-4)])
def test_far_field_reciprocity_of_gpu_solutions(LS, mixed, tol, bound):
    d, n, omega = 2, 64, 2 * math.pi * 6.0
    m = medium(d, n, 2)
    dirs = W.directions_circle(8)
    neg = [int(np.argmin(np.linalg.norm(dirs + dr, axis=1))) for dr in dirs]
    with LS.Solver(m, omega, mixed=mixed) as s:
        s.factor()
        g = s.rhs_plane_wave(dirs)
        u, info = s.solve(g, tol=tol)
        F = s.far_field(dirs, u, dirs)
    G = np.array([[F[neg[j], neg[i]] for j in range(8)] for i in range(8)])
    assert np.max(np.abs(F - G)) < bound * np.max(np.abs(F))
    assert np.max(np.abs(F)) > 1e-3


def test_far_field_bench_workload(LS):
    """2D n=256, 16 directions, 64 observation directions, on the solutions of the bench step."""
    w = W.bumps_2d(256, 32.0, 8, 16, 1002)
    m = W.enforce_buffer(w.m, 2)
    obs = W.directions_circle(64)
    with LS.Solver(m, w.omega, mixed=True) as s:
        s.factor()
        g = s.rhs_plane_wave(w.directions)
        u, info = s.solve(g, tol=1e-6)
        F = s.far_field(w.directions, u, obs)
    for r in (0, 7):
        ut = O.plane_wave(256, 2, w.omega, w.directions[r]) + u[r]
        ref = O.far_field(256, 2, w.omega, m, ut, obs[::8])
        assert np.max(np.abs(F[r, ::8] - ref)) < 1e-12 * np.max(np.abs(ref))


def test_far_field_refused_for_laplace(LS):
    w = W.laplace_3d(16, 1)
    with LS.Solver(W.enforce_buffer(w.V, 2), laplace=True) as s:
        with pytest.raises(LS.LsError) as e:
            s.far_field(np.array([[1.0, 0, 0]]), np.zeros((1, 16, 16, 16), complex), np.array([[1.0, 0, 0]]))
        assert e.value.status == LS.LS_ESTATE
