"""Parity of the higher-order weight of the singular point as a setup option
(ls_grid.k0_rule = LS_K0_CORRECTED, the one-point trapezoid correction of Sec. 2.1) with the
oracle given the same rule, through the C-ABI.

The library computes the weight on the host (its own lattice sum and Gauss-Legendre radial
quadrature) and the oracle with numpy / scipy; the two agree to ~1e-13 relative.  Every
other table entry and the stencils alpha are those of the default rule; C = alpha K(mu, mu)
moves by (k0_corrected - k0_ball) alpha.  Tolerances as in the other parity tests: the FP64
path takes the oracle's iterations and agrees to 1e-8, the mixed path reaches a true
relative residual <= 1e-6 and agrees with the oracle solved to 1e-10 within 1e-5.
"""

import numpy as np
import pytest

import oracle as O
from paper_1408_4495_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.late(1)]


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def medium(d, n, seed=0, amp=0.25):
    rng = np.random.default_rng(seed)
    nb = 3
    m = W.bumps(n, d, rng.uniform(-amp, amp, nb), rng.uniform(0.06, 0.12, nb), rng.uniform(0.3, 0.7, (nb, d)))
    return W.enforce_buffer(m, 2)


@pytest.fixture(scope="module")
def LS():
    from paper_1408_4495_gb300 import build, ls
    build.build()
    return ls


def _packed_c(d, mu0, c):
    out = np.zeros(3**d, complex)
    for t, cv in zip(mu0, c):
        out[sum((t[x] + 1) * 3 ** (d - 1 - x) for x in range(d))] = cv
    return out


@pytest.mark.parametrize("d,n,freq", [(2, 32, 4.0), (3, 16, 2.0), (3, 16, 0.0)])
def test_table_and_C_take_the_corrected_weight(LS, d, n, freq):
    omega = 2 * np.pi * freq
    lap = freq == 0.0
    m = medium(d, n)
    k0 = O.k0_corrected(d, omega, O.grid_h(n))
    with LS.Solver(m, omega, mixed=False, laplace=lap) as s:
        kb = s.kernel_table()
        Ab, Cb = s.stencils()
    with LS.Solver(m, omega, mixed=False, laplace=lap, k0_rule=LS.LS_K0_CORRECTED) as s:
        kc = s.kernel_table()
        Ac, Cc = s.stencils()
    assert abs(kc.flat[0] - k0) < 1e-11 * abs(k0)  # two independent quadratures (~2e-13 here)
    assert np.array_equal(kc.flat[1:], kb.flat[1:])
    assert np.max(np.abs(Ac - Ab)) < 1e-14
    _, (mu0, c) = O.all_stencils(n, d, omega, 2, k0=k0)
    ref = _packed_c(d, mu0, c)
    assert np.max(np.abs(Cc - ref)) < 1e-9 * np.max(np.abs(ref))
    assert np.max(np.abs(Cc - Cb)) > 1e-3 * np.max(np.abs(ref))


def test_plain_fp64_solve_with_the_corrected_weight(LS):
    w = W.plain_2d(32)
    m = W.enforce_buffer(w.m, 2)
    k0 = O.k0_corrected(2, w.omega, O.grid_h(w.n))
    ref = O.solve(w.n, 2, w.omega, m, w.directions, k0=k0)
    with LS.Solver(m, w.omega, mixed=False, k0_rule=LS.LS_K0_CORRECTED) as s:
        s.factor()
        g = s.rhs_plane_wave(w.directions)
        assert rel(g.reshape(1, -1), ref["g"]) < 1e-11
        u, info = s.solve(g, tol=1e-6)
    assert info[0].iters == ref["iters"][0]
    assert info[0].rel_resid <= 1e-6
    assert rel(u.reshape(1, -1), ref["u"]) < 1e-8


@pytest.mark.parametrize("d,n,freq,nrhs", [(2, 64, 8.0, 3), (3, 16, 2.0, 2)])
def test_mixed_solve_with_the_corrected_weight(LS, d, n, freq, nrhs):
    omega = 2 * np.pi * freq
    m = medium(d, n, seed=3)
    dirs = W.directions_circle(nrhs) if d == 2 else W.directions_sphere(nrhs, 7)
    k0 = O.k0_corrected(d, omega, O.grid_h(n))
    ref = O.solve(n, d, omega, m, dirs, tol=1e-10, k0=k0)
    ref6 = O.solve(n, d, omega, m, dirs, tol=1e-6, k0=k0)
    with LS.Solver(m, omega, mixed=True, k0_rule=LS.LS_K0_CORRECTED) as s:
        s.factor()
        g = s.rhs_plane_wave(dirs)
        u, info = s.solve(g, tol=1e-6)
    for j in range(nrhs):
        assert info[j].converged and info[j].rel_resid <= 1e-6
        assert rel(u[j].reshape(-1), ref["u"][j]) < 1e-5
        assert abs(info[j].iters - ref6["iters"][j]) <= 2


def test_laplace_solve_with_the_corrected_weight(LS):
    n = 16
    w = W.laplace_3d(n, 3, "gaussian", 1005)
    V = W.enforce_buffer(w.V, 2)
    k0 = O.k0_corrected(3, 0.0, O.grid_h(n))
    ref = O.laplace_solve(n, V, w.points, tol=1e-6, k0=k0)
    with LS.Solver(V, mixed=False, laplace=True, k0_rule=LS.LS_K0_CORRECTED) as s:
        s.factor()
        g = s.rhs_point_source(w.points)
        assert rel(g.reshape(len(w.points), -1), ref["g"]) < 1e-12
        u, info = s.solve(g, tol=1e-6)
    for j in range(len(w.points)):
        assert info[j].iters == ref["iters"][j]
        assert info[j].converged and info[j].rel_resid <= 1e-6
        assert rel(u[j].reshape(-1), ref["u"][j]) < 1e-8


def test_unknown_rule_is_refused(LS):
    with pytest.raises(LS.LsError) as e:
        LS.Solver(medium(2, 16), 2 * np.pi * 2, k0_rule=7)
    assert e.value.status == LS.LS_EINVAL
