"""The general-domain solve of Sec. 4 on the device, through the C-ABI (ls_general_support,
ls_general_sketch, ls_general_boundary_stencils, ls_general_setup, ls_factor, ls_solve).

The library keeps the box: every point off the unknowns Omega gets the identity row in M
and [A;B], so the preconditioner is diag(M_Omega^{-1} [A;B]_Omega, I), and the operator is
the box's (m vanishes off Omega, so A = [[A_OO, 0], [A_xO, I]] in the order Omega, rest).
The preconditioned operator is block lower triangular with an identity block, so GMRES on
the box takes at most one iteration more than the restricted method and its solution
restricted to Omega is the restricted solution (checked with the oracle's pieces on the CPU
for these cases: +1 iteration, agreement 1e-11 at tolerance 1e-10).

Checks against the oracle's restricted method (general_stencils / general_solve, same R):
the per-point stencil apply (FP64 to rounding, FP32 to 1e-6 relative), the preconditioner's
backward error, and the solve (FP64: the oracle's iterations or one more, solution within 1e-8 of
the oracle solved to 1e-10; mixed: within +-2 of that count, true relative residual
<= 1e-6, solution within 1e-5).  It runs after the established GPU tests (marker late).
"""

import itertools
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_1408_4495_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.late(3)]

CASES = [(2, 32, 4.0, "l2", 0.35), (2, 64, 8.0, "l1", 0.38), (3, 16, 2.0, "l2", 0.3)]
# backward error bounds of the preconditioner (FP64, FP32 fronts) per case, see below
BE_BOUND = {(2, 32, "l2"): (5e-13, 2e-5), (2, 64, "l1"): (1e-11, 6e-3), (3, 16, "l2"): (5e-13, 2e-5)}


@pytest.fixture(scope="module")
def LS():
    from paper_1408_4495_gb300 import build, ls
    build.build()
    return ls


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def case(d, n, freq, norm, rho):
    omega = 2 * math.pi * freq
    m = W.cavity(n, d, norm, rho=rho)
    idx = O.general_support(m, 2)
    R = np.random.default_rng(5).standard_normal((len(idx), 2 * 3**d))
    return omega, m, idx, R


def box_matrices(n, d, omega, m, st):
    """M and [A;B] of the box from the oracle's general-domain stencils: identity rows off
    Omega, boundary rows alpha_i, interior rows alpha + C omega^2 m."""
    idx, interior, bnd, (mu0, a0), (mu0c, c) = st
    N = n**d
    inter = np.zeros(N, dtype=bool)
    inter[idx[interior]] = True
    on = np.zeros(N, dtype=bool)
    on[idx] = True
    w2m = (omega**2 * m).reshape(-1)
    amap, cmap = dict(zip(mu0, a0)), dict(zip(mu0c, c))
    rows, cols, mv, sv = [], [], [], []
    for i in range(N):
        x = np.array(np.unravel_index(i, (n,) * d))
        if not on[i]:
            rows.append(i); cols.append(i); mv.append(1.0); sv.append(1.0)
            continue
        pairs = ([(t, amap[t]) for t in itertools.product((-1, 0, 1), repeat=d)] if inter[i]
                 else list(zip(*bnd[int(i)])))
        for t, a in pairs:
            j = int(np.ravel_multi_index(tuple(x + np.array(t)), (n,) * d))
            rows.append(i); cols.append(j); sv.append(a)
            mv.append(a + cmap[t] * w2m[j] if inter[i] else a)
    M = sp.csr_matrix((mv, (rows, cols)), shape=(N, N))
    S = sp.csr_matrix((sv, (rows, cols)), shape=(N, N))
    return M, S


def library_box_matrices(LS, s, n, d, omega, m, mask, alpha, bnd):
    """M and [A;B] of the box from the library's own rows (ls_general_rows of the stencils it
    derived from its device sketch), with the interior stencil and C of the context."""
    P3 = 3**d
    a_cls, c_int = s.stencils()
    rows, inter = LS.general_rows(mask, alpha, bnd, a_cls[(P3 - 1) // 2])
    offs = [np.array(t) for t in itertools.product((-1, 0, 1), repeat=d)]
    w2m = (omega**2 * m).reshape(-1)
    shape = (n,) * d
    ri, ci, mv, sv = [], [], [], []
    for i in range(n**d):
        x = np.array(np.unravel_index(i, shape))
        for t, tv in enumerate(offs):
            y = x + tv
            if np.any(y < 0) or np.any(y >= n) or rows[i, t] == 0:
                continue
            j = int(np.ravel_multi_index(tuple(y), shape))
            ri.append(i); ci.append(j); sv.append(rows[i, t])
            mv.append(rows[i, t] + (c_int[t] * w2m[j] if inter[i] else 0))
    N = n**d
    return sp.csr_matrix((mv, (ri, ci)), shape=(N, N)), sp.csr_matrix((sv, (ri, ci)), shape=(N, N))


@pytest.mark.parametrize("d,n,freq,norm,rho", CASES)
@pytest.mark.parametrize("mixed", [False, True])
def test_general_stencil_apply_and_preconditioner(LS, d, n, freq, norm, rho, mixed):
    """Two references.  (1) The library's rows: its stencil kernel must apply, and its
    factorization invert, exactly the rows its host step built from its device sketch, so the
    apply is held to rounding (FP64 1e-12, FP32 1e-6) and the preconditioner to the backward
    error of the rectangular path.  (2) The oracle's rows: the library's boundary stencils come
    from its own sketch and SVD and differ from the oracle's by at most delta = 1e-7 per
    coefficient (the bound test_gpu_general.py derives and checks for this route), so with
    |dalpha_i|_2 <= 3^(d/2) delta per row and every x_j in at most 3^d rows,
    |y - S_oracle x|_2 <= 3^d delta |x|_2.

    The backward error of the preconditioner grows like cond(F11) u (the sweeps multiply by
    the explicit inverse of every front's pivot block).  On the 2D n = 64 l1 cavity the
    diagonal boundary of Omega gives pivot blocks with cond ~ 1.5e4: measured on GB300
    1.7e-12 (FP64) and 1.2e-3 (FP32), whose ratio is u_32 / u_64, so that case takes about 5x
    those values as its bounds; the other cases keep the rectangular path's 5e-13 / 2e-5."""
    omega, m, idx, R = case(d, n, freq, norm, rho)
    st = O.general_stencils(n, d, omega, m, R)
    _, S_or = box_matrices(n, d, omega, m, st)
    rng = np.random.default_rng(17)
    x = rng.standard_normal((2,) + (n,) * d) + 1j * rng.standard_normal((2,) + (n,) * d)
    with LS.Solver(m, omega, dim=d, mixed=mixed) as s:
        mask = LS.general_support(m, 2)
        T = s.general_sketch(mask, R)
        alpha, bnd = LS.general_boundary_stencils(mask, T)
        s.general_setup(mask, alpha, bnd)
        M, S = library_box_matrices(LS, s, n, d, omega, m, mask, alpha, bnd)
        y = s.stencil_apply(x)
        s.factor()
        z = s.precond(x)
    normM = abs(M).sum(axis=1).max()
    be_bound = BE_BOUND[(d, n, norm)][1 if mixed else 0]
    for j in range(2):
        xj = x[j].reshape(-1)
        ref = S @ xj
        assert rel(y[j].reshape(-1), ref) < (1e-6 if mixed else 1e-12)
        dev = np.linalg.norm(y[j].reshape(-1) - S_or @ xj)
        assert dev <= 3**d * 1e-7 * np.linalg.norm(xj) + (1e-6 if mixed else 1e-12) * np.linalg.norm(ref), dev
        zj = z[j].reshape(-1)
        be = np.linalg.norm(M @ zj - ref) / (normM * np.linalg.norm(zj))
        print(f"general-domain preconditioner backward error d={d} n={n} {norm} mixed={mixed}: {be:.3g}")
        assert be < be_bound, be


@pytest.mark.parametrize("d,n,freq,norm,rho", CASES)
@pytest.mark.parametrize("mixed", [False, True])
def test_general_solve_matches_the_restricted_oracle(LS, d, n, freq, norm, rho, mixed):
    omega, m, idx, R = case(d, n, freq, norm, rho)
    dirs = W.directions_circle(2) if d == 2 else W.directions_sphere(2, 7)
    ref = O.general_solve(n, d, omega, m, dirs, R, tol=1e-10)
    ref6 = O.general_solve(n, d, omega, m, dirs, R, tol=1e-6)
    with LS.Solver(m, omega, dim=d, mixed=mixed) as s:
        mask = s.general_domain(m, R)
        s.factor()
        g = s.rhs_plane_wave(dirs)
        u, info = s.solve(g, tol=1e-6)
    assert np.array_equal(np.flatnonzero(mask.reshape(-1)), idx)
    for j in range(len(dirs)):
        assert rel(g[j].reshape(-1)[idx], ref["g"][j]) < 1e-11
        assert info[j].converged and info[j].rel_resid <= 1e-6
        if mixed:
            assert abs(info[j].iters - (ref6["iters"][j] + 1)) <= 2
            assert rel(u[j].reshape(-1)[idx], ref["u"][j]) < 1e-5
        else:
            assert ref6["iters"][j] <= info[j].iters <= ref6["iters"][j] + 1
            assert rel(u[j].reshape(-1)[idx], ref["u"][j]) < 1e-8


def test_general_setup_refuses_inconsistent_flags(LS):
    n, d = 32, 2
    omega, m, idx, R = case(d, n, 4.0, "l2", 0.35)
    with LS.Solver(m, omega, dim=d, mixed=False) as s:
        mask = LS.general_support(m, 2)
        T = s.general_sketch(mask, R)
        alpha, bnd = LS.general_boundary_stencils(mask, T)
        wrong = bnd.copy()
        wrong[np.flatnonzero(bnd)[0]] = False  # a boundary point claimed interior
        with pytest.raises(LS.LsError) as e:
            s.general_setup(mask, alpha, wrong)
        assert e.value.status == LS.LS_EINVAL
        s.general_setup(mask, alpha, bnd)
        with pytest.raises(LS.LsError) as e:  # the factorization was dropped
            s.solve(s.rhs_plane_wave(W.directions_circle(1)), tol=1e-6)
        assert e.value.status == LS.LS_ESTATE
