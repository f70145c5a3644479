"""Pins of the oracle's preconditioner (eq. PC), nested dissection, GMRES and whole solve."""

import json
import os

import numpy as np
import pytest

import oracle as O
from oracle.mie import mie_disk_scattered, mie_sphere_scattered
from paper_1408_4495_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _bump(n, d, A=-0.2, w=0.1):
    return W.enforce_buffer(W.bumps(n, d, [A], [w], [(0.5,) * d]), 2)


@pytest.mark.parametrize("d,n", [(2, 12), (3, 6)])
def test_preconditioner_is_identity_for_zero_medium(d, n):
    # m = 0: M = [A;B] = S, so P = M^{-1} S = I exactly (eq. PC)
    omega = 2 * np.pi * 2
    sten, cint = O.all_stencils(n, d, omega, 2)
    M, S = O.assemble(n, d, omega, np.zeros((n,) * d), sten, cint)
    P = O.Preconditioner(M, S, n, d)
    rng = np.random.default_rng(6)
    v = rng.standard_normal(n**d) + 1j * rng.standard_normal(n**d)
    assert np.linalg.norm(P(v) - v) < 1e-10 * np.linalg.norm(v)


def test_sparse_lu_equals_dense_solve():
    n, d = 16, 2
    omega = 2 * np.pi * 3
    m = _bump(n, d)
    sten, cint = O.all_stencils(n, d, omega, 2)
    M, S = O.assemble(n, d, omega, m, sten, cint)
    P = O.Preconditioner(M, S, n, d)
    rng = np.random.default_rng(7)
    r = rng.standard_normal(n * n) + 1j * rng.standard_normal(n * n)
    ref = np.linalg.solve(M.toarray(), r)
    assert np.linalg.norm(P.solve_M(r) - ref) < 1e-10 * np.linalg.norm(ref)


def test_assembly_rows_follow_the_stencils():
    n, d = 9, 2
    omega = 20.0
    m = np.zeros((n, n))
    m[4, 4] = 0.3
    sten, (mu0, c) = O.all_stencils(n, d, omega, 2)
    M, S = O.assemble(n, d, omega, m, sten, (mu0, c))
    Md, Sd = M.toarray(), S.toarray()
    idx = lambda a, b_: a * n + b_
    # interior row next to the perturbation: alpha + c * omega^2 m at the one column
    mu, alpha = sten[(0, 0)]
    for t, a in zip(mu, alpha):
        col = idx(3 + t[0], 3 + t[1])
        extra = c[mu0.index(t)] * omega**2 * m[3 + t[0], 3 + t[1]]
        assert abs(Md[idx(3, 3), col] - (a + extra)) < 1e-15
        assert Sd[idx(3, 3), col] == a
    # boundary rows: B only; nnz per row = |mu(i)|
    assert np.count_nonzero(Sd[idx(0, 0)]) == 4
    assert np.count_nonzero(Sd[idx(0, 4)]) == 6
    assert np.count_nonzero(Sd[idx(4, 4)]) == 9


@pytest.mark.parametrize("d,n", [(2, 37), (3, 11)])
def test_nd_order_is_a_permutation_with_separating_slabs(d, n):
    p = O.nd_order(n, d)
    assert np.array_equal(np.sort(p), np.arange(n**d))
    # top-level split of the cube along axis 0 at mid: the two halves are not adjacent
    mid = n // 2
    idx = np.indices((n,) * d).reshape(d, -1).T
    a0 = idx[:, 0]
    left = a0 < mid
    right = a0 > mid
    assert np.min(a0[right]) - np.max(a0[left]) == 2
    # the separator slab is eliminated last
    assert np.all(idx[p[-n ** (d - 1):], 0] == mid)


def test_gmres_matches_dense_solve_on_random_system():
    rng = np.random.default_rng(8)
    N = 60
    A = np.eye(N) + 0.3 * (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))) / np.sqrt(N)
    g = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    ref = np.linalg.solve(A, g)
    for restart in (50, 7):
        x, it, _ = O.gmres_right(lambda v: A @ v, lambda v: v, g, tol=1e-12, restart=restart, max_iter=2000)
        assert np.linalg.norm(x - ref) < 1e-10 * np.linalg.norm(ref)
    # a right preconditioner leaves the solution unchanged
    Pm = np.diag(1 + rng.uniform(0, 1, N))
    x, it, _ = O.gmres_right(lambda v: A @ v, lambda v: Pm @ v, g, tol=1e-12)
    assert np.linalg.norm(x - ref) < 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("d,n,freq", [(2, 24, 3.0), (2, 32, 4.0), (3, 8, 1.0)])
def test_whole_solve_matches_dense_discrete_system(d, n, freq):
    omega = 2 * np.pi * freq
    m = _bump(n, d)
    dirs = [(1.0, 0.0)] if d == 2 else [(0.0, 0.6, 0.8)]
    res = O.solve(n, d, omega, m, dirs, tol=1e-12)
    kt = O.kernel_table(n, d, omega)
    Kd = O.dense_K(kt, n, d)
    Adense = np.eye(n**d) + Kd * (omega**2 * m.reshape(-1))[None, :]
    g = O.rhs(kt, omega, m, dirs[0], direct=True).reshape(-1)
    ref = np.linalg.solve(Adense, g)
    assert np.linalg.norm(res["u"][0] - ref) < 1e-9 * np.linalg.norm(ref)
    assert res["resid"][0] < 1e-11


def test_zero_medium_gives_zero_solution_in_zero_iterations():
    n = 16
    res = O.solve(n, 2, 20.0, np.zeros((n, n)), [(1.0, 0.0)])
    assert res["iters"] == [0]
    assert np.all(res["u"] == 0)


def test_iteration_counts_in_the_papers_band():
    """The paper's rectangular-domain tables report 4..9 preconditioned GMRES iterations at
    tolerance 1e-6, essentially independent of omega (Sec. 3.3).  Qualitative band only."""
    with open(os.path.join(GOLDEN, "paper_rectangular_np.json")) as f:
        tab = json.load(f)
    lo = min(min(r["n_p"]) for r in tab["tables"])
    hi = max(max(r["n_p"]) for r in tab["tables"])
    its = []
    for freq, n in ((2.0, 24), (4.0, 48)):
        res = O.solve(n, 2, 2 * np.pi * freq, _bump(n, 2), [(0.0, -1.0)])
        its += res["iters"]
    assert all(1 <= i <= hi + 4 for i in its), (its, lo, hi)
    assert max(its) - min(its) <= 3


def test_discrete_solution_converges_to_mie_series():
    """Constant-contrast disk: the relative L2 error against the Mie series decreases as the
    grid is refined at fixed omega (discontinuous m, so no fixed order is asserted)."""
    omega = 2 * np.pi * 2
    errs = []
    for n in (32, 64):
        X = O.grid_coords(n, 2)
        r = np.hypot(X[0] - 0.5, X[1] - 0.5)
        m = np.where(r < 0.25, -0.3, 0.0)
        res = O.solve(n, 2, omega, m, [(1.0, 0.0)], tol=1e-10)
        ue = mie_disk_scattered(X[0], X[1], omega, -0.3, 0.25)
        errs.append(np.linalg.norm(res["u"][0].reshape(n, n) - ue) / np.linalg.norm(ue))
    assert errs[0] < 0.06
    assert errs[1] < 0.6 * errs[0]


def test_mie_series_satisfies_interface_conditions():
    # continuity of total field and radial derivative at r = R, and Helmholtz on each side
    omega, m0, R = 9.0, -0.3, 0.25
    th = np.linspace(0, 2 * np.pi, 7)
    eps = 1e-6
    for t in th:
        def tot(r):
            x, y = 0.5 + r * np.cos(t), 0.5 + r * np.sin(t)
            return mie_disk_scattered(np.array([x]), np.array([y]), omega, m0, R)[0] + np.exp(1j * omega * x)
        assert abs(tot(R - eps) - tot(R + eps)) < 1e-4
        dm = (tot(R - eps) - tot(R - 3 * eps)) / (2 * eps)
        dp = (tot(R + 3 * eps) - tot(R + eps)) / (2 * eps)
        assert abs(dm - dp) < 1e-2 * (1 + abs(dm))
    # Helmholtz inside with k1^2 = omega^2 (1 - m0)
    x0, y0, dl = 0.55, 0.47, 1e-3
    f = lambda x, y: mie_disk_scattered(np.array([x]), np.array([y]), omega, m0, R)[0] + np.exp(1j * omega * x)
    lap = (f(x0 + dl, y0) + f(x0 - dl, y0) + f(x0, y0 + dl) + f(x0, y0 - dl) - 4 * f(x0, y0)) / dl**2
    assert abs(lap + omega**2 * (1 - m0) * f(x0, y0)) < 1e-3 * omega**2


@pytest.mark.parametrize("d,n", [(2, 40), (3, 12)])
def test_M_approximates_stencil_times_operator(d, n):
    """eqs. (A), (B), (PCapp): [A;B](I + K w^2 m) ~ [A + C w^2 m; B].  The C w^2 m term must
    carry the part of [A;B] K w^2 m that survives: dropping it (M = S) or flipping its sign
    leaves a residual of the size of that part itself."""
    omega = 2 * np.pi * (3.0 if d == 2 else 1.0)
    m = _bump(n, d, A=-0.3, w=0.12)
    sten, cint = O.all_stencils(n, d, omega, 2)
    M, S = O.assemble(n, d, omega, m, sten, cint)
    kt = O.kernel_table(n, d, omega)
    rng = np.random.default_rng(9)
    x = (rng.standard_normal((n,) * d) + 1j * rng.standard_normal((n,) * d))
    SAx = S @ O.apply_operator(kt, omega, m, x).reshape(-1)
    Mx = M @ x.reshape(-1)
    Sx = S @ x.reshape(-1)
    part = np.linalg.norm(SAx - Sx)
    assert np.linalg.norm(SAx - Mx) < 0.05 * part


def test_sphere_mie_series_satisfies_interface_conditions():
    # continuity of the total field and of its radial derivative at r = R, and Helmholtz
    # inside (k1^2 = omega^2 (1 - m0)) and outside (omega^2), by finite differences
    omega, m0, R = 9.0, -0.3, 0.25
    eps = 1e-6

    def tot(x):
        return mie_sphere_scattered(*[np.array([v]) for v in x], omega, m0, R)[0] + np.exp(1j * omega * x[0])

    for t, p in ((0.3, 0.2), (1.4, 2.1), (2.7, 4.0)):
        e = np.array([np.cos(t), np.sin(t) * np.cos(p), np.sin(t) * np.sin(p)])
        at = lambda rr: tot(0.5 + rr * e)
        assert abs(at(R - eps) - at(R + eps)) < 1e-4
        dm = (at(R - eps) - at(R - 3 * eps)) / (2 * eps)
        dp = (at(R + 3 * eps) - at(R + eps)) / (2 * eps)
        assert abs(dm - dp) < 1e-2 * (1 + abs(dm))
    dl = 1e-3
    for x0, k2 in ((np.array([0.55, 0.47, 0.52]), omega**2 * (1 - m0)), (np.array([0.9, 0.3, 0.6]), omega**2)):
        lap = sum(tot(x0 + dl * np.eye(3)[a]) + tot(x0 - dl * np.eye(3)[a]) for a in range(3)) - 6 * tot(x0)
        lap /= dl**2
        assert abs(lap + k2 * tot(x0)) < 1e-3 * omega**2


def test_3d_discrete_solution_converges_to_the_sphere_mie_series():
    """Constant-contrast ball: the relative L2 error of the 3D solve against the Mie series
    decreases under refinement (measured 5.8e-2 at n = 15, 1.8e-2 at n = 31)."""
    omega = 2 * np.pi * 1.5
    errs = []
    for n in (15, 31):
        X = O.grid_coords(n, 3)
        r = np.sqrt(sum((X[a] - 0.5) ** 2 for a in range(3)))
        m = np.where(r < 0.25, -0.3, 0.0)
        res = O.solve(n, 3, omega, m, [(1.0, 0.0, 0.0)], tol=1e-10)
        ue = mie_sphere_scattered(X[0], X[1], X[2], omega, -0.3, 0.25)
        errs.append(np.linalg.norm(res["u"][0].reshape((n,) * 3) - ue) / np.linalg.norm(ue))
    assert errs[0] < 0.08
    assert errs[1] < 0.45 * errs[0]


def test_box_cavity_medium_and_its_iteration_counts():
    """The smoothed square / cubic cavities of Sec. 3.3 (Figs. R22, R32): the velocity
    c = (1 - m)^(-1/2) spans [2/3, 1] as the paper states, m is symmetric about the centre and
    vanishes outside the smoothed box, and at 6 points per wavelength of the homogeneous
    region the oracle's preconditioned GMRES stays within the band of the paper's tables and
    does not grow with omega (qualitative, as for the bump)."""
    with open(os.path.join(GOLDEN, "paper_rectangular_np.json")) as f:
        tab = json.load(f)
    hi = max(max(r["n_p"]) for r in tab["tables"])
    for d, n in ((2, 64), (3, 12)):
        m = W.box_cavity(n, d)
        c = (1 - m) ** -0.5
        assert abs(c.min() - 2 / 3) < 1e-12 and abs(c.max() - 1) < 1e-12
        assert np.allclose(m, np.flip(m, axis=0)) and np.allclose(m, np.swapaxes(m, 0, d - 1))
        x = W.grid_x(n)
        outside = np.abs(x - 0.5) > 0.2 + 0.05
        assert np.all(m[outside] == 0)
    its = []
    for n in (32, 64):
        m = W.enforce_buffer(W.box_cavity(n, 2), 2)
        res = O.solve(n, 2, 2 * np.pi * (n + 1) / 6, m, [(0.0, -1.0)])
        its += res["iters"]
    assert all(1 <= i <= hi + 4 for i in its), its
    assert max(its) - min(its) <= 2, its
