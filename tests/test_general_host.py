"""The library's host steps of the general-domain method (Sec. 4) against the oracle: the
unknowns (supp(m) with its b + 1 buffer) and the boundary stencils from a sketch T.  T is an
input of the library step (on the GPU path it comes from the operator passes applied to R);
here the test forms it with the oracle's FFT apply from a seeded R."""

import math

import numpy as np
import pytest

import oracle as O
from paper_1408_4495_gb300 import workloads as W


@pytest.fixture(scope="module")
def LS():
    from paper_1408_4495_gb300 import build, ls
    build.build()
    return ls


CASES = [(2, 32, 4.0, "l2", 0.35), (2, 32, 4.0, "l1", 0.38), (3, 12, 1.0, "l2", 0.25)]


@pytest.mark.parametrize("d,n,freq,norm,rho", CASES)
def test_general_support_matches_the_oracle(LS, d, n, freq, norm, rho):
    m = W.cavity(n, d, norm, rho=rho)
    mask = LS.general_support(m, 2)
    ref = np.zeros(n**d, dtype=bool)
    ref[O.general_support(m, 2)] = True
    assert np.array_equal(mask.reshape(-1), ref)


@pytest.mark.parametrize("d,n,freq,norm,rho", CASES)
def test_general_boundary_stencils_match_the_oracle(LS, d, n, freq, norm, rho):
    omega = 2 * math.pi * freq
    m = W.cavity(n, d, norm, rho=rho)
    idx = O.general_support(m, 2)
    R = np.random.default_rng(5).standard_normal((len(idx), 2 * 3**d))
    kt = O.kernel_table(n, d, omega)
    T = np.empty((len(idx), R.shape[1]), dtype=np.complex128)
    for q in range(R.shape[1]):
        full = np.zeros(n**d, dtype=np.complex128)
        full[idx] = R[:, q]
        T[:, q] = O.apply_K_fft(kt, (omega**2 * m.reshape(-1) * full).reshape((n,) * d)).reshape(-1)[idx]
    mask = np.zeros(n**d, dtype=np.uint8)
    mask[idx] = 1
    alpha, bnd = LS.general_boundary_stencils(mask.reshape((n,) * d), T)
    _, interior, ref, _, _ = O.general_stencils(n, d, omega, m, R)
    assert np.array_equal(bnd, ~interior)
    for k, i in enumerate(idx):
        if interior[k]:
            assert np.all(alpha[k] == 0)
            continue
        offs, a = ref[int(i)]
        row = np.zeros(3**d, dtype=np.complex128)
        for t, v in zip(offs, a):
            row[sum((t[x] + 1) * 3 ** (d - 1 - x) for x in range(d))] = v
        assert np.max(np.abs(alpha[k] - row)) < 1e-9, (k, np.max(np.abs(alpha[k] - row)))


def test_general_boundary_stencils_reject_a_short_sketch(LS):
    mask = np.ones((8, 8), dtype=np.uint8)
    with pytest.raises(LS.LsError):
        LS.general_boundary_stencils(mask, np.zeros((64, 4), dtype=np.complex128))


def _oracle_T(n, d, omega, m, R):
    return O.general_sketch(n, d, omega, m, R)


@pytest.mark.parametrize("d,n,freq,norm,rho", CASES)
def test_general_rows_embed_the_oracle_stencils_in_the_box(LS, d, n, freq, norm, rho):
    # the host step of ls_general_setup: identity rows off Omega, the oracle's boundary
    # stencils on the boundary of Omega, the rectangular interior stencil inside
    omega = 2 * math.pi * freq
    m = W.cavity(n, d, norm, rho=rho)
    idx = O.general_support(m, 2)
    R = np.random.default_rng(5).standard_normal((len(idx), 2 * 3**d))
    mask = LS.general_support(m, 2)
    alpha, bnd = LS.general_boundary_stencils(mask, _oracle_T(n, d, omega, m, R))
    _, interior, ref, (mu0, a0), _ = O.general_stencils(n, d, omega, m, R)
    code = lambda t: sum((t[x] + 1) * 3 ** (d - 1 - x) for x in range(d))
    a_int = np.zeros(3**d, dtype=np.complex128)
    for t, v in zip(mu0, a0):
        a_int[code(t)] = v
    rows, inter = LS.general_rows(mask, alpha, bnd, a_int)
    on = np.zeros(n**d, dtype=bool)
    on[idx] = True
    e0 = np.zeros(3**d)
    e0[(3**d - 1) // 2] = 1
    assert np.all(rows[~on] == e0)
    assert not np.any(inter[~on])
    assert np.array_equal(np.flatnonzero(inter), idx[interior])
    assert np.all(rows[idx[interior]] == a_int)
    for i in idx[~interior]:
        offs, a = ref[int(i)]
        want = np.zeros(3**d, dtype=np.complex128)
        for t, v in zip(offs, a):
            want[code(t)] = v
        assert np.max(np.abs(rows[i] - want)) < 1e-9


def test_general_rows_refuse_inconsistent_flags(LS):
    n, d, omega = 32, 2, 2 * math.pi * 4
    m = W.cavity(n, d, "l2", rho=0.35)
    idx = O.general_support(m, 2)
    R = np.random.default_rng(5).standard_normal((len(idx), 18))
    mask = LS.general_support(m, 2)
    alpha, bnd = LS.general_boundary_stencils(mask, _oracle_T(n, d, omega, m, R))
    a_int = np.zeros(9, dtype=np.complex128)
    a_int[4] = 1
    wrong = bnd.copy()
    wrong[np.flatnonzero(bnd)[0]] = False  # a boundary point claimed interior
    with pytest.raises(LS.LsError) as e:
        LS.general_rows(mask, alpha, wrong, a_int)
    assert e.value.status == LS.LS_EINVAL
    neg = alpha.copy()
    k = np.flatnonzero(bnd)[0]
    neg[k] = -neg[k]  # centre no longer positive
    with pytest.raises(LS.LsError):
        LS.general_rows(mask, neg, bnd, a_int)


@pytest.mark.parametrize("d,n,freq,rho", [(2, 32, 4.0, 0.35), (3, 12, 1.0, 0.25)])
def test_box_embedding_of_the_library_rows_gives_the_restricted_solution(LS, d, n, freq, rho):
    """The reading behind ls_general_setup, checked on the CPU with the library's own rows:
    M and [A;B] of the box built from ls_general_rows (identity off Omega), GMRES on the GPU machine
    operator, compared with the oracle's restricted method: same solution on Omega, at most one
    more iteration (the identity block of the block lower triangular preconditioned operator
    raises the degree of its minimal polynomial by at most one)."""
    import itertools

    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    omega = 2 * math.pi * freq
    P3, shape = 3**d, (n,) * d
    m = W.cavity(n, d, "l2", rho=rho)
    idx = O.general_support(m, 2)
    R = np.random.default_rng(5).standard_normal((len(idx), 2 * P3))
    mask = LS.general_support(m, 2)
    alpha, bnd = LS.general_boundary_stencils(mask, _oracle_T(n, d, omega, m, R))
    sten, (mu0c, c) = O.all_stencils(n, d, omega, 2)
    code = lambda t: sum((t[x] + 1) * 3 ** (d - 1 - x) for x in range(d))
    a_int = np.zeros(P3, dtype=np.complex128)
    for t, v in zip(*sten[(0,) * d]):
        a_int[code(t)] = v
    c_int = np.zeros(P3, dtype=np.complex128)
    for t, v in zip(mu0c, c):
        c_int[code(t)] = v
    rows, inter = LS.general_rows(mask, alpha, bnd, a_int)
    w2m = (omega**2 * m).reshape(-1)
    offs = [np.array(t) for t in itertools.product((-1, 0, 1), repeat=d)]
    ri, ci, mv, sv = [], [], [], []
    for i in range(n**d):
        x = np.array(np.unravel_index(i, shape))
        for t, tv in enumerate(offs):
            y = x + tv
            if np.any(y < 0) or np.any(y >= n):
                continue
            j = int(np.ravel_multi_index(tuple(y), shape))
            a = rows[i, t]
            v = a + (c_int[t] * w2m[j] if inter[i] else 0)
            if a != 0 or v != 0:
                ri.append(i); ci.append(j); sv.append(a); mv.append(v)
    M = sp.csc_matrix((mv, (ri, ci)), shape=(n**d, n**d))
    S = sp.csr_matrix((sv, (ri, ci)), shape=(n**d, n**d))
    lu = spla.splu(M)
    kt = O.kernel_table(n, d, omega)
    A = lambda v: O.apply_operator(kt, omega, m, v.reshape(shape)).reshape(-1)
    P = lambda v: lu.solve(S @ v)
    dr = (1.0, 0.0) if d == 2 else (0.0, 0.6, 0.8)
    ref = O.general_solve(n, d, omega, m, [dr], R, tol=1e-10)
    ref6 = O.general_solve(n, d, omega, m, [dr], R, tol=1e-6)
    g = O.rhs(kt, omega, m, dr).reshape(-1)
    u, it, _ = O.gmres_right(A, P, g, 1e-10, 50, 500)
    _, it6, _ = O.gmres_right(A, P, g, 1e-6, 50, 500)
    assert np.linalg.norm(u[idx] - ref["u"][0]) < 1e-8 * np.linalg.norm(ref["u"][0])
    assert ref6["iters"][0] <= it6 <= ref6["iters"][0] + 1
