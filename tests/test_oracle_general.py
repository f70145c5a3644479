"""Pins of the oracle's general-domain method (Sec. 4): unknowns on the support of m with
its buffer, the interior stencil of the rectangular method, randomized boundary stencils
from T = (K omega^2 m) R, and the preconditioned GMRES on the restricted system.

Pins: the restricted system's solution equals the full-grid solution on the same points
(m vanishes outside, so the Lippmann-Schwinger equation on supp(m) and its buffer is closed);
the boundary stencils are unit vectors attaining the smallest singular value of
T(mu(i), :) and no random unit vector beats them; interior rows of M equal the rectangular
method's rows at the same points; iteration counts in the band of the paper's Sec. 4 tables
and insensitive to the random draw.
"""

import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1408_4495_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _R(m, d, seed, mult=2):
    return np.random.default_rng(seed).standard_normal((len(O.general_support(m)), mult * 3**d))


@pytest.mark.parametrize("d,n,freq,norm,rho", [(2, 32, 4.0, "l2", 0.35), (2, 32, 4.0, "l1", 0.38),
                                               (3, 12, 1.0, "l2", 0.25)])
def test_general_solution_equals_the_full_grid_solution_on_omega(d, n, freq, norm, rho):
    omega = 2 * math.pi * freq
    m = W.cavity(n, d, norm, rho=rho)
    dirs = [np.eye(d)[-1] * -1.0]
    rg = O.general_solve(n, d, omega, m, dirs, _R(m, d, 0), tol=1e-11)
    rb = O.solve(n, d, omega, m, dirs, tol=1e-11)
    idx = rg["omega_idx"]
    ub = rb["u"][0][idx]
    assert np.linalg.norm(rg["u"][0] - ub) < 1e-8 * np.linalg.norm(ub)
    assert len(idx) < n**d  # a proper subset of the grid


def test_general_support_is_supp_m_with_its_buffer():
    n, d, b = 32, 2, 2
    m = W.cavity(n, d, "l1", rho=0.3)
    idx = O.general_support(m, b)
    inside = np.zeros(n**d, dtype=bool)
    inside[idx] = True
    inside = inside.reshape(n, n)
    sup = np.argwhere(m != 0)
    for x in np.argwhere(np.ones((n, n), dtype=bool)):
        dist = np.min(np.max(np.abs(sup - x), axis=1))
        assert inside[tuple(x)] == (dist <= b + 1)
    # m vanishes on every point of Omega within b of the complement (the buffer)
    out = np.argwhere(~inside)
    for x in np.argwhere(inside):
        if np.min(np.max(np.abs(out - x), axis=1)) <= b + 1:
            assert m[tuple(x)] == 0


@pytest.mark.parametrize("d,n,freq,rho", [(2, 24, 3.0, 0.35), (3, 10, 1.0, 0.25)])
def test_general_sketch_equals_the_direct_sum(d, n, freq, rho):
    # T = (K omega^2 m) R on Omega by the O(N^2) sum of the definition (dense K)
    omega = 2 * math.pi * freq
    m = W.cavity(n, d, "l2", rho=rho)
    R = _R(m, d, 4) + 1j * _R(m, d, 5)
    idx = O.general_support(m)
    T = O.general_sketch(n, d, omega, m, R)
    K = O.dense_K(O.kernel_table(n, d, omega), n, d)
    full = np.zeros((n**d, R.shape[1]), dtype=np.complex128)
    full[idx] = R
    ref = (K @ ((omega**2 * m.reshape(-1))[:, None] * full))[idx]
    assert T.shape == (len(idx), R.shape[1])
    assert np.linalg.norm(T - ref) < 1e-12 * np.linalg.norm(ref)


def test_general_boundary_stencils_attain_sigma_min():
    n, d, omega = 32, 2, 2 * math.pi * 4
    m = W.cavity(n, d, "l2", rho=0.35)
    R = _R(m, d, 3)
    idx, interior, bnd, _, _ = O.general_stencils(n, d, omega, m, R)
    # T = (K omega^2 m) R on Omega, recomputed by the direct sum of the definition
    K = O.dense_K(O.kernel_table(n, d, omega), n, d)
    full = np.zeros((n**d, R.shape[1]), dtype=np.complex128)
    full[idx] = R
    T = (K @ ((omega**2 * m.reshape(-1))[:, None] * full))[idx]
    pos = {int(i): k for k, i in enumerate(idx)}
    rng = np.random.default_rng(9)
    for i in list(bnd)[:: max(1, len(bnd) // 12)]:
        offs, alpha = bnd[i]
        x = np.array(np.unravel_index(i, (n,) * d))
        rows = [pos[int(np.ravel_multi_index(tuple(x + np.array(t)), (n,) * d))] for t in offs]
        Tm = T[rows]
        smin = np.linalg.svd(Tm, compute_uv=False)[-1]
        assert abs(np.linalg.norm(alpha) - 1) < 1e-13
        assert abs(np.linalg.norm(alpha @ Tm) - smin) < 1e-8 * np.linalg.norm(Tm, 2)
        for _ in range(50):
            beta = rng.standard_normal(len(offs)) + 1j * rng.standard_normal(len(offs))
            beta /= np.linalg.norm(beta)
            assert np.linalg.norm(beta @ Tm) >= np.linalg.norm(alpha @ Tm) * (1 - 1e-10)


def test_general_interior_rows_equal_the_rectangular_rows():
    n, d, omega = 32, 2, 2 * math.pi * 4
    m = W.cavity(n, d, "l2", rho=0.35)
    st = O.general_stencils(n, d, omega, m, _R(m, d, 1))
    Mg, Sg = O.general_assemble(n, d, omega, m, st)
    sten, cint = O.all_stencils(n, d, omega, 2)
    Mr, Sr = O.assemble(n, d, omega, m, sten, cint)
    idx, interior = st[0], st[1]
    Mr_omega = Mr[idx][:, idx]
    for k in np.flatnonzero(interior)[::7]:
        assert np.max(np.abs((Mg[k] - Mr_omega[k]).toarray())) < 1e-13
        # the full-grid row has no entries outside Omega for an interior point
        assert abs(Mr[idx[k]].sum() - Mr_omega[k].sum()) < 1e-12


@pytest.mark.parametrize("d,n,freq,rho", [(2, 64, 8.0, 0.35), (3, 16, 2.0, 0.28)])
def test_general_iterations_in_the_papers_band_and_stable_under_the_draw(d, n, freq, rho):
    """Sec. 4 tables report 4..9 iterations for smoothed l2 / l1 cavities; qualitative band."""
    with open(os.path.join(GOLDEN, "paper_general_np.json")) as f:
        tab = json.load(f)
    hi = max(max(t["n_p"]) for t in tab["tables"])
    for norm in ("l2", "l1"):
        m = W.cavity(n, d, norm, rho=rho)
        its = [O.general_solve(n, d, 2 * math.pi * freq, m, [np.eye(d)[-1] * -1.0], _R(m, d, s))["iters"][0]
               for s in (0, 1)]
        assert all(1 <= i <= hi + 3 for i in its), its
        assert abs(its[0] - its[1]) <= 1, its


def test_general_requires_the_grid_buffer():
    n = 32
    m = W.cavity(n, 2, "l2", rho=0.48)  # reaches into the b+1 outer layers
    with pytest.raises(ValueError):
        O.general_stencils(n, 2, 10.0, m, np.zeros((1, 1)))
