"""The general-domain method of Sec. 4 through the C-ABI: the sketch T = (K omega^2 m) R on
the unknowns, computed with the FP64 operator apply on the device (ls_general_sketch),
against the oracle's sketch (its own FFT of the circulant embedding), and the boundary
stencils the library's host step derives from that device sketch against the oracle's.

Tolerances: the sketch is an FP64 operator apply (relative <= 1e-11, as the FP64 operator
parity).  A stencil is the smallest singular vector of T(mu(i), :) and moves by about
|dT| / (gap between its two smallest singular values): on these cases a random relative
perturbation of 1e-12 in T moves the unit stencils by at most 1.5e-9 (2D) and 5e-8 (3D),
while the FP64 apply's rounding is of order 1e-14, so the comparison allows 1e-7 (absolute).
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_1408_4495_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.late(2)]


@pytest.fixture(scope="module")
def LS():
    from paper_1408_4495_gb300 import build, ls
    build.build()
    return ls


CASES = [(2, 32, 4.0, "l2", 0.35), (2, 64, 8.0, "l1", 0.38), (3, 16, 2.0, "l2", 0.3)]


@pytest.mark.parametrize("d,n,freq,norm,rho", CASES)
def test_sketch_matches_the_oracle(LS, d, n, freq, norm, rho):
    omega = 2 * math.pi * freq
    m = W.cavity(n, d, norm, rho=rho)
    mask = LS.general_support(m, 2)
    idx = O.general_support(m, 2)
    rng = np.random.default_rng(7)
    R = rng.standard_normal((len(idx), 2 * 3**d)) + 1j * rng.standard_normal((len(idx), 2 * 3**d))
    with LS.Solver(m, omega, dim=d, mixed=False) as s:
        T = s.general_sketch(mask, R)
    ref = O.general_sketch(n, d, omega, m, R)
    assert np.linalg.norm(T - ref) < 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("d,n,freq,norm,rho", CASES)
def test_boundary_stencils_from_the_device_sketch(LS, d, n, freq, norm, rho):
    omega = 2 * math.pi * freq
    m = W.cavity(n, d, norm, rho=rho)
    mask = LS.general_support(m, 2)
    idx = O.general_support(m, 2)
    R = np.random.default_rng(5).standard_normal((len(idx), 2 * 3**d))
    with LS.Solver(m, omega, dim=d, mixed=True) as s:
        T = s.general_sketch(mask, R)
    alpha, bnd = LS.general_boundary_stencils(mask, T)
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
        assert np.max(np.abs(alpha[k] - row)) < 1e-7, (k, np.max(np.abs(alpha[k] - row)))


def test_sketch_of_a_laplace_context_uses_the_potential(LS):
    n = 16
    w = W.laplace_3d(n, 1, "gaussian", 1005)
    V = W.enforce_buffer(w.V, 2)
    mask = LS.general_support(V, 2)
    idx = O.general_support(V, 2)
    R = np.random.default_rng(3).standard_normal((len(idx), 5)).astype(np.complex128)
    with LS.Solver(V, mixed=False, laplace=True) as s:
        T = s.general_sketch(mask, R)
    # the Laplace table with V in place of omega^2 m
    kt0 = O.kernel_table(n, 3, 0.0)
    full = np.zeros((n**3, R.shape[1]), dtype=np.complex128)
    full[idx] = R
    ref = np.stack([O.apply_K_fft(kt0, (V.reshape(-1) * full[:, q]).reshape((n,) * 3)).reshape(-1)[idx]
                    for q in range(R.shape[1])], axis=1)
    assert np.linalg.norm(T - ref) < 1e-11 * np.linalg.norm(ref)


def test_sketch_refuses_a_wrong_shape(LS):
    n = 32
    m = W.cavity(n, 2, "l2", rho=0.35)
    mask = LS.general_support(m, 2)
    with LS.Solver(m, 2 * math.pi * 4, mixed=False) as s:
        with pytest.raises(ValueError):
            s.general_sketch(mask, np.zeros((3, 4)))
