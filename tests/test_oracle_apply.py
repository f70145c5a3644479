"""Pins of the oracle's operator apply (eq. lsd / lso) and right-hand side (eq. ls)."""

import numpy as np
import pytest

import oracle as O


def _loop_K(kt, v):
    """Brute-force (K v)_i = sum_j k_{i-j} v_j with explicit Python loops (tiny n)."""
    n, d = v.shape[0], v.ndim
    out = np.zeros_like(v)
    pts = list(np.ndindex(*v.shape))
    for i in pts:
        acc = 0j
        for j in pts:
            t = tuple(i[a] - j[a] + n - 1 for a in range(d))
            acc += kt[t] * v[j]
        out[i] = acc
    return out


@pytest.mark.parametrize("d,n", [(2, 5), (3, 3)])
def test_dense_K_matches_python_loops(d, n):
    rng = np.random.default_rng(2)
    kt = O.kernel_table(n, d, 11.0)
    v = rng.standard_normal((n,) * d) + 1j * rng.standard_normal((n,) * d)
    assert np.allclose(O.apply_K_direct(kt, v), _loop_K(kt, v), rtol=1e-14, atol=1e-16)


@pytest.mark.parametrize("d,n", [(2, 8), (2, 32), (2, 33), (3, 6), (3, 12)])
def test_fft_apply_equals_direct_sum(d, n):
    rng = np.random.default_rng(3)
    omega = 2 * np.pi * 4
    kt = O.kernel_table(n, d, omega)
    v = rng.standard_normal((n,) * d) + 1j * rng.standard_normal((n,) * d)
    a = O.apply_K_fft(kt, v)
    b = O.apply_K_direct(kt, v)
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def test_apply_of_delta_is_kernel_column():
    n, d = 9, 2
    kt = O.kernel_table(n, d, 13.0)
    v = np.zeros((n, n), complex)
    j = (2, 6)
    v[j] = 1.0
    Kv = O.apply_K_fft(kt, v)
    for i in np.ndindex(n, n):
        assert abs(Kv[i] - kt[i[0] - j[0] + n - 1, i[1] - j[1] + n - 1]) < 1e-15 + 1e-12 * abs(Kv[i])


def test_operator_is_identity_when_m_zero():
    n = 16
    rng = np.random.default_rng(4)
    kt = O.kernel_table(n, 2, 20.0)
    u = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    assert np.array_equal(O.apply_operator(kt, 20.0, np.zeros((n, n)), u), u)


def test_rhs_definition_and_zero_medium():
    n = 12
    omega = 10.0
    kt = O.kernel_table(n, 2, omega)
    X = O.grid_coords(n, 2)
    m = 0.1 * np.exp(-((X[0] - 0.5) ** 2 + (X[1] - 0.5) ** 2) / 0.02)
    d = (0.6, 0.8)
    uI = np.exp(1j * omega * (0.6 * X[0] + 0.8 * X[1]))
    g = O.rhs(kt, omega, m, d, direct=True)
    assert np.allclose(g, _loop_K(kt, -(omega**2) * m * uI), rtol=1e-13, atol=1e-15)
    assert np.all(O.rhs(kt, omega, np.zeros((n, n)), d) == 0)


def test_plane_wave_solves_free_helmholtz():
    # (Delta_h + omega^2) u_I = O(h^2) on the grid: pins the phase convention exp(i w x.d)
    n, omega = 200, 10.0
    h = O.grid_h(n)
    d = np.array([0.28, 0.96])
    u = O.plane_wave(n, 2, omega, d)
    lap = (u[2:, 1:-1] + u[:-2, 1:-1] + u[1:-1, 2:] + u[1:-1, :-2] - 4 * u[1:-1, 1:-1]) / h**2
    assert np.max(np.abs(lap + omega**2 * u[1:-1, 1:-1])) < 0.01 * omega**2
    X = O.grid_coords(n, 2)
    assert abs(u[5, 7] - np.exp(1j * omega * (d[0] * X[0][5, 7] + d[1] * X[1][5, 7]))) < 1e-14
