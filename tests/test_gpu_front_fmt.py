"""ls_grid.front_fmt: the fronts' Schur products on the CUDA cores (LS_FRONT_FP32) give the
solution of the default 3xTF32 tensor-core products within the mixed path's tolerance, and
the formats that are not built are refused.  Tolerances as for the mixed parity tests:
relative residual <= 1e-6, 1e-5 from the oracle solved to 1e-10, iterations within 2."""

import numpy as np
import pytest

import oracle as O
from paper_1408_4495_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.late(1)]


@pytest.fixture(scope="module")
def LS():
    from paper_1408_4495_gb300 import build, ls
    build.build()
    return ls


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.mark.parametrize("d,n,freq,nrhs", [(2, 128, 16.0, 2), (3, 32, 4.0, 2)])
def test_cuda_core_fronts_solve_like_the_tensor_core_fronts(LS, d, n, freq, nrhs):
    omega = 2 * np.pi * freq
    rng = np.random.default_rng(9)
    m = W.enforce_buffer(W.bumps(n, d, rng.uniform(-0.2, 0.2, 3), rng.uniform(0.06, 0.12, 3),
                                 rng.uniform(0.3, 0.7, (3, d))), 2)
    dirs = W.directions_circle(nrhs) if d == 2 else W.directions_sphere(nrhs, 3)
    out = {}
    for fmt in (LS.LS_FRONT_3XTF32, LS.LS_FRONT_FP32):
        with LS.Solver(m, omega, mixed=True, front_fmt=fmt) as s:
            s.factor()
            g = s.rhs_plane_wave(dirs)
            out[fmt] = s.solve(g, tol=1e-6)
    for j in range(nrhs):
        for fmt in out:
            assert out[fmt][1][j].converged and out[fmt][1][j].rel_resid <= 1e-6
        assert abs(out[LS.LS_FRONT_FP32][1][j].iters - out[LS.LS_FRONT_3XTF32][1][j].iters) <= 2
        assert rel(out[LS.LS_FRONT_FP32][0][j], out[LS.LS_FRONT_3XTF32][0][j]) < 2e-5
    if d == 2:
        ref = O.solve(n, d, omega, m, dirs, tol=1e-10)
        for j in range(nrhs):
            assert rel(out[LS.LS_FRONT_FP32][0][j].reshape(-1), ref["u"][j]) < 1e-5


@pytest.mark.parametrize("fmt", [2, 3, 9])
def test_formats_not_built_are_refused(LS, fmt):
    m = np.zeros((16, 16))
    with pytest.raises(LS.LsError) as e:
        LS.Solver(m, 2 * np.pi * 2, mixed=True, front_fmt=fmt)
    assert e.value.status == LS.LS_EINVAL
