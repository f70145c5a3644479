"""The serving engine on the GPU (libls contexts on their own streams): a small seeded mix of
2D and 3D requests with shared media, served concurrently under a device-memory budget.
Every request converges, and each result equals the same request solved alone (a fresh
context, nothing else on the device) within 1e-5 relative L2 — the tolerance of the mixed
path against the oracle; contexts share no mutable device state, so the two differ only by
the run-to-run order of floating-point reductions."""

import numpy as np
import pytest

from paper_1408_4495_gb300 import serving as S
from paper_1408_4495_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.late(4)]


@pytest.fixture(scope="module")
def LS():
    from paper_1408_4495_gb300 import build, ls
    build.build()
    return ls


def test_served_results_equal_results_alone(LS):
    # 3D n = 24 takes the radix-3 FFT passes (2n = 48), like the n = 48 grid of the bench's mix
    stream = W.serving_stream(14, 1000.0, seed=11, grids=((2, 64), (2, 128), (3, 16), (3, 24)),
                              weights=(0.35, 0.35, 0.15, 0.15), max_dirs=6, pool=3)
    reqs = [S.Request(i, d, n, om, m, dirs, t) for i, (d, n, om, m, dirs, t) in enumerate(stream)]
    be = S.LibBackend(mixed=True, tol=1e-6)
    res, st = S.Engine(be, slots=3, budget_bytes=2 << 30).run(reqs)
    assert st["errors"] == 0, [r.error for r in res if r.error]
    assert st["all_converged"] and st["max_used_bytes"] <= 2 << 30
    assert st["max_concurrent"] >= 2
    assert st["p99_ms"] >= st["p50_ms"] > 0
    for q, r in zip(sorted(reqs, key=lambda q: q.arrival), res):
        with LS.Solver(q.m, q.omega, dim=q.d, mixed=True) as s:
            s.factor()
            g = s.rhs_plane_wave(np.ascontiguousarray(q.dirs))
            u, info = s.solve(g, 1e-6)
        assert all(i.converged for i in info)
        for j in range(len(q.dirs)):
            assert np.linalg.norm(r.u[j] - u[j]) <= 1e-5 * np.linalg.norm(u[j])
