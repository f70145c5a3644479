"""ls_set_medium: a sequence of media on one context gives the results of fresh contexts.

The potential tables are rewritten in place and everything that depends only on the grid
and the frequency is kept (including captured graphs), so a solve after ls_set_medium +
ls_factor must equal the solve of a context set up with that medium: the same kernels on the
same data (FP64 path to 1e-12, mixed path to 1e-5: the tolerances of the serving test, which
allow for the order of the reductions), and a rejected medium leaves the context as it was.
"""

import numpy as np
import pytest

from paper_1408_4495_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.late(1)]


@pytest.fixture(scope="module")
def LS():
    from paper_1408_4495_gb300 import build, ls
    build.build()
    return ls


def medium(d, n, seed):
    rng = np.random.default_rng(seed)
    m = W.bumps(n, d, rng.uniform(-0.25, 0.25, 3), rng.uniform(0.06, 0.12, 3), rng.uniform(0.3, 0.7, (3, d)))
    return W.enforce_buffer(m, 2)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("d,n,freq", [(2, 64, 8.0), (3, 16, 2.0)])
@pytest.mark.parametrize("mixed", [False, True])
def test_sequence_of_media_equals_fresh_contexts(LS, d, n, freq, mixed):
    omega = 2 * np.pi * freq
    dirs = W.directions_circle(2) if d == 2 else W.directions_sphere(2, 3)
    media = [medium(d, n, s) for s in (1, 2, 3)]
    fresh = []
    for m in media:
        with LS.Solver(m, omega, mixed=mixed) as s:
            s.factor()
            g = s.rhs_plane_wave(dirs)
            fresh.append((g, s.solve(g, tol=1e-6)[0]))
    with LS.Solver(media[0], omega, mixed=mixed) as s:
        for k, m in enumerate(media):
            if k:
                s.set_medium(m)
            s.factor()
            g = s.rhs_plane_wave(dirs)
            u, info = s.solve(g, tol=1e-6)
            assert all(i.converged for i in info)
            assert rel(g, fresh[k][0]) < 1e-12
            assert rel(u, fresh[k][1]) < (1e-5 if mixed else 1e-12)


def test_rejected_medium_leaves_the_context_unchanged(LS):
    n, omega = 32, 2 * np.pi * 4
    m = medium(2, n, 5)
    bad = m.copy()
    bad[0, 0] = 0.1  # inside the buffer
    with LS.Solver(m, omega, mixed=False) as s:
        s.factor()
        g = s.rhs_plane_wave(W.directions_circle(1))
        u0, _ = s.solve(g, tol=1e-8)
        with pytest.raises(LS.LsError) as e:
            s.set_medium(bad)
        assert e.value.status == LS.LS_EBUFFER
        u1, _ = s.solve(g, tol=1e-8)  # still factored with the old medium
        assert rel(u1, u0) < 1e-14
        s.set_medium(m)
        with pytest.raises(LS.LsError) as e:
            s.solve(g, tol=1e-8)
        assert e.value.status == LS.LS_ESTATE
