"""ls_export_factors / ls_import_factors: a factorization exported from one context and
imported into another of the same grid and medium solves like the original (the factored
fronts are the whole state the solves read; FP64 to 1e-12, mixed to 1e-5 as in the serving
test), and blobs of another medium, precision or format, or corrupted ones, are refused."""

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
    m = W.bumps(n, d, rng.uniform(-0.2, 0.2, 3), rng.uniform(0.06, 0.12, 3), rng.uniform(0.3, 0.7, (3, d)))
    return W.enforce_buffer(m, 2)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("d,n,freq", [(2, 64, 8.0), (3, 16, 2.0)])
@pytest.mark.parametrize("mixed", [False, True])
def test_imported_factors_solve_like_the_original(LS, d, n, freq, mixed):
    omega = 2 * np.pi * freq
    m = medium(d, n, 1)
    dirs = W.directions_circle(2) if d == 2 else W.directions_sphere(2, 3)
    with LS.Solver(m, omega, mixed=mixed) as a:
        a.factor()
        blob = a.export_factors()
        g = a.rhs_plane_wave(dirs)
        ua, ia = a.solve(g, tol=1e-6)
    with LS.Solver(m, omega, mixed=mixed) as b:
        b.import_factors(blob)
        ub, ib = b.solve(g, tol=1e-6)
    assert all(i.converged for i in ib)
    assert [i.iters for i in ia] == [i.iters for i in ib]
    assert rel(ub, ua) < (1e-5 if mixed else 1e-12)


def test_foreign_or_corrupted_blobs_are_refused(LS):
    n, omega = 32, 2 * np.pi * 4
    m = medium(2, n, 2)
    with LS.Solver(m, omega, mixed=True) as a:
        with pytest.raises(LS.LsError) as e:
            a.export_factors()
        assert e.value.status == LS.LS_ESTATE
        a.factor()
        blob = a.export_factors()
    for kwargs, mm in (({"mixed": True}, medium(2, n, 3)),        # another medium
                       ({"mixed": False}, m),                     # another precision
                       ({"mixed": True, "front_fmt": 1}, m)):     # another front format
        with LS.Solver(mm, omega, **kwargs) as c:
            with pytest.raises(LS.LsError) as e:
                c.import_factors(blob)
            assert e.value.status == LS.LS_EINVAL
    bad = blob.copy()
    bad[0] ^= 0xFF
    with LS.Solver(m, omega, mixed=True) as c:
        with pytest.raises(LS.LsError) as e:
            c.import_factors(bad)
        assert e.value.status == LS.LS_EINVAL
        with pytest.raises(LS.LsError) as e:
            c.import_factors(blob[:100])
        assert e.value.status == LS.LS_EINVAL
        c.import_factors(blob)  # the genuine one still works
        u, info = c.solve(c.rhs_plane_wave(W.directions_circle(1)), tol=1e-6)
        assert info[0].converged
