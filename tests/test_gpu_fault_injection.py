"""Error paths under host-side fault injection (ls_fault_alloc): a device allocation that
fails inside ls_setup, ls_factor or ls_solve is reported as LS_ENOMEM with its message, the
failed context is released or stays usable, and the library keeps serving afterwards.  No
GPU fault is induced: the refusal happens on the host before the allocator is asked."""

import numpy as np
import pytest

from paper_1408_4495_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.late(1)]


@pytest.fixture(scope="module")
def LS():
    from paper_1408_4495_gb300 import build, ls
    build.build()
    yield ls
    ls.fault_alloc(0)


def medium(n=32):
    rng = np.random.default_rng(4)
    m = W.bumps(n, 2, rng.uniform(-0.2, 0.2, 2), rng.uniform(0.06, 0.1, 2), rng.uniform(0.35, 0.65, (2, 2)))
    return W.enforce_buffer(m, 2)


@pytest.mark.parametrize("k", [1, 2, 5])
def test_failed_setup_reports_enomem_and_the_next_setup_works(LS, k):
    m, omega = medium(), 2 * np.pi * 4
    LS.fault_alloc(k)
    with pytest.raises(LS.LsError) as e:
        LS.Solver(m, omega, mixed=True)
    assert e.value.status == LS.LS_ENOMEM and "injected" in str(e.value)
    with LS.Solver(m, omega, mixed=True) as s:  # disarmed after firing
        s.factor()
        u, info = s.solve(s.rhs_plane_wave(W.directions_circle(2)), tol=1e-6)
    assert all(i.converged for i in info)


def test_failed_solve_leaves_the_context_usable(LS):
    m, omega = medium(), 2 * np.pi * 4
    with LS.Solver(m, omega, mixed=True) as s:
        s.factor()
        g = s.rhs_plane_wave(W.directions_circle(3))
        LS.fault_alloc(1)  # the solve's first new buffer
        with pytest.raises(LS.LsError) as e:
            s.solve(g, tol=1e-6)
        assert e.value.status == LS.LS_ENOMEM
        u, info = s.solve(g, tol=1e-6)
        assert all(i.converged for i in info)


def test_expired_tensor_core_wait_reports_etimeout_and_the_context_recovers(LS, monkeypatch):
    """The bounded mbarrier waits of the tensor-core front update: under the test hook
    LS_TEST_TC_TIMEOUT=1 no MMA is issued and the waits are short, so every wait expires with
    nothing in flight; the kernels free their tensor memory and return, the factorization
    reports LS_ETIMEOUT at the next call that reads it, and a factorization without the hook
    on the same context then solves normally.  No GPU fault is induced."""
    n = 128
    rng = np.random.default_rng(9)
    m = W.enforce_buffer(W.bumps(n, 2, rng.uniform(-0.2, 0.2, 3), rng.uniform(0.06, 0.1, 3),
                                 rng.uniform(0.35, 0.65, (3, 2))), 2)
    omega = 2 * np.pi * 16
    with LS.Solver(m, omega, mixed=True) as s:
        g = s.rhs_plane_wave(W.directions_circle(2))
        monkeypatch.setenv("LS_TEST_TC_TIMEOUT", "1")
        s.factor()
        with pytest.raises(LS.LsError) as e:
            s.solve(g, tol=1e-6)
        assert e.value.status == LS.LS_ETIMEOUT
        monkeypatch.delenv("LS_TEST_TC_TIMEOUT")
        s.factor()
        u, info = s.solve(g, tol=1e-6)
    assert all(i.converged and i.rel_resid <= 1e-6 for i in info)
