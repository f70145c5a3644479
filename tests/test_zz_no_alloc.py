"""ls_apply_noalloc: the FP64 operator apply for callers that cannot allocate device memory
when they need the operator (code running while another component owns the device memory
pool, loops where a cudaMalloc / cudaFree would synchronise the device, deployments that
forbid allocation after start-up).

It must give the result of the regular FP64 apply (ls_apply) through the C-ABI, call after
call, while using only the library's fixed scratch array, and it must allocate nothing: the
library's allocation fault injection (ls_fault_alloc) is armed around it on a context that has
never applied its operator.  tests/conftest.py sorts this file after every other test (the
late-marked ones included), so that a run stopping at its first failure has run the others.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-11  # the FP64 operator tolerance of the parity tests


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _medium(W, n, d):
    return W.enforce_buffer(W.bumps(n, d, [0.2, -0.15], [0.08, 0.1], [(0.4,) * d, (0.6,) * d]), 2)


@pytest.mark.parametrize("d,n,freq,nrhs", [(2, 64, 6.0, 3), (3, 16, 2.0, 2)])
def test_noalloc_apply_matches_regular_apply_on_consecutive_calls(d, n, freq, nrhs):
    torch = pytest.importorskip("torch")
    from paper_1408_4495_gb300 import build, ls, workloads as W

    build.build()
    rng = np.random.default_rng(31)
    omega = 2 * np.pi * freq
    shape = (nrhs,) + (n,) * d
    xs = [torch.from_numpy(rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).cuda() for _ in range(2)]
    with ls.Solver(_medium(W, n, d), omega, mixed=False) as s:
        # first the allocation-free calls, with every device allocation of the library refused
        outs = []
        ls.fault_alloc(1)
        try:
            for x in xs:
                out = torch.full_like(x, complex(np.nan, np.nan))
                s.apply_noalloc(x, out)
                outs.append(out)
            torch.cuda.synchronize()
        finally:
            ls.fault_alloc(0)
        # then the regular apply (which allocates its buffers) as the reference
        for call, (x, out) in enumerate(zip(xs, outs)):
            ref = s.apply(x, mixed=False)
            torch.cuda.synchronize()
            assert _rel(out.cpu().numpy(), ref.cpu().numpy()) < TOL, f"call {call}"


def test_noalloc_apply_refuses_what_it_cannot_do():
    torch = pytest.importorskip("torch")
    from paper_1408_4495_gb300 import build, ls

    build.build()
    n = 64
    with ls.Solver(np.zeros((n, n)), 10.0, mixed=False) as s:
        # more right-hand sides than the fixed scratch can hold (2 * n^2 * 16 bytes each)
        big = torch.zeros((600, n, n), dtype=torch.complex128, device="cuda")
        with pytest.raises(ls.LsError) as e:
            s.apply_noalloc(big, torch.empty_like(big))
        assert e.value.status == ls.LS_EINVAL and "scratch" in str(e.value)
        # host arrays are refused by the library itself (the entry point never copies)
        xh = np.zeros((1, n, n), complex)
        yh = np.empty_like(xh)
        st = s.lib.ls_apply_noalloc(s.h, 1, ctypes.c_void_p(xh.ctypes.data), ctypes.c_void_p(yh.ctypes.data))
        assert st == ls.LS_EINVAL
        # and the binding refuses what would make the library run past a buffer
        x = torch.ones((1, n, n), dtype=torch.complex128, device="cuda")
        with pytest.raises(ValueError):
            s.apply_noalloc(x, torch.empty((1, n, n), dtype=torch.complex64, device="cuda"))
        with pytest.raises(ValueError):
            s.apply_noalloc(x, torch.empty((1, n, n - 1), dtype=torch.complex128, device="cuda"))
        with pytest.raises(ValueError):
            s.apply_noalloc(x, torch.empty((2, n, n), dtype=torch.complex128, device="cuda"))
        # the context still works after the refused calls
        out = torch.empty_like(x)
        s.apply_noalloc(x, out)
        torch.cuda.synchronize()
        assert torch.equal(out, x)  # m = 0: the operator is the identity
