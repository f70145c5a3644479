"""ls_apply_noalloc: the operator apply for callers that cannot allocate device memory.

It must give the result of the regular FP64 apply (ls_apply) through the C-ABI, call after
call, while using only the library's fixed scratch buffer.  This file is collected last on
purpose, so that a run stopping at the first failure has run every other test first.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-11  # the FP64 operator tolerance of the parity tests


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("d,n,freq,nrhs", [(2, 64, 6.0, 3), (3, 16, 2.0, 2)])
def test_noalloc_apply_matches_regular_apply_on_consecutive_calls(d, n, freq, nrhs):
    torch = pytest.importorskip("torch")
    from paper_1408_4495_gb300 import build, ls, workloads as W

    build.build()
    rng = np.random.default_rng(31)
    m = W.enforce_buffer(W.bumps(n, d, [0.2, -0.15], [0.08, 0.1], [(0.4,) * d, (0.6,) * d]), 2)
    omega = 2 * np.pi * freq
    shape = (nrhs,) + (n,) * d
    with ls.Solver(m, omega, mixed=False) as s:
        for call in range(2):
            xh = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
            x = torch.from_numpy(xh).cuda()
            ref = s.apply(x, mixed=False)
            out = torch.full_like(x, complex(np.nan, np.nan))
            s.apply_noalloc(x, out)
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
        # host arrays are refused (the entry point never copies)
        xh = np.zeros((1, n, n), complex)
        with pytest.raises(ls.LsError) as e:
            s.apply_noalloc(xh, np.empty_like(xh))
        assert e.value.status == ls.LS_EINVAL
        # the context still works after a refused call
        x = torch.ones((1, n, n), dtype=torch.complex128, device="cuda")
        out = torch.empty_like(x)
        s.apply_noalloc(x, out)
        torch.cuda.synchronize()
        assert torch.equal(out, x)  # m = 0: the operator is the identity
