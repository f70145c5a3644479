"""Small, repeatable cases of single steps of the path, for profiling one kernel class under a
profiler (ncu) outside the benchmark.  Each case builds its context, runs the step twice (the
first run warms up) and exits; graphs are off, so every launch is a separate kernel.

    python -m paper_1408_4495_gb300.profile_cases precond --d 2 --n 1024 --nrhs 64
        ls_precond: one stencil apply + forward and backward sweeps per run (2D smoothed-noise
        medium at omega / 2 pi = n / 8, or 3D bumps)
    python -m paper_1408_4495_gb300.profile_cases apply --d 2 --n 1024 --nrhs 4
        ls_apply in FP32, then in float-float (the FFT row and column passes)
    python -m paper_1408_4495_gb300.profile_cases factor --d 3 --n 48
        ls_factor once (the front kernels, the tensor-core Schur products); prints the number
        of tensor-core GEMM launches of one factorization
    python -m paper_1408_4495_gb300.profile_cases solve --d 2 --n 1024 --nrhs 8
        ls_factor + ls_rhs_plane_wave + ls_solve at tolerance 1e-6 (the GMRES kernels)
"""

from __future__ import annotations

import argparse
import json
import os
import sys


def _medium(W, d, n):
    if d == 2:
        w = W.noise_2d(n, n / 8, 1, 1003) if n >= 1024 else W.bumps_2d(n, n / 8, 8, 1, 1002)
    else:
        w = W.bumps_3d(n, n / 8, 6, 1, 1004)
    return W.enforce_buffer(w.m, 2), w.omega


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["precond", "apply", "factor", "solve"])
    ap.add_argument("--d", type=int, default=2)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--nrhs", type=int, default=16)
    ap.add_argument("--tune", default=None, help="launch-shape choices to apply (JSON object, as ls_set_tune takes)")
    a = ap.parse_args(argv)
    os.environ["LS_GRAPHS"] = "0"  # read by ls_setup: every launch stays a separate kernel
    import torch

    from paper_1408_4495_gb300 import ls, workloads as W

    m, omega = _medium(W, a.d, a.n)
    s = ls.Solver(torch.tensor(m, device="cuda"), omega, dim=a.d, mixed=True)
    if a.tune:
        s.set_tune(json.loads(a.tune))
    shape = (a.nrhs,) + (a.n,) * a.d
    x = torch.randn(shape, dtype=torch.complex128, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    out = {"case": a.case, "d": a.d, "n": a.n, "nrhs": a.nrhs}
    if a.case == "precond":
        s.factor()
        for _ in range(2):
            s.precond(x)
    elif a.case == "apply":
        for _ in range(2):
            s.apply(x, prec=ls.LS_PREC_MIXED)
            s.apply(x, prec=ls.LS_PREC_FF)
    elif a.case == "solve":
        dirs = W.directions_circle(a.nrhs) if a.d == 2 else W.directions_sphere(a.nrhs, 1004)
        for _ in range(2):
            s.factor()
            u, info = s.solve(s.rhs_plane_wave(dirs), tol=1e-6)
        out["iters"] = [i.iters for i in info]
    else:
        ls.profile_start(None)
        s.factor()
        s.precond(x[:1])  # waits for the factorization and reads its error flag
        torch.cuda.synchronize()
        out["tc_launches"] = ls.profile_stop()["counts"].get("nd_gemm_tc_c64", 0)
    torch.cuda.synchronize()
    s.close()
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
