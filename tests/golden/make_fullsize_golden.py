"""Writes the oracle's reference values for the full-size parity tests (tests/test_gpu_fullsize.py).

Only oracle/ and the seeded input generators (paper_1408_4495_gb300/workloads.py, which hold
no arithmetic of the method) are used: for each full-size workload and a few of its incident
directions, the oracle's preconditioned GMRES (Secs. 2-3: SVD stencils, SuperLU of the
nested-dissection ordered M, right-preconditioned GMRES(50)) is run to relative residual 1e-6
for the iteration count and to 1e-10 for the reference solution, whose values are stored at
seeded sample points (the whole vector is millions of entries).  The SuperLU factorization
takes minutes (2D n = 1024) to about an hour (3D n = 64) on a 2 GHz host, which is why the
values are stored instead of recomputed in the GPU tests.

    python tests/golden/make_fullsize_golden.py 2d_n1024   # writes fullsize_2d_n1024.json
    python tests/golden/make_fullsize_golden.py 3d_n64     # writes fullsize_3d_n64.json
"""

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_1408_4495_gb300 import workloads as W  # noqa: E402

CASES = {
    # name: (workload builder, its arguments, directions solved, samples per direction)
    "2d_n1024": ("noise_2d", (1024, 128.0, 64, 1003), [0, 37], 1024),
    "3d_n64": ("bumps_3d", (64, 8.0, 6, 8, 1004), [0, 5], 1024),
}
SAMPLE_SEED = 2024


def sample_points(N, count):
    """Seeded flat grid indices of the stored solution values (also used by the tests)."""
    return np.sort(np.random.default_rng(SAMPLE_SEED).choice(N, size=count, replace=False))


def main(name):
    fn, args, sel, count = CASES[name]
    w = getattr(W, fn)(*args)
    m = W.enforce_buffer(w.m, 2)
    n, d, omega = w.n, w.d, w.omega
    t0 = time.time()
    ktab = O.kernel_table(n, d, omega)
    sten, cint = O.all_stencils(n, d, omega, 2)
    M, S = O.assemble(n, d, omega, m, sten, cint)
    P = O.Preconditioner(M, S, n, d)
    t_fac = time.time() - t0
    shape = (n,) * d
    A = lambda x: O.apply_operator(ktab, omega, m, x.reshape(shape), workers=-1).reshape(-1)
    idx = sample_points(n**d, count)
    out = {"source": "oracle/ (tests/golden/make_fullsize_golden.py): preconditioned GMRES(50), x0 = 0; "
                     "iterations at relative residual 1e-6, solution at 1e-10 sampled at seeded points",
           "workload": [fn, list(args)], "directions": sel, "sample_seed": SAMPLE_SEED, "samples": count,
           "factor_seconds": t_fac, "sample_idx": [int(i) for i in idx], "iters_1e-6": [], "iters_1e-10": [],
           "resid_1e-10": [], "u_norm": [], "u_re": [], "u_im": []}
    for j in sel:
        g = O.rhs(ktab, omega, m, w.directions[j], workers=-1).reshape(-1)
        _, it6, _ = O.gmres_right(A, P, g, 1e-6, 50, 500)
        u, it10, _ = O.gmres_right(A, P, g, 1e-10, 50, 500)
        out["iters_1e-6"].append(int(it6))
        out["iters_1e-10"].append(int(it10))
        out["resid_1e-10"].append(float(np.linalg.norm(g - A(u)) / np.linalg.norm(g)))
        out["u_norm"].append(float(np.linalg.norm(u)))
        out["u_re"].append([float(v) for v in u[idx].real])
        out["u_im"].append([float(v) for v in u[idx].imag])
        print(name, "direction", j, "iterations", it6, it10, flush=True)
    with open(os.path.join(HERE, f"fullsize_{name}.json"), "w") as f:
        json.dump(out, f)
        f.write("\n")


def add_sample_idx(name):
    """Adds the sample indices to a file written before they were stored (same generator)."""
    path = os.path.join(HERE, f"fullsize_{name}.json")
    with open(path) as f:
        out = json.load(f)
    fn, args, _, count = CASES[name]
    w = getattr(W, fn)(*args)
    out["sample_idx"] = [int(i) for i in sample_points(w.n**w.d, count)]
    with open(path, "w") as f:
        json.dump(out, f)
        f.write("\n")


if __name__ == "__main__":
    if len(sys.argv) > 2 and sys.argv[2] == "--add-sample-idx":
        add_sample_idx(sys.argv[1])
    else:
        main(sys.argv[1])
