#!/usr/bin/env python
"""Throughput of the sparsifying-preconditioned Lippmann-Schwinger solve on one GB300.

Headline workload (the largest single-GPU configuration, 2D large batched): unit square,
n = 1024 (h = 1/1025), omega = 2 pi 128, medium = seeded white noise convolved with a
Gaussian of width 4h, scaled to max|m| = 0.2, times a smooth cutoff; 64 plane waves evenly
spaced on the circle, GMRES(50) to relative residual 1e-6, mixed precision (FP32 operator /
stencil / fronts with 3xTF32 tensor-core Schur products, FP64 Arnoldi coefficients and the
refinement residual).  One step = ls_factor (assembly + nested-dissection LU of the medium) +
ls_rhs_plane_wave (64 right-hand sides) + ls_solve (64 right-hand sides).  The tables that
depend only on (n, omega) -- the Nystrom symbol and the SVD stencils -- are built once by
ls_setup before timing, as the library caches them per (n, omega).

Beside it, in the same line: the identical FP64 GPU path on that workload ("plain_fp64"),
the 2D n = 256 (16 waves) and 3D n = 64 (8 waves) batched workloads with their FP64 paths
("configs"), the Sec. 5 Laplace workload, the far-field pattern, the serving stream, a
cuFFT-based convolution of the same padded size as a comparison point for the library's FFT
passes (timing only), the end-to-end rate through the public API with host buffers, and the
FP64 CPU oracle on a bounded sample.

Metric: solves/s = right-hand sides converged to 1e-6 per second, whole job.

--impl reference times the FP64 CPU oracle (oracle/) on the headline workload: each step is
one right-hand side (its plane-wave right-hand side and preconditioned GMRES solve), the
assembly + sparse LU of the medium done once before the steps and amortised over the
workload's 64 right-hand sides in the reported rate.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "solves/s at rel. residual 1e-6, mixed vs plain FP64 on 1 GB300; p50/p99 latency"
TOL = 1e-6
L2_FLUSH_BYTES = 256 << 20

# name -> (builder, description); "2d_noise_n1024" is the headline
WORKLOADS = {
    "2d_noise_n1024_omega2pi128_64rhs": ("noise_2d", (1024, 128.0, 64, 1003)),
    "2d_bumps_n256_omega2pi32_16rhs": ("bumps_2d", (256, 32.0, 8, 16, 1002)),
    "3d_bumps_n64_omega2pi8_8rhs": ("bumps_3d", (64, 8.0, 6, 8, 1004)),
}
HEADLINE = "2d_noise_n1024_omega2pi128_64rhs"


def workload(name=HEADLINE):
    from paper_1408_4495_gb300 import workloads as W
    fn, a = WORKLOADS[name]
    w = getattr(W, fn)(*a)
    w.m = W.enforce_buffer(w.m, w.buffer_b)
    w.name = name
    return w


def config(w, extra=None):
    c = {"workload": w.name, "d": w.d, "n": w.n, "N": w.n ** w.d,
         "omega": w.omega, "nrhs": w.nrhs, "tol": TOL, "restart": w.restart,
         "precision": "mixed: FP32 complex operator/stencil/fronts (3xTF32 tensor-core Schur products), "
                      "FP64 Arnoldi coefficients + refinement residual",
         "step": f"ls_factor + ls_rhs_plane_wave + ls_solve (all {w.nrhs} right-hand sides)",
         "cached_per_n_omega": "Nystrom symbol and SVD stencils (built by ls_setup before timing)",
         "l2": "flushed between timed steps (256 MiB device write outside the events)",
         "parallelism": "replicas"}
    if extra:
        c.update(extra)
    return c


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, device_id):
        self.device_id = device_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.device_id)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------ distributed
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, device, world):
    """The largest x over the ranks of the process group (x itself when world == 1)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_rank * world / seconds


# ------------------------------------------------------------------------------ oracle timing
class OracleRun:
    """The FP64 CPU oracle on one workload: assembly + sparse LU of the medium once (timed),
    then right-hand sides one at a time (plane-wave right-hand side + preconditioned GMRES)."""

    def __init__(self, w, workers):
        import oracle as O
        self.O, self.w, self.workers = O, w, workers
        self.ktab = O.kernel_table(w.n, w.d, w.omega)
        self.sten, self.cint = O.all_stencils(w.n, w.d, w.omega, w.buffer_b)
        t0 = time.perf_counter()
        M, S = O.assemble(w.n, w.d, w.omega, w.m, self.sten, self.cint)
        self.P = O.Preconditioner(M, S, w.n, w.d)
        self.t_factor = time.perf_counter() - t0
        self.shape = (w.n,) * w.d

    def A(self, x):
        return self.O.apply_operator(self.ktab, self.w.omega, self.w.m, x.reshape(self.shape),
                                     workers=self.workers).reshape(-1)

    def solve_rhs(self, j):
        """One right-hand side; returns (seconds, iterations)."""
        O, w = self.O, self.w
        t0 = time.perf_counter()
        g = O.rhs(self.ktab, w.omega, w.m, w.directions[j % w.nrhs], workers=self.workers).reshape(-1)
        _, it, _ = O.gmres_right(self.A, self.P, g, TOL, w.restart)
        return time.perf_counter() - t0, it

    def rate(self, t_rhs):
        """solves/s of the whole workload: the factorization amortised over its right-hand sides."""
        return self.w.nrhs / (self.t_factor + self.w.nrhs * t_rhs)


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(name, cores):
    """Bounded sample for the GPU arm's cpu_baseline: the factorization once and 2 right-hand
    sides, extrapolated linearly to the workload's right-hand sides.  Runs in a process of its
    own (spawned before the first GPU call) while the GPU measurements proceed."""
    w = workload(name)
    orc = OracleRun(w, cores)
    ts = [orc.solve_rhs(j)[0] for j in range(2)]
    t_rhs = sum(ts) / len(ts)
    return {"value": orc.rate(t_rhs), "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"assembly + SuperLU factorization of the medium ({orc.t_factor:.1f} s, once) + 2 of the "
                      f"{w.nrhs} right-hand sides ({t_rhs:.1f} s each: plane-wave RHS + preconditioned GMRES), "
                      f"extrapolated linearly to {w.nrhs} (marked extrapolated); scipy.fft workers={cores}, "
                      f"SuperLU serial; run in a separate host process concurrently with the GPU measurements",
            "extrapolated": True}


def start_oracle_sample(name, cores):
    """Spawns the cpu_baseline process (spawn: no CUDA state is inherited)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    ex = cf.ProcessPoolExecutor(max_workers=1, mp_context=mp.get_context("spawn"))
    return ex, ex.submit(oracle_sample, name, cores)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = workload()
    cores = cpu_cores()
    orc = OracleRun(w, cores)
    for k in range(args.warmup):
        orc.solve_rhs(k)
    times, its = [], []
    for k in range(args.steps):
        t, it = orc.solve_rhs(args.warmup + k)
        times.append(t)
        its.append(it)
    t_rhs = sum(times) / len(times)
    value = orc.rate(t_rhs)
    sample = (f"each step one of the {w.nrhs} right-hand sides (plane-wave RHS + GMRES with the SuperLU "
              f"preconditioner); the assembly + SuperLU factorization of the medium ({orc.t_factor:.1f} s) runs once "
              f"before the steps and is amortised over the {w.nrhs} right-hand sides in value; "
              f"scipy.fft workers={cores}, SuperLU serial; Nystrom table and stencils built before timing")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_rhs,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(w, {"precision": "FP64 (CPU oracle)",
                                                        "step": "one right-hand side (factorization amortised)",
                                                        "l2": "not applicable (host run, no device)"}),
            "iters": {"min": min(its), "max": max(its)}, "factor_s": orc.t_factor,
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------ GPU arm
# the per-iteration HBM-bound kernel classes of the FP32 path (FFT passes, stencil, sweeps):
# the roofline object reports the one with the largest share of device time among them.  The
# float-float classes (_cff: right-hand side and refinement residual) are FP32-ALU bound and
# appear in roofline_by_class only.
HBM_CLASSES = ("fft_row_fwd_c64", "fft_col_sym_c64", "fft_col_fwd_c64", "fft_col_inv_c64", "fft_row_inv_c64",
               "stencil_c64", "nd_fwd_c64", "nd_bwd_c64")
MODELED = ("fft_row_fwd", "fft_col_sym", "fft_col_fwd", "fft_col_inv", "fft_row_inv", "stencil", "nd_fwd", "nd_bwd")


def live_rhs(infos):
    """Average number of right-hand sides a GMRES iteration's launches carry: converged
    right-hand sides are compacted out, so over one cycle the iterations move sum_j iters_j
    right-hand sides in max_j iters_j launch sets (per step; ``infos`` holds one list of
    per-right-hand-side iteration counts per step)."""
    tot = sum(sum(step) for step in infos)
    sets = sum(max(step) for step in infos if step)
    return tot / sets if sets else 0.0


# classes launched once per GMRES iteration on the live right-hand sides only; the others
# (float-float residual and right-hand-side passes) carry every right-hand side
PER_ITERATION = ("fft_row_fwd_c64", "fft_col_sym_c64", "fft_col_fwd_c64", "fft_col_inv_c64", "fft_row_inv_c64",
                 "stencil", "nd_fwd", "nd_bwd")


def algorithmic_bytes(cls, w, nd, counts, steps, rhs=None):
    """Average bytes one launch of a kernel class must move (reads + writes): the per-unit
    figures of the pass design, FP32 complex = 8 B, FP64 / float-float complex = 16 B.
      2D row pass forward (scale, pad, FFT along the last axis): read u N c, write 2N c, weights N c/2 once
      2D column pass (FFT, x symbol, inverse, crop):            read 2N c, write 2N c, symbol (n+1)^2 c once
      2D row pass inverse (+u):                                 read 2N c + N c, write N c
      3D passes: row fwd N -> 2N, column fwd 2N -> 4N, symbol pass 4N -> 4N, column inv 4N -> 2N,
                 row inv 2N + N -> N (per right-hand side, times c)
      stencil: read v N c, write r N c
      nested-dissection sweeps: every factor block once per sweep + each right-hand side's vector
                 read and written once (N c each), spread over the sweep's launches (one per level
                 on the CUDA cores, three -- gather, tensor-core product, scatter -- per level on
                 the tensor cores: the launches per sweep come from ``counts``, one application
                 being one nd_items_out launch after its sweeps; one per level without counts).
    ``rhs``: right-hand sides per launch (default: all of the workload's)."""
    n, N, R = w.n, w.n ** w.d, (w.nrhs if rhs is None else rhs)
    c = 8 if cls.endswith("_c64") else 16
    wb = c // 2
    if w.d == 2:
        if cls.startswith("fft_row_fwd"):
            return R * N * c * 3 + N * wb
        if cls.startswith("fft_col_sym"):
            return R * 2 * (n * 2 * n) * c + (n + 1) ** 2 * c
        if cls.startswith("fft_row_inv"):
            return R * N * c * 4
    else:
        if cls.startswith("fft_row_fwd"):
            return R * N * c * 3 + N * wb
        if cls.startswith("fft_col_fwd"):
            return R * N * c * 6
        if cls.startswith("fft_col_sym"):
            return R * N * c * 8 + (n + 1) ** 3 * c
        if cls.startswith("fft_col_inv"):
            return R * N * c * 6
        if cls.startswith("fft_row_inv"):
            return R * N * c * 4
    if cls.startswith("stencil"):
        return R * N * c * 2
    if cls.startswith("nd_fwd") or cls.startswith("nd_bwd"):
        return sweep_bytes(cls, w, nd, rhs) / sweep_launches(cls, nd, counts)
    raise ValueError(cls)


def sweep_bytes(cls, w, nd, rhs=None):
    """Algorithmic bytes of one forward or backward sweep (see algorithmic_bytes)."""
    N, R = w.n ** w.d, (w.nrhs if rhs is None else rhs)
    c = 8 if cls.endswith("_c64") else 16
    key = "fwd" if cls.startswith("nd_fwd") else "bwd"
    return nd[f"{key}_factor_bytes"] + R * N * c * 2


def sweep_launches(cls, nd, counts):
    """Launches per sweep: from the class counts when they include the applications' item
    output launches (one per application), else one per level."""
    apps = (counts or {}).get("nd_items_out" + cls[6:], 0)
    if apps and (counts or {}).get(cls, 0):
        return counts[cls] / apps
    return nd["levels"]


# ncu DRAM traffic of one sweep (all its launches) on the headline workload, valid while the
# kernels' sources are unchanged: the sha1 of their source regions (the text between two
# markers of a file, or the whole file) taken when the counters were captured
# (profiles/nd_sweep_2d_n1024_64rhs.md).  "rhs": the right-hand sides of the capture; the
# line scales the bytes to the live count of the timed launches with the byte model's ratio
# (factor bytes fixed, vector bytes in proportion) and divides them over the sweep's launches.
SWEEP_SRC = [("paper_1408_4495_gb300/csrc/nd.cu", "template <typename C> struct SweepK {",
              "template <typename C, int RC>\nstatic void solve_chunk"),
             ("paper_1408_4495_gb300/csrc/tc_gemm.cu", None, None),
             ("paper_1408_4495_gb300/csrc/common.cuh", None, None)]
TRAFFIC = {
    "nd_fwd_c64": {"src": SWEEP_SRC, "sha1": "dbe70b303e8aa4d939eaf9785ba2d610664e5412", "bytes_per_sweep": 6082.2e6,
                   "rhs": 64},
    "nd_bwd_c64": {"src": SWEEP_SRC, "sha1": "dbe70b303e8aa4d939eaf9785ba2d610664e5412", "bytes_per_sweep": 3786.4e6,
                   "rhs": 64},
}


def source_sha1(src):
    import hashlib
    h = hashlib.sha1()
    for path, begin, end in src:
        with open(os.path.join(ROOT, path), encoding="utf-8") as f:
            text = f.read()
        if begin is not None:
            i = text.find(begin)
            j = text.find(end, i + 1) if i >= 0 else -1
            if i < 0 or j < 0:
                return None
            text = text[i:j]
        h.update(text.encode())
    return h.hexdigest()


def recorded_traffic(cls, w=None, nd=None, rhs=None, counts=None):
    """Recorded DRAM bytes per launch of a sweep class: the sweep's bytes scaled to ``rhs``
    right-hand sides by the byte model, over its launches; None when there is no record or a
    kernel changed since."""
    rec = TRAFFIC.get(cls)
    if not rec or not rec["sha1"] or not rec["bytes_per_sweep"]:
        return None
    if source_sha1(rec["src"]) != rec["sha1"]:
        return None
    per_sweep = rec["bytes_per_sweep"]
    if w is not None and rhs is not None:
        per_sweep *= sweep_bytes(cls, w, nd, rhs) / sweep_bytes(cls, w, nd, rec["rhs"])
    return per_sweep / sweep_launches(cls, nd, counts) if nd is not None else per_sweep


class GpuBench:
    def __init__(self, args):
        import torch
        from paper_1408_4495_gb300 import ls
        self.torch, self.ls, self.args = torch, ls, args
        self.rank, self.world, self.local = dist_env()
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl")
        torch.cuda.set_device(self.local)
        self.dev = torch.device("cuda", self.local)
        self.stream = torch.cuda.Stream(device=self.dev)
        self.flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=self.dev)

    def solver(self, w, mixed, m=None):
        t0 = time.perf_counter()
        s = self.ls.Solver(self.torch.tensor(w.m, device=self.dev) if m is None else m, w.omega, dim=w.d,
                           buffer_b=w.buffer_b, restart=w.restart, mixed=mixed, stream=self.stream)
        return s, time.perf_counter() - t0

    def buffers(self, w):
        torch = self.torch
        shape = (w.nrhs,) + (w.n,) * w.d
        dirs = torch.tensor(w.directions, device=self.dev)
        g = torch.empty(shape, dtype=torch.complex128, device=self.dev)
        u = torch.empty(shape, dtype=torch.complex128, device=self.dev)
        return dirs, g, u

    def timed(self, s, steps, warmup, step_fn, prof_class=None, clocks=False):
        torch, ls = self.torch, self.ls
        for _ in range(warmup):
            step_fn(s)
        if self.world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local_uuid(torch, self.local)) if clocks else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        ls.profile_start(prof_class)
        evs, infos = [], []
        for _ in range(steps):
            with torch.cuda.stream(self.stream):
                self.flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            infos.append(step_fn(s))
            e1.record(self.stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        prof = ls.profile_stop()
        ck = sampler.stop() if sampler else None
        total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), self.dev, self.world)
        if self.world > 1:
            torch.distributed.barrier()
        return total_ms, infos, prof, ck

    def plane_wave_step(self, w):
        dirs, g, u = self.buffers(w)

        def step(s):
            s.factor()
            s.rhs_plane_wave(dirs, out=g)
            _, info = s.solve(g, TOL, out=u)
            return info
        return step, dirs, g, u

    def rooflines(self, w, s, nd, steps):
        """Every launch bracketed by CUDA events on its stream (graphs bypassed while launches
        are timed); per-class device-time shares and the byte model per class."""
        step, _, _, _ = self.plane_wave_step(w)
        roof_ms, rinfos, rprof, _ = self.timed(s, steps, 1, step, prof_class="*")
        r_live = live_rhs([[i.iters for i in inf] for inf in rinfos])
        by_cls = rprof.get("ms_by_class", {})
        tot_cls = sum(by_cls.values()) or 1.0
        shares = {k: round(v / tot_cls, 4) for k, v in sorted(by_cls.items(), key=lambda x: -x[1])}
        peak, peak_src = measured_hbm_peak()
        by_model = {}
        for c2 in sorted(by_cls):
            if c2.startswith(MODELED) and rprof["counts"].get(c2, 0) > 0:
                avg2 = by_cls[c2] / rprof["counts"][c2]
                ab2 = algorithmic_bytes(c2, w, nd, rprof["counts"], steps,
                                        rhs=r_live if c2.startswith(PER_ITERATION) else None)
                by_model[c2] = {"achieved_gbs": ab2 / (avg2 / 1e3) / 1e9, "frac": ab2 / (avg2 / 1e3) / 1e9 / peak,
                                "avg_launch_us": avg2 * 1e3, "algorithmic_bytes_per_launch": ab2,
                                "launches": rprof["counts"][c2], "share": by_cls[c2] / tot_cls,
                                "bound": "hbm" if c2 in HBM_CLASSES else "fp32 alu (float-float)"}
        cls = self.args.profile_class or max((k for k in by_cls if k in HBM_CLASSES), key=lambda k: by_cls[k],
                                             default=None)
        roof = None
        if cls and cls in by_model:
            bm = by_model[cls]
            roof = {"kernel": cls, "bound": "hbm", "achieved": bm["achieved_gbs"], "peak": peak, "unit": "GB/s",
                    "frac": bm["achieved_gbs"] / peak,
                    "traffic": recorded_traffic(cls, w, nd, r_live, rprof["counts"]),
                    "traffic_note": "ncu dram__bytes_read + write of whole sweeps (64 right-hand sides), scaled to "
                                    "the live count by the byte model, per launch of the sweep",
                    "peak_source": peak_src,
                    "algorithmic_bytes_per_launch": bm["algorithmic_bytes_per_launch"],
                    "avg_launch_us": bm["avg_launch_us"], "launches_timed": bm["launches"], "steps_timed": steps,
                    "share_of_kernel_time": bm["share"], "live_rhs_per_iteration": r_live,
                    "class_scope": "largest device-time share among the per-iteration HBM-bound classes "
                                   "(FP32 FFT passes, stencil, nested-dissection sweeps)"}
        return roof, by_model, shares, rprof["counts"]

    def config_line(self, name, steps, fp64_steps):
        """Secondary workload: mixed and FP64 steps, iterations and the mixed / FP64 ratio."""
        w = workload(name)
        step, _, _, _ = self.plane_wave_step(w)
        s, _ = self.solver(w, True)
        ms, infos, _, _ = self.timed(s, steps, 2, step)
        nd = s.nd_stats()
        s.close()
        s64, _ = self.solver(w, False)
        ms64, infos64, _, _ = self.timed(s64, fp64_steps, 1, step)
        s64.close()
        its = [i.iters for inf in infos for i in inf]
        its64 = [i.iters for inf in infos64 for i in inf]
        v = job_rate(w.nrhs * steps, self.world, ms / 1e3)
        v64 = job_rate(w.nrhs * fp64_steps, self.world, ms64 / 1e3)
        return {"workload": name, "value": v, "unit": "solves/s", "ms_per_step": ms / steps, "steps": steps,
                "iters": {"min": min(its), "max": max(its)},
                "max_rel_resid": max(i.rel_resid for inf in infos for i in inf),
                "all_converged": all(i.converged for inf in infos for i in inf),
                "plain_fp64": {"value": v64, "unit": "solves/s", "ms_per_step": ms64 / fp64_steps,
                               "steps": fp64_steps, "iters": {"min": min(its64), "max": max(its64)}},
                "mixed_over_fp64": v / v64, "factor_flops": nd["factor_flops"], "max_front": nd["max_front"]}

    def cufft_comparison(self, w, s):
        """The library's FP32 operator apply on every right-hand side (sum of its FFT pass
        classes, CUDA events per launch) beside a cuFFT convolution of the same padded size
        and batch through torch.fft: scale, zero-pad, 2D/3D FFT, symbol product, inverse FFT,
        crop, + u.  Timing only: nothing of it is on the library's path."""
        torch, ls = self.torch, self.ls
        shape = (w.nrhs,) + (w.n,) * w.d
        gen = torch.Generator(device=self.dev).manual_seed(7)
        x = torch.randn(shape, dtype=torch.complex128, device=self.dev, generator=gen)
        s.apply(x, mixed=True)
        torch.cuda.synchronize()
        ls.profile_start("*")
        reps = 3
        for _ in range(reps):
            s.apply(x, mixed=True)
        torch.cuda.synchronize()
        prof = ls.profile_stop()
        lib_ms = sum(v for k, v in prof.get("ms_by_class", {}).items() if k.startswith("fft_")) / reps
        x32 = x.to(torch.complex64)
        L = 2 * w.n
        dims = tuple(range(1, w.d + 1))
        sym = torch.randn((L,) * w.d, dtype=torch.complex64, device=self.dev, generator=gen)
        wgt = torch.randn((w.n,) * w.d, dtype=torch.float32, device=self.dev, generator=gen)
        crop = (slice(None),) + (slice(0, w.n),) * w.d

        def conv():
            f = torch.fft.fftn(x32 * wgt, s=(L,) * w.d, dim=dims)
            f *= sym
            return torch.fft.ifftn(f, dim=dims)[crop] + x32

        with torch.cuda.stream(self.stream):
            conv()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            for _ in range(reps):
                y = conv()
            e1.record(self.stream)
        torch.cuda.synchronize()
        del y
        cufft_ms = e0.elapsed_time(e1) / reps
        return {"library_fft_ms": lib_ms, "cufft_ms": cufft_ms, "library_over_cufft_time": lib_ms / cufft_ms,
                "nrhs": w.nrhs, "padded": [L] * w.d,
                "includes": "library: sum of its FFT pass launches of one FP32 ls_apply (CUDA events per launch); "
                            "cuFFT: torch.fft fftn (zero-padded) + symbol product + ifftn + crop + u in complex64, "
                            "CUDA events, timing only"}

    def e2e(self, w):
        """End to end through the public API with host buffers (pinned): ls_setup (medium from
        host) + factor + right-hand sides (directions from host) + solve (solution to host) + free."""
        torch, ls = self.torch, self.ls
        shape = (w.nrhs,) + (w.n,) * w.d
        m_host = torch.tensor(w.m).pin_memory()
        dirs_host = torch.tensor(w.directions).pin_memory()
        u_host = torch.empty(shape, dtype=torch.complex128).pin_memory()
        g = torch.empty(shape, dtype=torch.complex128, device=self.dev)
        steps = max(1, min(self.args.steps, 3))

        def e2e_step():
            with ls.Solver(m_host.numpy(), w.omega, dim=w.d, buffer_b=w.buffer_b, restart=w.restart, mixed=True,
                           stream=self.stream) as s:
                s.factor()
                s.rhs_plane_wave(dirs_host.numpy(), out=g)
                s.solve(g, TOL, out=u_host.numpy())
            return float(np.abs(u_host.numpy()[:, :1]).max())

        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            e2e_step()
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, self.dev, self.world)
        out = {"value": job_rate(w.nrhs * steps, self.world, e2e_s), "unit": "solves/s", "steps": steps,
               "h2d_bytes_per_step": int(m_host.numel() * 8 + dirs_host.numel() * 8),
               "d2h_bytes_per_step": int(u_host.numel() * 16),
               "includes": "ls_setup (medium from pinned host) + ls_factor + ls_rhs_plane_wave + ls_solve "
                           "(solution to pinned host) + ls_free, wall clock"}
        # the same on one context that takes a new medium every step (ls_set_medium)
        try:
            with ls.Solver(m_host.numpy(), w.omega, dim=w.d, buffer_b=w.buffer_b, restart=w.restart, mixed=True,
                           stream=self.stream) as s:
                def same_grid_step():
                    s.set_medium(m_host.numpy())
                    s.factor()
                    s.rhs_plane_wave(dirs_host.numpy(), out=g)
                    s.solve(g, TOL, out=u_host.numpy())

                same_grid_step()
                same_grid_step()  # graphs are captured on the second run
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(steps):
                    same_grid_step()
                torch.cuda.synchronize()
                sg_s = max_over_ranks(time.perf_counter() - t0, self.dev, self.world)
            out["same_grid"] = {"value": job_rate(w.nrhs * steps, self.world, sg_s), "unit": "solves/s",
                                "h2d_bytes_per_step": out["h2d_bytes_per_step"],
                                "d2h_bytes_per_step": out["d2h_bytes_per_step"],
                                "includes": "ls_set_medium (medium from pinned host) + ls_factor + ls_rhs_plane_wave "
                                            "+ ls_solve (solution to pinned host) on one context, wall clock"}
        except Exception as e:  # reported in the line instead of losing the headline
            out["same_grid"] = {"error": f"{type(e).__name__}: {e}"}
        return out

    def laplace(self):
        """Sec. 5 Laplace variant: 3D n = 64, Gaussian potential with max|V| ~ 1/h^2, 8 delta
        sources; one step = ls_factor + ls_rhs_point_source + ls_solve."""
        torch, ls = self.torch, self.ls
        from paper_1408_4495_gb300 import workloads as W
        lw = W.laplace_3d(64, 8, "gaussian", 1005)
        V_dev = torch.tensor(W.enforce_buffer(lw.V, 2), device=self.dev)
        pts_dev = torch.tensor(lw.points.astype(np.int32), device=self.dev)
        lshape = (lw.nrhs,) + (lw.n,) * 3
        gl = torch.empty(lshape, dtype=torch.complex128, device=self.dev)
        ul = torch.empty(lshape, dtype=torch.complex128, device=self.dev)
        out = {}
        for mixed in (True, False):
            s_lap = ls.Solver(V_dev, dim=3, buffer_b=lw.buffer_b, restart=lw.restart, mixed=mixed,
                              stream=self.stream, laplace=True)

            def lap_step(s):
                s.factor()
                s.rhs_point_source(pts_dev, out=gl)
                _, info = s.solve(gl, TOL, out=ul)
                return info

            kl = max(2, min(self.args.steps, 5)) if mixed else 1
            ms_l, infos_l, _, _ = self.timed(s_lap, kl, 2 if mixed else 1, lap_step)
            nd_l = s_lap.nd_stats()
            s_lap.close()
            rec = {"value": job_rate(lw.nrhs * kl, self.world, ms_l / 1e3), "unit": "solves/s",
                   "ms_per_step": ms_l / kl, "steps": kl,
                   "iters": {"min": min(i.iters for inf in infos_l for i in inf),
                             "max": max(i.iters for inf in infos_l for i in inf)},
                   "max_rel_resid": max(i.rel_resid for inf in infos_l for i in inf),
                   "all_converged": all(i.converged for inf in infos_l for i in inf)}
            if mixed:
                out.update(rec)
                out.update({"workload": f"{lw.name}_{lw.nrhs}src", "factor_flops": nd_l["factor_flops"],
                            "max_front": nd_l["max_front"],
                            "step": "ls_factor + ls_rhs_point_source + ls_solve (all sources), mixed precision"})
            else:
                out["plain_fp64"] = rec
        return out

    def far_field(self, w, s, dirs, u):
        torch = self.torch
        nobs = 64
        obs = (np.array([[math.cos(2 * math.pi * k / nobs), math.sin(2 * math.pi * k / nobs)] for k in range(nobs)])
               if w.d == 2 else W_sphere(nobs))
        obs_dev = torch.tensor(obs, device=self.dev)
        ff_out = torch.empty((w.nrhs, nobs), dtype=torch.complex128, device=self.dev)
        s.far_field(dirs, u, obs_dev, out=ff_out)
        torch.cuda.synchronize()
        fe0, fe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fe0.record(self.stream)
        for _ in range(3):
            s.far_field(dirs, u, obs_dev, out=ff_out)
        fe1.record(self.stream)
        torch.cuda.synchronize()
        return {"ms": fe0.elapsed_time(fe1) / 3, "nrhs": w.nrhs, "nobs": nobs,
                "includes": "ls_far_field with device buffers (copies of its inputs, one FP64 kernel)"}


def W_sphere(count):
    from paper_1408_4495_gb300 import workloads as W
    return W.directions_sphere(count, 11)


def run_gpu(args):
    rank, world, _ = dist_env()
    cpu_job = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # two host cores stay with the process that drives the GPU
        cpu_job = start_oracle_sample(HEADLINE, max(1, cpu_cores() - 2))
    B = GpuBench(args)
    torch, ls = B.torch, B.ls
    w = workload()
    step, dirs_dev, g, u = B.plane_wave_step(w)

    # ---- mixed precision on the headline workload; the autotuner picks the launch shapes of
    # its factorization and sweeps first (untimed; the choice also serves the later contexts
    # of this grid and precision, e.g. the end-to-end ones)
    s_mix, setup_s = B.solver(w, True)
    t0 = time.perf_counter()
    if args.tune:
        # fixed launch shapes (profiling runs: timings under a profiler would mislead the tuner)
        s_mix.set_tune(json.loads(args.tune))
        s_mix.factor()
        tune = {"choice": s_mix.tune(), "factor_ms": [], "solve_ms": []}
    else:
        tune = s_mix.autotune(w.nrhs)
    tune_s = time.perf_counter() - t0
    nd = s_mix.nd_stats()
    # headline region: launches counted, replayed through the library's CUDA graphs
    total_ms, infos, prof, clocks = B.timed(s_mix, args.steps, args.warmup, step, clocks=True)
    value = job_rate(w.nrhs * args.steps, B.world, total_ms / 1e3)
    its = [i.iters for inf in infos for i in inf]
    refs = [i.refinements for inf in infos for i in inf]
    res = [i.rel_resid for inf in infos for i in inf]
    conv = all(i.converged for inf in infos for i in inf)
    launches = prof["total"]
    # roofline region: the same steps again, every launch timed
    roof, by_model, shares, counts_roof = B.rooflines(w, s_mix, nd, max(3, min(args.steps, 5)))
    far = B.far_field(w, s_mix, dirs_dev, u)

    if args.only_mixed:
        if B.rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "solves/s", "only_mixed": True,
                              "ms_per_step": total_ms / args.steps, "iters": {"min": min(its), "max": max(its)},
                              "gpu_launches": launches, "roofline": roof, "roofline_by_class": by_model,
                              "device_time_shares": shares}), flush=True)
        s_mix.close()
        return 0
    cufft = B.cufft_comparison(w, s_mix)
    s_mix.close()

    # ---- plain FP64 path on the same workload
    s64, _ = B.solver(w, False)
    k64 = max(1, min(args.steps, 2))
    ms64, infos64, _, _ = B.timed(s64, k64, 1, step)
    value64 = job_rate(w.nrhs * k64, B.world, ms64 / 1e3)
    its64 = [i.iters for inf in infos64 for i in inf]
    s64.close()

    # ---- the other batched workloads, each with its FP64 path
    others = {}
    for name, ks, k64s in (("2d_bumps_n256_omega2pi32_16rhs", max(3, min(args.steps, 10)), 3),
                           ("3d_bumps_n64_omega2pi8_8rhs", max(3, min(args.steps, 5)), 1)):
        try:
            others[name] = B.config_line(name, ks, k64s)
        except Exception as e:  # reported in the line instead of losing the headline
            others[name] = {"error": f"{type(e).__name__}: {e}"}
    try:
        lap = B.laplace()
    except Exception as e:
        lap = {"error": f"{type(e).__name__}: {e}"}

    # ---- serving: a seeded Poisson stream through the continuous-batching engine
    try:
        serving = run_serving(np, torch)
    except Exception as e:  # reported in the line instead of losing the headline
        serving = {"error": f"{type(e).__name__}: {e}"}

    e2e = B.e2e(w)

    # ---- CPU oracle on the host cores (rank 0, N = 1), started before the GPU work
    cpu = None
    if cpu_job is not None:
        ex, fut = cpu_job
        try:
            cpu = fut.result()
        except Exception as e:  # reported in the line instead of losing the headline
            cpu = {"error": f"{type(e).__name__}: {e}"}
        ex.shutdown()

    if B.rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": B.world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c64+c128", "data": "synthetic",
                "config": config(w), "iters": {"min": min(its), "max": max(its)},
                "refinements": {"min": min(refs), "max": max(refs)},
                "max_rel_resid": max(res), "all_converged": conv,
                "plain_fp64": {"value": value64, "unit": "solves/s", "ms_per_step": ms64 / k64, "steps": k64,
                               "iters": {"min": min(its64), "max": max(its64)}},
                "mixed_over_fp64": value / value64, "configs": others, "laplace_3d": lap, "far_field": far,
                "cufft": cufft, "serving": serving, "setup_ms": setup_s * 1e3, "nd": nd,
                "autotune": {"choice": tune["choice"], "seconds": tune_s, "factor_ms": tune["factor_ms"],
                             "solve_ms": tune["solve_ms"]},
                "roofline": roof, "roofline_by_class": by_model, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches,
                "launches_by_class": prof["counts"], "device_time_shares": shares, "clocks": clocks}
        print(json.dumps(line), flush=True)
    if B.world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_serving(np, torch, count=500, seed=1006):
    """The serving mix (2D n in {128, 256, 512} 70 %, 3D n in {32, 48} 30 %, omega / 2 pi = n / 8,
    1-32 plane waves, 4-8 bumps with max|m| <= 0.3) as a seeded Poisson stream through the
    continuous-batching engine.  ``count`` requests (500 by default instead of the mix's 2000,
    so that the whole bench run stays within a few minutes; the rate is calibrated on a
    saturated warm-up and the arrival process is the same)."""
    from paper_1408_4495_gb300 import serving as S
    from paper_1408_4495_gb300 import workloads as W

    free, _ = torch.cuda.mem_get_info()
    budget = int(min(60 << 30, 0.5 * free))

    def reqs(n_req, rate, sd):
        st = W.serving_stream(n_req, rate, sd, max_dirs=32, pool=16)
        return [S.Request(i, d, n, om, m, dirs, t) for i, (d, n, om, m, dirs, t) in enumerate(st)]

    be = S.LibBackend(mixed=True, tol=TOL)
    eng = S.Engine(be, slots=4, budget_bytes=budget)
    # saturated warm-up (everything arrives at once): calibrates the arrival rate
    warm, wst = eng.run(reqs(32, 1e9, seed + 1))
    rate = 0.8 * len(warm) / wst["wall_s"]
    res, st = eng.run(reqs(count, rate, seed))
    # the same requests alone on a fresh context each, for the mix-vs-alone difference
    worst = 0.0
    for q, r in list(zip(sorted(reqs(count, rate, seed), key=lambda q: q.arrival), res))[:6]:
        if r.error:
            continue
        with be.ls.Solver(q.m, q.omega, dim=q.d, mixed=True) as s_alone:
            s_alone.factor()
            g = s_alone.rhs_plane_wave(np.ascontiguousarray(q.dirs))
            u, _ = s_alone.solve(g, TOL)
        for j in range(len(q.dirs)):
            worst = max(worst, float(np.linalg.norm(r.u[j] - u[j]) / np.linalg.norm(u[j])))
    # plain FP64 path, one request at a time, on the first requests of the stream
    be64 = S.LibBackend(mixed=False, tol=TOL)
    sub = reqs(8, 1e9, seed)
    res64, st64 = S.Engine(be64, slots=1, budget_bytes=budget, keep_factors=False).run(sub)
    grids = {}
    for q in reqs(count, rate, seed):
        key = f"{q.d}d_n{q.n}"
        grids[key] = grids.get(key, 0) + 1
    return {"requests": st["requests"], "errors": st["errors"], "solves": st["solves"],
            "value": st["solves_per_s"], "unit": "solves/s", "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "arrival_rate_per_s": rate, "slots": 4, "budget_bytes": budget, "cache_hits": st["cache_hits"],
            "evictions": st["evictions"], "retargets": st.get("retargets", 0), "max_concurrent": st["max_concurrent"],
            "max_used_bytes": st["max_used_bytes"], "all_converged": st["all_converged"],
            "mix_vs_alone_max_rel_l2": worst, "requests_by_grid": grids,
            "fp64_one_at_a_time": {"requests": st64["requests"], "value": st64["solves_per_s"], "unit": "solves/s",
                                   "p50_ms": st64["p50_ms"], "p99_ms": st64["p99_ms"]},
            "workload": f"Poisson stream of {count} requests (the mix's 2000 scaled to keep the bench within a few "
                        "minutes): 2D n in {128, 256, 512} (70 %), 3D n in {32, 48} (30 %), omega / 2 pi = n / 8, "
                        "4-8 bumps with max|m| <= 0.3 from a pool of 16 media per grid, 1-32 plane waves per "
                        "request; arrival rate 0.8x the saturated warm-up throughput"}


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def local_uuid(torch, local):
    try:
        u = torch.cuda.get_device_properties(local).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            return vis.split(",")[local]
        return local


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--profile-class", default=None,
                    help="kernel class whose roofline is reported (the largest share of device time)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-mixed", action="store_true",
                    help="time the mixed-precision steps only (short runs under a profiler)")
    ap.add_argument("--tune", default=None,
                    help="apply these launch shapes (JSON object, as ls_set_tune takes) instead of autotuning")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
