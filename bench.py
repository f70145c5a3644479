#!/usr/bin/env python
"""Throughput of the sparsifying-preconditioned Lippmann-Schwinger solve on one GB300.

Workload (the 2D batched configuration): unit square, n = 256 (h = 1/257), omega = 2 pi 32,
medium = 8 seeded Gaussian bumps (A ~ U[-0.3, 0.3], w ~ U[0.03, 0.1], c ~ U[0.2, 0.8]^2)
times a smooth cutoff, 16 plane waves evenly spaced on the circle, GMRES(50) to relative
residual 1e-6, mixed precision (FP32 operator / stencil / fronts, FP64 Arnoldi and FP64
refinement).  One step = ls_factor (assembly + nested-dissection LU of the medium) +
ls_rhs_plane_wave (16 right-hand sides) + ls_solve (16 right-hand sides).  The tables that
depend only on (n, omega) -- the Nystrom symbol and the SVD stencils -- are built once by
ls_setup before timing, as the library caches them per (n, omega).

Metric: solves/s = right-hand sides converged to 1e-6 per second, whole job.
The identical FP64 GPU path is timed beside it ("plain_fp64").

--impl reference times the FP64 CPU oracle (oracle/) on the same workload and step.
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


def workload():
    from paper_1408_4495_gb300 import workloads as W
    w = W.bumps_2d(256, 32.0, 8, 16, 1002)
    w.m = W.enforce_buffer(w.m, w.buffer_b)
    return w


def config(w, extra=None):
    c = {"workload": "2d_bumps_n256_omega2pi32_16rhs", "d": w.d, "n": w.n, "N": w.n ** w.d,
         "omega": w.omega, "nrhs": w.nrhs, "tol": TOL, "restart": w.restart,
         "precision": "mixed: FP32 complex operator/stencil/fronts, FP64 Arnoldi + refinement",
         "step": "ls_factor + ls_rhs_plane_wave + ls_solve (all 16 right-hand sides)",
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
def oracle_step(w, ktab, sten, cint, nrhs=None, workers=None):
    """One step of the workload on the CPU oracle: assembly + sparse LU of the medium, the
    right-hand sides and the preconditioned GMRES solves.  Returns (seconds, iterations)."""
    import oracle as O
    nr = w.nrhs if nrhs is None else nrhs
    t0 = time.perf_counter()
    M, S = O.assemble(w.n, w.d, w.omega, w.m, sten, cint)
    P = O.Preconditioner(M, S, w.n, w.d)
    shape = (w.n,) * w.d

    def A(x):
        return O.apply_operator(ktab, w.omega, w.m, x.reshape(shape), workers=workers).reshape(-1)

    its = []
    for j in range(nr):
        g = O.rhs(ktab, w.omega, w.m, w.directions[j], workers=workers).reshape(-1)
        _, it, _ = O.gmres_right(A, P, g, TOL, w.restart)
        its.append(it)
    return time.perf_counter() - t0, its


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_tables(w):
    import oracle as O
    return O.kernel_table(w.n, w.d, w.omega), *O.all_stencils(w.n, w.d, w.omega, w.buffer_b)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = workload()
    cores = cpu_cores()
    ktab, sten, cint = oracle_tables(w)
    for _ in range(args.warmup):
        oracle_step(w, ktab, sten, cint, workers=cores)
    times, its = [], []
    for _ in range(args.steps):
        t, it = oracle_step(w, ktab, sten, cint, workers=cores)
        times.append(t)
        its += it
    total = sum(times)
    value = w.nrhs * args.steps / total
    sample = (f"full step ({w.nrhs} right-hand sides, assembly + SuperLU factor + GMRES) per step; "
              f"scipy.fft workers={cores}, SuperLU serial; Nystrom table and stencils built before timing")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(w, {"precision": "FP64 (CPU oracle)",
                                                                 "l2": "not applicable (host run, no device)"}),
            "iters": {"min": min(its), "max": max(its)},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------ GPU arm
MODELED = ("fft_row_fwd", "fft_col_sym", "fft_row_inv", "stencil", "nd_fwd", "nd_bwd")


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
PER_ITERATION = ("fft_row_fwd_c64", "fft_col_sym_c64", "fft_row_inv_c64", "stencil", "nd_fwd", "nd_bwd")


def algorithmic_bytes(cls, w, nd, counts, steps, rhs=None):
    """Average bytes one launch of a kernel class must move (reads + writes), from the pass
    design: FP32 complex = 8 B, FP64 complex = 16 B, lines of n (grid) or L = 2n (padded).
    The nested-dissection sweeps read every factor block once and move the front vectors;
    one launch per level, so the per-launch figure is a sweep's bytes / its launches.
    ``rhs``: right-hand sides per launch (default: all of the workload's)."""
    n, N, R = w.n, w.n ** w.d, (w.nrhs if rhs is None else rhs)
    c = 8 if cls.endswith("_c64") else 16
    wb = 4 if c == 8 else 8
    if cls.startswith("fft_row_fwd"):      # read u (n per line), weights once; write L per line
        return R * N * c * 3 + N * wb
    if cls.startswith("fft_col_sym"):      # read and write n x L per right-hand side, symbol once
        return R * 2 * (n * 2 * n) * c + (n + 1) ** 2 * c
    if cls.startswith("fft_row_inv"):      # read L per line + u, write y
        return R * N * c * 4
    if cls.startswith("stencil"):
        return R * N * (16 + c)             # read FP64 v, write r
    if cls.startswith("nd_fwd") or cls.startswith("nd_bwd"):
        key = "fwd" if cls.startswith("nd_fwd") else "bwd"
        per_sweep = nd[f"{key}_factor_bytes"] + R * nd[f"{key}_bytes_per_rhs"]
        return per_sweep / nd["levels"]  # one launch per level in both sweeps
    raise ValueError(cls)


# ncu DRAM traffic per launch of a kernel class, valid while the kernel's source is unchanged:
# the sha1 of its source region (the text between two markers of the file) and of the
# header it includes for its arithmetic, taken when the counters were captured; see profiles/.
SWEEP_SRC = [("paper_1408_4495_gb300/csrc/nd.cu", "template <typename C> struct SweepK {",
              "// r[rhs][N] -> T[group][N][RC]"),
             ("paper_1408_4495_gb300/csrc/common.cuh", None, None)]
TRAFFIC = {
    "nd_fwd_c64": {"src": SWEEP_SRC, "sha1": "2dfd35c36927992687d1a8cf6d3ebbad7a7353a0", "bytes": 5847217},
    "nd_bwd_c64": {"src": SWEEP_SRC, "sha1": "2dfd35c36927992687d1a8cf6d3ebbad7a7353a0", "bytes": 8079202},
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


def recorded_traffic(cls):
    rec = TRAFFIC.get(cls)
    if not rec or not rec["sha1"]:
        return None
    if source_sha1(rec["src"]) != rec["sha1"]:
        return None
    return rec["bytes"]


def run_gpu(args):
    import torch
    from paper_1408_4495_gb300 import ls

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload()
    stream = torch.cuda.Stream(device=dev)
    m_dev = torch.tensor(w.m, device=dev)
    dirs_dev = torch.tensor(w.directions, device=dev)
    shape = (w.nrhs,) + (w.n,) * w.d
    g = torch.empty(shape, dtype=torch.complex128, device=dev)
    u = torch.empty(shape, dtype=torch.complex128, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def make(mixed):
        t0 = time.perf_counter()
        s = ls.Solver(m_dev, w.omega, dim=w.d, buffer_b=w.buffer_b, restart=w.restart, mixed=mixed, stream=stream)
        return s, time.perf_counter() - t0

    def step(s):
        s.factor()
        s.rhs_plane_wave(dirs_dev, out=g)
        _, info = s.solve(g, TOL, out=u)
        return info

    def timed(s, steps, warmup, prof_class=None, clocks=False, step_fn=None):
        step_fn = step_fn or step
        for _ in range(warmup):
            step_fn(s)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local_uuid(torch, local)) if clocks else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        ls.profile_start(prof_class)
        evs, infos = [], []
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos.append(step_fn(s))
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        prof = ls.profile_stop()
        ck = sampler.stop() if sampler else None
        total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), dev, world)
        if world > 1:
            torch.distributed.barrier()
        return total_ms, infos, prof, ck

    # ---- mixed precision (the headline)
    s_mix, setup_s = make(True)
    nd = s_mix.nd_stats()
    # headline region: launches counted, replayed through the library's CUDA graphs
    total_ms, infos, prof, clocks = timed(s_mix, args.steps, args.warmup, None, clocks=True)
    value = job_rate(w.nrhs * args.steps, world, total_ms / 1e3)
    its = [i.iters for inf in infos for i in inf]
    res = [i.rel_resid for inf in infos for i in inf]
    conv = all(i.converged for inf in infos for i in inf)
    launches = prof["total"]

    # roofline region: the same steps again, every launch bracketed by CUDA events on its
    # stream (graphs are bypassed while launches are timed); per-class device time shares
    roof = None
    k_roof = max(3, min(args.steps, 10))
    roof_ms, rinfos, rprof, _ = timed(s_mix, k_roof, 1, "*")
    r_live = live_rhs([[i.iters for i in inf] for inf in rinfos])
    by_cls = rprof.get("ms_by_class", {})
    tot_cls = sum(by_cls.values()) or 1.0
    shares = {k: round(v / tot_cls, 4) for k, v in sorted(by_cls.items(), key=lambda x: -x[1])}
    # the kernel class with the largest share of device time among those with a byte model
    cls = args.profile_class or max((k for k in by_cls if k.startswith(MODELED)), key=lambda k: by_cls[k],
                                    default="nd_fwd_c64")
    if by_cls.get(cls, 0) > 0 and rprof["counts"].get(cls, 0) > 0:
        nlaunch = rprof["counts"][cls]
        avg_ms = by_cls[cls] / nlaunch
        abytes = algorithmic_bytes(cls, w, nd, rprof["counts"], k_roof,
                                   rhs=r_live if cls.startswith(PER_ITERATION) else None)
        achieved = abytes / (avg_ms / 1e3) / 1e9
        peak, peak_src = measured_hbm_peak()
        roof = {"kernel": cls, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": recorded_traffic(cls), "peak_source": peak_src,
                "algorithmic_bytes_per_launch": abytes, "avg_launch_us": avg_ms * 1e3,
                "launches_timed": nlaunch, "steps_timed": k_roof,
                "share_of_kernel_time": by_cls[cls] / tot_cls, "live_rhs_per_iteration": r_live}
    # the same model for every class that has one (HBM-bound passes and sweeps)
    by_model = {}
    for c2 in sorted(by_cls):
        if c2.startswith(MODELED) and rprof["counts"].get(c2, 0) > 0:
            avg2 = by_cls[c2] / rprof["counts"][c2]
            ab2 = algorithmic_bytes(c2, w, nd, rprof["counts"], k_roof,
                                    rhs=r_live if c2.startswith(PER_ITERATION) else None)
            pk, _ = measured_hbm_peak()
            by_model[c2] = {"achieved_gbs": ab2 / (avg2 / 1e3) / 1e9, "frac": ab2 / (avg2 / 1e3) / 1e9 / pk,
                            "avg_launch_us": avg2 * 1e3, "algorithmic_bytes_per_launch": ab2}

    # exterior evaluation after the step: far-field pattern of the 16 solutions in 64 directions
    obs_dev = torch.tensor(np.array([[math.cos(2 * math.pi * k / 64), math.sin(2 * math.pi * k / 64)] for k in range(64)])
                           if w.d == 2 else np.eye(3), device=dev)
    ff_out = torch.empty((w.nrhs, obs_dev.shape[0]), dtype=torch.complex128, device=dev)
    s_mix.far_field(dirs_dev, u, obs_dev, out=ff_out)
    torch.cuda.synchronize()
    fe0, fe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fe0.record(stream)
    for _ in range(5):
        s_mix.far_field(dirs_dev, u, obs_dev, out=ff_out)
    fe1.record(stream)
    torch.cuda.synchronize()
    far = {"ms": fe0.elapsed_time(fe1) / 5, "nrhs": w.nrhs, "nobs": int(obs_dev.shape[0]),
           "includes": "ls_far_field with device buffers (copies of its inputs, one FP64 kernel)"}

    if args.only_mixed:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "solves/s", "only_mixed": True,
                              "ms_per_step": total_ms / args.steps, "iters": {"min": min(its), "max": max(its)},
                              "gpu_launches": launches, "roofline": roof}), flush=True)
        s_mix.close()
        return 0

    # ---- plain FP64 path beside it
    s64, _ = make(False)
    k64 = max(1, min(args.steps, 5))
    ms64, infos64, _, _ = timed(s64, k64, 1)
    value64 = job_rate(w.nrhs * k64, world, ms64 / 1e3)
    its64 = [i.iters for inf in infos64 for i in inf]
    s64.close()

    # ---- Sec. 5 Laplace variant beside it: 3D n = 64, Gaussian potential with max|V| ~ 1/h^2,
    # 8 delta sources; one step = ls_factor + ls_rhs_point_source + ls_solve
    from paper_1408_4495_gb300 import workloads as W
    lw = W.laplace_3d(64, 8, "gaussian", 1005)
    V_dev = torch.tensor(W.enforce_buffer(lw.V, 2), device=dev)
    pts_dev = torch.tensor(lw.points.astype(np.int32), device=dev)
    lshape = (lw.nrhs,) + (lw.n,) * 3
    gl = torch.empty(lshape, dtype=torch.complex128, device=dev)
    ul = torch.empty(lshape, dtype=torch.complex128, device=dev)
    s_lap = ls.Solver(V_dev, dim=3, buffer_b=lw.buffer_b, restart=lw.restart, mixed=True, stream=stream, laplace=True)

    def lap_step(s):
        s.factor()
        s.rhs_point_source(pts_dev, out=gl)
        _, info = s.solve(gl, TOL, out=ul)
        return info

    kl = max(2, min(args.steps, 5))
    ms_l, infos_l, _, _ = timed(s_lap, kl, 2, step_fn=lap_step)
    nd_l = s_lap.nd_stats()
    fe0, fe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s_lap.solve(gl, TOL, out=ul)  # completes any pending factorization before the events
    fe0.record(stream)
    s_lap.factor()
    fe1.record(stream)
    s_lap.precond(gl[:1].clone())  # waits for the factorization (it reports its errors)
    torch.cuda.synchronize()
    fac_ms = fe0.elapsed_time(fe1)
    s_lap.close()
    lap = {"workload": f"{lw.name}_{lw.nrhs}src", "value": job_rate(lw.nrhs * kl, world, ms_l / 1e3),
           "unit": "solves/s", "ms_per_step": ms_l / kl, "steps": kl, "warmup": 2,
           "step": "ls_factor + ls_rhs_point_source + ls_solve (all sources), mixed precision",
           "iters": {"min": min(i.iters for inf in infos_l for i in inf),
                     "max": max(i.iters for inf in infos_l for i in inf)},
           "max_rel_resid": max(i.rel_resid for inf in infos_l for i in inf),
           "all_converged": all(i.converged for inf in infos_l for i in inf),
           "factor_ms": fac_ms, "factor_flops": nd_l["factor_flops"],
           "factor_tflops": nd_l["factor_flops"] / (fac_ms / 1e3) / 1e12, "max_front": nd_l["max_front"]}

    # ---- serving: a seeded Poisson stream of 2D / 3D requests through the continuous-batching
    # engine (concurrent contexts on their own streams, factor cache, memory budget), at 0.8x
    # the throughput measured on a saturated warm-up; p50 / p99 latency beside throughput; a
    # few requests re-solved alone for the mix-vs-alone difference; the plain FP64 path one
    # request at a time beside it
    try:
        serving = run_serving(np, torch)
    except Exception as e:  # reported in the line instead of losing the headline
        serving = {"error": f"{type(e).__name__}: {e}"}

    # ---- end to end through the public API with host buffers (pinned)
    m_host = torch.tensor(w.m).pin_memory()
    dirs_host = torch.tensor(w.directions).pin_memory()
    u_host = torch.empty(shape, dtype=torch.complex128).pin_memory()
    e2e_steps = max(1, min(args.steps, 5))

    def e2e_step():
        with ls.Solver(m_host.numpy(), w.omega, dim=w.d, buffer_b=w.buffer_b, restart=w.restart, mixed=True,
                       stream=stream) as s:
            s.factor()
            s.rhs_plane_wave(dirs_host.numpy(), out=g)
            s.solve(g, TOL, out=u_host.numpy())
        return float(np.abs(u_host.numpy()).max())

    e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev, world)
    e2e = {"value": job_rate(w.nrhs * e2e_steps, world, e2e_s), "unit": "solves/s",
           "h2d_bytes_per_step": int(m_host.numel() * 8 + dirs_host.numel() * 8),
           "d2h_bytes_per_step": int(u_host.numel() * 16),
           "includes": "ls_setup (medium from pinned host) + ls_factor + ls_rhs_plane_wave + ls_solve "
                       "(solution to pinned host) + ls_free, wall clock"}

    # ---- the same on one context that takes a new medium every step (ls_set_medium), the
    # form a serving loop uses for a sequence of media on one grid
    sg_local, sg_err = 0.0, None
    try:
        with ls.Solver(m_host.numpy(), w.omega, dim=w.d, buffer_b=w.buffer_b, restart=w.restart, mixed=True,
                       stream=stream) as s:
            def same_grid_step():
                s.set_medium(m_host.numpy())
                s.factor()
                s.rhs_plane_wave(dirs_host.numpy(), out=g)
                s.solve(g, TOL, out=u_host.numpy())
                return float(np.abs(u_host.numpy()).max())

            same_grid_step()
            same_grid_step()  # graphs are captured on the second run
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                same_grid_step()
            torch.cuda.synchronize()
            sg_local = time.perf_counter() - t0
    except Exception as e:  # reported in the line instead of losing the headline
        sg_err = f"{type(e).__name__}: {e}"
    sg_s = max_over_ranks(sg_local, dev, world)
    e2e["same_grid"] = ({"error": sg_err} if sg_err else
                        {"value": job_rate(w.nrhs * e2e_steps, world, sg_s), "unit": "solves/s",
                         "h2d_bytes_per_step": e2e["h2d_bytes_per_step"],
                         "d2h_bytes_per_step": e2e["d2h_bytes_per_step"],
                         "includes": "ls_set_medium (medium from pinned host) + ls_factor + ls_rhs_plane_wave + "
                                     "ls_solve (solution to pinned host) on one context, wall clock"})

    # ---- CPU oracle on the host cores (rank 0, N = 1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = cpu_cores()
        ktab, sten, cint = oracle_tables(w)
        t, _ = oracle_step(w, ktab, sten, cint, nrhs=4, workers=cores)
        t_fac = oracle_factor_time(w, sten, cint)
        per_rhs = (t - t_fac) / 4
        step_s = t_fac + per_rhs * w.nrhs
        cpu = {"value": w.nrhs / step_s, "unit": "solves/s", "cores": cores, "kind": "oracle",
               "sample": f"assembly + SuperLU factor + 4 of the {w.nrhs} right-hand sides (GMRES), "
                         f"per-RHS time scaled to {w.nrhs}; scipy.fft workers={cores}, SuperLU serial"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c64+c128", "data": "synthetic",
                "config": config(w), "iters": {"min": min(its), "max": max(its)},
                "max_rel_resid": max(res), "all_converged": conv,
                "plain_fp64": {"value": value64, "unit": "solves/s", "ms_per_step": ms64 / k64, "steps": k64,
                               "iters": {"min": min(its64), "max": max(its64)}},
                "mixed_over_fp64": value / value64, "laplace_3d": lap, "far_field": far, "serving": serving,
                "setup_ms": setup_s * 1e3, "nd": nd,
                "roofline": roof, "roofline_by_class": by_model, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches,
                "launches_by_class": prof["counts"], "device_time_shares": shares, "clocks": clocks}
        print(json.dumps(line), flush=True)
    s_mix.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_serving(np, torch, count=64, seed=1006):
    from paper_1408_4495_gb300 import serving as S
    from paper_1408_4495_gb300 import workloads as W

    free, _ = torch.cuda.mem_get_info()
    budget = int(min(40 << 30, 0.5 * free))
    grids = ((2, 128), (2, 256), (3, 16), (3, 32))
    weights = (0.35, 0.35, 0.15, 0.15)

    def reqs(n_req, rate, sd):
        st = W.serving_stream(n_req, rate, sd, grids=grids, weights=weights, max_dirs=16, pool=16)
        return [S.Request(i, d, n, om, m, dirs, t) for i, (d, n, om, m, dirs, t) in enumerate(st)]

    be = S.LibBackend(mixed=True, tol=TOL)
    eng = S.Engine(be, slots=4, budget_bytes=budget)
    # saturated warm-up (everything arrives at once): calibrates the arrival rate
    warm, wst = eng.run(reqs(16, 1e9, seed + 1))
    rate = 0.8 * len(warm) / wst["wall_s"]
    res, st = eng.run(reqs(count, rate, seed))
    # the same requests alone on a fresh context each, for the mix-vs-alone difference
    worst = 0.0
    for q, r in list(zip(sorted(reqs(count, rate, seed), key=lambda q: q.arrival), res))[:4]:
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
    return {"requests": st["requests"], "errors": st["errors"], "solves": st["solves"],
            "value": st["solves_per_s"], "unit": "solves/s", "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "arrival_rate_per_s": rate, "slots": 4, "budget_bytes": budget, "cache_hits": st["cache_hits"],
            "evictions": st["evictions"], "retargets": st.get("retargets", 0), "max_concurrent": st["max_concurrent"],
            "max_used_bytes": st["max_used_bytes"], "all_converged": st["all_converged"],
            "mix_vs_alone_max_rel_l2": worst,
            "fp64_one_at_a_time": {"requests": st64["requests"], "value": st64["solves_per_s"], "unit": "solves/s",
                                   "p50_ms": st64["p50_ms"], "p99_ms": st64["p99_ms"]},
            "workload": "Poisson stream: 2D n in {128, 256} (70 %), 3D n in {16, 32} (30 %), omega / 2 pi = n / 8, "
                        "4-8 bumps with max|m| <= 0.3 from a pool of 16 media per grid, 1-16 plane waves per "
                        "request; arrival rate 0.8x the saturated warm-up throughput"}


def oracle_factor_time(w, sten, cint):
    import oracle as O
    t0 = time.perf_counter()
    M, S = O.assemble(w.n, w.d, w.omega, w.m, sten, cint)
    O.Preconditioner(M, S, w.n, w.d)
    return time.perf_counter() - t0


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
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
