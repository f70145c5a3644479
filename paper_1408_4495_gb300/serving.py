"""Continuous-batching request loop over libls: the serving form of the solver.

A request is one scattering problem: a grid (d, n), an angular frequency, a medium m sampled
on the grid and 1..k incident plane-wave directions.  Requests arrive over time.  The engine
admits a request as soon as a worker slot is free and its device-memory footprint fits the
budget, keeps each medium's factorization resident afterwards (keyed by grid, frequency and a
hash of the medium, evicted least-recently-used when memory is needed), and runs admitted
requests concurrently: every context owns its CUDA stream, so one request's factorization
overlaps another's FFTs and sweeps on the device.  Each result is the same as the request
solved alone: contexts share no mutable state on the device.

When memory must be freed for a new medium and an idle context of the same grid and
frequency is resident, the engine gives that context the new medium (``retarget``:
ls_set_medium, which keeps the stencils, the symbol, the nested-dissection structure and the
buffers) instead of closing it and setting up a new one.  With ``host_cache_bytes`` the
factorization of a context that leaves the device is kept in host memory
(ls_export_factors, least recently used out) and imported when its medium returns, so that
request skips the factorization.

The engine itself is host logic (threads, a condition variable, the admission queue); the
device work goes through a backend, ``LibBackend`` for libls.  Latency is arrival to result
on the host; the run reports p50 / p99 and the throughput in solves/s (incident directions
solved to the tolerance per second of wall clock).
"""

from __future__ import annotations

import collections
import hashlib
import threading
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    d: int
    n: int
    omega: float
    m: np.ndarray = field(repr=False)  # medium on the grid, host float64
    dirs: np.ndarray = field(repr=False)  # (k, d) incident directions
    arrival: float = 0.0  # seconds after the start of the run
    key: str = ""  # cache key: grid, frequency and a hash of the medium

    def __post_init__(self):
        if not self.key:
            h = hashlib.sha1(np.ascontiguousarray(self.m, dtype=np.float64).tobytes()).hexdigest()[:16]
            self.key = f"{self.d}:{self.n}:{self.omega!r}:{h}"


@dataclass
class Result:
    rid: int
    u: np.ndarray | None = field(default=None, repr=False)  # (k,) + (n,) * d scattered fields
    iters: list = field(default_factory=list)
    rel_resid: list = field(default_factory=list)
    converged: bool = False
    cache_hit: bool = False
    arrival: float = 0.0
    start: float = 0.0
    end: float = 0.0
    error: str = ""

    @property
    def latency(self) -> float:
        return self.end - self.arrival


class LibBackend:
    """libls contexts: ``open`` runs ls_setup, ``footprint`` estimates the device bytes of the
    factorization and the Krylov space from the nested-dissection statistics, ``factor`` and
    ``solve`` run ls_factor and ls_rhs_plane_wave + ls_solve on the context's own stream."""

    def __init__(self, mixed: bool = True, tol: float = 1e-6, restart: int = 50):
        from . import ls
        self.ls = ls
        self.mixed, self.tol, self.restart = mixed, tol, restart

    def open(self, req: Request):
        return self.ls.Solver(req.m, req.omega, dim=req.d, restart=self.restart, mixed=self.mixed)

    def footprint(self, ctx, req: Request) -> int:
        st = ctx.nd_stats()
        elem = 8 if self.mixed else 16
        N = req.n ** req.d
        k = len(req.dirs)
        # fronts and front vectors, plus per right-hand side the Krylov basis of about 12
        # FP64 vectors, the FP32 preconditioned vectors and the FFT scratch
        return int(st["factor_entries"] * elem * 1.1 + k * N * (12 * 16 + 12 * elem + 64))

    def factor(self, ctx):
        ctx.factor()

    def retarget(self, ctx, req: Request):
        ctx.set_medium(req.m)

    def export_factors(self, ctx):
        return ctx.export_factors()

    def import_factors(self, ctx, blob):
        ctx.import_factors(blob)

    def solve(self, ctx, req: Request):
        g = ctx.rhs_plane_wave(np.ascontiguousarray(req.dirs, dtype=np.float64))
        u, info = ctx.solve(g, self.tol, raise_on_noconv=False)
        return u, [i.iters for i in info], [i.rel_resid for i in info], all(i.converged for i in info)

    def close(self, ctx):
        ctx.close()


class Engine:
    """Admission by free slot and device-memory budget, FIFO order, factor cache, concurrent
    execution on ``slots`` worker threads."""

    def __init__(self, backend, slots: int = 4, budget_bytes: int = 16 << 30, keep_factors: bool = True,
                 host_cache_bytes: int = 0):
        self.backend = backend
        self.slots = slots
        self.budget = budget_bytes
        self.keep = keep_factors
        # second level of the factor cache: factorizations of evicted contexts kept in host
        # memory (ls_export_factors) and imported when their medium comes back
        self.host_cache = host_cache_bytes if hasattr(backend, "export_factors") else 0

    def run(self, requests, clock=time.perf_counter):
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        cv = threading.Condition()
        pending = collections.deque()
        cache = collections.OrderedDict()  # key -> [ctx, bytes, busy, factored, grid]
        jobs = collections.deque()
        results = {}
        stats = {"max_used_bytes": 0, "max_concurrent": 0, "evictions": 0, "cache_hits": 0, "retargets": 0,
                 "spills": 0, "host_hits": 0}
        spill = collections.OrderedDict()  # key -> exported factorization (host bytes)
        self._spill_store = spill
        state = {"used": 0, "running": 0, "done": 0, "stop": False}
        t0 = clock()

        def worker():
            while True:
                with cv:
                    while not jobs and not state["stop"]:
                        cv.wait()
                    if state["stop"] and not jobs:
                        return
                    req, ent, res = jobs.popleft()
                try:
                    if not ent[3]:
                        self.backend.factor(ent[0])
                        ent[3] = True
                    u, its, rr, conv = self.backend.solve(ent[0], req)
                    res.u, res.iters, res.rel_resid, res.converged = u, its, rr, conv
                except Exception as e:  # reported per request; the engine keeps serving
                    res.error = f"{type(e).__name__}: {e}"
                res.end = clock() - t0
                with cv:
                    ent[2] = False
                    state["running"] -= 1
                    state["done"] += 1
                    if not self.keep or res.error:
                        self._drop(cache, req.key, state)
                    results[req.rid] = res
                    cv.notify_all()

        threads = [threading.Thread(target=worker, daemon=True) for _ in range(self.slots)]
        for t in threads:
            t.start()
        nxt = 0
        with cv:
            while state["done"] < len(reqs):
                now = clock() - t0
                while nxt < len(reqs) and reqs[nxt].arrival <= now:
                    pending.append(reqs[nxt])
                    nxt += 1
                # admit from the head of the queue while a slot is free and memory fits
                while pending and state["running"] < self.slots:
                    req = pending[0]
                    res = Result(req.rid, arrival=req.arrival)
                    ent = cache.get(req.key)
                    if ent is not None and ent[2]:
                        break  # the medium's context is in use: keep FIFO order
                    if ent is None:
                        grid = (req.d, req.n, req.omega)
                        ctx = None
                        try:
                            cand = self._idle_same_grid(cache, grid)
                            if cand is not None:
                                need = self.backend.footprint(cand[1][0], req)
                                if need <= self.budget and state["used"] + need > self.budget:
                                    # room must be made anyway: the idle context takes the medium
                                    del cache[cand[0]]
                                    state["used"] -= cand[1][1]
                                    self._spill(cand[0], cand[1], stats)
                                    try:
                                        self.backend.retarget(cand[1][0], req)
                                    except Exception:
                                        self.backend.close(cand[1][0])
                                        raise
                                    ctx = cand[1][0]
                                    stats["retargets"] += 1
                            if ctx is None:
                                ctx = self.backend.open(req)
                                need = self.backend.footprint(ctx, req)
                        except Exception as e:
                            res.error = f"{type(e).__name__}: {e}"
                            res.end = clock() - t0
                            results[req.rid] = res
                            state["done"] += 1
                            pending.popleft()
                            continue
                        if need > self.budget:
                            self.backend.close(ctx)
                            res.error = f"footprint {need} B exceeds the budget {self.budget} B"
                            res.end = clock() - t0
                            results[req.rid] = res
                            state["done"] += 1
                            pending.popleft()
                            continue
                        while state["used"] + need > self.budget and self._evict_one(cache, state, stats):
                            pass
                        if state["used"] + need > self.budget:
                            self.backend.close(ctx)
                            break  # wait for running requests to release memory
                        ent = [ctx, need, False, False, grid]
                        blob = spill.pop(req.key, None)
                        if blob is not None:
                            try:
                                self.backend.import_factors(ctx, blob)
                                ent[3] = True
                                stats["host_hits"] += 1
                            except Exception:
                                pass  # factored afresh by the worker
                        cache[req.key] = ent
                        state["used"] += need
                        stats["max_used_bytes"] = max(stats["max_used_bytes"], state["used"])
                    else:
                        res.cache_hit = True
                        stats["cache_hits"] += 1
                    cache.move_to_end(req.key)
                    pending.popleft()
                    ent[2] = True
                    res.start = clock() - t0
                    state["running"] += 1
                    stats["max_concurrent"] = max(stats["max_concurrent"], state["running"])
                    jobs.append((req, ent, res))
                    cv.notify_all()
                if state["done"] >= len(reqs):
                    break
                wait = None
                if nxt < len(reqs):
                    wait = max(0.0, reqs[nxt].arrival - (clock() - t0))
                cv.wait(timeout=wait if wait is not None else 0.05)
            state["stop"] = True
            cv.notify_all()
        for t in threads:
            t.join()
        for ent in cache.values():
            self.backend.close(ent[0])
        cache.clear()
        out = [results[r.rid] for r in reqs]
        ok = [r for r in out if not r.error]
        lat = np.array([r.latency for r in ok]) if ok else np.zeros(1)
        solved = sum(len(q.dirs) for q, r in zip(reqs, out) if not r.error and r.converged)
        span = (max(r.end for r in out) - min(q.arrival for q in reqs)) if out else 0.0
        stats.update({
            "requests": len(out), "errors": sum(1 for r in out if r.error),
            "solves": solved, "wall_s": span, "solves_per_s": solved / span if span > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "all_converged": all(r.converged for r in ok),
        })
        return out, stats

    def _idle_same_grid(self, cache, grid):
        """The least recently used idle entry of this grid and frequency, if the backend can
        give a context a new medium."""
        if not hasattr(self.backend, "retarget"):
            return None
        for key, ent in cache.items():
            if not ent[2] and ent[4] == grid:
                return key, ent
        return None

    def _spill(self, key, ent, stats):
        """Keeps the factorization of an idle context that leaves the device in host memory."""
        if not self.host_cache or not ent[3]:
            return
        try:
            blob = self.backend.export_factors(ent[0])
        except Exception:
            return
        if len(blob) > self.host_cache:
            return
        spill = self._spill_store
        spill[key] = blob
        spill.move_to_end(key)
        while sum(len(b) for b in spill.values()) > self.host_cache:
            spill.popitem(last=False)
        stats["spills"] += 1

    def _evict_one(self, cache, state, stats) -> bool:
        for key, ent in cache.items():  # least recently used first
            if not ent[2]:
                self._spill(key, ent, stats)
                self.backend.close(ent[0])
                state["used"] -= ent[1]
                del cache[key]
                stats["evictions"] += 1
                return True
        return False

    def _drop(self, cache, key, state):
        ent = cache.get(key)
        if ent is not None and not ent[2]:
            self.backend.close(ent[0])
            state["used"] -= ent[1]
            del cache[key]
