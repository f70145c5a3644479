"""Host logic of the serving engine (paper_1408_4495_gb300/serving.py) on CPU, with a fake
backend whose 'device work' is a deterministic function of the request plus a sleep: every
request is served and its result equals the result alone, admission keeps the device-memory
footprint within the budget, media are served from the factor cache, an oversize request is
reported without stopping the others, the slots run concurrently, and the latency statistics
follow the schedule."""

import threading
import time

import numpy as np
import pytest

from paper_1408_4495_gb300 import serving as S
from paper_1408_4495_gb300 import workloads as W


class FakeBackend:
    def __init__(self, solve_s=0.004, factor_s=0.003, bytes_per_point=1000):
        self.solve_s, self.factor_s, self.bpp = solve_s, factor_s, bytes_per_point
        self.lock = threading.Lock()
        self.open_bytes = 0
        self.max_open_bytes = 0
        self.factored = 0

    def open(self, req):
        return {"key": req.key, "bytes": self.footprint(None, req)}

    def footprint(self, ctx, req):
        return req.n ** req.d * self.bpp

    def factor(self, ctx):
        time.sleep(self.factor_s)
        with self.lock:
            self.factored += 1

    def solve(self, ctx, req):
        time.sleep(self.solve_s)
        u = np.exp(1j * np.outer(req.dirs.sum(axis=1), req.m.reshape(-1))).reshape((len(req.dirs),) + req.m.shape)
        return u, [3] * len(req.dirs), [1e-7] * len(req.dirs), True

    def close(self, ctx):
        pass


def requests(count, rate, pool=None, seed=3):
    out = []
    for i, (d, n, om, m, dirs, t) in enumerate(W.serving_stream(count, rate, seed, grids=((2, 16), (2, 32)),
                                                                weights=(0.5, 0.5), max_dirs=4, pool=pool)):
        out.append(S.Request(i, d, n, om, m, dirs, t))
    return out


def test_every_request_served_and_equal_to_alone():
    be = FakeBackend()
    reqs = requests(30, 400.0)
    res, st = S.Engine(be, slots=4, budget_bytes=10 << 20).run(reqs)
    assert st["errors"] == 0 and st["requests"] == 30 and st["all_converged"]
    for q, r in zip(sorted(reqs, key=lambda q: q.arrival), res):
        ref = be.solve(None, q)[0]
        assert np.array_equal(r.u, ref)
        assert r.end >= r.start >= r.arrival - 1e-9


def test_budget_is_never_exceeded_and_factors_are_cached():
    be = FakeBackend()
    reqs = requests(40, 2000.0, pool=3)
    budget = 3 * 32 * 32 * 1000  # room for three of the largest media
    res, st = S.Engine(be, slots=4, budget_bytes=budget).run(reqs)
    assert st["errors"] == 0
    assert st["max_used_bytes"] <= budget
    assert st["cache_hits"] > 0
    # a medium is factored once per residency in the cache
    assert be.factored == len(reqs) - st["cache_hits"]


def test_evictions_under_a_small_budget():
    be = FakeBackend()
    reqs = requests(30, 2000.0, pool=4)
    budget = 32 * 32 * 1000  # one large medium at a time
    res, st = S.Engine(be, slots=3, budget_bytes=budget).run(reqs)
    assert st["errors"] == 0 and st["max_used_bytes"] <= budget
    assert st["evictions"] > 0


def test_oversize_request_is_reported_and_the_rest_served():
    be = FakeBackend()
    reqs = requests(10, 1000.0)
    big = S.Request(99, 2, 64, 10.0, np.zeros((64, 64)), np.array([[1.0, 0.0]]), 0.001)
    res, st = S.Engine(be, slots=2, budget_bytes=32 * 32 * 1000).run(reqs + [big])
    errs = [r for r in res if r.error]
    assert [r.rid for r in errs] == [99] and "budget" in errs[0].error
    assert st["requests"] == 11 and st["errors"] == 1


@pytest.mark.parametrize("slots", [1, 4])
def test_slots_run_concurrently(slots):
    be = FakeBackend(solve_s=0.03)
    reqs = [S.Request(i, 2, 16, 12.0, np.full((16, 16), 0.1 * (i + 1)), np.array([[1.0, 0.0]]), 0.0)
            for i in range(8)]
    t0 = time.perf_counter()
    res, st = S.Engine(be, slots=slots, budget_bytes=1 << 30).run(reqs)
    wall = time.perf_counter() - t0
    assert st["max_concurrent"] == slots
    # 8 solves of 30 ms (+3 ms factor): serial ~0.26 s, four slots ~0.07 s
    if slots == 4:
        assert wall < 0.24
    else:
        assert wall > 0.25


def test_latency_statistics_follow_the_schedule():
    be = FakeBackend(solve_s=0.02, factor_s=0.0)
    reqs = [S.Request(i, 2, 16, 12.0, np.full((16, 16), 0.01 * (i + 1)), np.array([[1.0, 0.0]]), 0.0)
            for i in range(10)]
    res, st = S.Engine(be, slots=1, budget_bytes=1 << 30).run(reqs)
    lat = sorted(r.latency for r in res)
    # one slot, all arriving at once: the k-th result waits for k solves of 20 ms
    for k, l in enumerate(lat):
        assert l >= 0.02 * (k + 1) - 1e-3
    assert abs(st["p50_ms"] - np.percentile(lat, 50) * 1e3) < 1e-6
    assert st["p99_ms"] >= st["p50_ms"]
    assert st["solves"] == 10 and st["solves_per_s"] > 0


class RetargetBackend(FakeBackend):
    """Fake backend that can give an open context a new medium (as ls_set_medium does)."""

    def __init__(self, **kw):
        super().__init__(**kw)
        self.opened = 0
        self.retargeted = 0

    def open(self, req):
        with self.lock:
            self.opened += 1
        return {"key": req.key, "grid": (req.d, req.n, req.omega)}

    def retarget(self, ctx, req):
        assert ctx["grid"] == (req.d, req.n, req.omega)
        with self.lock:
            self.retargeted += 1
        ctx["key"] = req.key

    def solve(self, ctx, req):
        assert ctx["key"] == req.key  # the context holds this request's medium
        return super().solve(ctx, req)


def test_idle_contexts_of_the_same_grid_take_new_media():
    be = RetargetBackend()
    reqs = requests(40, 2000.0)  # every medium unique
    budget = 2 * 32 * 32 * 1000  # two large media at a time
    res, st = S.Engine(be, slots=2, budget_bytes=budget).run(reqs)
    assert st["errors"] == 0 and st["all_converged"]
    assert st["max_used_bytes"] <= budget
    assert st["retargets"] > 0 and be.retargeted == st["retargets"]
    assert be.opened + be.retargeted == len(reqs)  # no cache hits: every request got a context
    for q, r in zip(sorted(reqs, key=lambda q: q.arrival), res):
        assert np.array_equal(r.u, be.solve({"key": q.key}, q)[0])


def test_no_retarget_while_memory_fits():
    be = RetargetBackend()
    reqs = requests(10, 2000.0)
    res, st = S.Engine(be, slots=2, budget_bytes=1 << 30).run(reqs)
    assert st["errors"] == 0 and st["retargets"] == 0 and be.opened == len(reqs)


def test_a_failed_retarget_is_reported_and_the_engine_keeps_serving():
    class Flaky(RetargetBackend):
        def retarget(self, ctx, req):
            if req.rid % 3 == 0:
                raise RuntimeError("set_medium refused")
            super().retarget(ctx, req)

    be = Flaky()
    reqs = requests(30, 2000.0)
    budget = 2 * 32 * 32 * 1000
    res, st = S.Engine(be, slots=2, budget_bytes=budget).run(reqs)
    assert st["requests"] == 30 and st["max_used_bytes"] <= budget
    failed = [r for r in res if r.error]
    assert failed and all("set_medium refused" in r.error for r in failed)
    assert all(r.rid % 3 == 0 for r in failed)
    for q, r in zip(sorted(reqs, key=lambda q: q.arrival), res):
        if not r.error:
            assert np.array_equal(r.u, be.solve({"key": q.key}, q)[0])


class SpillBackend(FakeBackend):
    """Fake backend whose contexts can export and import their factorization."""

    def __init__(self, **kw):
        super().__init__(**kw)
        self.imported = 0

    def open(self, req):
        return {"key": req.key, "factored": False}

    def factor(self, ctx):
        super().factor(ctx)
        ctx["factored"] = True

    def export_factors(self, ctx):
        assert ctx["factored"]
        return ("blob:" + ctx["key"]).encode()

    def import_factors(self, ctx, blob):
        assert blob == ("blob:" + ctx["key"]).encode()  # the medium's own factorization
        with self.lock:
            self.imported += 1
        ctx["factored"] = True

    def solve(self, ctx, req):
        assert ctx["factored"] and ctx["key"] == req.key
        return super().solve(ctx, req)


def test_evicted_factorizations_come_back_from_host_memory():
    be = SpillBackend()
    reqs = requests(40, 2000.0, pool=4)
    budget = 32 * 32 * 1000  # one large medium at a time on the device
    res, st = S.Engine(be, slots=2, budget_bytes=budget, host_cache_bytes=1 << 20).run(reqs)
    assert st["errors"] == 0 and st["all_converged"] and st["max_used_bytes"] <= budget
    assert st["spills"] > 0 and st["host_hits"] > 0 and be.imported == st["host_hits"]
    # every request is a device hit, a host hit or a fresh factorization
    assert be.factored + st["host_hits"] + st["cache_hits"] == len(reqs)
    for q, r in zip(sorted(reqs, key=lambda q: q.arrival), res):
        assert np.array_equal(r.u, be.solve({"key": q.key, "factored": True}, q)[0])


def test_host_cache_is_bounded():
    be = SpillBackend()
    reqs = requests(40, 2000.0, pool=6)
    blob = len(be.export_factors({"key": reqs[0].key, "factored": True}))
    eng = S.Engine(be, slots=1, budget_bytes=32 * 32 * 1000, host_cache_bytes=2 * blob + 1)
    res, st = eng.run(reqs)
    assert st["errors"] == 0
    assert sum(len(b) for b in eng._spill_store.values()) <= 2 * blob + 1
