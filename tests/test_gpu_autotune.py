"""The autotuner (ls_autotune) through the C-ABI: it times the launch-shape alternatives on a
context, applies the fastest, keeps them for later contexts of the same grid and precision
and writes them to LS_TUNE_FILE; every alternative factors and solves the same system, so
the solve after tuning matches the oracle like any other (mixed-precision tolerances)."""

import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1408_4495_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.late(1)]


@pytest.fixture(scope="module")
def LS():
    from paper_1408_4495_gb300 import build, ls
    build.build()
    return ls


def test_autotune_applies_keeps_and_persists_its_choice(LS, tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("LS_TUNE_FILE", str(path))
    n, d = 64, 2
    rng = np.random.default_rng(12)
    m = W.enforce_buffer(W.bumps(n, d, rng.uniform(-0.2, 0.2, 3), rng.uniform(0.06, 0.1, 3),
                                 rng.uniform(0.35, 0.65, (3, 2))), 2)
    omega = 2 * np.pi * 8
    dirs = W.directions_circle(3)
    with LS.Solver(m, omega, mixed=True) as s:
        rep = s.autotune(4)
        choice = rep["choice"]
        assert s.tune() == choice
        assert len(rep["factor_ms"]) >= 4 and all(ms > 0 for _, ms in rep["factor_ms"])
        # sweep split: the base and 2 alternatives; forward and backward solve levels on the
        # tensor cores: 5 more each (the base is automatic); the one-CTA-per-front levels: 5 more
        assert len(rep["solve_ms"]) == 18 and all(ms > 0 for _, ms in rep["solve_ms"])
        # left factored with the chosen shapes
        g = s.rhs_plane_wave(dirs)
        u, info = s.solve(g, tol=1e-6)
    ref = O.solve(n, d, omega, m, dirs, tol=1e-10)
    ref6 = O.solve(n, d, omega, m, dirs, tol=1e-6)
    for j in range(len(dirs)):
        assert info[j].converged and abs(info[j].iters - ref6["iters"][j]) <= 2
        assert np.linalg.norm(u[j].reshape(-1) - ref["u"][j]) < 1e-5 * np.linalg.norm(ref["u"][j])
    # the file holds the entry, and a later context of the same grid and precision takes it
    lines = [json.loads(x) for x in path.read_text().splitlines() if x.strip()]
    ent = [e for e in lines if e["d"] == d and e["n"] == n and e["prec"] == LS.LS_PREC_MIXED]
    assert len(ent) == 1 and ent[0]["sweep_ctas"] == choice["sweep_ctas"]
    with LS.Solver(m, omega, mixed=True) as s2:
        assert s2.tune() == choice
    with LS.Solver(m, omega, mixed=False) as s3:  # another precision keeps the defaults
        assert s3.tune()["sweep_ctas"] == 2


def test_set_tune_validates_and_applies(LS):
    n, d = 32, 2
    m = W.enforce_buffer(W.bumps(n, d, [0.1], [0.1], [[0.5, 0.5]]), 2)
    with LS.Solver(m, 2 * np.pi * 4, mixed=True) as s:
        base = s.tune()
        s.set_tune({"tcs_min_rows": 128, "sweep_ctas": 4, "unknown": 1})
        t = s.tune()
        assert t["tcs_min_rows"] == 128 and t["sweep_ctas"] == 4
        assert {k: v for k, v in t.items() if k not in ("tcs_min_rows", "sweep_ctas")} == \
            {k: v for k, v in base.items() if k not in ("tcs_min_rows", "sweep_ctas")}
        for bad in ({"sweep_ctas": 5}, {"gj_max_own": 0}, {"two_level_min": -1}, {"tcs_min_rows": 1.5},
                    {"small_max_k": 257}, {"small_max_k": -2}, {"tcs_bwd_min_rows": 0}):
            with pytest.raises(LS.LsError) as e:
                s.set_tune(bad)
            assert e.value.status == LS.LS_EINVAL
        assert s.tune() == t
        # -1: the automatic choice (the default)
        assert base["tcs_min_rows"] == base["tcs_bwd_min_rows"] == base["small_max_k"] == -1
        s.set_tune({"tcs_min_rows": -1})
        assert s.tune()["tcs_min_rows"] == -1
