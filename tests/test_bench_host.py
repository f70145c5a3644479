"""Host-side arithmetic of bench.py's roofline model (no GPU): the live right-hand-side count
of the GMRES iterations and the per-launch algorithmic bytes."""

import numpy as np

import bench
from paper_1408_4495_gb300 import workloads as W


def test_live_rhs_counts_compacted_iterations():
    # 16 right-hand sides, 12 converge after 3 iterations and 4 after 4: the first three
    # iterations carry 16, the fourth carries 4, i.e. 52 right-hand sides in 4 launch sets
    step = [3] * 12 + [4] * 4
    assert bench.live_rhs([step]) == 52 / 4
    assert bench.live_rhs([step, [2] * 16]) == (52 + 32) / (4 + 2)
    assert bench.live_rhs([]) == 0.0


def test_algorithmic_bytes_scale_with_the_right_hand_sides():
    w = W.bumps_2d(64, 8.0, 3, 16, 1)
    nd = {"fwd_factor_bytes": 1e6, "bwd_factor_bytes": 2e6, "fwd_bytes_per_rhs": 1e4,
          "bwd_bytes_per_rhs": 2e4, "levels": 10}
    n, N = 64, 64 * 64
    assert bench.algorithmic_bytes("fft_row_fwd_c64", w, nd, None, None) == 16 * N * 8 * 3 + N * 4
    assert bench.algorithmic_bytes("fft_row_fwd_c64", w, nd, None, None, rhs=8) == 8 * N * 8 * 3 + N * 4
    assert bench.algorithmic_bytes("fft_col_sym_cff", w, nd, None, None) == 16 * 2 * (n * 2 * n) * 16 + (n + 1) ** 2 * 16
    # sweeps: every factor block once + each live right-hand side's vector read and written once
    assert bench.algorithmic_bytes("nd_fwd_c64", w, nd, None, None, rhs=4) == (1e6 + 4 * N * 8 * 2) / 10
    assert bench.algorithmic_bytes("stencil_c64", w, nd, None, None, rhs=2) == 2 * N * 8 * 2
    assert "stencil_c64".startswith(bench.PER_ITERATION)
    assert not "fft_row_fwd_cff".startswith(bench.PER_ITERATION)
    assert "fft_col_sym_cff" not in bench.HBM_CLASSES and "nd_bwd_c64" in bench.HBM_CLASSES


def test_3d_pass_bytes():
    w = W.bumps_3d(16, 2.0, 2, 4, 1)
    N = 16**3
    assert bench.algorithmic_bytes("fft_col_fwd_c64", w, {}, None, None) == 4 * N * 8 * 6
    assert bench.algorithmic_bytes("fft_col_sym_c64", w, {}, None, None) == 4 * N * 8 * 8 + 17**3 * 8


def test_sweep_launches_follow_the_counts():
    """A sweep is one launch per level on the CUDA cores; a tensor-core level adds its gather
    and scatter: the launches per sweep come from the class counts over the applications
    (one nd_items_out launch each, whether the items came from a transposition launch or
    from the fused stencil), else one per level."""
    nd = {"levels": 10, "fwd_factor_bytes": 1e6, "bwd_factor_bytes": 2e6}
    assert bench.sweep_launches("nd_fwd_c64", nd, None) == 10
    assert bench.sweep_launches("nd_fwd_c64", nd, {"nd_fwd_c64": 42, "nd_items_out_c64": 3}) == 14
    assert bench.sweep_launches("nd_fwd_c64", nd, {"nd_fwd_c64": 42, "nd_items_c64": 1, "nd_items_out_c64": 3}) == 14
    w = bench.workload("2d_bumps_n256_omega2pi32_16rhs")
    N = w.n ** 2
    per = (1e6 + 16 * N * 8 * 2) / 14
    assert bench.algorithmic_bytes("nd_fwd_c64", w, nd, {"nd_fwd_c64": 42, "nd_items_out_c64": 3}, 3) == per


def test_recorded_traffic_follows_the_sources(monkeypatch):
    """The recorded ncu traffic of a sweep is used only while the sources it was captured with
    are unchanged (sha1 of their regions), and is scaled to the live right-hand sides by the
    byte model and spread over the sweep's launches."""
    rec = dict(bench.TRAFFIC["nd_fwd_c64"])
    rec["sha1"] = bench.source_sha1(rec["src"])
    assert rec["sha1"] is not None
    monkeypatch.setitem(bench.TRAFFIC, "nd_fwd_c64", rec)
    assert bench.recorded_traffic("nd_fwd_c64") == rec["bytes_per_sweep"]
    nd = {"levels": 17, "fwd_factor_bytes": 1e9, "bwd_factor_bytes": 1.2e9}
    w = bench.workload("2d_noise_n1024_omega2pi128_64rhs")
    counts = {"nd_fwd_c64": 41 * 9, "nd_items_out_c64": 9}
    per = bench.recorded_traffic("nd_fwd_c64", w, nd, 32, counts)
    scale = bench.sweep_bytes("nd_fwd_c64", w, nd, 32) / bench.sweep_bytes("nd_fwd_c64", w, nd, rec["rhs"])
    assert np.isclose(per, rec["bytes_per_sweep"] * scale / 41)
    stale = dict(rec, sha1="0" * 40)
    monkeypatch.setitem(bench.TRAFFIC, "nd_fwd_c64", stale)
    assert bench.recorded_traffic("nd_fwd_c64") is None
