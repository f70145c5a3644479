"""Host logic of bench.py under N > 1 ranks, on CPU with the gloo backend (world size 2):
the timed region's max over ranks, the whole-job rate, and the reference arm running on
rank 0 only.  The GPU path shards as independent replicas with no data-path collective,
so these are the only cross-rank steps."""

import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r"""
import os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
rank, world, _ = bench.dist_env()
dist.init_process_group("gloo", rank=rank, world_size=world)
# each rank "times" a different region; the job time is the slowest rank's
t = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu", world)
assert t == 10.0 + 5.0 * (world - 1), t
# whole-job throughput: every rank's units over that time
assert abs(bench.job_rate(16 * 3, world, t) - 16 * 3 * world / t) < 1e-12
dist.barrier()
dist.destroy_process_group()
print("ok", rank, flush=True)
"""


def _spawn(code, world, extra_env=None):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            p.kill()
            out, err = p.communicate()
        outs.append((p.returncode, out, err))
    return outs


def test_max_over_ranks_and_job_rate_gloo_world2():
    pytest.importorskip("torch")
    outs = _spawn(WORKER, 2)
    for r, (rc, out, err) in enumerate(outs):
        assert rc == 0, err
        assert f"ok {r}" in out


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, "cpu", 1) == 3.5
    assert bench.job_rate(16, 1, 2.0) == 8.0


def test_reference_arm_runs_on_rank0_only():
    # a non-zero rank exits 0 at once, without touching the oracle or printing a line
    code = ("import sys; sys.path.insert(0, sys.argv[1]); import bench; "
            "sys.argv = ['bench.py', '--impl', 'reference', '--gpus', '2', '--steps', '1', '--warmup', '3']; "
            "sys.exit(bench.main())")
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, "-c", code, ROOT], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""
