"""The multi-rank path of bench.py on CPU (gloo, world size 2): the barrier and
max-over-ranks timing, the whole-job aggregation of independent replicas, and
the reference arm under torchrun (rank 0 alone prints its line)."""
import json
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


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_setup()
    ms = 100.0 + 50.0 * r           # rank 1 is the slow one
    bench.barrier()
    ms_max = bench.allreduce(ms, "max")
    launches = bench.allreduce(7 + r, "sum")
    rate = bench.replica_rate(2 * 8 * 64 * 64 * 3, w, ms_max)
    out.put((r, w, ms_max, launches, rate))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_gloo_two_ranks_timing_and_aggregation():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, ms_max, launches, rate in res:
        assert w == 2
        assert ms_max == 150.0             # the slowest rank's time, on every rank
        assert launches == 15.0            # 7 + 8
        # both replicas' outputs over the slowest rank's time
        assert rate == pytest.approx(2 * (2 * 8 * 64 * 64 * 3) / 0.150)


def test_reference_arm_under_torchrun_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--N", "64", "--steps", "1", "--warmup", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
