"""Multi-rank bench path on CPU: two `gloo` ranks stand in for two GPUs.

The solve does not shard, so N ranks run independent replicas; what the
ranks share is the timing contract: a barrier on both sides of the timed
region, the job time taken as the maximum over ranks, and the value as all
ranks' solves over that time.  The reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    dist.barrier()
    t = bench.job_time_ms(100.0 * (rank + 1), ws)        # rank r "took" 100 (r + 1) ms
    v = bench.job_value(5, ws, t)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, v))


def test_two_rank_job_time_is_max_and_value_counts_all_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, v in got:
        assert t == 200.0                       # the slower rank's time, on every rank
        assert v == pytest.approx(2 * 5 / 0.2)  # 10 solves in 0.2 s


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time_ms(12.5, 1) == 12.5
    assert bench.job_value(4, 1, 500.0) == pytest.approx(8.0)


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
