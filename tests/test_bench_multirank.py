"""The N > 1 launch of bench.py (replicas, one per GPU), exercised on CPU with
two gloo ranks: the slowest rank's step time bounds the job, every rank's
environments count, and the reference arm prints on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [100.0, 250.0][rank]
    e2e_ms = [120.0, 260.0][rank]
    out = bench.aggregate(ms, e2e_ms, 100, world, dist, "cpu")
    dist.destroy_process_group()
    q.put((rank, out))


def test_two_gloo_ranks_take_the_slowest_step():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        ms, e_ms, value, e2e = res[r]
        assert ms == 250.0 and e_ms == 260.0
        assert abs(value - 2 * 100 / 0.25) < 1e-9
        assert abs(e2e - 2 * 100 / 0.26) < 1e-9


def test_single_rank_aggregate_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ms, e_ms, value, e2e = bench.aggregate(50.0, 60.0, 100, 1)
    assert (ms, e_ms) == (50.0, 60.0) and abs(value - 2000.0) < 1e-9


def test_reference_arm_prints_on_rank0_only(tmp_path):
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
