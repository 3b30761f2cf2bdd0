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


def test_set_cost_model_counts_the_operations():
    """One environment set of an L x L lattice: 4 sweeps of L-1 absorbs, each
    (L-1) right environments + 2 half-sweeps of L site steps; 2L passes of
    2(L-1) environment steps and L open sites."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.set_cost_model(3, 1.0, 0.0) == 4 * 2 * (2 + 6) + 2 * 3 * 4
    assert bench.set_cost_model(3, 0.0, 1.0) == 2 * 3 * 3
    assert bench.set_cost_model(20, 2.0, 5.0) == 4 * 19 * 59 * 2.0 + 40 * (38 * 2.0 + 20 * 5.0)


def test_reference_arm_step_time_is_the_time_of_its_value():
    """The reference arm's ms_per_step is the time of one whole environment set
    at the throughput it reports (not the time of its sample)."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "c2",
                        "--steps", "1", "--warmup", "0", "--ref-budget", "1"],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "envs/s"
    assert abs(line["ms_per_step"] - 1e3 * 100 / line["value"]) <= 1e-3 * line["ms_per_step"] + 0.1
    assert line["e2e"]["value"] == line["value"] and line["cpu_baseline"]["kind"] == "oracle"
