"""Cluster windows sharded over ranks (Section 5.2: independent clusters on
separate processors): the anchor partition, and the assembly of the
per-rank density matrices by one all-reduce, run as two gloo ranks on the
CPU with the oracle computing each rank's windows."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_partition_covers_every_anchor_once_and_balances():
    from paper_1311_6696_gb300 import shard
    for (Ly, Lx, n, world) in ((14, 14, 4, 2), (14, 14, 6, 8), (20, 20, 2, 3), (5, 7, 3, 4), (3, 3, 2, 16)):
        parts = shard.partition(Ly, Lx, n, world)
        assert len(parts) == world and parts[0][0] == 0 and parts[-1][1] == Ly * Lx
        for (a0, a1), (b0, _) in zip(parts, parts[1:]):
            assert a0 <= a1 == b0
        cost = [shard.window_cost(Ly, Lx, n, a // Lx, a % Lx) for a in range(Ly * Lx)]
        share = sum(cost) / world
        for a0, a1 in parts:
            assert sum(cost[a0:a1]) <= share + max(cost) + 1e-9


def test_window_extent_is_the_clipped_window():
    from oracle import peps_oracle as O
    from paper_1311_6696_gb300 import shard
    for L in (1, 4, 9):
        for n in (1, 2, 3, 6, 20):
            for i in range(L):
                lo, hi = O.window_bounds(L, i, n)
                assert shard.window_extent(L, i, n) == hi - lo + 1


def test_owned_masks_give_each_entry_one_owner():
    from paper_1311_6696_gb300 import shard
    Ly, Lx = 5, 6
    parts = shard.partition(Ly, Lx, 3, 3)
    tot = [0, 0, 0]
    for a0, a1 in parts:
        for i, m in enumerate(shard.owned_masks(Ly, Lx, a0, a1)):
            tot[i] = tot[i] + m.astype(int)
    for t in tot:
        assert np.all(t == 1)


def _oracle_parts(A, n, chi, a0, a1):
    """What one rank contributes: its anchors' normalised density matrices,
    zeros elsewhere (the oracle stands in for the GPU)."""
    from oracle import peps_oracle as O
    Ly, Lx = A.shape[:2]
    anchors = [(a // Lx, a % Lx) for a in range(a0, a1)]
    env = O.env_cluster(A, n=n, chi=chi, mode="var", anchors=anchors)
    d = A.shape[2]
    out = {"site": np.zeros((Ly * Lx, d, d)), "hbond": np.zeros((Ly * (Lx - 1), d * d, d * d)),
           "vbond": np.zeros(((Ly - 1) * Lx, d * d, d * d))}
    for (y, x) in anchors:
        out["site"][y * Lx + x] = env["rho_site"][y][x]
        if x + 1 < Lx:
            out["hbond"][y * (Lx - 1) + x] = env["rho_h"][y][x].reshape(d * d, d * d)
        if y + 1 < Ly:
            out["vbond"][y * Lx + x] = env["rho_v"][y][x].reshape(d * d, d * d)
    return out


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1311_6696_gb300 import shard, synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A = synth.peps_gauss(4, 5, 2, 2, seed=81)
    a0, a1 = shard.partition(4, 5, 2, world)[rank]
    full = shard.gather_rhos(_oracle_parts(A, 2, 6, a0, a1), dist)
    dist.destroy_process_group()
    q.put((rank, (a0, a1), full))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_assemble_the_whole_cluster_environment():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict((r, (rng, full)) for r, rng, full in (q.get(timeout=300) for _ in ps))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(4, 5, 2, 2, seed=81)
    whole = _oracle_parts(A, 2, 6, 0, 20)
    (r0, f0), (r1, f1) = res[0], res[1]
    assert r0[1] == r1[0] and r0[0] == 0 and r1[1] == 20 and r0[1] - r0[0] > 0 and r1[1] - r1[0] > 0
    for k in ("site", "hbond", "vbond"):
        assert np.array_equal(f0[k], f1[k])
        assert np.array_equal(f0[k], whole[k])


# ------------------------------------------------------------------ the tensor update over ranks (Section 5.4)
def test_row_partition_keeps_strips_whole_and_balances():
    from oracle import update_oracle as U
    from paper_1311_6696_gb300 import shard
    for (Ly, Lx, world) in ((6, 5, 2), (6, 5, 3), (20, 20, 8), (4, 4, 16)):
        for s in U.trotter_sets(Ly, Lx):
            parts = shard.row_partition(s, world)
            assert len(parts) == world
            assert sorted(b for p in parts for b in p) == sorted(s)
            strips = {}
            for r, p in enumerate(parts):
                for kind, y, x in p:
                    strips.setdefault((kind, y if kind == 0 else x), set()).add(r)
            assert all(len(v) == 1 for v in strips.values())
            biggest = max(sum(1 for b in s if (b[1] if b[0] == 0 else b[2]) == k[1]) for k in strips)
            for p in parts:
                assert len(p) <= len(s) / world + biggest


def _update_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from oracle import update_oracle as U
    from paper_1311_6696_gb300 import shard, synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A = synth.peps_simple_update(5, 4, 2, seed=7, steps=40)
    G = U.heisenberg_gate(0.05)
    out = []
    for s in U.trotter_sets(5, 4):
        mine = shard.row_partition(s, world)[rank]
        new, _ = U.update_bonds_cluster(A, G, mine, 1, chi=8, mode="var") if mine else (A, [])
        merged = shard.merge_updates(torch.from_numpy(A), torch.from_numpy(np.asarray(new)),
                                     shard.bond_sites(mine), dist)
        out.append(merged.numpy())
    dist.destroy_process_group()
    q.put((rank, out))


def test_two_gloo_ranks_reproduce_one_cluster_update_of_each_set():
    """Each rank refits its strips' bonds (the oracle stands in for the GPU);
    the merged lattice equals one update of the whole set, bit for bit."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    from oracle import update_oracle as U
    from paper_1311_6696_gb300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    ps = [ctx.Process(target=_update_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=300) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    A = synth.peps_simple_update(5, 4, 2, seed=7, steps=40)
    G = U.heisenberg_gate(0.05)
    for i, s in enumerate(U.trotter_sets(5, 4)):
        whole, _ = U.update_bonds_cluster(A, G, s, 1, chi=8, mode="var")
        assert np.array_equal(res[0][i], whole) and np.array_equal(res[1][i], whole)
