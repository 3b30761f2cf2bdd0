"""Cluster environments sharded over processes (one per GPU).

The paper's cluster scheme makes every window independent: separate
processors contract their own clusters and exchange only the small
separable-boundary tensors (Section 5.2).  Here each rank

1. takes a contiguous range of anchors (row-major y*Lx + x) whose estimated
   cost is its share of the whole (``partition``),
2. computes the CU_0 boundaries itself (they are cheap, so nothing is
   exchanged before the windows) and the windows of its anchors
   (``peps_env_cluster_range``),
3. and the density matrices of all anchors are assembled on every rank by one
   all-reduce (sum) of arrays in which each rank filled only its own anchors
   (``gather_rhos``): every entry has exactly one owner, so the sum is exact.

The tensor update shards the same way (Section 5.4: with the cluster update
different rows or columns are updated simultaneously on different processors,
and only small tensors are exchanged after each set of Trotter gates).  Each
rank updates the bonds of whole row (column) strips of one set
(``row_partition``) from the input state -- recomputing the CU_0 boundaries
itself -- and the updated site tensors are assembled on every rank by one
all-reduce in which each site has one owner (``merge_updates``).

Only the partitions and the assembly live here; every contraction runs in the
library.
"""
from __future__ import annotations

import numpy as np


def window_extent(L: int, i: int, n: int) -> int:
    """Rows (or columns) of the window around index i: n, clipped at the edge
    (rows i - ceil(n/2) + 1 .. i - ceil(n/2) + n)."""
    h = -(-n // 2)
    lo = i - h + 1
    return min(lo + n - 1, L - 1) - max(lo, 0) + 1


def window_cost(Ly: int, Lx: int, n: int, y: int, x: int) -> float:
    """Relative device time of the window around (y, x): (window sites)^1.6, the
    model the library's own lane scheduler uses for one window."""
    return float(window_extent(Ly, y, n) * window_extent(Lx, x, n)) ** 1.6


def partition(Ly: int, Lx: int, n: int, world: int):
    """Contiguous anchor ranges [(a0, a1)] * world covering 0 .. Ly*Lx, each
    holding about 1/world of the total window cost (a range may be empty)."""
    assert world >= 1
    cost = np.array([window_cost(Ly, Lx, n, a // Lx, a % Lx) for a in range(Ly * Lx)])
    cum = np.concatenate([[0.0], np.cumsum(cost)])
    total = cum[-1]
    cuts = [0]
    for r in range(1, world):
        cuts.append(int(np.searchsorted(cum, total * r / world, side="left")))
    cuts.append(Ly * Lx)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def owned_masks(Ly: int, Lx: int, a0: int, a1: int):
    """Boolean masks (site [Ly*Lx], hbond [Ly*(Lx-1)], vbond [(Ly-1)*Lx]) of the
    entries an anchor range owns: site (y,x) and its bonds to (y,x+1), (y+1,x)."""
    a = np.arange(Ly * Lx)
    site = (a >= a0) & (a < a1)
    hb = np.array([a0 <= y * Lx + x < a1 for y in range(Ly) for x in range(Lx - 1)], dtype=bool)
    vb = np.array([a0 <= y * Lx + x < a1 for y in range(Ly - 1) for x in range(Lx)], dtype=bool)
    return site, hb, vb


def gather_rhos(parts: dict, dist, device="cpu") -> dict:
    """All-reduce (sum) of zero-filled per-rank density-matrix arrays
    {"site": [Ly*Lx, d, d], "hbond": [...], "vbond": [...]} into the full
    arrays on every rank (exact: each entry has one owner)."""
    import torch
    out = {}
    for k in ("site", "hbond", "vbond"):
        t = torch.as_tensor(np.ascontiguousarray(parts[k]), dtype=torch.float64, device=device)
        if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
        out[k] = t.cpu().numpy()
    return out


def env_cluster_sharded(A, n: int, chi: int, rank: int, world: int, dist=None, device="cpu", **kw) -> dict:
    """Every anchor's site / bond density matrices of the cluster scheme,
    computed over `world` ranks (this one computing partition(...)[rank]) and
    assembled on every rank.  kw: the options of peps.env_cluster."""
    from . import peps
    Ly, Lx = int(A.shape[0]), int(A.shape[1])
    a0, a1 = partition(Ly, Lx, n, world)[rank]
    env = peps.env_cluster(A, n=n, chi=chi, anchors=(a0, a1), **kw)
    parts = {k: env.rho(k) for k in ("site", "hbond", "vbond")}
    return gather_rhos(parts, dist, device)


def row_partition(bonds, world: int):
    """The bonds of one Trotter set grouped by the strip they are updated in
    (horizontal bonds by row, vertical bonds by column), the strips dealt to
    the ranks in contiguous blocks of about equal bond count."""
    assert world >= 1
    rows = {}
    for b in bonds:
        kind, y, x = (int(v) for v in b)
        rows.setdefault((kind, y if kind == 0 else x), []).append((kind, y, x))
    keys = sorted(rows)
    total = sum(len(rows[k]) for k in keys)
    parts = [[] for _ in range(world)]
    acc, r = 0, 0
    for k in keys:
        while r < world - 1 and acc >= total * (r + 1) / world:
            r += 1
        parts[r].extend(rows[k])
        acc += len(rows[k])
    return parts


def bond_sites(bonds):
    """The sites the bonds touch."""
    out = []
    for kind, y, x in bonds:
        out.append((y, x))
        out.append((y, x + 1) if kind == 0 else (y + 1, x))
    return out


def merge_updates(A_old, A_new, mine, dist):
    """The lattice with every rank's updated sites: A_new's sites listed in
    ``mine`` (this rank's), A_old's where no rank updated.  One all-reduce of
    the owned values and one of the ownership mask; each site has at most one
    owner, so the assembly is exact.  Torch tensors, any device."""
    import torch
    contrib = torch.zeros_like(A_new)
    mask = torch.zeros(A_new.shape[:2], dtype=A_new.dtype, device=A_new.device)
    for y, x in mine:
        contrib[y, x] = A_new[y, x]
        mask[y, x] = 1.0
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(contrib, op=dist.ReduceOp.SUM)
        dist.all_reduce(mask, op=dist.ReduceOp.SUM)
    return torch.where(mask[:, :, None, None, None, None, None] > 0, contrib, A_old)


def bond_update_sharded(A, gate, bonds, chi: int, rank: int, world: int, dist=None, delta=None, **kw):
    """One Trotter set updated over ``world`` ranks (this one updating
    row_partition(...)[rank]) and assembled on every rank; the same result as
    one call of peps.bond_update over all the bonds.  A: CUDA tensor
    (Ly,Lx,d,D,D,D,D), not modified; returns the new lattice.  kw: the
    options of peps.bond_update."""
    from . import peps
    mine = row_partition(bonds, world)[rank]
    new = A.clone()
    if mine:
        peps.bond_update(A, gate, mine, chi, out=new, delta=delta, **kw)
    return merge_updates(A, new, bond_sites(mine), dist)
