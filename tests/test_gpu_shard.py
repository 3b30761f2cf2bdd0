"""Anchor ranges of the cluster scheme on the GPU: calls whose ranges
partition the anchors reproduce one full call, and bad ranges fail."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def peps():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1311_6696_gb300 import peps as P
    return P


@pytest.mark.parametrize("precision", ["fp64", "tf32x3"])
def test_partitioned_ranges_reproduce_the_full_call(peps, precision):
    from paper_1311_6696_gb300 import shard, synth
    A = synth.peps_gauss(6, 7, 2, 3, seed=91)
    full = peps.env_cluster(A, n=3, chi=9, mode="var", precision=precision)
    tol = 1e-12 if precision == "fp64" else 1e-6
    for world in (2, 3):
        acc = {k: np.zeros_like(full.rho(k)) for k in ("site", "hbond", "vbond")}
        for a0, a1 in shard.partition(6, 7, 3, world):
            part = peps.env_cluster(A, n=3, chi=9, mode="var", precision=precision, anchors=(a0, a1))
            masks = shard.owned_masks(6, 7, a0, a1)
            for (k, m) in zip(("site", "hbond", "vbond"), masks):
                r = part.rho(k)
                assert np.all(r[~m] == 0.0)            # nothing outside the range
                acc[k] += r
        for k in acc:
            f = full.rho(k)
            assert np.max(np.abs(acc[k] - f)) <= tol * np.max(np.abs(f)), (world, k)


def test_sharded_helper_on_one_rank_is_the_full_call(peps):
    from paper_1311_6696_gb300 import shard, synth
    A = synth.peps_gauss(5, 5, 2, 2, seed=92)
    full = peps.env_cluster(A, n=2, chi=4, mode="var")
    got = shard.env_cluster_sharded(A, n=2, chi=4, rank=0, world=1, mode="var")
    for k in ("site", "hbond", "vbond"):
        assert np.max(np.abs(got[k] - full.rho(k))) <= 1e-12 * np.max(np.abs(full.rho(k)))


def test_bad_anchor_ranges_are_einval(peps):
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(3, 3, 2, 2, seed=93)
    for rng in ((-1, 3), (4, 2), (0, 10)):
        with pytest.raises(peps.PepsError) as e:
            peps.env_cluster(A, n=2, chi=4, anchors=rng)
        assert e.value.code == peps.EINVAL
    e = peps.env_cluster(A, n=2, chi=4, anchors=(0, 0))          # empty: nothing computed
    assert np.all(e.rho("site") == 0.0)


@pytest.mark.parametrize("delta", [None, 1])
def test_update_shares_merged_equal_one_update(peps, delta):
    """The tensor update of a Trotter set split into row strips for 3 ranks
    (Section 5.4), each share computed from the same input and merged, equals
    one call over the whole set."""
    import torch
    from oracle import update_oracle as U
    from paper_1311_6696_gb300 import shard, synth
    A = torch.from_numpy(synth.peps_simple_update(6, 5, 3, seed=5, steps=40)).cuda()
    G = U.heisenberg_gate(0.05)
    for s in U.trotter_sets(6, 5):
        whole, _ = peps.bond_update(A, G, s, chi=12, mode="var", out=torch.empty_like(A), delta=delta)
        merged = A.clone()
        for r in range(3):
            new = shard.bond_update_sharded(A, G, s, 12, r, 3, None, delta=delta, mode="var")
            merged = shard.merge_updates(merged, new, shard.bond_sites(shard.row_partition(s, 3)[r]), None)
        assert torch.max(torch.abs(merged - whole)).item() < 1e-12
