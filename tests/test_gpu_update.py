"""The full update's tensor update on the GPU (peps_bond_update) against the
FP64 oracle (oracle/update_oracle.py): Section 2's reduced-tensor ALS, every
bond of a Trotter set from the environment of the same state (Sections 4.4,
5.2), and the imaginary-time evolution against the paper's FU energy."""
from __future__ import annotations

import os

import numpy as np
import pytest

from oracle import bruteforce as BF
from oracle import peps_oracle as O
from oracle import update_oracle as U

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_6696_gb300 import peps
    return torch, peps


def _pair_products(A, bonds):
    """The two-site tensor of every bond (bond gauge summed out)."""
    out = []
    for kind, y, x in bonds:
        a = A[y, x]
        if kind == 0:
            out.append(np.einsum("sulnr,tvrmq->sulntvmq", a, A[y, x + 1]))
        else:
            out.append(np.einsum("sulnr,tnvmq->sulrtvmq", a, A[y + 1, x]))
    return out


def _untouched(bonds, Ly, Lx):
    used = set()
    for kind, y, x in bonds:
        used.add((y, x))
        used.add((y, x + 1) if kind == 0 else (y + 1, x))
    return [(y, x) for y in range(Ly) for x in range(Lx) if (y, x) not in used]


def _compare(got, want, bonds, tol):
    for pg, pw in zip(_pair_products(got, bonds), _pair_products(want, bonds)):
        assert np.max(np.abs(pg - pw)) < tol * np.max(np.abs(pw))


@pytest.mark.parametrize("mode", ["svd", "var"])
@pytest.mark.parametrize("set_index", [0, 1, 2, 3])
def test_fp64_bond_update_matches_the_oracle(env, mode, set_index):
    torch, peps = env
    from paper_1311_6696_gb300 import synth
    A = synth.peps_simple_update(5, 4, 3, seed=11, steps=60)
    G = U.heisenberg_gate(0.05)
    bonds = U.trotter_sets(5, 4)[set_index]
    want, wcost = U.update_bonds(A, G, bonds, chi=12, mode=mode, iters=6)
    At = torch.from_numpy(A).cuda()
    out, cost = peps.bond_update(At, G, bonds, chi=12, mode=mode, iters=6, out=torch.empty_like(At))
    got = out.cpu().numpy()
    _compare(got, want, bonds, 1e-9)
    assert np.max(np.abs(np.array(cost) - np.array(wcost))) < 1e-9
    for y, x in _untouched(bonds, 5, 4):
        assert np.array_equal(got[y, x], A[y, x])
    assert np.array_equal(At.cpu().numpy(), A)        # the input was not written


def test_update_in_place_and_f32(env):
    torch, peps = env
    from paper_1311_6696_gb300 import synth
    A = synth.peps_simple_update(4, 4, 2, seed=3, steps=40)
    G = U.heisenberg_gate(0.02)
    bonds = U.trotter_sets(4, 4)[2]
    want, _ = U.update_bonds(A, G, bonds, chi=16, mode="svd", iters=4)
    At = torch.from_numpy(A).cuda()
    peps.bond_update(At, G, bonds, chi=16, mode="svd", iters=4)
    _compare(At.cpu().numpy(), want, bonds, 1e-9)
    A32 = torch.from_numpy(A.astype(np.float32)).cuda()
    peps.bond_update(A32, G, bonds, chi=16, mode="svd", iters=4)
    _compare(A32.cpu().numpy().astype(np.float64), want, bonds, 1e-5)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_tensor_core_environment_update_matches_the_oracle(env, prec):
    """8x8 D=4 at chi=16: the norm matrices from the tensor-core contraction,
    the ALS in FP64."""
    torch, peps = env
    from paper_1311_6696_gb300 import synth
    A = synth.peps_simple_update(8, 8, 4, seed=5, steps=60)
    G = U.heisenberg_gate(0.05)
    bonds = U.trotter_sets(8, 8)[0]
    want, wcost = U.update_bonds(A, G, bonds, chi=16, mode="var", iters=6)
    At = torch.from_numpy(A).cuda()
    out, cost = peps.bond_update(At, G, bonds, chi=16, mode="var", precision=prec, iters=6,
                                 out=torch.empty_like(At))
    _compare(out.cpu().numpy(), want, bonds, 2e-4)


def test_exact_gate_reproduces_the_brute_force_state(env):
    """A bond carrying one Schmidt value: the gated state is held exactly."""
    torch, peps = env
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(3, 3, 2, 4, 23)
    y, x = 1, 1
    A[y, x, :, :, :, :, 1:] = 0.0
    A[y, x + 1, :, :, 1:, :, :] = 0.0
    G = U.heisenberg_gate(0.7) @ np.diag([1.0, 2.0, 0.5, 1.5])
    At = torch.from_numpy(A).cuda()
    _, cost = peps.bond_update(At, G, [(0, y, x)], chi=64, mode="svd", iters=6)
    psi = BF.state_vector(BF.dense_lattice(A)).reshape([2] * 9)
    i1, i2 = 4, 5
    P = np.moveaxis(psi, (i1, i2), (0, 1))
    sh = P.shape
    want = np.moveaxis((G @ P.reshape(4, -1)).reshape(sh), (0, 1), (i1, i2)).ravel()
    got = BF.state_vector(BF.dense_lattice(At.cpu().numpy()))
    c = abs(float(got @ want)) / (np.linalg.norm(got) * np.linalg.norm(want))
    assert 1.0 - c < 1e-12 and cost[0] < 1e-12


def test_bond_update_input_errors(env):
    torch, peps = env
    from paper_1311_6696_gb300 import synth
    A = torch.from_numpy(synth.peps_gauss(3, 3, 2, 2, 1)).cuda()
    G = np.eye(4)
    with pytest.raises(peps.PepsError):
        peps.bond_update(A, G, [(0, 0, 0), (0, 0, 1)], chi=8)          # shared site
    with pytest.raises(peps.PepsError):
        peps.bond_update(A, G, [(0, 0, 2)], chi=8)                      # outside
    with pytest.raises(peps.PepsError):
        peps.bond_update(A, G, [(2, 0, 0)], chi=8)                      # kind
    with pytest.raises(peps.PepsError):
        peps.bond_update(A, np.full((4, 4), np.nan), [(0, 0, 0)], chi=8)
    # the context is still usable
    peps.bond_update(A, G, [(0, 0, 0)], chi=8)


def _e_fu_table(kind="D"):
    for line in open(os.path.join(GOLDEN, "fu_heisenberg_4x4_table.txt")):
        p = line.split()
        if p and p[0] == kind and p[1] == "2":
            return float(p[5]), float(p[7])


def test_gpu_full_update_reaches_the_paper_fu_energy_at_4x4_D2(env):
    """The parallel FU on the GPU from the simple-update state (D' = 4 as in
    Table EFU), energy per site from the GPU's full environment at chi = 64."""
    torch, peps = env
    from paper_1311_6696_gb300 import synth
    A = torch.from_numpy(synth.peps_simple_update(4, 4, 2, seed=0)).cuda()
    G = U.heisenberg_gate(0.01)
    peps.evolve(A, G, steps=160, chi=4, mode="svd", iters=6)
    e = peps.env_full(A, chi=64, mode="svd")
    h = np.concatenate([e.expect("hbond", O.SDOTS), e.expect("vbond", O.SDOTS)])
    e_site = float(np.sum(h)) / 16
    e_tab, tol = _e_fu_table()
    assert abs(e_site - e_tab) < tol, (e_site, e_tab)


# ------------------------------------------------------------------ cluster update CU_delta (Section 5)
@pytest.mark.parametrize("delta", [0, 1, 2])
@pytest.mark.parametrize("set_index", [0, 3])
def test_fp64_cluster_update_matches_the_oracle(env, delta, set_index):
    torch, peps = env
    from paper_1311_6696_gb300 import synth
    A = synth.peps_simple_update(5, 4, 3, seed=11, steps=60)
    G = U.heisenberg_gate(0.05)
    bonds = U.trotter_sets(5, 4)[set_index]
    want, wcost = U.update_bonds_cluster(A, G, bonds, delta, chi=12, mode="var", iters=6)
    At = torch.from_numpy(A).cuda()
    out, cost = peps.bond_update(At, G, bonds, chi=12, mode="var", iters=6, out=torch.empty_like(At), delta=delta)
    got = out.cpu().numpy()
    _compare(got, want, bonds, 1e-9)
    assert np.max(np.abs(np.array(cost) - np.array(wcost))) < 1e-9
    for y, x in _untouched(bonds, 5, 4):
        assert np.array_equal(got[y, x], A[y, x])


def test_cluster_covering_the_lattice_is_the_full_update_on_the_gpu(env):
    torch, peps = env
    from paper_1311_6696_gb300 import synth
    A = torch.from_numpy(synth.peps_simple_update(5, 4, 3, seed=11, steps=60)).cuda()
    G = U.heisenberg_gate(0.05)
    for bonds in U.trotter_sets(5, 4):
        a, ca = peps.bond_update(A, G, bonds, chi=12, mode="var", iters=6, out=torch.empty_like(A))
        b, cb = peps.bond_update(A, G, bonds, chi=12, mode="var", iters=6, out=torch.empty_like(A), delta=4)
        assert torch.max(torch.abs(a - b)).item() < 1e-12
        assert np.max(np.abs(ca - cb)) < 1e-12


def test_cluster_update_rejects_a_negative_delta(env):
    torch, peps = env
    from paper_1311_6696_gb300 import synth
    A = torch.from_numpy(synth.peps_gauss(3, 3, 2, 2, 1)).cuda()
    with pytest.raises(peps.PepsError):
        peps.bond_update(A, np.eye(4), [(0, 0, 0)], chi=8, delta=-1)


def test_gpu_cu1_reaches_the_paper_energy_at_4x4_D2(env):
    """The parallel CU_1 on the GPU (D' = 4, Table ECU1)."""
    torch, peps = env
    from paper_1311_6696_gb300 import synth
    A = torch.from_numpy(synth.peps_simple_update(4, 4, 2, seed=0)).cuda()
    G = U.heisenberg_gate(0.01)
    peps.evolve(A, G, steps=160, chi=4, mode="svd", iters=6, delta=1)
    e = peps.env_full(A, chi=64, mode="svd")
    h = np.concatenate([e.expect("hbond", O.SDOTS), e.expect("vbond", O.SDOTS)])
    e_tab, tol = _e_fu_table("CU1")
    assert abs(float(np.sum(h)) / 16 - e_tab) < tol
