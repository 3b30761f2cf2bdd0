"""Pins of the tensor-update oracle (Section 2: ALS with N_l A_l = b_l on the
reduced tensors; Sections 4.4 / 5.2: the bonds of a Trotter set updated
from one environment), against things the oracle's own formulas do not fix:

* the norm matrix N against the brute-force norm network with the reduced
  tensors removed (state vectors, no boundary MPS);
* exact gates: a gate whose result the new bond can hold (a product gate, or
  any gate on a bond that carried one Schmidt value) must reproduce the
  brute-force state G|psi> exactly;
* Eckart-Young: with N the identity the ALS fixed point is the truncated SVD;
* stationarity of the ALS result for a general N;
* the imaginary-time evolution against the paper's FU energy of the 4x4
  Heisenberg model at D=2 (Table EFU) and the variational bound (exact
  energy, Appendix A);
* the cluster update CU_delta (Section 5): delta >= L-1 is the full update
  bit for bit, an exact gate stays exact with a cluster environment, and the
  CU_1 and CU_0 evolutions reach the paper's energies (Tables ECU1, ECU0).
"""
from __future__ import annotations

import os

import numpy as np
import pytest

from oracle import bruteforce as BF
from oracle import peps_oracle as O
from oracle import update_oracle as U
from paper_1311_6696_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_lattice(Ly, Lx, d, D, seed):
    return synth.peps_gauss(Ly, Lx, d, D, seed)


def _norm_matrix_bruteforce(Ad, p1, p2, X1site, X2site):
    """Sum over every physical index but the pair's of psi_X psi_X, where psi_X
    is the lattice with the pair's sites replaced by the isometry tensors
    (their reduced leg in place of the physical one)."""
    rows = BF.dense_lattice(Ad)
    rows[p1[0]][p1[1]] = X1site
    rows[p2[0]][p2[1]] = X2site
    psi = BF.state_vector(rows)
    dims = [t.shape[0] for row in rows for t in row]
    psi = psi.reshape(dims)
    Lx = len(rows[0])
    i1, i2 = p1[0] * Lx + p1[1], p2[0] * Lx + p2[1]
    others = [i for i in range(len(dims)) if i not in (i1, i2)]
    P = np.transpose(psi, [i1, i2] + others).reshape(dims[i1], dims[i2], -1)
    return np.einsum("abx,cdx->abcd", P, P)


def _exact_bond_norm(Ad, kind, y, x, chi=64):
    lat = O.lattice_from_dense(Ad)
    o = O.orientations(lat)
    src, H = (o[0], Ad.shape[0]) if kind == 0 else (o[2], Ad.shape[1])
    r, c = (y, x) if kind == 0 else (x, y)
    tb, _ = O.boundary_sweep(src, chi, "svd", 2, 0, 0, upto=H - 1)
    bb, _ = O.boundary_sweep(o[1] if kind == 0 else o[3], chi, "svd", 2, 0, 1, upto=H - 1)
    T, B = tb[r], bb[H - 1 - r]
    L, R = O.row_envs(T, B, src, r)
    A1, A2 = src.A[r][c], src.A[r][c + 1]
    X1, a1 = U.split_left(A1)
    X2, a2 = U.split_right(A2)
    N = U.bond_norm(L[c], R[c + 1], T[c], X1, B[c], T[c + 1], X2, B[c + 1])
    return N, X1, X2, a1, a2


@pytest.mark.parametrize("kind,y,x", [(0, 1, 0), (0, 2, 1), (1, 0, 1), (1, 1, 2)])
def test_norm_matrix_is_the_norm_network_without_the_reduced_tensors(kind, y, x):
    Ad = _rand_lattice(3, 3, 2, 2, seed=41)
    N, X1, X2, _, _ = _exact_bond_norm(Ad, kind, y, x)
    # the isometries in the original orientation
    X1s, X2s = U.x_site_left(X1), U.x_site_right(X2)
    if kind == 1:
        X1s, X2s = X1s.transpose(0, 2, 1, 4, 3), X2s.transpose(0, 2, 1, 4, 3)
    p1, p2 = (y, x), ((y, x + 1) if kind == 0 else (y + 1, x))
    ref = _norm_matrix_bruteforce(Ad, p1, p2, X1s, X2s)
    scale = np.sum(N * ref) / np.sum(ref * ref)
    assert scale > 0
    assert np.max(np.abs(N - scale * ref)) < 1e-12 * np.max(np.abs(N))


def test_split_reproduces_the_site_tensors():
    A = np.random.default_rng(3).standard_normal((2, 3, 4, 2, 3))
    X, a = U.split_left(A)
    assert np.allclose(U.join_left(X, a), A, atol=1e-13)
    k = X.shape[-1]
    Xm = X.reshape(-1, k)
    assert np.allclose(Xm.T @ Xm, np.eye(k), atol=1e-13)
    X, a = U.split_right(A)
    assert np.allclose(U.join_right(X, a), A, atol=1e-13)


def _apply_two_site(psi, dims, i1, i2, G):
    d = dims[i1]
    P = np.moveaxis(psi.reshape(dims), (i1, i2), (0, 1))
    sh = P.shape
    P = (G @ P.reshape(d * d, -1)).reshape(sh)
    return np.moveaxis(P, (0, 1), (i1, i2)).ravel()


def _overlap_distance(a, b):
    a = a / np.linalg.norm(a)
    b = b / np.linalg.norm(b)
    return 1.0 - abs(float(a @ b))


@pytest.mark.parametrize("kind", [0, 1])
def test_a_product_gate_is_applied_exactly(kind):
    rng = np.random.default_rng(5)
    Ad = _rand_lattice(3, 3, 2, 2, seed=17)
    g1, g2 = rng.standard_normal((2, 2)), rng.standard_normal((2, 2))
    G = np.kron(g1, g2)
    y, x = (1, 0) if kind == 0 else (0, 1)
    new, cost = U.update_bonds(Ad, G, [(kind, y, x)], chi=64, mode="svd", iters=6)
    p1, p2 = (y, x), ((y, x + 1) if kind == 0 else (y + 1, x))
    dims = [2] * 9
    want = _apply_two_site(BF.state_vector(BF.dense_lattice(Ad)), dims, p1[0] * 3 + p1[1], p2[0] * 3 + p2[1], G)
    got = BF.state_vector(BF.dense_lattice(new))
    assert cost[0] < 1e-12
    assert _overlap_distance(got, want) < 1e-13


@pytest.mark.parametrize("kind", [0, 1])
def test_an_entangling_gate_on_a_product_bond_is_applied_exactly(kind):
    """The bond carried one Schmidt value, so the gate's result has bond
    rank <= d^2 = 4 = D and is held exactly."""
    Ad = _rand_lattice(3, 3, 2, 4, seed=23)
    y, x = (1, 1) if kind == 0 else (1, 1)
    if kind == 0:
        Ad[y, x, :, :, :, :, 1:] = 0.0
        Ad[y, x + 1, :, :, 1:, :, :] = 0.0
    else:
        Ad[y, x, :, :, :, 1:, :] = 0.0
        Ad[y + 1, x, :, 1:, :, :, :] = 0.0
    G = U.heisenberg_gate(0.7)
    G = G @ np.diag([1.0, 2.0, 0.5, 1.5])          # not symmetric in (s, t)
    new, cost = U.update_bonds(Ad, G, [(kind, y, x)], chi=256, mode="svd", iters=6)
    p1, p2 = (y, x), ((y, x + 1) if kind == 0 else (y + 1, x))
    want = _apply_two_site(BF.state_vector(BF.dense_lattice(Ad)), [2] * 9, p1[0] * 3 + p1[1],
                           p2[0] * 3 + p2[1], G)
    got = BF.state_vector(BF.dense_lattice(new))
    assert cost[0] < 1e-12
    assert _overlap_distance(got, want) < 1e-12


def test_identity_metric_gives_the_truncated_svd():
    """Eckart-Young: with N = 1 the best pair of rank Dn is the truncated SVD of
    Theta, and ALS reaches it."""
    rng = np.random.default_rng(9)
    k1, k2, d, D = 3, 4, 2, 2
    aL = rng.standard_normal((k1, d, 3))
    aR = rng.standard_normal((k2, d, 3))
    G = rng.standard_normal((d * d, d * d))
    N = np.einsum("ik,jl->ijkl", np.eye(k1), np.eye(k2))
    bL, bR, c = U.als(N, aL, aR, G, D, iters=60)
    Th = U.apply_gate(G, aL, aR).reshape(k1 * d, d * k2)
    s = np.linalg.svd(Th, compute_uv=False)
    assert abs(c - np.sum(s[D:] ** 2) / np.sum(s ** 2)) < 1e-10


def test_als_result_is_stationary():
    """Both gradients of d vanish at the ALS result for a general positive N."""
    Ad = _rand_lattice(3, 4, 2, 2, seed=29)
    N, X1, X2, a1, a2 = _exact_bond_norm(Ad, 0, 1, 1)
    N = U.positive_part(N)
    G = U.heisenberg_gate(0.3)
    bL, bR, c = U.als(N, a1, a2, G, 2, iters=200)
    Th = U.apply_gate(G, a1, a2)
    R = U.pair(bL, bR) - Th
    gL = np.einsum("ijkl,istj,ltq->ksq", N, R, bR)
    gR = np.einsum("ijkl,istj,ksq->ltq", N, R, bL)
    ref = np.einsum("ijkl,istj,ltq->ksq", N, Th, bR)
    assert np.max(np.abs(gL)) < 1e-7 * np.max(np.abs(ref))
    assert np.max(np.abs(gR)) < 1e-7 * np.max(np.abs(ref))
    # and the fit beats its start (the Euclidean truncated SVD)
    Dn = bL.shape[2]
    Us, S, V = U._svd_pair(Th, Dn)
    assert c <= U.cost(N, Th, Us * S[None, None, :], V) + 1e-14


def test_bonds_of_one_set_must_not_share_a_site():
    Ad = _rand_lattice(3, 3, 2, 2, seed=1)
    with pytest.raises(ValueError):
        U.update_bonds(Ad, np.eye(4), [(0, 0, 0), (0, 0, 1)], chi=8)


def _e_exact():
    for line in open(os.path.join(GOLDEN, "heisenberg_4x4_ed.txt")):
        if line.startswith("e0_per_site"):
            return float(line.split()[1])


def _e_fu_table(kind="D"):
    for line in open(os.path.join(GOLDEN, "fu_heisenberg_4x4_table.txt")):
        p = line.split()
        if p and p[0] == kind and p[1] == "2":
            return float(p[5]), float(p[7])


def test_full_update_reaches_the_paper_fu_energy_at_4x4_D2():
    """Imaginary time from the simple-update state with the parallel FU
    (D' = 4 as in Table EFU); energy per site at D' = 64 (exact here).
    The evolution converges to -0.544582 after 400 steps; 160 steps are
    within 3e-5 of it."""
    A = synth.peps_simple_update(4, 4, 2, seed=0)
    e_su = U.energy(A, chi=64) / 16
    A = U.evolve(A, tau=0.01, steps=160, chi=4, mode="svd", iters=6)
    e_fu = U.energy(A, chi=64) / 16
    e_tab, tol = _e_fu_table()
    assert _e_exact() < e_fu < e_su
    assert abs(e_fu - e_tab) < tol, (e_fu, e_tab, e_su)


@pytest.mark.parametrize("set_index", [0, 2])
def test_cluster_covering_the_lattice_is_the_full_update(set_index):
    A = synth.peps_simple_update(4, 4, 2, seed=0, steps=30)
    G = U.heisenberg_gate(0.05)
    s = U.trotter_sets(4, 4)[set_index]
    a, ca = U.update_bonds(A, G, s, chi=16, mode="var")
    b, cb = U.update_bonds_cluster(A, G, s, 3, chi=16, mode="var")
    assert np.array_equal(a, b) and ca == cb


@pytest.mark.parametrize("delta", [0, 1])
def test_exact_gate_is_exact_with_a_cluster_environment(delta):
    """Any positive N holds the gated pair exactly when the bond can."""
    Ad = _rand_lattice(3, 3, 2, 4, seed=23)
    y, x = 1, 1
    Ad[y, x, :, :, :, :, 1:] = 0.0
    Ad[y, x + 1, :, :, 1:, :, :] = 0.0
    G = U.heisenberg_gate(0.7) @ np.diag([1.0, 2.0, 0.5, 1.5])
    new, cost = U.update_bonds_cluster(Ad, G, [(0, y, x)], delta, chi=64, mode="svd", iters=6)
    want = _apply_two_site(BF.state_vector(BF.dense_lattice(Ad)), [2] * 9, 4, 5, G)
    got = BF.state_vector(BF.dense_lattice(new))
    assert cost[0] < 1e-12 and _overlap_distance(got, want) < 1e-12


def test_cu1_reaches_the_paper_energy_at_4x4_D2():
    """CU_1 with D' = 4 from the simple-update state (Table ECU1); 150 steps
    are within 3e-5 of the evolution's limit."""
    A = synth.peps_simple_update(4, 4, 2, seed=0)
    A = U.evolve(A, tau=0.01, steps=150, chi=4, mode="svd", iters=6, delta=1)
    e = U.energy(A, chi=64) / 16
    e_tab, tol = _e_fu_table("CU1")
    assert abs(e - e_tab) < tol, (e, e_tab)


def test_cu0_keeps_the_paper_energy_at_4x4_D2():
    """CU_0 (a generalised simple update) from the simple-update state stays at
    Table ECU0's energy."""
    A = synth.peps_simple_update(4, 4, 2, seed=0)
    A = U.evolve(A, tau=0.01, steps=30, chi=4, mode="svd", iters=6, delta=0)
    e = U.energy(A, chi=64) / 16
    e_tab, tol = _e_fu_table("CU0")
    assert abs(e - e_tab) < tol, (e, e_tab)
