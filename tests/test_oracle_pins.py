"""Pins for the FP64 oracle: checks against things other than itself.

* brute-force state vectors (the PEPS definition, Section 2) on 4x4 and 4x5;
* exactness: chi >= (D^2)^(Lx/2) reproduces the exact contraction;
* closed forms for D=1 product states;
* a cluster covering the lattice is the full method (Section 5: CU_{L-1});
* cluster windows with CU_0 closures vs brute force of the closed window;
* CU_0 positivity (Section 5.1) and its fixed point checked as a stationary
  point of the overlap, computed with dense vectors;
* the var local update vs a dense least-squares solve (Section 2, N A = b);
* gauge invariance, and top-down vs bottom-up norms;
* the paper's exact 4x4 Heisenberg energy (Appendix A) pins the S.S
  operator and the brute-force bond observables.
"""
import math
import os

import numpy as np
import pytest

from oracle import bruteforce as BF
from oracle import peps_oracle as O
from paper_1311_6696_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _bf_all(A):
    Ly, Lx = A.shape[:2]
    psi = BF.state_vector(BF.dense_lattice(A))
    dims = [A.shape[2]] * (Ly * Lx)
    site = lambda op: [BF.expect_site(psi, dims, i, op) for i in range(Ly * Lx)]
    hb = [BF.expect_bond(psi, dims, y * Lx + x, y * Lx + x + 1, O.SDOTS)
          for y in range(Ly) for x in range(Lx - 1)]
    vb = [BF.expect_bond(psi, dims, y * Lx + x, (y + 1) * Lx + x, O.SDOTS)
          for y in range(Ly - 1) for x in range(Lx)]
    return dict(lnN=math.log(BF.norm(psi)), sz=site(O.SZ), sx=site(O.SX), hb=hb, vb=vb)


def _maxdiff(a, b):
    return max(abs(x - y) for x, y in zip(a, b))


def _check_env_vs_bf(env, bf, tol):
    assert abs(env["ln_norm"] - bf["lnN"]) < tol
    assert env["sign"] == 1
    assert _maxdiff(O.expect_all(env, "site", O.SZ), bf["sz"]) < tol
    assert _maxdiff(O.expect_all(env, "site", O.SX), bf["sx"]) < tol
    assert _maxdiff(O.expect_all(env, "hbond", O.SDOTS), bf["hb"]) < tol
    assert _maxdiff(O.expect_all(env, "vbond", O.SDOTS), bf["vb"]) < tol


# ---------------------------------------------------------------- golden
def test_golden_heisenberg_4x4_energy_pins_sdots_and_bonds():
    sp = pytest.importorskip("scipy.sparse")
    sla = pytest.importorskip("scipy.sparse.linalg")
    vals = {}
    for line in open(os.path.join(GOLDEN, "heisenberg_4x4_ed.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    L = int(vals["L"])
    N = L * L
    # Hamiltonian from Pauli matrices directly (independent of O.SDOTS).
    sx = sp.csr_matrix([[0.0, 1.0], [1.0, 0.0]])
    sy_im = sp.csr_matrix([[0.0, -1.0], [1.0, 0.0]])      # sigma_y = i * sy_im
    sz = sp.csr_matrix([[1.0, 0.0], [0.0, -1.0]])

    def op(o, i):
        return sp.kron(sp.kron(sp.identity(2 ** i), o), sp.identity(2 ** (N - i - 1)), format="csr")

    bonds = [(y * L + x, y * L + x + 1) for y in range(L) for x in range(L - 1)] + \
            [(y * L + x, (y + 1) * L + x) for y in range(L - 1) for x in range(L)]
    H = sp.csr_matrix((2 ** N, 2 ** N))
    for i, j in bonds:
        # sigma_y x sigma_y = (i*sy_im) x (i*sy_im) = - sy_im x sy_im
        H = H + 0.25 * (op(sx, i) @ op(sx, j) - op(sy_im, i) @ op(sy_im, j) + op(sz, i) @ op(sz, j))
    w, v = sla.eigsh(H, k=1, which="SA")
    e0 = w[0] / N
    assert abs(e0 - vals["e0_per_site"]) < 0.6 * 10 ** (-vals["digits"])
    psi = v[:, 0]
    e_bf = sum(BF.expect_bond(psi, [2] * N, i, j, O.SDOTS) for i, j in bonds) / N
    assert abs(e_bf - e0) < 1e-10


# ---------------------------------------------------------------- brute force / exactness
@pytest.mark.parametrize("mode", ["svd", "var"])
def test_4x4_D2_exact_chi_matches_bruteforce(mode):
    A = synth.workload("4x4_D2")            # uniform[0,1) from seed 1, unit-norm tensors
    env = O.env_full(A, chi=16, mode=mode)  # (D^2)^(Lx/2) = 16: exact
    _check_env_vs_bf(env, _bf_all(A), 1e-12)


@pytest.mark.parametrize("mode", ["svd", "var"])
def test_4x5_D2_exact_chi_matches_bruteforce(mode):
    A = synth.peps_gauss(4, 5, 2, 2, seed=11)
    env = O.env_full(A, chi=16, mode=mode)  # (D^2)^floor(5/2) = 16
    _check_env_vs_bf(env, _bf_all(A), 1e-12)


def test_3x3_D3_exact_chi_matches_bruteforce():
    A = synth.peps_gauss(3, 3, 2, 3, seed=12)
    env = O.env_full(A, chi=9, mode="svd")  # (D^2)^1 = 9
    _check_env_vs_bf(env, _bf_all(A), 1e-12)


def test_truncation_error_decreases_with_chi():
    A = synth.peps_uniform(4, 5, 2, 2, seed=13)
    bf = _bf_all(A)
    errs = [_maxdiff(O.expect_all(O.env_full(A, chi=c, mode="svd"), "site", O.SZ), bf["sz"])
            for c in (2, 4, 8)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-5


# ---------------------------------------------------------------- D = 1 closed forms
@pytest.mark.parametrize("mode", ["svd", "var"])
def test_product_state_closed_forms(mode):
    A = synth.peps_product(3, 4, 2, seed=5)
    a = A[:, :, :, 0, 0, 0, 0]
    env = O.env_full(A, chi=4, mode=mode)
    lnN = float(np.sum(np.log(np.sum(a * a, axis=2))))
    assert abs(env["ln_norm"] - lnN) < 1e-12
    n2 = np.sum(a * a, axis=2)
    z = (a[..., 0] ** 2 - a[..., 1] ** 2) / n2
    x = 2 * a[..., 0] * a[..., 1] / n2
    assert _maxdiff(O.expect_all(env, "site", O.SZ), z.ravel()) < 1e-13
    assert _maxdiff(O.expect_all(env, "site", O.SX), x.ravel()) < 1e-13
    hb = [(x[i, j] * x[i, j + 1] + z[i, j] * z[i, j + 1]) / 4 for i in range(3) for j in range(3)]
    vb = [(x[i, j] * x[i + 1, j] + z[i, j] * z[i + 1, j]) / 4 for i in range(2) for j in range(4)]
    assert _maxdiff(O.expect_all(env, "hbond", O.SDOTS), hb) < 1e-13
    assert _maxdiff(O.expect_all(env, "vbond", O.SDOTS), vb) < 1e-13
    # CU_0 is exact for product states: every cluster size gives the same values.
    for n in (1, 2):
        ec = O.env_cluster(A, n=n, chi=4, mode=mode)
        assert _maxdiff(O.expect_all(ec, "site", O.SZ), z.ravel()) < 1e-13
    assert _maxdiff(O.expect_all(ec, "hbond", O.SDOTS), hb) < 1e-13
    assert _maxdiff(O.expect_all(ec, "vbond", O.SDOTS), vb) < 1e-13


# ---------------------------------------------------------------- clusters
@pytest.mark.parametrize("mode", ["svd", "var"])
def test_cluster_covering_lattice_is_full(mode):
    A = synth.peps_gauss(4, 4, 2, 2, seed=7)
    ef = O.env_full(A, chi=6, mode=mode)     # truncated on purpose
    ec = O.env_cluster(A, n=8, chi=6, mode=mode)
    for k in ("rho_site", "rho_h", "rho_v"):
        for ra, rb in zip(ef[k], ec[k]):
            for a, b in zip(ra, rb):
                assert np.array_equal(a, b)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_cluster_window_matches_bruteforce_of_closed_window(n):
    A = synth.peps_gauss(4, 5, 2, 2, seed=8)
    lat = O.lattice_from_dense(A)
    cu0 = O.cu0_all(lat)
    for (y, x) in [(0, 0), (1, 1), (2, 3), (3, 4), (1, 4), (3, 0)]:
        W, (r0, r1, c0, c1) = O.window_lattice(lat, cu0, y, x, n)
        s, h, v = O.cluster_anchor(W, y - r0, x - c0, 64, "svd", 2, 0)
        rows, extra = BF.absorb_closures(W.A, W.top, W.bottom, W.left, W.right)
        psi = BF.state_vector(rows)
        dims = [2 * extra[i][j] for i in range(W.Ly) for j in range(W.Lx)]
        i = (y - r0) * W.Lx + (x - c0)
        assert abs(O.expect(s, O.SZ) - BF.expect_site(psi, dims, i, O.SZ)) < 1e-12
        assert abs(O.expect(s, O.SX) - BF.expect_site(psi, dims, i, O.SX)) < 1e-12
        if h is not None:
            assert abs(O.expect(h, O.SDOTS) - BF.expect_bond(psi, dims, i, i + 1, O.SDOTS)) < 1e-12
        if v is not None:
            assert abs(O.expect(v, O.SDOTS) - BF.expect_bond(psi, dims, i, i + W.Lx, O.SDOTS)) < 1e-12


def test_window_shape_clipped_not_shifted():
    assert O.window_bounds(14, 0, 6) == (0, 3)
    assert O.window_bounds(14, 7, 6) == (5, 10)
    assert O.window_bounds(14, 13, 6) == (11, 13)
    assert O.window_bounds(14, 5, 2) == (5, 6)
    assert O.window_bounds(14, 13, 2) == (13, 13)
    assert O.window_bounds(14, 3, 28) == (0, 13)


# ---------------------------------------------------------------- CU_0
def test_cu0_positive_symmetric_and_init_independent():
    A = synth.peps_gauss(5, 4, 2, 3, seed=9)
    lat = O.lattice_from_dense(A)
    s1 = O.cu0_sweep(lat)
    s2 = O.cu0_sweep(lat, init="random", init_seed=4)
    for r1, r2 in zip(s1[1:], s2[1:]):
        for a, b in zip(r1, r2):
            assert np.max(np.abs(a - b)) < 1e-10
            assert np.max(np.abs(a - a.T)) < 1e-14
            assert np.linalg.eigvalsh(a).min() > -1e-14


def test_cu0_fixed_point_is_stationary_overlap():
    """The D'=1 fixed point maximises the overlap locally: each sigma_x is
    parallel to the derivative of <Sigma|T> w.r.t. sigma_x, where T is the
    row applied to the previous separable boundary, built as a dense vector."""
    A = synth.peps_gauss(3, 3, 2, 2, seed=10)
    lat = O.lattice_from_dense(A)
    sig = O.cu0_sweep(lat)
    for r in range(2):
        prev, new = sig[r], sig[r + 1]
        # dense target T over (n_0, o_0, n_1, o_1, n_2, o_2)
        t = None
        for x in range(3):
            a = lat.A[r][x]
            site = np.einsum("uv,sulnr,svmoq->lmnorq", prev[x], a, a)
            if t is None:
                t = site[0, 0]                          # left legs of dim 1
            else:
                t = np.einsum("...rq,rqnoRQ->...noRQ", t, site)
        t = t[..., 0, 0]
        for x in range(3):
            # contract every other site's sigma into the dense target
            idx = "abcdef"
            specs, ops = [], []
            for k in range(3):
                if k != x:
                    specs.append(idx[2 * k] + idx[2 * k + 1])
                    ops.append(new[k])
            out = idx[2 * x] + idx[2 * x + 1]
            g = np.einsum(idx + "," + ",".join(specs) + "->" + out, t, *ops)
            g = g / np.linalg.norm(g)
            assert np.max(np.abs(g - new[x])) < 1e-9


def test_cu0_exact_for_product_state():
    A = synth.peps_product(3, 3, 2, seed=2)
    lat = O.lattice_from_dense(A)
    sig = O.cu0_sweep(lat)
    for r in range(1, 3):
        for m in sig[r]:
            assert m.shape == (1, 1) and abs(m[0, 0] - 1.0) < 1e-15


# ---------------------------------------------------------------- var local update
def test_var_local_update_is_dense_least_squares():
    """b_0 from the chain equals the least-squares optimum of ||T' - O T||^2
    over the first tensor of T' with the others right-orthonormal (Section 2)."""
    A = synth.peps_gauss(3, 3, 2, 2, seed=14)
    lat = O.lattice_from_dense(A)
    T, _ = O.boundary_sweep(lat, chi=4, mode="svd", upto=1)
    T1 = T[1]
    y = 1
    Lx = 3
    A1 = lat.A[y]
    phys = [A1[x].shape[3] ** 2 for x in range(Lx)]
    prod = [T1[k].shape[3] * A1[k].shape[4] ** 2 for k in range(Lx - 1)]
    caps = O.bond_caps(phys, prod, 3)
    N = O.right_canonicalize(O.var_init(T1, caps, [A1[x].shape[3] for x in range(Lx)], 0, 0, y))
    R = [None] * Lx
    R[Lx - 1] = O.closure_right(lat.right[y])
    for x in range(Lx - 1, 0, -1):
        R[x - 1] = O.renv_prev(O.chain_right(R[x], T1[x], A1[x]), N[x])
    b0 = O.close_left(O.chain_left(O.closure_left(lat.left[y]), T1[0], A1[0]), R[0])
    # dense target O T
    P = O.product_mps(T1, lat, y)
    target = P[0]
    for k in range(1, Lx):
        target = np.tensordot(target, P[k], axes=([target.ndim - 1], [0]))
    target = target.reshape(-1)
    # dense T' as a linear map of N[0]
    rest = N[1]
    for k in range(2, Lx):
        rest = np.tensordot(rest, N[k], axes=([rest.ndim - 1], [0]))
    rest = rest.reshape(rest.shape[0], -1)                  # [e, rest]
    c, n, o, e = N[0].shape
    cols = []
    for idx in range(c * n * o * e):
        unit = np.zeros(c * n * o * e)
        unit[idx] = 1.0
        U = unit.reshape(c, n, o, e)
        v = np.tensordot(U, rest, axes=([3], [0])).reshape(-1)
        cols.append(v)
    Jd = np.stack(cols, axis=1)
    sol, *_ = np.linalg.lstsq(Jd, target, rcond=None)
    assert np.max(np.abs(sol.reshape(b0.shape) - b0)) < 1e-12 * max(1.0, np.max(np.abs(b0)))


def test_var_fit_start_from_canonical_boundary_needs_no_gauge_pass():
    """A var fit that ends on a right-to-left half-sweep leaves sites 1..L-1
    right-orthonormal (Section 2, orthonormal gauge).  When the next row's
    bond caps equal its bonds, the next fit starts from a plain copy of it,
    and the start's right-canonicalisation changes only the signs of the bond
    bases: every entry keeps its magnitude and the state is the same."""
    A = synth.peps_gauss(5, 5, 2, 2, seed=41)
    lat = O.lattice_from_dense(A)
    bounds, _ = O.boundary_sweep(lat, chi=8, mode="var", upto=3)
    T = bounds[3]
    Lx = 5
    for x in range(1, Lx):
        M = T[x].reshape(T[x].shape[0], -1)
        assert np.max(np.abs(M @ M.T - np.eye(M.shape[0]))) < 1e-12
    y = 3
    A3 = lat.A[y]
    phys = [A3[x].shape[3] ** 2 for x in range(Lx)]
    prod = [T[k].shape[3] * A3[k].shape[4] ** 2 for k in range(Lx - 1)]
    caps = O.bond_caps(phys, prod, 8)
    assert caps == [T[k].shape[3] for k in range(Lx - 1)] and max(caps) == 8
    N0 = O.var_init(T, caps, [A3[x].shape[3] for x in range(Lx)], 0, 0, y)
    assert all(np.array_equal(N0[x], T[x]) for x in range(Lx))
    N1 = O.right_canonicalize(N0)

    def dense(N):
        v = N[0]
        for k in range(1, Lx):
            v = np.tensordot(v, N[k], axes=([v.ndim - 1], [0]))
        return v.reshape(-1)

    for x in range(Lx):
        assert np.max(np.abs(np.abs(N1[x]) - np.abs(N0[x]))) < 1e-12
    v0, v1 = dense(N0), dense(N1)
    assert np.max(np.abs(v1 - v0)) < 1e-12 * np.max(np.abs(v0))


# ---------------------------------------------------------------- consistency
def test_top_down_and_bottom_up_norms_agree_at_exact_chi():
    A = synth.peps_gauss(4, 4, 2, 2, seed=15)
    lat = O.lattice_from_dense(A)
    l1, s1 = O.norm(lat, chi=16)
    l2, s2 = O.norm(O.flip_ud(lat), chi=16)
    l3, s3 = O.norm(O.transpose(lat), chi=16)
    assert abs(l1 - l2) < 1e-12 and abs(l1 - l3) < 1e-12 and s1 == s2 == s3 == 1


def _gauged(A, G, horizontal=True, vertical=True):
    Gi = np.linalg.inv(G)
    B = A.copy()
    if horizontal:   # bond (1,1)-(1,2): G on the right leg, G^-1 on the left leg
        B[1, 1] = np.einsum("sulnr,rk->sulnk", B[1, 1], G)
        B[1, 2] = np.einsum("kl,sulnr->suknr", Gi, B[1, 2])
    if vertical:     # bond (0,2)-(1,2): G on the down leg, G^-1 on the up leg
        B[0, 2] = np.einsum("sulnr,nk->sulkr", B[0, 2], G)
        B[1, 2] = np.einsum("ku,sulnr->sklnr", Gi, B[1, 2])
    return B


def test_gauge_invariance_exact_chi():
    A = synth.peps_gauss(4, 4, 2, 2, seed=16)
    B = _gauged(A, synth.random_gauge(2, seed=17))
    e1 = O.env_full(A, chi=16, mode="svd")
    e2 = O.env_full(B, chi=16, mode="svd")
    assert abs(e1["ln_norm"] - e2["ln_norm"]) < 1e-12
    for kind, op in (("site", O.SZ), ("hbond", O.SDOTS), ("vbond", O.SDOTS)):
        assert _maxdiff(O.expect_all(e1, kind, op), O.expect_all(e2, kind, op)) < 1e-12


def test_horizontal_gauge_leaves_truncated_top_down_norm_unchanged():
    """A gauge on a bond inside a row only changes the gauge of the product
    MPS bond, which the canonical form removes before truncation."""
    A = synth.peps_gauss(4, 4, 2, 3, seed=16)
    B = _gauged(A, synth.random_gauge(3, seed=17), vertical=False)
    l1, _ = O.norm(A, chi=6, mode="svd")
    l2, _ = O.norm(B, chi=6, mode="svd")
    assert abs(l1 - l2) < 1e-12


# ---------------------------------------------------------------- planted mistakes
def test_planted_mistake_in_chain_is_caught(monkeypatch):
    """A transposed operand in the ket stage must fail the brute-force pin."""
    A = synth.peps_gauss(3, 3, 2, 2, seed=18)
    bf = _bf_all(A)
    good = O.chain_left

    def bad(L, M, Aa):
        X1 = O._ein("clma,auvb->clmuvb", L, M)
        X2 = O._ein("clmuvb,slunr->cmvbsnr", X1, Aa)    # u and l swapped
        return O._ein("cmvbsnr,svmoq->cbnroq", X2, Aa)

    monkeypatch.setattr(O, "chain_left", bad)
    env = O.env_full(A, chi=9, mode="svd")
    monkeypatch.setattr(O, "chain_left", good)
    assert _maxdiff(O.expect_all(env, "site", O.SZ), bf["sz"]) > 1e-6


def test_planted_mistake_in_noise_free_cu0_is_caught(monkeypatch):
    """A dropped right environment in the CU_0 update breaks stationarity."""
    A = synth.peps_gauss(3, 3, 2, 2, seed=10)
    lat = O.lattice_from_dense(A)
    good = O.cu0_local
    monkeypatch.setattr(O, "cu0_local", lambda Lm, S, Aa, Rm: good(Lm, S, Aa, np.eye(Rm.shape[0])))
    bad = O.cu0_sweep(lat)
    monkeypatch.setattr(O, "cu0_local", good)
    ok = O.cu0_sweep(lat)
    assert max(np.max(np.abs(a - b)) for ra, rb in zip(ok[1:], bad[1:]) for a, b in zip(ra, rb)) > 1e-6


def test_cluster_error_shrinks_with_window_size():
    """Section 5.2: the cluster scheme interpolates between CU_0 and the full
    update -- on a simple-update state the deviation of every bond's <S.S>
    from the full environments falls as the window grows and vanishes once
    the window covers the lattice (same chi, svd mode)."""
    from paper_1311_6696_gb300 import synth
    A = synth.peps_simple_update(6, 6, 2, seed=31, steps=150)
    full = O.env_full(A, chi=16, mode="svd")

    def bonds(e):
        return np.concatenate([np.ravel(O.expect_all(e, "hbond", O.SDOTS)),
                               np.ravel(O.expect_all(e, "vbond", O.SDOTS))])

    ref = bonds(full)
    errs = [float(np.mean(np.abs(bonds(O.env_cluster(A, n=n, chi=16, mode="svd")) - ref))) for n in (2, 3, 4, 6)]
    assert all(a > 2 * b for a, b in zip(errs, errs[1:])), errs
    assert float(np.max(np.abs(bonds(O.env_cluster(A, n=12, chi=16, mode="svd")) - ref))) == 0.0


def _dense_top_boundary(Ad, rows):
    """The exact boundary below the first `rows` rows as a dense vector over
    the sites' (ket down leg, bra down leg) pairs, site 0 most significant:
    the ket of those rows with open physical and down legs (brute force, no
    MPS), contracted with its own copy over every physical index."""
    from oracle import bruteforce as BF
    Lx, D = Ad.shape[1], Ad.shape[3]
    lat = BF.dense_lattice(Ad[:rows].copy())
    # the last kept row's down legs are interior: give them their real dimension
    last = [np.array(Ad[rows - 1, x, :, :(1 if rows == 1 else D), :(1 if x == 0 else D), :D,
                        :(1 if x == Lx - 1 else D)]) for x in range(Lx)]
    lat[rows - 1] = last
    psi = np.ones((1, 1))                                   # [S so far, open down legs]
    for row in lat:
        R = BF._row_tensor(row)                             # [S, U, N]
        psi = np.einsum("pu,sun->psn", psi, R).reshape(-1, R.shape[2])
    B = psi.T @ psi                                         # [N ket, N bra]
    B = B.reshape([D] * Lx + [D] * Lx)
    order = [i for x in range(Lx) for i in (x, Lx + x)]     # (n_x, o_x) per site
    return B.transpose(order).reshape(-1)


def _mps_to_dense(P):
    v = P[0]
    for M in P[1:]:
        v = np.tensordot(v, M, axes=([v.ndim - 1], [0]))
    return v.reshape(-1)


def test_svd_truncation_is_sequential_eckart_young_on_the_dense_boundary():
    """svd mode at truncated chi (Section 2: the new boundary is the best MPS
    of bond chi, here by the SVD sweep): after the two top rows of a 3x5 D=2
    lattice the product boundary has bond 16 and chi=8 truncates cuts 1 and
    2.  A right-to-left SVD sweep over a left-canonical MPS is, cut by cut,
    the best rank-k approximation (Eckart-Young) of the current state across
    that cut; the same truncations done on the dense 4^5 vector with nothing
    but a matrix SVD must give the oracle's boundary."""
    from oracle import peps_oracle as O
    from paper_1311_6696_gb300 import synth
    Ad = synth.peps_gauss(3, 5, 2, 2, seed=31, mean=0.0, std=1.0)   # far from a product state
    chi = 8
    bounds, _ = O.boundary_sweep(O.lattice_from_dense(Ad), chi, "svd", upto=2)
    got = _mps_to_dense(bounds[2])
    assert [M.shape[3] for M in bounds[2][:-1]] == [4, 8, 8, 4]
    psi = _dense_top_boundary(Ad, 2)
    Lx, p = 5, 4
    caps = [4, 8, 8, 4]
    for k in range(Lx - 2, -1, -1):                          # cut k: sites 0..k | k+1..
        M = psi.reshape(p ** (k + 1), -1)
        U, S, Vt = np.linalg.svd(M, full_matrices=False)
        r = caps[k]
        psi = ((U[:, :r] * S[:r]) @ Vt[:r]).reshape(-1)
    # something was truncated (the test is not the exact case)
    assert np.linalg.norm(psi - _dense_top_boundary(Ad, 2)) > 1e-3 * np.linalg.norm(psi)
    want = psi / np.linalg.norm(psi)
    got = got / np.linalg.norm(got)
    assert np.max(np.abs(got - want)) < 1e-10


def _dense_row_transfer(row):
    """The double-layer transfer matrix of one row (ket and bra, physical
    index traced, left/right legs of dimension 1 at the row's ends), as a
    dense matrix from the up-leg pairs (u_x, v_x) to the down-leg pairs
    (n_x, o_x), sites in order, site 0 most significant."""
    W = None
    for A in row:
        w = np.einsum("sulnr,svmoq->uvnolmrq", A, A)      # one site, (u,v) -> (n,o), (l,m) | (r,q)
        du, dn, dl, dr = A.shape[1], A.shape[3], A.shape[2], A.shape[4]
        w = w.reshape(du * du, dn * dn, dl * dl, dr * dr)
        if W is None:
            assert dl == 1
            W = w[:, :, 0, :]                                 # [U, N, right]
        else:
            W = np.einsum("UNk,unkr->UuNnr", W, w)
            W = W.reshape(W.shape[0] * W.shape[1], W.shape[2] * W.shape[3], W.shape[4])
    assert W.shape[2] == 1
    return W[:, :, 0]


def test_boundary_fidelity_matches_dense_transfer_matrices():
    """Fig. Fid's distance 1 - f, pinned by dense linear algebra on a 4x4 D=2
    lattice: the exact environment of the left-most column is the product of
    the dense row transfer matrices of the right-to-left sweep applied to the
    trivial boundary; the cluster form applies only delta of them to the CU_0
    product vector.  At exact chi the oracle's MPS form must agree."""
    from oracle import peps_oracle as O
    from paper_1311_6696_gb300 import synth
    Ad = synth.peps_gauss(4, 4, 2, 2, seed=71, mean=0.2, std=1.0)
    lat = O.lattice_from_dense(Ad)
    o = O.orientations(lat)[3]
    L = o.Ly
    T = [_dense_row_transfer(o.A[r]) for r in range(L)]
    ones = np.ones(1)
    ref = ones
    for r in range(L - 1):
        ref = ref @ T[r]
    cu0 = O.cu0_sweep(o)
    for delta in (1, 2):
        r0 = L - 1 - delta
        v = np.ones(1)
        for m in cu0[r0]:
            v = np.kron(v, m.ravel())
        for r in range(r0, L - 1):
            v = v @ T[r]
        f = abs(ref @ v) / (np.linalg.norm(ref) * np.linalg.norm(v))
        got = O.boundary_fidelity(Ad, delta, chi=64, chi_ref=64, mode="svd")
        assert abs(got - (1.0 - f)) < 1e-12, (delta, got, 1.0 - f)
        assert got > 1e-6                       # the cluster form is not the full one here
    assert O.boundary_fidelity(Ad, L - 1, chi=64, chi_ref=64, mode="svd") < 1e-13


def test_boundary_fidelity_falls_with_the_cluster_size():
    """Section 5.2 / Fig. Fid: at a large boundary bond the distance drops
    with every added column and vanishes when the cluster holds them all."""
    from oracle import peps_oracle as O
    from paper_1311_6696_gb300 import synth
    A = synth.peps_simple_update(6, 6, 2, seed=3, steps=100)
    d = [O.boundary_fidelity(A, delta, chi=16, chi_ref=32) for delta in (1, 2, 3, 4)]
    assert all(d[i + 1] < 0.5 * d[i] for i in range(3)), d
    assert O.boundary_fidelity(A, 5, chi=32, chi_ref=32) < 1e-14


def _finite_copies(A, L):
    """An L x L OBC lattice with A on every site, its outward legs cut to index 0."""
    Ad = np.zeros((L, L) + A.shape)
    for y in range(L):
        for x in range(L):
            sl = (slice(None), slice(0, 1) if y == 0 else slice(None), slice(0, 1) if x == 0 else slice(None),
                  slice(0, 1) if y == L - 1 else slice(None), slice(0, 1) if x == L - 1 else slice(None))
            Ad[(y, x) + sl] = A[sl]
    return Ad


def test_infinite_cu0_is_the_finite_cu0_deep_inside_a_large_lattice():
    """Section 5.4: the dominant D'=1 boundary of the infinite lattice is what
    the finite CU_0 (Section 5.1, pinned above) converges to far from every
    edge of a lattice of copies; checked in all four directions."""
    from oracle import peps_oracle as O
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(3, 3, 2, 3, seed=5)[1, 1]
    L = 16
    lat = O.lattice_from_dense(_finite_copies(A, L))
    for o, (lo, Ao) in enumerate(zip(O.orientations(lat), O.ipeps_orientations(A))):
        sig = O.cu0_infinite(Ao)
        fin = O.cu0_sweep(lo)
        assert np.max(np.abs(fin[L // 2][L // 2] - sig)) < 1e-12, o


def test_ipeps_cluster_of_a_product_state_is_the_closed_form():
    from oracle import peps_oracle as O
    rng = np.random.default_rng(3)
    a = rng.uniform(-1, 1, 2)
    A = a.reshape(2, 1, 1, 1, 1)
    r = O.ipeps_cluster(A, 3, 1)
    z = (a[0] ** 2 - a[1] ** 2) / (a @ a)
    x = 2 * a[0] * a[1] / (a @ a)
    assert abs(O.expect(r["rho_site"], O.SZ) - z) < 1e-14
    assert abs(O.expect(r["rho_site"], O.SX) - x) < 1e-14
    for k in ("rho_h", "rho_v"):
        assert abs(O.expect(r[k], O.SDOTS) - (x * x + z * z) / 4) < 1e-14


def test_ipeps_cluster_matches_the_finite_cluster_deep_inside():
    """The iPEPS cluster density matrices equal the finite cluster scheme's at
    the centre of a large lattice of copies (same window, same closures there)."""
    from oracle import peps_oracle as O
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(3, 3, 2, 2, seed=8)[1, 1]
    L = 20          # far enough from the edges (the distance decays exponentially: 1e-10 at 14, 1e-13 at 18)
    fin = O.env_cluster(_finite_copies(A, L), n=3, chi=8, mode="var", anchors=[(L // 2, L // 2)])
    inf = O.ipeps_cluster(A, 3, 8)
    c = L // 2
    for got, want in ((inf["rho_site"], fin["rho_site"][c][c]), (inf["rho_h"], fin["rho_h"][c][c]),
                      (inf["rho_v"], fin["rho_v"][c][c])):
        g = got.reshape(got.shape[0] if got.ndim == 2 else 4, -1)
        w = want.reshape(g.shape)
        assert np.max(np.abs(g / np.trace(g) - w / np.trace(w))) < 1e-11


# ------------------------------------------------------------------ var mode at truncated chi
def _var_fit_trace(seed, Ly, Lx, D, chi, halves):
    """Distance |P - F|^2 / |P|^2 of the var fit F (after h half-sweeps) from
    the exact product MPS P of the second absorb, and the projection defect
    (<P|F> - <F|F>) / |P|^2, for h = 1 .. halves."""
    A = synth.peps_gauss(Ly, Lx, 2, D, seed, mean=0.0, std=1.0)
    lat = O.lattice_from_dense(A)
    T, _ = O.absorb_compress(O.closure_mps(lat.top), lat, 0, 64, "svd", 2, 0, 0)
    y = 1
    P = O.product_mps(T, lat, y)
    Ax = lat.A[y]
    phys = [Ax[x].shape[3] ** 2 for x in range(Lx)]
    prod = [T[k].shape[3] * Ax[k].shape[4] ** 2 for k in range(Lx - 1)]
    caps = O.bond_caps(phys, prod, chi)
    assert any(prod[k] > caps[k] for k in range(Lx - 1))          # it truncates
    pp = O.mps_overlap(P, P)
    out = []
    for h in range(1, halves + 1):
        F, _ = O.var_compress(T, lat, y, caps, h, 0, 0)
        pf, ff = O.mps_overlap(P, F), O.mps_overlap(F, F)
        out.append(((pp + ff - 2 * pf) / pp, (pf - ff) / pp))
    return out


@pytest.mark.parametrize("seed,Ly,Lx,D,chi", [(5, 4, 5, 2, 3), (7, 4, 6, 2, 4), (9, 3, 5, 3, 5)])
def test_var_fit_at_truncated_chi_is_monotone_and_a_projection(seed, Ly, Lx, D, chi):
    """Section 2's one-site ALS with N_l = 1: every local step replaces the
    centre tensor by the projection b_l, so |P - F| never grows from one
    half-sweep to the next, and after each half-sweep <P|F> = <F|F>."""
    tr = _var_fit_trace(seed, Ly, Lx, D, chi, 6)
    for (d0, _), (d1, _) in zip(tr, tr[1:]):
        assert d1 <= d0 + 1e-12
    assert tr[-1][0] < tr[0][0]                                     # it does improve
    for _, defect in tr:
        assert abs(defect) < 1e-12


def test_var_fit_pins_catch_a_swapped_environment(monkeypatch):
    """The same pins fail when the local vector uses the right environment
    with its ket and bra legs swapped (a plausible index slip)."""
    real = O.close_left
    monkeypatch.setattr(O, "close_left", lambda X3, R: real(X3, R.transpose(0, 2, 1, 3)))
    tr = _var_fit_trace(5, 4, 5, 2, 3, 4)
    broken = any(d1 > d0 + 1e-12 for (d0, _), (d1, _) in zip(tr, tr[1:])) or \
        any(abs(g) > 1e-12 for _, g in tr)
    assert broken
