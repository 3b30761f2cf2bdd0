"""FP64 CPU oracle for the tensor update of the full / cluster update.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  It shares no
code with the CUDA path and the CUDA path never calls it.

What it computes (Lubasch, Cirac, Banuls, "Unifying PEPS contractions"):

* Section 2: imaginary-time evolution applies Trotter gates one bond at a
  time; after a gate O acts on the PEPS |phi>, the new PEPS |psi> minimises
  d = || |psi> - O|phi> ||^2 by alternating least squares, one tensor at a
  time, the optimal tensor solving N_l A_l = b_l.  N_l is <psi|psi> with A_l
  and A_l* left out, b_l is <psi|O|phi> with A_l* left out.
* Section 2 (footnote on the cost of the tensor update): the variational
  parameters are restricted to the reduced tensors, which makes the linear
  systems O(D^6).  Each site tensor of the bond is split by a QR into an
  isometry X carrying the legs the gate does not touch and a reduced tensor
  a carrying the physical leg and the shared bond: A_l = X_l a_l.
* The environment of the pair is the norm network with the two reduced
  tensors removed; its value on the reduced legs is the norm matrix
  N[k1, k2, k1', k2'] (ket legs k1 k2, bra legs k1' k2').  It is the
  two-site density-matrix network of Section 5.3 with X_l in place of the
  site tensors and the reduced leg k in place of the physical leg.
* Sections 4.4 and 5.2 (parallel CU): the bonds of one Trotter set are
  updated independently, every one from the environment of the same state.
* Section 5 (cluster update CU_delta): the environment of a row's (column's)
  bonds is the exact contraction of the rows (columns) within distance delta,
  closed beyond them by the separable CU_0 boundaries of Section 5.1.

Readings where the paper is silent (the CUDA path follows the same rules,
written out here and in its own code, never shared):

* QR split: left site A[s,u,l,n,r] as the matrix (u l n) x (s r); right
  site A[t,u,l,n,r] as (u n r) x (t l); thin Householder QR (LAPACK's
  reflector signs); k = min(rows, cols).
* N is symmetrised over (ket, bra) and replaced by its positive part (the
  eigenvalues below zero, a product of the environment's approximation, are
  set to zero).
* Theta = O applied to the reduced pair: Theta[k1,s,t,k2] =
  sum G[s,t,s',t'] a_l[k1,s',r] a_r[k2,t',r], gate G[(s t),(s' t')].
* ALS start: the truncated SVD of Theta as (k1 s) x (t k2) keeping
  Dn = min(D, k1 d, k2 d) triplets, a_l = U S, a_r = V.
* ALS: ``iters`` rounds, each solving for a_l (a_r fixed) then for a_r (a_l
  fixed).  The normal equations are block diagonal in the free physical
  index; each block is solved by Cholesky with the shift
  1e-12 * trace / size added to the diagonal.
* Result: the product psi = a_l a_r is split again by an SVD into
  a_l = U sqrt(S), a_r = V sqrt(S) (Dn triplets; each U column's largest
  entry made positive, V's column flipped with it), then A_l = X_l a_l,
  A_r = X_r a_r, each scaled to unit Frobenius norm; bond slots beyond Dn
  are zero.
* Reported cost: d / <Theta|N|Theta> with the (positive) N.
* Vertical bonds use the transposed lattice (rows of the transpose are the
  columns), as the density matrices of vertical bonds do.
* CU_delta: the cluster of a row is rows r - delta .. r + delta clipped at
  the lattice edge, all columns, closed by the CU_0 matrices of the cuts
  above and below it (at the lattice edge these are the lattice's own
  closures) and on the sides by the lattice's closures; var noise keyed by
  the strip's own rows.

Index conventions as in ``peps_oracle``: A[s, u, l, n, r].
"""
from __future__ import annotations

import numpy as np

from . import peps_oracle as O


# ---------------------------------------------------------------------------
# Reduced tensors (Section 2, footnote: restrict the update to them)
# ---------------------------------------------------------------------------
def split_left(A):
    """A[s,u,l,n,r] -> (X[u,l,n,k], a[k,s,r]) with A = X a (sum over k)."""
    s, u, l, n, r = A.shape
    M = A.transpose(1, 2, 3, 0, 4).reshape(u * l * n, s * r)
    Q, R = np.linalg.qr(M)
    k = Q.shape[1]
    return Q.reshape(u, l, n, k), R.reshape(k, s, r)


def split_right(A):
    """A[t,u,l,n,r] -> (X[u,n,r,k], a[k,t,l]) with A = X a (sum over k)."""
    t, u, l, n, r = A.shape
    M = A.transpose(1, 3, 4, 0, 2).reshape(u * n * r, t * l)
    Q, R = np.linalg.qr(M)
    k = Q.shape[1]
    return Q.reshape(u, n, r, k), R.reshape(k, t, l)


def join_left(X, a):
    """A[s,u,l,n,r] = sum_k X[u,l,n,k] a[k,s,r]."""
    return np.einsum("ulnk,ksr->sulnr", X, a)


def join_right(X, a):
    """A[t,u,l,n,r] = sum_k X[u,n,r,k] a[k,t,l]."""
    return np.einsum("unrk,ktl->tulnr", X, a)


def x_site_left(X):
    """X[u,l,n,k] as a site tensor with physical leg k and a right leg of dim 1."""
    return X.transpose(3, 0, 1, 2)[..., None]


def x_site_right(X):
    """X[u,n,r,k] as a site tensor with physical leg k and a left leg of dim 1."""
    return X.transpose(3, 0, 1, 2)[:, :, None, :, :]


# ---------------------------------------------------------------------------
# The norm matrix of a bond (Section 2: environment of the pair)
# ---------------------------------------------------------------------------
def bond_norm(Lv, Rv, M1, X1, B1, M2, X2, B2):
    """N[k1,k2,k1',k2'] of the horizontal pair whose left / right sites are
    replaced by the isometries X1[u,l,n,k] and X2[u,n,r,k]; Lv / Rv the row
    environments left of the pair and right of it, M / B the boundary MPS
    sites above / below the two columns."""
    return O.rho_hbond(Lv, Rv, M1, x_site_left(X1), B1, M2, x_site_right(X2), B2)


def quad(N, X, Y):
    """<X|N|Y> = sum N[i,j,k,l] X[i,s,t,j] Y[k,s,t,l]: ket X, bra Y."""
    return float(np.einsum("ijkl,istj,kstl->", N, X, Y, optimize=True))


def positive_part(N):
    """Symmetrise N over (ket, bra) and keep its non-negative spectrum."""
    k1, k2 = N.shape[0], N.shape[1]
    m = N.reshape(k1 * k2, k1 * k2)
    m = 0.5 * (m + m.T)
    w, V = np.linalg.eigh(m)
    return ((V * np.where(w > 0.0, w, 0.0)) @ V.T).reshape(k1, k2, k1, k2)


# ---------------------------------------------------------------------------
# ALS on the reduced pair (Section 2: N_l A_l = b_l, one tensor at a time)
# ---------------------------------------------------------------------------
def apply_gate(G, aL, aR):
    """Theta[k1,s,t,k2] = sum G[s,t,s',t'] aL[k1,s',r] aR[k2,t',r]."""
    d = aL.shape[1]
    G4 = G.reshape(d, d, d, d)
    return np.einsum("stuv,aur,bvr->astb", G4, aL, aR, optimize=True)


def _svd_pair(P, Dn):
    """Truncated SVD of P[k1,s,t,k2] as (k1 s) x (t k2): U (k1,s,Dn), S, V (k2,t,Dn)."""
    k1, d, _, k2 = P.shape
    U, S, Vt = np.linalg.svd(P.reshape(k1 * d, d * k2), full_matrices=False)
    U, S, Vt = U[:, :Dn], S[:Dn], Vt[:Dn]
    return U.reshape(k1, d, Dn), S, Vt.reshape(Dn, d, k2).transpose(2, 1, 0)


def _chol_solve(A, B):
    """Solve (A + eps I) X = B, eps = 1e-12 trace(A)/n, by Cholesky."""
    n = A.shape[0]
    eps = 1e-12 * np.trace(A) / n
    C = np.linalg.cholesky(A + eps * np.eye(n))
    Y = np.linalg.solve(C, B)
    return np.linalg.solve(C.T, Y)


def als_left(N, Theta, aR):
    """a_l minimising d with a_r fixed: for each s,
    sum_{i,r} Nt[(k r'),(i r)] a[i,s,r] = b[k,s,r']."""
    k1 = N.shape[0]
    Dn = aR.shape[2]
    d = Theta.shape[1]
    Nt = np.einsum("ijkl,jtr,ltq->kqir", N, aR, aR, optimize=True).reshape(k1 * Dn, k1 * Dn)
    b = np.einsum("ijkl,istj,ltq->kqs", N, Theta, aR, optimize=True).reshape(k1 * Dn, d)
    x = _chol_solve(Nt, b)                         # [(i r), s]
    return x.reshape(k1, Dn, d).transpose(0, 2, 1)


def als_right(N, Theta, aL):
    """a_r minimising d with a_l fixed: for each t,
    sum_{j,r} Nt[(l r'),(j r)] a[j,t,r] = b[l,t,r']."""
    k2 = N.shape[1]
    Dn = aL.shape[2]
    d = Theta.shape[2]
    Nt = np.einsum("ijkl,isr,ksq->lqjr", N, aL, aL, optimize=True).reshape(k2 * Dn, k2 * Dn)
    b = np.einsum("ijkl,istj,ksq->lqt", N, Theta, aL, optimize=True).reshape(k2 * Dn, d)
    x = _chol_solve(Nt, b)
    return x.reshape(k2, Dn, d).transpose(0, 2, 1)


def pair(aL, aR):
    """psi[k1,s,t,k2] = sum_r aL[k1,s,r] aR[k2,t,r]."""
    return np.einsum("asr,btr->astb", aL, aR)


def cost(N, Theta, aL, aR):
    """d / <Theta|N|Theta> for the pair aL aR."""
    diff = pair(aL, aR) - Theta
    return quad(N, diff, diff) / quad(N, Theta, Theta)


def als(N, aL0, aR0, G, D, iters):
    """The reduced pair after the gate G (Section 2), and its relative cost.

    N must already be the positive part.  Returns (aL, aR, cost) with aL
    (k1, d, Dn), aR (k2, d, Dn) split in the balanced gauge."""
    Theta = apply_gate(G, aL0, aR0)
    k1, d, _, k2 = Theta.shape
    Dn = min(D, k1 * d, k2 * d)
    U, S, V = _svd_pair(Theta, Dn)
    aL, aR = U * S[None, None, :], V
    for _ in range(iters):
        aL = als_left(N, Theta, aR)
        aR = als_right(N, Theta, aL)
    U, S, V = _svd_pair(pair(aL, aR), Dn)
    for i in range(Dn):
        col = U[:, :, i].ravel()
        if col[np.argmax(np.abs(col))] < 0:
            U[:, :, i] *= -1.0
            V[:, :, i] *= -1.0
    sq = np.sqrt(S)
    aL, aR = U * sq[None, None, :], V * sq[None, None, :]
    return aL, aR, cost(N, Theta, aL, aR)


# ---------------------------------------------------------------------------
# One parallel update of a set of bonds (Sections 2, 4.4, 5.2)
# ---------------------------------------------------------------------------
def _pad_site(A, D):
    out = np.zeros((A.shape[0], D, D, D, D))
    out[:, :A.shape[1], :A.shape[2], :A.shape[3], :A.shape[4]] = A
    return out


def update_pair(Lv, Rv, M1, A1, B1, M2, A2, B2, G, D, iters):
    """The horizontal pair (A1, A2) after the gate, from its environment."""
    X1, a1 = split_left(A1)
    X2, a2 = split_right(A2)
    N = positive_part(bond_norm(Lv, Rv, M1, X1, B1, M2, X2, B2))
    aL, aR, c = als(N, a1, a2, G, D, iters)
    Dn = aL.shape[2]
    n1 = join_left(X1, aL)
    n2 = join_right(X2, aR.transpose(0, 1, 2))
    # bond slots beyond Dn stay zero; shapes follow the old tensors' bond dims
    B1n = np.zeros(A1.shape)
    B1n[..., :Dn] = n1
    B2n = np.zeros(A2.shape)
    B2n[:, :, :Dn] = n2
    return B1n / np.linalg.norm(B1n), B2n / np.linalg.norm(B2n), c


def _check_disjoint(bonds):
    seen = set()
    for kind, y, x in bonds:
        a, b = (y, x), ((y, x + 1) if kind == 0 else (y + 1, x))
        if a in seen or b in seen:
            raise ValueError("a site is in two bonds")
        seen.update([a, b])


def _store(out, D, kind, y, x, n1, n2):
    """New tensors of the pair (computed in the frame of ``kind``) into the
    dense lattice."""
    if kind == 1:
        n1, n2 = n1.transpose(0, 2, 1, 4, 3), n2.transpose(0, 2, 1, 4, 3)
        p1, p2 = (y, x), (y + 1, x)
    else:
        p1, p2 = (y, x), (y, x + 1)
    out[p1] = _pad_site(n1, D)
    out[p2] = _pad_site(n2, D)


def update_bonds(Ad, G, bonds, chi, mode="var", sweeps=2, seed=0, iters=8):
    """Apply the two-site gate G (d^2 x d^2) to every bond of ``bonds`` and
    refit, all from the full environment of the input state (the parallel
    schedule).  bonds: (kind, y, x) with kind 0 = (y,x)-(y,x+1) and 1 =
    (y,x)-(y+1,x); no site may be in two bonds.  Returns the new dense
    lattice and the relative cost of every bond."""
    Ad = np.asarray(Ad, dtype=np.float64)
    Ly, Lx, d, D = Ad.shape[0], Ad.shape[1], Ad.shape[2], Ad.shape[3]
    _check_disjoint(bonds)
    lat = O.lattice_from_dense(Ad)
    o = O.orientations(lat)
    out = Ad.copy()
    costs = [None] * len(bonds)
    for kind in (0, 1):
        sel = [(i, y, x) for i, (k, y, x) in enumerate(bonds) if k == kind]
        if not sel:
            continue
        # kind 1: the transposed lattice, where the bond is horizontal in row x
        src = o[0] if kind == 0 else o[2]
        H = Ly if kind == 0 else Lx
        tb, _ = O.boundary_sweep(src, chi, mode, sweeps, seed, 0 if kind == 0 else 2, upto=H - 1)
        bb, _ = O.boundary_sweep(o[1] if kind == 0 else o[3], chi, mode, sweeps, seed,
                                 1 if kind == 0 else 3, upto=H - 1)
        for i, y, x in sel:
            r, c = (y, x) if kind == 0 else (x, y)
            T, B = tb[r], bb[H - 1 - r]
            L, R = O.row_envs(T, B, src, r)
            A1, A2 = src.A[r][c], src.A[r][c + 1]
            n1, n2, costs[i] = update_pair(L[c], R[c + 1], T[c], A1, B[c], T[c + 1], A2, B[c + 1], G, D, iters)
            _store(out, D, kind, y, x, n1, n2)
    return out, costs


# ---------------------------------------------------------------------------
# Cluster update CU_delta (Section 5: a cluster of size delta around a row is
# every row within distance delta of it, and likewise for columns; outside it
# the environment is the separable CU_0 boundary of Section 5.1)
# ---------------------------------------------------------------------------
def strip_lattice(lat, cu0, r, delta, frame):
    """Rows r - delta .. r + delta (clipped) of ``lat`` with every column,
    closed above and below by the CU_0 matrices of those cuts and on the
    sides by the lattice's own closures.  frame 0: lat's rows; frame 1: the
    rows of the transposed lattice (columns of lat), with cu0 the CU_0
    matrices of lat's four orientations (top, bottom, left, right)."""
    sT, sB, sL, sR = cu0 if frame == 0 else (cu0[2], cu0[3], cu0[0], cu0[1])
    src = lat if frame == 0 else O.transpose(lat)
    H, W = src.Ly, src.Lx
    r0, r1 = max(0, r - delta), min(H - 1, r + delta)
    A = [[src.A[i][c] for c in range(W)] for i in range(r0, r1 + 1)]
    top = [sT[r0][c] for c in range(W)]
    bottom = [sB[H - 1 - r1][c] for c in range(W)]
    left = [sL[0][i] for i in range(r0, r1 + 1)]
    right = [sR[0][i] for i in range(r0, r1 + 1)]
    return O.Lat(A, top, bottom, left, right), r0


def update_bonds_cluster(Ad, G, bonds, delta, chi, mode="var", sweeps=2, seed=0, iters=8,
                         tol=1e-13, max_half=200):
    """As update_bonds, but every bond's environment is the cluster of size
    delta around its row (horizontal bonds) or column (vertical bonds):
    delta = 0 is CU_0 (a generalised simple update), delta >= L - 1 the full
    update.  All bonds use the CU_0 boundaries and clusters of the input state
    (the parallel CU of Section 5.4)."""
    Ad = np.asarray(Ad, dtype=np.float64)
    D = Ad.shape[3]
    _check_disjoint(bonds)
    if delta < 0:
        raise ValueError("delta must be >= 0")
    lat = O.lattice_from_dense(Ad)
    cu0 = O.cu0_all(lat, tol, max_half)
    out = Ad.copy()
    costs = [None] * len(bonds)
    rows = {}
    for i, (kind, y, x) in enumerate(bonds):
        r, c = (y, x) if kind == 0 else (x, y)
        rows.setdefault((kind, r), []).append((i, y, x, c))
    for (kind, r), sel in rows.items():
        S, r0 = strip_lattice(lat, cu0, r, delta, kind)
        rr = r - r0
        so = O.orientations(S)
        tag = 0 if kind == 0 else 2
        tb, _ = O.boundary_sweep(so[0], chi, mode, sweeps, seed, tag, upto=rr)
        bb, _ = O.boundary_sweep(so[1], chi, mode, sweeps, seed, tag + 1, upto=S.Ly - 1 - rr)
        T, B = tb[rr], bb[S.Ly - 1 - rr]
        L, R = O.row_envs(T, B, S, rr)
        for i, y, x, c in sel:
            A1, A2 = S.A[rr][c], S.A[rr][c + 1]
            n1, n2, costs[i] = update_pair(L[c], R[c + 1], T[c], A1, B[c], T[c + 1], A2, B[c + 1], G, D, iters)
            _store(out, D, kind, y, x, n1, n2)
    return out, costs


# ---------------------------------------------------------------------------
# Imaginary-time driver (Section 2; the CU of Sections 4.4 and 5)
# ---------------------------------------------------------------------------
def trotter_sets(Ly, Lx):
    """Four bond sets with no shared site: horizontal even / odd columns,
    vertical even / odd rows (first-order Trotter order)."""
    sets = []
    for par in (0, 1):
        sets.append([(0, y, x) for y in range(Ly) for x in range(par, Lx - 1, 2)])
    for par in (0, 1):
        sets.append([(1, y, x) for y in range(par, Ly - 1, 2) for x in range(Lx)])
    return sets


def heisenberg_gate(tau):
    """exp(-tau h) for h = S.S on one bond, as a (d^2 x d^2) matrix."""
    h = np.array([[0.25, 0, 0, 0], [0, -0.25, 0.5, 0], [0, 0.5, -0.25, 0], [0, 0, 0, 0.25]])
    w, v = np.linalg.eigh(h)
    return (v * np.exp(-tau * w)) @ v.T


def energy(Ad, chi, mode="svd"):
    """<H>/bonds of the Heisenberg model from the full environment."""
    env = O.env_full(Ad, chi, mode)
    h = np.array([[0.25, 0, 0, 0], [0, -0.25, 0.5, 0], [0, 0.5, -0.25, 0], [0, 0, 0, 0.25]])
    e = [O.expect(r, h) for row in env["rho_h"] for r in row]
    e += [O.expect(r, h) for row in env["rho_v"] for r in row]
    return float(np.sum(e))


def evolve(Ad, tau, steps, chi, mode="var", iters=8, sweeps=2, seed=0, delta=None):
    """``steps`` first-order Trotter steps of exp(-tau H), every set updated
    in parallel from its own environment: the full one (delta None) or the
    clusters of size delta."""
    G = heisenberg_gate(tau)
    A = np.asarray(Ad, dtype=np.float64)
    for _ in range(steps):
        for s in trotter_sets(A.shape[0], A.shape[1]):
            if delta is None:
                A, _ = update_bonds(A, G, s, chi, mode, sweeps, seed, iters)
            else:
                A, _ = update_bonds_cluster(A, G, s, delta, chi, mode, sweeps, seed, iters)
    return A
