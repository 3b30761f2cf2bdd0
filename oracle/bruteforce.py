"""Brute-force state vectors of small PEPS: the plain definition, written out.

TEST INFRASTRUCTURE ONLY (see the oracle package header).

psi[s_1 .. s_N] = F(A_1^{s_1} ... A_N^{s_N}) with F the contraction of every
virtual index (Section 2, the PEPS definition and Fig. 1).  Norms and local
expectation values follow from psi directly.  Nothing here uses boundary
MPS, truncation or environments, so it pins the boundary-MPS oracle
independently.

Closures (a window's outward legs closed by positive matrices C = X X^T,
Section 5.2) are handled by absorbing X into the ket and the bra: the
column index of X becomes an extra physical index of that site.
"""
from __future__ import annotations

import numpy as np


def _row_tensor(row):
    """Contract one row's horizontal legs: R[S, U, Dn] with S, U, Dn the
    row-major products of the sites' physical, up and down indices."""
    t = row[0]                                   # [s,u,l,n,r], l has dim 1
    d, u, l, n, r = t.shape
    assert l == 1
    cur = t.reshape(d, u, n, r)                  # [S, U, N, r]
    for A in row[1:]:
        d2, u2, l2, n2, r2 = A.shape
        x = np.einsum("SUNr,surnq->SsUuNnq", cur, A)   # contract r with the left leg
        S, U, N = cur.shape[0] * d2, cur.shape[1] * u2, cur.shape[2] * n2
        cur = x.reshape(S, U, N, r2)
    assert cur.shape[3] == 1
    return cur[:, :, :, 0]


def state_vector(A):
    """psi as a flat vector, sites in row-major order, site 0 most significant.

    ``A`` is a list of rows of tensors [s,u,l,n,r] whose outward legs have
    dimension 1 (apply :func:`absorb_closures` first for a closed window).
    """
    psi = np.ones((1, 1))                         # [S_so_far, U_of_next_row]
    for row in A:
        R = _row_tensor(row)                      # [S, U, N]
        psi = np.einsum("pu,sun->psn", psi, R).reshape(-1, R.shape[2])
    assert psi.shape[1] == 1
    return psi[:, 0]


def dense_lattice(Ad):
    """Rows of tensors from the dense C-ABI array (OBC legs sliced to dim 1)."""
    Ly, Lx, d, D = Ad.shape[:4]
    rows = []
    for y in range(Ly):
        row = []
        for x in range(Lx):
            du = 1 if y == 0 else D
            dl = 1 if x == 0 else D
            dd = 1 if y == Ly - 1 else D
            dr = 1 if x == Lx - 1 else D
            row.append(np.array(Ad[y, x, :, :du, :dl, :dd, :dr]))
        rows.append(row)
    return rows


def _sqrt_psd(C):
    w, V = np.linalg.eigh(0.5 * (C + C.T))
    return V * np.sqrt(np.clip(w, 0.0, None))


def absorb_closures(A, top, bottom, left, right):
    """Fold closure matrices into the edge tensors; returns (rows, extra) where
    extra[y][x] is the dimension of the extra physical index of site (y,x)."""
    Ly, Lx = len(A), len(A[0])
    rows, extra = [], []
    for y in range(Ly):
        row, ex = [], []
        for x in range(Lx):
            t = np.array(A[y][x])                 # [s,u,l,n,r]
            e = 1
            for side, mats, idx in (("u", top, x), ("d", bottom, x), ("l", left, y), ("r", right, y)):
                if side == "u" and y != 0:
                    continue
                if side == "d" and y != Ly - 1:
                    continue
                if side == "l" and x != 0:
                    continue
                if side == "r" and x != Lx - 1:
                    continue
                X = _sqrt_psd(np.asarray(mats[idx], dtype=np.float64))
                ax = {"u": 1, "l": 2, "d": 3, "r": 4}[side]
                t = np.moveaxis(np.tensordot(t, X, axes=([ax], [0])), -1, ax)
                # move the new (closure) index into the physical slot
                s = t.shape
                t = np.moveaxis(t, ax, 1)          # [s, k, ...rest]
                t = t.reshape((s[0] * s[ax],) + t.shape[2:])
                t = np.expand_dims(t, ax)          # outward leg of dimension 1
                e *= s[ax]
            row.append(t)
            ex.append(e)
        rows.append(row)
        extra.append(ex)
    return rows, extra


def norm(psi):
    return float(psi @ psi)


def _site_op(psi, dims, i, O):
    """(O acting on the leading factor of site i's index) applied to psi."""
    pre = int(np.prod(dims[:i]))
    post = int(np.prod(dims[i + 1:]))
    d = O.shape[0]
    ex = dims[i] // d
    p = psi.reshape(pre, d, ex, post)
    return np.einsum("ts,psqr->ptqr", O, p).reshape(-1)


def expect_site(psi, dims, i, O):
    """<O_i> with O acting on the physical (leading) part of site i's index."""
    return float(psi @ _site_op(psi, dims, i, O)) / norm(psi)


def expect_bond(psi, dims, i, j, O2, d=2):
    """<O_{ij}> for a d^2 x d^2 operator on sites i < j, rows (s_i, s_j)."""
    O4 = O2.reshape(d, d, d, d)                  # [t_i, t_j, s_i, s_j]
    # reshape psi so that sites i and j are explicit axes
    pre = int(np.prod(dims[:i]))
    mid = int(np.prod(dims[i + 1:j]))
    post = int(np.prod(dims[j + 1:]))
    ei, ej = dims[i] // d, dims[j] // d
    p = psi.reshape(pre, d, ei, mid, d, ej, post)
    q = np.einsum("tusv,psamvbr->ptamubr", O4, p)
    return float(psi @ q.reshape(-1)) / norm(psi)
