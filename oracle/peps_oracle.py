"""FP64 CPU oracle for the boundary-MPS contraction of finite OBC PEPS.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  It shares no
code with the CUDA path and the CUDA path never calls it.

What it computes (Lubasch, Cirac, Banuls, "Unifying PEPS contractions"):

* Sandwich contraction (Section 2, Fig. 2): the norm network <psi|psi> is
  swept row by row; each row (ket A, bra A*, physical index traced) is
  absorbed into a boundary MPS, which is then approximated by an MPS of bond
  dimension chi (the paper's D').  Absorption is done ket first, then bra, so
  the D^8 double-layer tensor is never formed.
* Compression (Section 2, "optimally approximated by a MPS of fixed bond
  dimension D'"): ``svd`` = QR sweep to left-canonical form, then an SVD
  sweep keeping the largest chi singular values; ``var`` = one-site
  alternating least squares with the local equation N_l A_l = b_l of
  Section 2, where the orthonormal gauge makes N_l the identity.
* Environments and local reduced density matrices (Section 2: environment of
  a site; Section 5.3: local expectation values).
* CU_0 separable boundaries (Section 5.1, Figs. 7-8): a D'=1 boundary whose
  local ALS update is proportional to b_l, and stays positive.
* Cluster environments (Section 5, 5.2, 5.3): inside a window around a site
  the contraction is done as in the full method; outside it the environment
  is the product of CU_0 matrices.

Readings where the paper is silent (fixed here, and shared with the CUDA
path only as a written rule, never as code):

* bond cap at cut k: min(chi, product of physical dims left of the cut,
  the same on the right, bond of the product MPS), made consistent so no
  site matrix is rank-deficient by shape;
* var: warm start from the previous boundary (copied where it fits), with
  SplitMix64 noise of relative size 1e-3 on every other entry; the start is
  right-canonicalised; each half-sweep visits every site; two half-sweeps
  (L->R, R->L) by default; if no cut needs truncation the product MPS is
  only left-canonicalised;
* after every absorb+compress the boundary's centre tensor is scaled to
  unit Frobenius norm and the log of the factor is accumulated;
* the norm is the top-down sweep with the last row contracted exactly;
* vertical-bond densities come from the transposed lattice;
* a cluster window is n x n around its anchor (rows y-ceil(n/2)+1 ..),
  clipped (not shifted) at the lattice edge; CU_0 matrices start from the
  identity and stop when no matrix changes by 1e-13 in a half-sweep.

Index conventions (all tensors real float64):
  site tensor        A[s, u, l, n, r]   (physical, up, left, down, right)
  boundary MPS site  M[a, u, v, b]      (left bond, ket leg, bra leg, right bond)
  left environment   L[c, l, m, a]      (closing-MPS bond, ket leg, bra leg, open-MPS bond)
  right environment  R[b, r, q, c]      (open-MPS bond, ket leg, bra leg, closing-MPS bond)
  closure matrix     C[k, k']           (ket leg, bra leg) on an outward leg
"""
from __future__ import annotations

import math

import numpy as np


class OracleNotConverged(RuntimeError):
    """A CU_0 fixed-point iteration hit its half-sweep cap."""


def _ein(spec, a, b):
    # One pairwise contraction; the library routine is a step, nothing more.
    return np.einsum(spec, a, b, optimize=True)


# ---------------------------------------------------------------------------
# Lattices
# ---------------------------------------------------------------------------
class Lat:
    """A finite square-lattice network with a closure matrix on every outward leg.

    For the full lattice the outward legs have dimension 1 and the closures
    are [[1]] (open boundary conditions, Section 2).  A cluster window keeps
    the real dimension D on its outward legs and closes them with CU_0
    matrices (Section 5.2).
    """

    def __init__(self, A, top, bottom, left, right):
        self.A = A              # A[y][x] -> (d, Du, Dl, Dd, Dr)
        self.top = top          # top[x]    (Du, Du) on the up legs of row 0
        self.bottom = bottom    # bottom[x] (Dd, Dd) on the down legs of the last row
        self.left = left        # left[y]   (Dl, Dl) on the left legs of column 0
        self.right = right      # right[y]  (Dr, Dr) on the right legs of the last column

    @property
    def Ly(self):
        return len(self.A)

    @property
    def Lx(self):
        return len(self.A[0])


def lattice_from_dense(Ad: np.ndarray) -> Lat:
    """Dense (Ly, Lx, d, D, D, D, D) array -> Lat with OBC legs of dimension 1."""
    Ly, Lx, d, D = Ad.shape[0], Ad.shape[1], Ad.shape[2], Ad.shape[3]
    A = []
    for y in range(Ly):
        row = []
        for x in range(Lx):
            du = 1 if y == 0 else D
            dl = 1 if x == 0 else D
            dd = 1 if y == Ly - 1 else D
            dr = 1 if x == Lx - 1 else D
            row.append(np.array(Ad[y, x, :, :du, :dl, :dd, :dr], dtype=np.float64))
        A.append(row)
    one = lambda: np.ones((1, 1))
    return Lat(A, [one() for _ in range(Lx)], [one() for _ in range(Lx)],
               [one() for _ in range(Ly)], [one() for _ in range(Ly)])


def flip_ud(lat: Lat) -> Lat:
    """Mirror rows (a top-down sweep of the result is a bottom-up sweep)."""
    Ly = lat.Ly
    A = [[lat.A[Ly - 1 - y][x].transpose(0, 3, 2, 1, 4) for x in range(lat.Lx)]
         for y in range(Ly)]
    return Lat(A, list(lat.bottom), list(lat.top),
               [lat.left[Ly - 1 - y] for y in range(Ly)],
               [lat.right[Ly - 1 - y] for y in range(Ly)])


def transpose(lat: Lat) -> Lat:
    """Swap rows and columns (rows of the result are columns of the input)."""
    A = [[lat.A[y][x].transpose(0, 2, 1, 4, 3) for y in range(lat.Ly)]
         for x in range(lat.Lx)]
    return Lat(A, list(lat.left), list(lat.right), list(lat.top), list(lat.bottom))


def orientations(lat: Lat):
    """The four sweep directions: top-down, bottom-up, left-right, right-left."""
    t = transpose(lat)
    return [lat, flip_ud(lat), t, flip_ud(t)]


# ---------------------------------------------------------------------------
# Counter-based noise for the var initialisation (SplitMix64, Steele et al.
# 2014), keyed by (seed, orientation tag, row, column, entry index).
# ---------------------------------------------------------------------------
_MASK = (1 << 64) - 1
_GOLD = 0x9E3779B97F4A7C15


def init_noise(seed: int, tag: int, y: int, x: int, n: int) -> np.ndarray:
    """n values in [-1, 1): entry i is mix(key + i + golden) with
    key = seed*golden + (tag<<56 | y<<44 | x<<32), all mod 2^64."""
    key = (seed * _GOLD + ((tag << 56) | (y << 44) | (x << 32))) & _MASK
    with np.errstate(over="ignore"):
        z = np.uint64(key) + np.arange(n, dtype=np.uint64) + np.uint64(_GOLD)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -52) - 1.0


# ---------------------------------------------------------------------------
# The absorb chain (Section 2, Fig. 2(b)): ket contraction, then bra.
# ---------------------------------------------------------------------------
def chain_left(L, M, A):
    """X3[c,b,n,r,o,q] = sum L[c,l,m,a] M[a,u,v,b] A[s,u,l,n,r] A[s,v,m,o,q]."""
    X1 = _ein("clma,auvb->clmuvb", L, M)            # boundary  x environment
    X2 = _ein("clmuvb,sulnr->cmvbsnr", X1, A)       # ket layer
    return _ein("cmvbsnr,svmoq->cbnroq", X2, A)     # bra layer, s traced


def chain_right(R, M, A):
    """Y3[a,c,l,n,m,o] = sum M[a,u,v,b] A[s,u,l,n,r] A[s,v,m,o,q] R[b,r,q,c]."""
    Y1 = _ein("auvb,brqc->auvrqc", M, R)
    Y2 = _ein("auvrqc,sulnr->avqcsln", Y1, A)
    return _ein("avqcsln,svmoq->aclnmo", Y2, A)


def close_left(X3, R):
    """Local vector b[c,n,o,e] = sum X3[c,b,n,r,o,q] R[b,r,q,e]."""
    return _ein("cbnroq,brqe->cnoe", X3, R)


def close_right(L, Y3):
    """Local vector b[c,n,o,e] = sum L[c,l,m,a] Y3[a,e,l,n,m,o]."""
    return _ein("clma,aelnmo->cnoe", L, Y3)


def lenv_next(X3, Q):
    """L'[e,r,q,b] = sum X3[c,b,n,r,o,q] Q[c,n,o,e] (Q closes the bottom side)."""
    return _ein("cbnroq,cnoe->erqb", X3, Q)


def renv_prev(Y3, Q):
    """R'[a,l,m,c] = sum Y3[a,e,l,n,m,o] Q[c,n,o,e]."""
    return _ein("aelnmo,cnoe->almc", Y3, Q)


def closure_left(C):
    return C[None, :, :, None]


def closure_right(C):
    return C[None, :, :, None]


def closure_mps(mats):
    """A product boundary (bond 1) whose site matrices are the given closures."""
    return [m[None, :, :, None].astype(np.float64) for m in mats]


# ---------------------------------------------------------------------------
# Bond caps (reading of Section 2: chi bounds every bond; an exact MPS never
# needs more than the smaller of the two physical dimensions across a cut).
# ---------------------------------------------------------------------------
def bond_caps(phys, prod, chi):
    """caps[k] for cut k (between sites k and k+1).

    phys[x] = physical dimension (Dv^2) of site x; prod[k] = bond of the
    product MPS at cut k.  cap = min(chi, left product, right product,
    product bond), then made consistent so every site matrix has at least as
    many rows (columns) as its right (left) bond.
    """
    Lx = len(phys)
    caps = []
    for k in range(Lx - 1):
        lp = 1
        for x in range(k + 1):
            lp = min(lp * phys[x], 1 << 62)
        rp = 1
        for x in range(k + 1, Lx):
            rp = min(rp * phys[x], 1 << 62)
        caps.append(min(chi, lp, rp, prod[k]))
    for k in range(1, Lx - 1):
        caps[k] = min(caps[k], caps[k - 1] * phys[k])
    for k in range(Lx - 3, -1, -1):
        caps[k] = min(caps[k], caps[k + 1] * phys[k + 1])
    return caps


# ---------------------------------------------------------------------------
# svd mode
# ---------------------------------------------------------------------------
def product_mps(T, lat: Lat, y: int):
    """P[x] = boundary x row y (Fig. 2(b), left), bonds fused (a,l,l') / (b,r,r').

    The left closure of row y is absorbed into site 0 and the right closure
    into the last site, so the end bonds of P are 1.
    """
    Lx = lat.Lx
    P = []
    for x in range(Lx):
        A = lat.A[y][x]
        t1 = _ein("auvb,sulnr->avbslnr", T[x], A)     # ket
        t2 = _ein("avbslnr,svmoq->almnobrq", t1, A)                     # bra
        if x == 0:
            t2 = _ein("lm,almnobrq->anobrq", lat.left[y], t2)
            a = t2.shape[0]
        else:
            a = t2.shape[0] * t2.shape[1] * t2.shape[2]
        if x == Lx - 1:
            t2 = _ein("...brq,rq->...b", t2, lat.right[y])
        shp = t2.shape
        if x == 0:
            n, o = shp[1], shp[2]
        else:
            n, o = shp[3], shp[4]
        P.append(t2.reshape(a, n, o, -1))
    return P


def left_canonicalize(P):
    """QR sweep left to right; the last site carries the norm."""
    P = list(P)
    for x in range(len(P) - 1):
        a, n, o, b = P[x].shape
        Q, R = np.linalg.qr(P[x].reshape(a * n * o, b))
        P[x] = Q.reshape(a, n, o, Q.shape[1])
        P[x + 1] = np.tensordot(R, P[x + 1], axes=([1], [0]))
    return P


def svd_truncate(P, caps):
    """SVD sweep right to left keeping exactly min(cap, rank) triplets;
    singular values are absorbed leftward, so site 0 carries the norm."""
    P = list(P)
    for x in range(len(P) - 1, 0, -1):
        a, n, o, b = P[x].shape
        U, S, Vt = np.linalg.svd(P[x].reshape(a, n * o * b), full_matrices=False)
        k = min(caps[x - 1], S.shape[0])
        P[x] = Vt[:k].reshape(k, n, o, b)
        P[x - 1] = np.tensordot(P[x - 1], U[:, :k] * S[:k], axes=([3], [0]))
    return P


# ---------------------------------------------------------------------------
# var mode: one-site ALS with N_l = identity (Section 2)
# ---------------------------------------------------------------------------
def var_init(T, caps, pdim, seed, tag, y):
    """Warm start from the previous boundary, copied where it fits, with
    counter-based noise on every entry outside the copied block."""
    Lx = len(T)
    new = []
    for x in range(Lx):
        c = 1 if x == 0 else caps[x - 1]
        e = 1 if x == Lx - 1 else caps[x]
        D = pdim[x]
        N = np.zeros((c, D, D, e))
        M = T[x]
        a, u, _, b = M.shape
        ca, cu, cb = min(a, c), min(u, D), min(b, e)
        N[:ca, :cu, :cu, :cb] = M[:ca, :cu, :cu, :cb]
        mask = np.ones(N.shape, dtype=bool)
        mask[:ca, :cu, :cu, :cb] = False
        if mask.any():
            z = init_noise(seed, tag, y, x, N.size).reshape(N.shape)
            scale = 1e-3 * np.linalg.norm(M) / math.sqrt(N.size)
            N[mask] += scale * z[mask]
        new.append(N)
    return new


def right_canonicalize(N):
    """LQ sweep right to left (QR of the transpose); site 0 carries the norm."""
    N = list(N)
    for x in range(len(N) - 1, 0, -1):
        c, n, o, e = N[x].shape
        Q, R = np.linalg.qr(N[x].reshape(c, n * o * e).T)
        k = Q.shape[1]
        N[x] = Q.T.reshape(k, n, o, e)
        N[x - 1] = np.tensordot(N[x - 1], R.T, axes=([3], [0]))
    return N


def var_compress(T, lat: Lat, y: int, caps, sweeps: int, seed: int, tag: int):
    """One-site ALS fit of the new boundary to (row y) x T.

    Each half-sweep visits every site; at site x the optimal tensor is the
    local vector b_x (the norm matrix is the identity because every other
    site is orthonormal), then it is orthonormalised by QR (left-to-right)
    or LQ (right-to-left) and the environment is moved.  Returns the new
    MPS with the centre at site 0 (even ``sweeps``) or the last site.
    """
    Lx = lat.Lx
    A = lat.A[y]
    pdim = [A[x].shape[3] for x in range(Lx)]
    N = right_canonicalize(var_init(T, caps, pdim, seed, tag, y))
    R = [None] * Lx
    L = [None] * Lx
    R[Lx - 1] = closure_right(lat.right[y])
    for x in range(Lx - 1, 0, -1):
        R[x - 1] = renv_prev(chain_right(R[x], T[x], A[x]), N[x])
    L[0] = closure_left(lat.left[y])
    centre = 0
    for h in range(sweeps):
        if h % 2 == 0:
            for x in range(Lx):
                X3 = chain_left(L[x], T[x], A[x])
                b = close_left(X3, R[x])
                if x < Lx - 1:
                    c, n, o, e = b.shape
                    Q, _ = np.linalg.qr(b.reshape(c * n * o, e))
                    N[x] = Q.reshape(c, n, o, Q.shape[1])
                    L[x + 1] = lenv_next(X3, N[x])
                else:
                    N[x] = b
            centre = Lx - 1
        else:
            for x in range(Lx - 1, -1, -1):
                Y3 = chain_right(R[x], T[x], A[x])
                b = close_right(L[x], Y3)
                if x > 0:
                    c, n, o, e = b.shape
                    Q, _ = np.linalg.qr(b.reshape(c, n * o * e).T)
                    N[x] = Q.T.reshape(Q.shape[1], n, o, e)
                    R[x - 1] = renv_prev(Y3, N[x])
                else:
                    N[x] = b
            centre = 0
    return N, centre


# ---------------------------------------------------------------------------
# One absorb + compress step and the boundary sweep (Section 2)
# ---------------------------------------------------------------------------
def absorb_compress(T, lat: Lat, y: int, chi: int, mode: str, sweeps: int,
                    seed: int, tag: int):
    """Returns (new boundary, ln of the normalisation removed from it)."""
    Lx = lat.Lx
    A = lat.A[y]
    phys = [A[x].shape[3] ** 2 for x in range(Lx)]
    prod = [T[k].shape[3] * A[k].shape[4] ** 2 for k in range(Lx - 1)]
    caps = bond_caps(phys, prod, chi)
    if mode == "svd":
        P = svd_truncate(left_canonicalize(product_mps(T, lat, y)), caps)
        centre = 0
    elif mode == "var":
        if all(prod[k] <= caps[k] for k in range(Lx - 1)):
            P = left_canonicalize(product_mps(T, lat, y))   # exact: no fit needed
            centre = Lx - 1
        else:
            P, centre = var_compress(T, lat, y, caps, sweeps, seed, tag)
    else:
        raise ValueError(mode)
    nrm = np.linalg.norm(P[centre])
    P[centre] = P[centre] / nrm
    return P, math.log(nrm)


def boundary_sweep(lat: Lat, chi: int, mode: str = "svd", sweeps: int = 2,
                   seed: int = 0, tag: int = 0, upto: int | None = None):
    """Top-down boundaries: out[y] is the boundary above row y (out[0] is the
    top closure).  Rows 0 .. upto-1 are absorbed (default: all but the last)."""
    Ly = lat.Ly
    stop = Ly - 1 if upto is None else upto
    T = closure_mps(lat.top)
    bounds, lns = [T], [0.0]
    for y in range(stop):
        T, ln = absorb_compress(T, lat, y, chi, mode, sweeps, seed, tag)
        bounds.append(T)
        lns.append(ln)
    return bounds, lns


# ---------------------------------------------------------------------------
# Row environments and local reduced density matrices (Sections 2 and 5.3)
# ---------------------------------------------------------------------------
def row_envs(T, B, lat: Lat, y: int):
    """Left/right environments along row y between top boundary T and bottom
    boundary B (B's physical legs are the down legs of row y).  Each is
    divided by its Frobenius norm, which cancels in every ratio."""
    Lx = lat.Lx
    A = lat.A[y]
    L = [None] * Lx
    R = [None] * Lx
    L[0] = closure_left(lat.left[y])
    for x in range(Lx - 1):
        t = lenv_next(chain_left(L[x], T[x], A[x]), B[x])
        L[x + 1] = t / np.linalg.norm(t)
    R[Lx - 1] = closure_right(lat.right[y])
    for x in range(Lx - 1, 0, -1):
        t = renv_prev(chain_right(R[x], T[x], A[x]), B[x])
        R[x - 1] = t / np.linalg.norm(t)
    return L, R


def _open_site(Lv, M, A, Bv):
    """W[e,r,q,b,s,t]: left environment pushed through one site with its
    physical index left open (s ket, t bra)."""
    X1 = _ein("clma,auvb->clmuvb", Lv, M)
    X2 = _ein("clmuvb,sulnr->cmvbsnr", X1, A)
    X3 = _ein("cmvbsnr,tvmoq->cbsnrtoq", X2, A)
    return _ein("cbsnrtoq,cnoe->erqbst", X3, Bv)


def rho_site(Lv, Rv, M, A, Bv):
    """rho[s,t] of one site (unnormalised)."""
    W = _open_site(Lv, M, A, Bv)
    return _ein("erqbst,brqe->st", W, Rv)


def rho_hbond(Lv, Rv, M1, A1, B1, M2, A2, B2):
    """rho[s1,s2,t1,t2] of two horizontally adjacent sites (unnormalised)."""
    W = _open_site(Lv, M1, A1, B1)                        # [c,l,m,a,s1,t1]
    X1 = _ein("clmaij,auvb->clmuvbij", W, M2)
    X2 = _ein("clmuvbij,sulnr->cmvbsnrij", X1, A2)
    X3 = _ein("cmvbsnrij,tvmoq->cbsnrtoqij", X2, A2)
    X4 = _ein("cbsnrtoqij,cnoe->erqbstij", X3, B2)
    return _ein("erqbstij,brqe->isjt", X4, Rv)


def expect(rho, op):
    """<O> = Tr(rho O) / Tr(rho) for rho[ket..., bra...] flattened to a matrix."""
    k = int(round(math.sqrt(rho.size)))
    r = rho.reshape(k, k)
    return float(np.sum(r * op.T) / np.trace(r))


def _row_rhos(lat: Lat, T, B, y: int, xs=None, bonds=True):
    """rho_site at the columns in xs (default all) and rho_hbond to their right."""
    L, R = row_envs(T, B, lat, y)
    Lx = lat.Lx
    xs = range(Lx) if xs is None else xs
    A = lat.A[y]
    rs, rh = {}, {}
    for x in xs:
        rs[x] = rho_site(L[x], R[x], T[x], A[x], B[x])
        if bonds and x + 1 < Lx:
            rh[x] = rho_hbond(L[x], R[x + 1], T[x], A[x], B[x],
                              T[x + 1], A[x + 1], B[x + 1])
    return rs, rh


# ---------------------------------------------------------------------------
# Full environments (sandwich contraction from all four sides)
# ---------------------------------------------------------------------------
def _norm_from_top(lat: Lat, T, lns):
    """ln|<psi|psi>| and its sign: the last row contracted exactly between the
    last top boundary and the bottom closures (reading: top-down only)."""
    Ly, Lx = lat.Ly, lat.Lx
    y = Ly - 1
    A = lat.A[y]
    B = closure_mps(lat.bottom)
    Lv = closure_left(lat.left[y])
    ln = sum(lns)
    for x in range(Lx):
        Lv = lenv_next(chain_left(Lv, T[x], A[x]), B[x])
        if x < Lx - 1:
            nr = np.linalg.norm(Lv)
            Lv = Lv / nr
            ln += math.log(nr)
    s = float(_ein("erqb,rq->", Lv, lat.right[y]))
    return ln + math.log(abs(s)), (1 if s > 0 else -1)


def env_full(Ad_or_lat, chi: int, mode: str = "svd", sweeps: int = 2, seed: int = 0):
    """All local reduced density matrices and the norm of a finite PEPS.

    Returns dict with rho_site[y][x] (d,d), rho_h[y][x] for bond
    (y,x)-(y,x+1) as (d,d,d,d)=[s1,s2,t1,t2], rho_v[y][x] for bond
    (y,x)-(y+1,x), ln_norm and sign.
    """
    lat = Ad_or_lat if isinstance(Ad_or_lat, Lat) else lattice_from_dense(Ad_or_lat)
    Ly, Lx = lat.Ly, lat.Lx
    o = orientations(lat)
    bt, lnt = boundary_sweep(o[0], chi, mode, sweeps, seed, 0, upto=Ly - 1)
    bb, _ = boundary_sweep(o[1], chi, mode, sweeps, seed, 1, upto=Ly - 1)
    bl, _ = boundary_sweep(o[2], chi, mode, sweeps, seed, 2, upto=Lx - 1)
    br, _ = boundary_sweep(o[3], chi, mode, sweeps, seed, 3, upto=Lx - 1)
    rho_s = [[None] * Lx for _ in range(Ly)]
    rho_h = [[None] * (Lx - 1) for _ in range(Ly)]
    rho_v = [[None] * Lx for _ in range(Ly - 1)]
    for y in range(Ly):
        rs, rh = _row_rhos(lat, bt[y], bb[Ly - 1 - y], y)
        for x in range(Lx):
            rho_s[y][x] = rs[x]
            if x < Lx - 1:
                rho_h[y][x] = rh[x]
    t = o[2]
    for x in range(Lx):
        _, rh = _row_rhos(t, bl[x], br[Lx - 1 - x], x)
        for y in range(Ly - 1):
            rho_v[y][x] = rh[y]
    ln, sg = _norm_from_top(lat, bt[Ly - 1], lnt)
    return dict(rho_site=rho_s, rho_h=rho_h, rho_v=rho_v, ln_norm=ln, sign=sg)


def norm(Ad_or_lat, chi: int, mode: str = "svd", sweeps: int = 2, seed: int = 0):
    """(ln|<psi|psi>|, sign) by the top-down sweep."""
    lat = Ad_or_lat if isinstance(Ad_or_lat, Lat) else lattice_from_dense(Ad_or_lat)
    bt, lnt = boundary_sweep(lat, chi, mode, sweeps, seed, 0)
    return _norm_from_top(lat, bt[lat.Ly - 1], lnt)


# ---------------------------------------------------------------------------
# CU_0: separable (D'=1) boundaries (Section 5.1)
# ---------------------------------------------------------------------------
def cu0_local(Lm, S, A, Rm):
    """b[n,o] = sum Lm[l,m] S[u,v] A[s,u,l,n,r] A[s,v,m,o,q] Rm[r,q]; O(dD^5)."""
    Y = _ein("lm,sulnr->smunr", Lm, A)
    Z = _ein("smunr,uv->smvnr", Y, S)
    Z = _ein("smvnr,rq->smvnq", Z, Rm)
    return _ein("smvnq,svmoq->no", Z, A)


def cu0_lenv(Lm, S, A, N):
    """L'[r,q] = sum Lm[l,m] S[u,v] A[s,u,l,n,r] A[s,v,m,o,q] N[n,o]."""
    Y = _ein("lm,sulnr->smunr", Lm, A)
    Z = _ein("smunr,uv->smvnr", Y, S)
    Z = _ein("smvnr,no->smvor", Z, N)
    return _ein("smvor,svmoq->rq", Z, A)


def cu0_renv(Rm, S, A, N):
    """R'[l,m] = sum Rm[r,q] S[u,v] A[s,u,l,n,r] A[s,v,m,o,q] N[n,o]."""
    Y = _ein("rq,sulnr->sulnq", Rm, A)
    Z = _ein("sulnq,uv->svlnq", Y, S)
    Z = _ein("svlnq,no->svloq", Z, N)
    return _ein("svloq,svmoq->lm", Z, A)


def _fro(m):
    return m / np.linalg.norm(m)


def cu0_sweep(lat: Lat, tol: float = 1e-13, max_half: int = 200,
              init: str = "identity", init_seed: int = 0):
    """Top-down separable boundaries.  out[r] (r = 0..Ly-1) is the list of
    D x D matrices on the up legs of row r (out[0] = top closures).

    For each cut the D'=1 boundary is found by ALS: each local update is
    b_l itself (norm matrix proportional to the identity, Fig. 8), scaled to
    unit Frobenius norm; half-sweeps alternate L->R and R->L until the
    largest change of any matrix is below ``tol``.  Initial matrices are the
    identity (or X X^T with X from ``init_seed`` when init='random'), so they
    are positive and stay positive (Section 5.1).
    """
    Ly, Lx = lat.Ly, lat.Lx
    sig = [np.array(m, dtype=np.float64) for m in lat.top]
    out = [sig]
    rng = np.random.default_rng(init_seed)
    for r in range(Ly - 1):
        A = lat.A[r]
        new = []
        for x in range(Lx):
            D = A[x].shape[3]
            if init == "random":
                X = rng.uniform(-1, 1, (D, D))
                new.append(_fro(X @ X.T))
            else:
                new.append(_fro(np.eye(D)))
        Rm = [None] * Lx
        Lm = [None] * Lx
        Rm[Lx - 1] = lat.right[r]
        for x in range(Lx - 1, 0, -1):
            Rm[x - 1] = _fro(cu0_renv(Rm[x], sig[x], A[x], new[x]))
        Lm[0] = lat.left[r]
        done = False
        for h in range(max_half):
            change = 0.0
            if h % 2 == 0:
                for x in range(Lx):
                    b = _fro(cu0_local(Lm[x], sig[x], A[x], Rm[x]))
                    change = max(change, float(np.linalg.norm(b - new[x])))
                    new[x] = b
                    if x < Lx - 1:
                        Lm[x + 1] = _fro(cu0_lenv(Lm[x], sig[x], A[x], new[x]))
            else:
                for x in range(Lx - 1, -1, -1):
                    b = _fro(cu0_local(Lm[x], sig[x], A[x], Rm[x]))
                    change = max(change, float(np.linalg.norm(b - new[x])))
                    new[x] = b
                    if x > 0:
                        Rm[x - 1] = _fro(cu0_renv(Rm[x], sig[x], A[x], new[x]))
            if change < tol:
                done = True
                break
        if not done:
            raise OracleNotConverged(f"CU0 cut {r}: change {change:.3e} after {max_half} half-sweeps")
        sig = new
        out.append(sig)
    return out


def cu0_all(lat: Lat, tol: float = 1e-13, max_half: int = 200):
    """Separable boundaries from all four sides, in the orientations' frames."""
    return [cu0_sweep(o, tol, max_half) for o in orientations(lat)]


# ---------------------------------------------------------------------------
# Cluster environments (Section 5; window shape per Section 5.3 "around the
# individual terms"; n x n window clipped at the lattice edge)
# ---------------------------------------------------------------------------
def window_bounds(L: int, i: int, n: int):
    h = -(-n // 2)
    lo = i - h + 1
    return max(lo, 0), min(lo + n - 1, L - 1)


def window_lattice(lat: Lat, cu0, y: int, x: int, n: int):
    """The window around (y, x) with its outward legs closed by CU_0 matrices."""
    Ly, Lx = lat.Ly, lat.Lx
    r0, r1 = window_bounds(Ly, y, n)
    c0, c1 = window_bounds(Lx, x, n)
    sT, sB, sL, sR = cu0
    A = [[lat.A[r][c] for c in range(c0, c1 + 1)] for r in range(r0, r1 + 1)]
    top = [sT[r0][c] for c in range(c0, c1 + 1)]
    bottom = [sB[Ly - 1 - r1][c] for c in range(c0, c1 + 1)]
    left = [sL[c0][r] for r in range(r0, r1 + 1)]
    right = [sR[Lx - 1 - c1][r] for r in range(r0, r1 + 1)]
    return Lat(A, top, bottom, left, right), (r0, r1, c0, c1)


def cluster_anchor(W: Lat, yw: int, xw: int, chi: int, mode: str, sweeps: int, seed: int):
    """rho_site, rho_h (to the right) and rho_v (downwards) at window site
    (yw, xw), computed with the full routine restricted to the window."""
    Hh, Ww = W.Ly, W.Lx
    o = orientations(W)
    bt, _ = boundary_sweep(o[0], chi, mode, sweeps, seed, 0, upto=yw)
    bb, _ = boundary_sweep(o[1], chi, mode, sweeps, seed, 1, upto=Hh - 1 - yw)
    rs, rh = _row_rhos(W, bt[yw], bb[Hh - 1 - yw], yw, xs=[xw])
    rv = None
    if yw + 1 < Hh:
        bl, _ = boundary_sweep(o[2], chi, mode, sweeps, seed, 2, upto=xw)
        br, _ = boundary_sweep(o[3], chi, mode, sweeps, seed, 3, upto=Ww - 1 - xw)
        _, rhv = _row_rhos(o[2], bl[xw], br[Ww - 1 - xw], xw, xs=[yw])
        rv = rhv[yw]
    return rs[xw], rh.get(xw), rv


def env_cluster(Ad_or_lat, n: int, chi: int, mode: str = "svd", sweeps: int = 2,
                seed: int = 0, tol: float = 1e-13, max_half: int = 200, anchors=None):
    """Cluster environments for every site (or the given anchors).

    Returns the same dict layout as env_full (entries None where not
    computed), with ln_norm absent.
    """
    lat = Ad_or_lat if isinstance(Ad_or_lat, Lat) else lattice_from_dense(Ad_or_lat)
    Ly, Lx = lat.Ly, lat.Lx
    cu0 = cu0_all(lat, tol, max_half)
    rho_s = [[None] * Lx for _ in range(Ly)]
    rho_h = [[None] * (Lx - 1) for _ in range(Ly)]
    rho_v = [[None] * Lx for _ in range(Ly - 1)]
    if anchors is None:
        anchors = [(y, x) for y in range(Ly) for x in range(Lx)]
    for (y, x) in anchors:
        W, (r0, _, c0, _) = window_lattice(lat, cu0, y, x, n)
        s, h, v = cluster_anchor(W, y - r0, x - c0, chi, mode, sweeps, seed)
        rho_s[y][x] = s
        if x + 1 < Lx:
            rho_h[y][x] = h
        if y + 1 < Ly:
            rho_v[y][x] = v
    return dict(rho_site=rho_s, rho_h=rho_h, rho_v=rho_v)


# ---------------------------------------------------------------------------
# Boundary fidelity (Section 5.2, Fig. Fid): distance of the environment of
# the left-most column, computed with a cluster of delta columns, from the
# full contraction of the other columns at a large reference bond.
# ---------------------------------------------------------------------------
def mps_overlap(P, Q):
    """<P|Q> of two boundary MPS with the same physical legs (real)."""
    E = np.ones((1, 1))
    for a, b in zip(P, Q):
        E = _ein("ab,auvc->buvc", E, a)
        E = _ein("buvc,buvd->cd", E, b)
    return float(E[0, 0])


def left_column_boundary(lat: Lat, delta: int, chi: int, mode: str = "var", sweeps: int = 2, seed: int = 0):
    """The boundary MPS on the right legs of column 0 (the environment of the
    left-most column).  delta >= Lx-1: the full contraction of columns
    Lx-1 .. 1 (Section 2).  Otherwise the cluster form (Section 5.2):
    columns delta .. 1 are absorbed at bond chi into the CU_0 separable
    boundary (Section 5.1) of the columns right of column delta.  The sweep
    is the right-to-left one (orientation 3, rows = columns from the right);
    var noise is keyed by the rows of the part that is absorbed."""
    o = orientations(lat)[3]
    L = o.Ly
    if delta >= L - 1:
        b, _ = boundary_sweep(o, chi, mode, sweeps, seed, 3, upto=L - 1)
        return b[L - 1]
    r0 = L - 1 - delta
    sep = cu0_sweep(o)[r0]
    part = Lat(o.A[r0:], list(sep), list(o.bottom), list(o.left[r0:]), list(o.right[r0:]))
    b, _ = boundary_sweep(part, chi, mode, sweeps, seed, 3, upto=delta)
    return b[delta]


def boundary_fidelity(Ad_or_lat, delta: int, chi: int, chi_ref: int, mode: str = "var", sweeps: int = 2,
                      seed: int = 0) -> float:
    """1 - f with f = |tr(rho_ref^T rho)| for unit-norm rho_ref, rho (Fig. Fid):
    rho = left_column_boundary(delta, chi), rho_ref = the full contraction at chi_ref."""
    lat = Ad_or_lat if isinstance(Ad_or_lat, Lat) else lattice_from_dense(Ad_or_lat)
    ref = left_column_boundary(lat, lat.Lx, chi_ref, mode, sweeps, seed)
    rho = left_column_boundary(lat, delta, chi, mode, sweeps, seed)
    f = abs(mps_overlap(ref, rho)) / math.sqrt(mps_overlap(ref, ref) * mps_overlap(rho, rho))
    return 1.0 - f


# ---------------------------------------------------------------------------
# Infinite PEPS (Section 5.4): a CU procedure needs only the dominant D'=1
# boundary of the infinite lattice (O(dD^5)), followed by a cluster
# contraction as in the finite case.  Single-site unit cell: every site holds
# the same tensor A[s,u,l,n,r], every leg has dimension D.
# ---------------------------------------------------------------------------
def ipeps_orientations(A):
    """A as seen by the top-down, bottom-up, left-right and right-left sweeps
    (the leg permutations of flip_ud and transpose)."""
    tr = A.transpose(0, 2, 1, 4, 3)
    return [A, A.transpose(0, 3, 2, 1, 4), tr, tr.transpose(0, 3, 2, 1, 4)]


def cu0_infinite(A, tol: float = 1e-13, max_iter: int = 5000):
    """Dominant separable (D'=1) boundary of the infinite lattice from the top:
    sigma with sigma ~ b(sigma), b the local CU_0 update (Section 5.1) of a
    row of copies of A between sigma above and sigma below, its horizontal
    environments the dominant left / right fixed points of that row.  Each
    step updates the left environment, the right environment and sigma once,
    all scaled to unit Frobenius norm, from identities; it stops when none
    moves by tol."""
    D = A.shape[1]
    sig = _fro(np.eye(D))
    Lm = _fro(np.eye(D))
    Rm = _fro(np.eye(D))
    for _ in range(max_iter):
        Ln = _fro(cu0_lenv(Lm, sig, A, sig))
        Rn = _fro(cu0_renv(Rm, sig, A, sig))
        b = _fro(cu0_local(Ln, sig, A, Rn))
        change = max(float(np.linalg.norm(Ln - Lm)), float(np.linalg.norm(Rn - Rm)),
                     float(np.linalg.norm(b - sig)))
        Lm, Rm, sig = Ln, Rn, b
        if change < tol:
            return sig
    raise OracleNotConverged(f"infinite CU0: change {change:.3e} after {max_iter} steps")


def ipeps_cluster(A, n: int, chi: int, mode: str = "var", sweeps: int = 2, seed: int = 0, tol: float = 1e-13):
    """Density matrices of one site, its right bond and its down bond of the
    infinite PEPS: an n x n window of copies of A (anchor at row and column
    ceil(n/2)-1, as for interior windows of the finite lattice) closed by the
    four infinite separable boundaries, contracted by the full routine at chi.
    Returns dict(rho_site, rho_h, rho_v, sigma) with sigma the four boundary
    matrices (top, bottom, left, right)."""
    A = np.asarray(A, dtype=np.float64)
    sig = [cu0_infinite(Ao, tol) for Ao in ipeps_orientations(A)]
    rows = [[A for _ in range(n)] for _ in range(n)]
    W = Lat(rows, [sig[0]] * n, [sig[1]] * n, [sig[2]] * n, [sig[3]] * n)
    a = -(-n // 2) - 1
    s, h, v = cluster_anchor(W, a, a, chi, mode, sweeps, seed)
    return dict(rho_site=s, rho_h=h, rho_v=v, sigma=sig)


# ---------------------------------------------------------------------------
# Operators (eq. 1 and eq. 2 conventions: Pauli matrices, S = sigma/2)
# ---------------------------------------------------------------------------
SZ = np.array([[1.0, 0.0], [0.0, -1.0]])
SX = np.array([[0.0, 1.0], [1.0, 0.0]])
SDOTS = 0.25 * np.array([[1.0, 0, 0, 0], [0, -1.0, 2.0, 0], [0, 2.0, -1.0, 0], [0, 0, 0, 1.0]])


def expect_all(env, kind: str, op):
    """Expectation values of op at every site / bond, as a flat list in
    row-major order (None where the environment was not computed)."""
    key = {"site": "rho_site", "hbond": "rho_h", "vbond": "rho_v"}[kind]
    out = []
    for row in env[key]:
        for r in row:
            out.append(None if r is None else expect(r, op))
    return out
