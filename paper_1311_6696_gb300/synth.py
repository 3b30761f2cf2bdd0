"""Seeded synthetic PEPS inputs.

This module only draws numbers and lays them out; it holds none of the
boundary-MPS arithmetic.  The CUDA path and the CPU oracle both take their
inputs from here, so the same seed gives bit-identical tensors to both.

Layout of a lattice (the C-ABI layout): a dense float64 array of shape
``(Ly, Lx, d, D, D, D, D)`` with legs ``[s, up, left, down, right]``
(Section 2, Fig. 1(b): one tensor per site, a physical index ``s`` and four
virtual indices).  Open boundary conditions give edge tensors fewer virtual
legs (Section 2, footnote on OBC); a leg that points out of the lattice uses
index 0 only and every other entry on it is zero.

Generators
----------
* :func:`splitmix64_stream` -- the published SplitMix64 generator (Steele,
  Lea & Flood, OOPSLA 2014), used as a sequential stream.
* :func:`peps_uniform` -- entries i.i.d. uniform[0,1), each tensor scaled to
  unit Frobenius norm (the 4x4 D=2 workload).
* :func:`peps_gauss` -- entries ``0.5 + 0.1*N(0,1)`` by Box-Muller on the same
  stream, unit Frobenius norm (the 10x10 D=4 and 14x14 D=6 workloads).
* :func:`peps_product` -- a D=1 product state (closed-form test cases).
* :func:`peps_simple_update` -- a seeded simple-update (Section 3) Heisenberg
  ground-state approximation (the 20x20 D=8 and 16x16 D=4 workloads).

Tensors are filled in site-row-major order, each in C order over its ragged
(effective) shape, drawing from one stream that continues across sites.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64_stream(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+n-1`` of SplitMix64 seeded with ``seed``.

    Output i is ``mix(seed + (i+1)*golden)`` (mod 2^64), i.e. the state is
    advanced by the golden-ratio increment before each mix.
    """
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        return _mix(s + i * _GOLDEN)


def uniform01(seed: int, n: int, start: int = 0) -> np.ndarray:
    """n doubles in [0,1) from the top 53 bits of each SplitMix64 output."""
    z = splitmix64_stream(seed, n, start)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, n: int) -> np.ndarray:
    """n standard normals by Box-Muller on consecutive uniform pairs."""
    m = (n + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]                      # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:n]


def site_dims(Ly: int, Lx: int, y: int, x: int, D: int):
    """Effective (up, left, down, right) dimensions of site (y, x) under OBC."""
    return (1 if y == 0 else D, 1 if x == 0 else D,
            1 if y == Ly - 1 else D, 1 if x == Lx - 1 else D)


def _fill(Ly: int, Lx: int, d: int, D: int, values: np.ndarray) -> np.ndarray:
    A = np.zeros((Ly, Lx, d, D, D, D, D))
    pos = 0
    for y in range(Ly):
        for x in range(Lx):
            du, dl, dd, dr = site_dims(Ly, Lx, y, x, D)
            n = d * du * dl * dd * dr
            t = values[pos:pos + n].reshape(d, du, dl, dd, dr)
            pos += n
            nrm = np.linalg.norm(t)
            A[y, x, :, :du, :dl, :dd, :dr] = t / nrm
    return A


def _count(Ly: int, Lx: int, d: int, D: int) -> int:
    n = 0
    for y in range(Ly):
        for x in range(Lx):
            n += d * int(np.prod(site_dims(Ly, Lx, y, x, D)))
    return n


def peps_uniform(Ly: int, Lx: int, d: int, D: int, seed: int) -> np.ndarray:
    """Entries i.i.d. uniform[0,1), each tensor scaled to unit norm."""
    return _fill(Ly, Lx, d, D, uniform01(seed, _count(Ly, Lx, d, D)))


def peps_gauss(Ly: int, Lx: int, d: int, D: int, seed: int,
               mean: float = 0.5, std: float = 0.1) -> np.ndarray:
    """Entries ``mean + std*N(0,1)``, each tensor scaled to unit norm."""
    z = normal(seed, _count(Ly, Lx, d, D))
    return _fill(Ly, Lx, d, D, mean + std * z)


def peps_product(Ly: int, Lx: int, d: int, seed: int) -> np.ndarray:
    """A D=1 product state: site vectors a_i with entries uniform[-1,1)."""
    u = uniform01(seed, Ly * Lx * d) * 2.0 - 1.0
    return u.reshape(Ly, Lx, d, 1, 1, 1, 1).copy()


def random_gauge(D: int, seed: int, eps: float = 0.3) -> np.ndarray:
    """A well-conditioned invertible D x D matrix ``I + eps*U`` (gauge tests)."""
    u = uniform01(seed, D * D).reshape(D, D) * 2.0 - 1.0
    return np.eye(D) + eps * u / max(1.0, np.linalg.norm(u, 2))


# Named workloads: (Ly, Lx, d, D, generator).
WORKLOADS = {
    "4x4_D2": dict(Ly=4, Lx=4, d=2, D=2, gen="uniform", seed=1),
    "10x10_D4": dict(Ly=10, Lx=10, d=2, D=4, gen="gauss", seed=2),
    "14x14_D6": dict(Ly=14, Lx=14, d=2, D=6, gen="gauss", seed=3),
    "20x20_D8": dict(Ly=20, Lx=20, d=2, D=8, gen="gauss", seed=4),
    "16x16_D4": dict(Ly=16, Lx=16, d=2, D=4, gen="gauss", seed=5),
    "20x20_D8_su": dict(Ly=20, Lx=20, d=2, D=8, gen="su", seed=4),
    "16x16_D4_su": dict(Ly=16, Lx=16, d=2, D=4, gen="su", seed=5),
    "20x20_D4_su": dict(Ly=20, Lx=20, d=2, D=4, gen="su", seed=6),
}


def workload(name: str, seed: int | None = None) -> np.ndarray:
    w = WORKLOADS[name]
    s = w["seed"] if seed is None else seed
    if w["gen"] == "uniform":
        return peps_uniform(w["Ly"], w["Lx"], w["d"], w["D"], s)
    if w["gen"] == "su":
        return peps_simple_update(w["Ly"], w["Lx"], w["D"], s)
    return peps_gauss(w["Ly"], w["Lx"], w["d"], w["D"], s)


# ---------------------------------------------------------------------------
# Simple-update imaginary-time evolution (input generator for the 20x20 D=8
# and 16x16 D=4 workloads).  Section 3: tensors Gamma with diagonal bond
# weights lambda; a nearest-neighbour gate acts on a pair using only the six
# lambdas around it.  First-order Trotter over four bond sets (horizontal even
# / odd columns, vertical even / odd rows); lambda normalised to lambda_1 = 1;
# the start is a Neel product state whose zero entries are replaced by uniform
# noise in [-0.01, 0.01] (Appendix B).  The PEPS handed out is A = Gamma with
# sqrt(lambda) absorbed on every bond, each tensor scaled to unit norm.
# Dense padded storage: outward (OBC) legs carry lambda = (1, 0, ..., 0).
# ---------------------------------------------------------------------------
def _heisenberg_gate(tau: float) -> np.ndarray:
    """exp(-tau S.S) as a 4x4 matrix on (s_1, s_2)."""
    h = 0.25 * np.array([[1.0, 0, 0, 0], [0, -1.0, 2.0, 0], [0, 2.0, -1.0, 0], [0, 0, 0, 1.0]])
    w, v = np.linalg.eigh(h)
    return (v * np.exp(-tau * w)) @ v.T


def _qr_pos(M):
    """Batched thin QR with a non-negative diagonal of R: the factors no longer
    depend on the sign convention of the LAPACK that computes them."""
    Q, R = np.linalg.qr(M)
    s = np.where(np.diagonal(R, axis1=1, axis2=2) < 0, -1.0, 1.0)
    return Q * s[:, None, :], R * s[:, :, None]


def _svd_signed(M):
    """Batched SVD with the largest-magnitude entry of every left singular
    vector positive (the right vectors flipped with them)."""
    U, S, Vt = np.linalg.svd(M)
    idx = np.argmax(np.abs(U), axis=1)                                  # (n, k)
    piv = np.take_along_axis(U, idx[:, None, :], axis=1)[:, 0, :]
    s = np.where(piv < 0, -1.0, 1.0)
    return U * s[:, None, :], S, Vt * s[:, :, None]


def _su_pair(Ga, Gb, lam_a, lam_b, lam_ab, gate, D):
    """Batched simple update of horizontal pairs.

    Ga, Gb: (n, d, D, D, D, D) [s, u, l, dn, r]; lam_a = (up, left, down) of the
    left site, lam_b = (up, down, right) of the right site, each (n, D);
    lam_ab: (n, D).  Returns new Ga, Gb, lam_ab.
    """
    n, d = Ga.shape[0], Ga.shape[1]
    inv = lambda l: np.where(l > 0, 1.0 / np.where(l > 0, l, 1.0), 0.0)
    lu, ll, ld = lam_a
    ru, rd, rr = lam_b
    A = Ga * lu[:, None, :, None, None, None] * ll[:, None, None, :, None, None] \
        * ld[:, None, None, None, :, None] * lam_ab[:, None, None, None, None, :]
    B = Gb * ru[:, None, :, None, None, None] * rd[:, None, None, None, :, None] \
        * rr[:, None, None, None, None, :]
    # QR-reduce the outer legs: A -> [(u,l,dn), (s,r)], B -> [(u,dn,r), (t,l)]
    Am = A.transpose(0, 2, 3, 4, 1, 5).reshape(n, D ** 3, d * D)
    Bm = B.transpose(0, 2, 4, 5, 1, 3).reshape(n, D ** 3, d * D)
    Qa, Ra = _qr_pos(Am)                              # Ra: (n, k, d*D)
    Qb, Rb = _qr_pos(Bm)
    k = Ra.shape[1]
    # shared bond contracted: th[a,s,b,t] = sum_r Ra[a,s,r] Rb[b,t,r]
    th = np.matmul(Ra.reshape(n, k * d, D), Rb.reshape(n, k * d, D).transpose(0, 2, 1))
    # gate on (s, t): th'[a,p,b,q] = sum_st G[p,q,s,t] th[a,s,b,t]
    th = th.reshape(n, k, d, k, d).transpose(0, 1, 3, 2, 4).reshape(n * k * k, d * d)
    th = (th @ gate.T).reshape(n, k, k, d, d).transpose(0, 1, 3, 2, 4).reshape(n, k * d, k * d)
    U, S, Vt = _svd_signed(th)
    S = S[:, :D]
    lam = S / S[:, :1]
    Ua = U[:, :, :D]                                  # [(a, s'), r]
    Vb = Vt[:, :D, :]                                 # [r, (b, t')]
    # back to site tensors: An[i,s',r] = sum_a Qa[i,a] Ua[a,s',r], Bn[i,t',r] likewise
    An = np.matmul(Qa, Ua.reshape(n, k, d * D)).reshape(n, D, D, D, d, D)
    Bn = np.matmul(Qb, Vb.reshape(n, D, k, d).transpose(0, 2, 3, 1).reshape(n, k, d * D)).reshape(n, D, D, D, d, D)
    Ga = An.transpose(0, 4, 1, 2, 3, 5) * inv(lu)[:, None, :, None, None, None] \
        * inv(ll)[:, None, None, :, None, None] * inv(ld)[:, None, None, None, :, None]
    # Bn: [(u, dn, r), t, l] -> [t, u, l, dn, r]
    Gb = Bn.transpose(0, 4, 1, 5, 2, 3) * inv(ru)[:, None, :, None, None, None] \
        * inv(rd)[:, None, None, None, :, None] * inv(rr)[:, None, None, None, None, :]
    return Ga, Gb, lam


_POOL = None


def _su_pairs(Ga, Gb, lam_a, lam_b, lam_ab, gate, D):
    """_su_pair over chunks of the independent pairs on a thread pool (numpy's
    batched linear algebra runs one matrix at a time and releases the GIL);
    every pair's arithmetic is the same as in one batch."""
    global _POOL
    import concurrent.futures as cf
    import os
    n = Ga.shape[0]
    workers = min(16, os.cpu_count() or 1)
    if workers <= 1 or n < 2 * workers:
        return _su_pair(Ga, Gb, lam_a, lam_b, lam_ab, gate, D)
    if _POOL is None:
        _POOL = cf.ThreadPoolExecutor(max_workers=workers)
    cuts = np.linspace(0, n, workers + 1).astype(int)
    parts = [(a, b) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
    futs = [_POOL.submit(_su_pair, Ga[a:b], Gb[a:b], tuple(l[a:b] for l in lam_a),
                         tuple(l[a:b] for l in lam_b), lam_ab[a:b], gate, D) for a, b in parts]
    res = [f.result() for f in futs]
    return tuple(np.concatenate([r[i] for r in res]) for i in range(3))


def peps_simple_update(Ly: int, Lx: int, D: int, seed: int, tau: float = 0.01, steps: int = 400,
                       d: int = 2) -> np.ndarray:
    """Seeded simple-update ground-state approximation of the spin-1/2
    Heisenberg model (eq. 2), returned as dense OBC tensors."""
    assert d == 2
    rng_u = uniform01(seed, Ly * Lx * d * D ** 4) * 0.02 - 0.01
    G = rng_u.reshape(Ly, Lx, d, D, D, D, D).copy()
    for y in range(Ly):
        for x in range(Lx):
            du, dl, dd, dr = site_dims(Ly, Lx, y, x, D)
            mask = np.zeros((d, D, D, D, D), dtype=bool)
            mask[:, :du, :dl, :dd, :dr] = True
            G[y, x][~mask] = 0.0
            G[y, x, (x + y) % 2, 0, 0, 0, 0] = 1.0        # Neel product state
    e1 = np.zeros(D)
    e1[0] = 1.0
    lh = np.zeros((Ly, max(Lx - 1, 0), D))
    lh[..., :] = 1.0
    lv = np.ones((max(Ly - 1, 0), Lx, D))
    gate = _heisenberg_gate(tau)

    def lam_up(y, x):
        return lv[y - 1, x] if y > 0 else e1

    def lam_dn(y, x):
        return lv[y, x] if y < Ly - 1 else e1

    def lam_lt(y, x):
        return lh[y, x - 1] if x > 0 else e1

    def lam_rt(y, x):
        return lh[y, x] if x < Lx - 1 else e1

    def hset(par):
        return [(y, x) for y in range(Ly) for x in range(par, Lx - 1, 2)]

    def vset(par):
        return [(y, x) for y in range(par, Ly - 1, 2) for x in range(Lx)]

    for _ in range(steps):
        for par in (0, 1):
            bonds = hset(par)
            if bonds:
                ys, xs = zip(*bonds)
                ys, xs = np.array(ys), np.array(xs)
                Ga, Gb = G[ys, xs], G[ys, xs + 1]
                la = (np.stack([lam_up(y, x) for y, x in bonds]), np.stack([lam_lt(y, x) for y, x in bonds]),
                      np.stack([lam_dn(y, x) for y, x in bonds]))
                lb = (np.stack([lam_up(y, x + 1) for y, x in bonds]), np.stack([lam_dn(y, x + 1) for y, x in bonds]),
                      np.stack([lam_rt(y, x + 1) for y, x in bonds]))
                Ga, Gb, lam = _su_pairs(Ga, Gb, la, lb, lh[ys, xs], gate, D)
                G[ys, xs], G[ys, xs + 1], lh[ys, xs] = Ga, Gb, lam
        for par in (0, 1):
            bonds = vset(par)
            if bonds:
                # a vertical pair is a horizontal pair of the transposed lattice:
                # [s,u,l,dn,r] -> [s,l,u,r,dn]
                ys, xs = zip(*bonds)
                ys, xs = np.array(ys), np.array(xs)
                Ga = G[ys, xs].transpose(0, 1, 3, 2, 5, 4)
                Gb = G[ys + 1, xs].transpose(0, 1, 3, 2, 5, 4)
                la = (np.stack([lam_lt(y, x) for y, x in bonds]), np.stack([lam_up(y, x) for y, x in bonds]),
                      np.stack([lam_rt(y, x) for y, x in bonds]))
                lb = (np.stack([lam_lt(y + 1, x) for y, x in bonds]), np.stack([lam_rt(y + 1, x) for y, x in bonds]),
                      np.stack([lam_dn(y + 1, x) for y, x in bonds]))
                Ga, Gb, lam = _su_pairs(Ga, Gb, la, lb, lv[ys, xs], gate, D)
                G[ys, xs] = Ga.transpose(0, 1, 3, 2, 5, 4)
                G[ys + 1, xs] = Gb.transpose(0, 1, 3, 2, 5, 4)
                lv[ys, xs] = lam
    A = G.copy()
    for y in range(Ly):
        for x in range(Lx):
            t = A[y, x]
            t = t * np.sqrt(lam_up(y, x))[None, :, None, None, None] * np.sqrt(lam_lt(y, x))[None, None, :, None, None] \
                * np.sqrt(lam_dn(y, x))[None, None, None, :, None] * np.sqrt(lam_rt(y, x))[None, None, None, None, :]
            A[y, x] = t / np.linalg.norm(t)
    return A


def gram4(A: np.ndarray) -> float:
    """Fingerprint of a dense lattice that survives a change of bond gauge: a
    weighted sum over sites and legs k of Tr(G_k^2), G_k = M_k M_k^T with M_k
    the site tensor matricised as (leg k) x (the other legs).  Inserting an
    orthogonal matrix and its transpose on a bond leaves it unchanged.  The
    simple-update generator fixes a bond's gauge only up to such a rotation
    inside a block of equal singular values (the Heisenberg model's spin
    symmetry makes them), and which rotation LAPACK returns there differs
    between platforms: the bytes are not portable, this sum is."""
    Ly, Lx = A.shape[:2]
    w = uniform01(98, Ly * Lx * 5).reshape(Ly, Lx, 5)
    tot = 0.0
    for y in range(Ly):
        for x in range(Lx):
            T = A[y, x]
            for k in range(5):
                M = np.moveaxis(T, k, 0).reshape(T.shape[k], -1)
                G = M @ M.T
                tot += float(w[y, x, k] * np.sum(G * G))
    return tot
