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
}


def workload(name: str, seed: int | None = None) -> np.ndarray:
    w = WORKLOADS[name]
    s = w["seed"] if seed is None else seed
    if w["gen"] == "uniform":
        return peps_uniform(w["Ly"], w["Lx"], w["d"], w["D"], s)
    return peps_gauss(w["Ly"], w["Lx"], w["d"], w["D"], s)
