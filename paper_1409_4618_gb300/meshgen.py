"""Seeded synthetic meshes and per-element / per-DOF input vectors.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle's tests. It holds no finite-element arithmetic: it only lays out
node coordinates and element connectivity and draws random numbers.

Mesh families (the workloads of Sec. 3.3, Tables 1-2, and Sec. 4):

* ``kuhn_cube(n)``: the unit cube split into n^3 cubes, each cut into six
  tetrahedra along the main diagonal (Kuhn / Freudenthal split). The level-L
  cube of Table 2 is n = 6 * 2**(L-1): its face and edge counts are exactly
  the matrix sizes printed there.
* ``kuhn_square(n)``: the unit square split into n^2 squares, each cut into
  two triangles along the "/" diagonal (Tables 3 and 5 use this family).
* ``lshape(level)``: the L-shaped domain (0,1)^2 minus (1/2,1)^2 of Table 1,
  6 * 4**level triangles.

Numbering: node id = i + (n+1)*(j + (n+1)*k) (x fastest); cube id =
i + n*(j + n*k); the six tetrahedra of a cube follow the axis permutations
(0,1,2), (0,2,1), (1,0,2), (1,2,0), (2,0,1), (2,1,0) and list their nodes in
path order from the cube's lower corner, so half of them have det B_K < 0.

Randomness is counter based (SplitMix64 finaliser applied to seed, stream and
index), so every value can be regenerated independently of how many others
were drawn.  Streams: 0-2 jitter of x/y/z, 3 element coefficient, 4-5 the
vector ``u``, 6-7 the vector ``v``, 8 batched mesh sizes.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_JITTER = 0
STREAM_COEFF = 3
STREAM_U = 4
STREAM_V = 6
STREAM_SIZES = 8

_KUHN_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea, Flood 2014)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, index) -> np.ndarray:
    """U[0,1) doubles for the given counters (53 random bits each)."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        key = _mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + _GOLDEN * np.uint64(stream + 1))
        z = _mix64(key + _GOLDEN * (idx + np.uint64(1)))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """N(0,1) doubles by Box-Muller from two uniform streams (stream, stream+1)."""
    i = np.arange(n, dtype=np.uint64)
    u1 = 1.0 - uniform(seed, stream, i)          # (0, 1]
    u2 = uniform(seed, stream + 1, i)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def log_uniform_coeff(seed: int, n_elems: int, lo: float = 0.1, hi: float = 10.0) -> np.ndarray:
    """Per-element coefficient, log-uniform in [lo, hi]."""
    u = uniform(seed, STREAM_COEFF, np.arange(n_elems, dtype=np.uint64))
    return np.exp(np.log(lo) + (np.log(hi) - np.log(lo)) * u)


def _jitter(nodes: np.ndarray, interior: np.ndarray, amount: float, seed: int) -> np.ndarray:
    ids = np.nonzero(interior)[0].astype(np.uint64)
    for c in range(nodes.shape[1]):
        u = uniform(seed, STREAM_JITTER + c, ids)
        nodes[interior, c] += (2.0 * u - 1.0) * amount
    return nodes


def kuhn_cube(n: int, jitter: float = 0.0, seed: int = 0):
    """Unit cube, n^3 cubes x 6 tetrahedra. ``jitter`` is a fraction of h = 1/n
    applied uniformly to each coordinate of interior nodes only.

    Returns (nodes float64 [V,3], elems int32 [T,4])."""
    if n < 1:
        raise ValueError("n must be >= 1")
    h = 1.0 / n
    m = n + 1
    k, j, i = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    nodes = np.stack([i.ravel() * h, j.ravel() * h, k.ravel() * h], axis=1).astype(np.float64)
    # exact boundary values (the domain stays the unit cube)
    nodes[np.stack([i.ravel(), j.ravel(), k.ravel()], 1) == n] = 1.0
    if jitter:
        ii, jj, kk = i.ravel(), j.ravel(), k.ravel()
        interior = (ii > 0) & (ii < n) & (jj > 0) & (jj < n) & (kk > 0) & (kk < n)
        nodes = _jitter(nodes, interior, jitter * h, seed)
    ck, cj, ci = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    step = (1, m, m * m)
    base = ci + m * (cj + m * ck)
    elems = np.empty((n ** 3, 6, 4), dtype=np.int64)
    for t, perm in enumerate(_KUHN_PERMS):
        cur = base.copy()
        elems[:, t, 0] = cur
        for s, ax in enumerate(perm):
            cur = cur + step[ax]
            elems[:, t, s + 1] = cur
    return nodes, elems.reshape(-1, 4).astype(np.int32)


def kuhn_square(n: int, jitter: float = 0.0, seed: int = 0):
    """Unit square, n^2 squares x 2 triangles along the "/" diagonal.

    Returns (nodes float64 [V,2], elems int32 [T,3])."""
    if n < 1:
        raise ValueError("n must be >= 1")
    h = 1.0 / n
    m = n + 1
    j, i = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    nodes = np.stack([i.ravel() * h, j.ravel() * h], axis=1).astype(np.float64)
    nodes[np.stack([i.ravel(), j.ravel()], 1) == n] = 1.0
    if jitter:
        ii, jj = i.ravel(), j.ravel()
        interior = (ii > 0) & (ii < n) & (jj > 0) & (jj < n)
        nodes = _jitter(nodes, interior, jitter * h, seed)
    cj, ci = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    base = (ci + m * cj).ravel()
    elems = np.empty((n * n, 2, 3), dtype=np.int64)
    step = (1, m)
    for t, perm in enumerate(((0, 1), (1, 0))):
        cur = base.copy()
        elems[:, t, 0] = cur
        for s, ax in enumerate(perm):
            cur = cur + step[ax]
            elems[:, t, s + 1] = cur
    return nodes, elems.reshape(-1, 3).astype(np.int32)


def lshape(level: int):
    """L-shaped domain (0,1)^2 minus (1/2,1)^2 of Table 1: a 2m x 2m grid of
    squares (m = 2**level) without the upper-right m x m block, two triangles
    per square, 6 * 4**level triangles."""
    m = 2 ** level
    nodes_full, elems_full = kuhn_square(2 * m)
    g = 2 * m + 1
    # drop the squares whose lower corner is in the removed quadrant
    sq = np.arange((2 * m) ** 2)
    si, sj = sq % (2 * m), sq // (2 * m)
    keep_sq = ~((si >= m) & (sj >= m))
    keep_el = np.repeat(keep_sq, 2)
    elems = elems_full[keep_el]
    used = np.zeros(g * g, dtype=bool)
    used[elems.ravel()] = True
    new_id = np.cumsum(used) - 1
    return nodes_full[used].copy(), new_id[elems].astype(np.int32)


def batch_sizes(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Grid sizes n_b ~ U{lo..hi} for a batch of cube meshes."""
    u = uniform(seed, STREAM_SIZES, np.arange(count, dtype=np.uint64))
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


def shuffle_local_order(elems: np.ndarray, seed: int) -> np.ndarray:
    """Randomly permute the local node order of every element (changes the
    sign of det B_K for odd permutations)."""
    T, nv = elems.shape
    keys = uniform(seed, 9, np.arange(T * nv, dtype=np.uint64)).reshape(T, nv)
    order = np.argsort(keys, axis=1, kind="stable")
    return np.take_along_axis(elems, order, axis=1).astype(np.int32)
