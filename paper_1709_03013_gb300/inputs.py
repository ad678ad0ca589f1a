"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds workload recipes only -- sizes, seeds, arrival times and a few
hand-made orders given as 0/1 matrices -- and none of the method's arithmetic.
The sprinkled coordinates themselves are drawn by each side's own counter-based
generator from (seed, seq); this module only decides which (d, N, seed, seq)
each set or request gets.

Workloads (the paper's own benchmarks use synthetic sprinkles, Sec. 5.1):
  * single sets: d=2 N=2048 seed 0; d=4 N=65536 seed 1; d=2 N=131072 seed 2
  * batch: 4096 diamonds, d alternating 2/4 (even index -> d=2), N log-uniform in
    [256, 8192] from seed 3, set s sprinkled with (seed=3, seq=s)
  * serve: 20000 requests, d in {2,4} 50/50, N log-uniform in [1024, 65536], Poisson
    arrivals, from seed 4; request r sprinkled with (seed=4, seq=r)
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SINGLE_CONFIGS = {
    "d2_n2048": dict(d=2, N=2048, seed=0),
    "d4_n65536": dict(d=4, N=65536, seed=1),
    "d2_n131072": dict(d=2, N=131072, seed=2),
}


@dataclass(frozen=True)
class SetSpec:
    d: int
    N: int
    seed: int
    seq: int


def log_uniform_sizes(n: int, lo: int, hi: int, rng: np.random.Generator) -> np.ndarray:
    """N = floor(exp(U[ln lo, ln hi])), clipped to [lo, hi]."""
    x = rng.uniform(np.log(lo), np.log(hi), size=n)
    return np.clip(np.floor(np.exp(x)).astype(np.int64), lo, hi)


def batch_workload(n_sets: int = 4096, seed: int = 3, lo: int = 256, hi: int = 8192) -> list[SetSpec]:
    """Many independent diamonds of uneven size: d alternates 2/4, N log-uniform."""
    rng = np.random.default_rng(seed)
    sizes = log_uniform_sizes(n_sets, lo, hi, rng)
    return [SetSpec(d=2 if s % 2 == 0 else 4, N=int(sizes[s]), seed=seed, seq=s)
            for s in range(n_sets)]


@dataclass(frozen=True)
class Request:
    arrival_s: float
    spec: SetSpec


def serve_workload(n_req: int = 20000, rate_per_s: float = 90.0, seed: int = 4,
                   lo: int = 1024, hi: int = 65536) -> list[Request]:
    """Poisson arrivals (exponential gaps at the given rate), d in {2,4} 50/50,
    N log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    ds = np.where(rng.random(n_req) < 0.5, 2, 4)
    sizes = log_uniform_sizes(n_req, lo, hi, rng)
    gaps = rng.exponential(1.0 / rate_per_s, size=n_req)
    t = np.cumsum(gaps) - gaps[0]
    return [Request(float(t[r]), SetSpec(int(ds[r]), int(sizes[r]), seed, r)) for r in range(n_req)]


# ------------------------------------------------------------ hand-made orders

def chain_rel(N: int) -> np.ndarray:
    """A total order: every pair related (symmetric 0/1 matrix, zero diagonal)."""
    rel = np.ones((N, N), dtype=np.uint8)
    np.fill_diagonal(rel, 0)
    return rel


def antichain_rel(N: int) -> np.ndarray:
    """No pair related."""
    return np.zeros((N, N), dtype=np.uint8)


def rel_from_edges(N: int, edges) -> np.ndarray:
    rel = np.zeros((N, N), dtype=np.uint8)
    for i, j in edges:
        rel[i, j] = rel[j, i] = 1
    return rel


def random_upper_rel(N: int, p: float, seed: int) -> np.ndarray:
    """Symmetric 0/1 matrix whose upper triangle is Bernoulli(p): an arbitrary
    time-ordered relation matrix (not transitively closed), the kind of input
    the action accepts from any source (Sec. 1.3: any adjacency matrix)."""
    rng = np.random.default_rng(seed)
    up = np.triu((rng.random((N, N)) < p).astype(np.uint8), 1)
    return up | up.T


def layered_order_rel(N: int, seed: int, p: float = 0.5) -> np.ndarray:
    """A three-layer order in the style of Kleitman-Rothschild (sizes N/4, N/2, N/4):
    random relations between adjacent layers, all pairs of layers 1 and 3 related."""
    rng = np.random.default_rng(seed)
    a, b = N // 4, N // 4 + N // 2
    rel = np.zeros((N, N), dtype=np.uint8)
    rel[:a, a:b] = rng.random((a, b - a)) < p
    rel[a:b, b:] = rng.random((b - a, N - b)) < p
    rel[:a, b:] = 1
    return rel | rel.T


def pack_rows(rel: np.ndarray, stride_words: int) -> np.ndarray:
    """Bit-pack a 0/1 matrix into uint64 rows: bit k of row i at word k//64,
    bit k%64 (LSB first), rows padded with zero words to stride_words."""
    N = rel.shape[0]
    bits = np.zeros((N, stride_words * 64), dtype=np.uint8)
    bits[:, :N] = rel
    packed = np.packbits(bits, axis=1, bitorder="little")
    return packed.view(np.uint64).reshape(N, stride_words).copy()


# ------------------------------------------------------- light-cone stress sets

def light_cone_coords(d: int, N: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Unsorted coordinates [4, N] crowded onto light cones, for the link's tie-breaking.

    A quarter of the elements are base points on a dyadic grid (multiples of 2^-21 in
    [-1/2, 1/2]); every other element copies a base point and moves it by an exactly null
    displacement (d=4: along an axis, or along 3-4-5 and 1-2-2 directions; d=2: a step in
    u or v only), after which a third of them are nudged by one unit in the last place in
    one coordinate, and a few are exact duplicates or carry signed zeros.  Products of the
    grid values with `scale` (1 or an integer below 2^31) stay exact.  d=4 rows are
    t, x, y, z; d=2 rows are t, x, u, v with t = (u + v) / 2, x = (v - u) / 2.
    """
    rng = np.random.default_rng(seed)
    g = 2.0 ** -21
    nb = max(1, N // 4)
    c = np.zeros((4, N), dtype=np.float64)
    if d == 4:
        c[:, :nb] = rng.integers(-2 ** 20, 2 ** 20, size=(4, nb)) * g
        for e in range(nb, N):
            b = int(rng.integers(0, nb))
            p = c[:, b].copy()
            mode = int(rng.integers(0, 4))
            if mode == 0:                                   # along an axis
                dt = int(rng.integers(1, 2 ** 18)) * g
                a = 1 + int(rng.integers(0, 3))
                p[0] += dt
                p[a] += dt if rng.random() < 0.5 else -dt
            elif mode == 1:                                 # 3-4-5 direction
                dl = int(rng.integers(1, 2 ** 15)) * g
                ax = rng.permutation(3)[:2] + 1
                p[0] += 5 * dl
                p[ax[0]] += 3 * dl * (1 if rng.random() < 0.5 else -1)
                p[ax[1]] += 4 * dl * (1 if rng.random() < 0.5 else -1)
            elif mode == 2:                                 # 1-2-2 direction
                dl = int(rng.integers(1, 2 ** 15)) * g
                sg = np.where(rng.random(3) < 0.5, 1.0, -1.0)
                p[0] += 3 * dl
                p[1:] += dl * sg * np.array([1.0, 2.0, 2.0])
            # mode 3: exact duplicate of the base point
            if mode != 3 and rng.random() < 1 / 3:
                a = int(rng.integers(0, 4))
                p[a] = np.nextafter(p[a], np.inf if rng.random() < 0.5 else -np.inf)
            c[:, e] = p
    else:
        uv = rng.integers(-2 ** 20, 2 ** 20, size=(2, nb)) * g
        c[2:, :nb] = uv
        for e in range(nb, N):
            b = int(rng.integers(0, nb))
            u, v = c[2, b], c[3, b]
            mode = int(rng.integers(0, 4))
            step = int(rng.integers(1, 2 ** 18)) * g
            if mode == 0:
                v += step                                   # equal u: null, unrelated
            elif mode == 1:
                u += step                                   # equal v
            elif mode == 2:                                 # u equal in float, not in double
                u += 2.0 ** -45
                v += step
            if rng.random() < 1 / 3:
                v = np.nextafter(v, np.inf if rng.random() < 0.5 else -np.inf)
            c[2, e], c[3, e] = u, v
        zs = rng.choice(N, size=max(1, N // 50), replace=False)
        c[2, zs[: len(zs) // 2]] = -0.0
        c[2, zs[len(zs) // 2:]] = 0.0
        c[0] = (c[2] + c[3]) / 2
        c[1] = (c[3] - c[2]) / 2
    return c * scale
