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
