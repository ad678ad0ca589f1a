"""CPU oracle for the causal-set hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct statement of what the GPU library computes
(Cunningham & Krioukov, arXiv:1709.03013, Secs. 2.1-2.2 and 4.1-4.2, Eq. s_local),
written in plain C (``csg_oracle.c``) and loaded here with ctypes.  Only the
test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It shares no code with the CUDA library, and the
library never imports it.

Every array crossing this module is a numpy array on the host:
  coords   float64 [4, N]  (d=2 rows t, x, u, v; d=4 rows t, x, y, z)
  rel      uint8   [N, N]  symmetric 0/1 adjacency matrix, zero diagonal
  words    uint64  [N, stride] bit-packed rows (bit k of row i at word k//64)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csg_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libcsg_oracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, EREJECT = 0, -1, -2, -3
DS2 = 3  # geometry code of the 1+1 de Sitter slab (Sec. 5.1); 2 and 4 are the flat diamonds


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FMA contraction) and return the .so path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    # -O3 lets gcc vectorise the integer triple loop (integer sums are exact in any order);
    # floating-point code keeps its written order (no fast-math, no contraction)
    cmd = ["gcc", "-O3", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, u64, i32, dbl = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
        vp = ctypes.c_void_p
        lib.orc_philox4x64_10.argtypes = [vp, vp, vp]
        lib.orc_philox4x64_10.restype = None
        lib.orc_sprinkle.argtypes = [i32, i64, u64, u64, vp, vp]
        lib.orc_sort.argtypes = [i32, i64, vp, vp]
        lib.orc_link.argtypes = [i32, i64, vp, vp, i32]
        lib.orc_link_row.argtypes = [i32, i64, vp, i64, vp]
        lib.orc_related.argtypes = [i32, i64, vp, i64, i64]
        lib.orc_pack.argtypes = [i64, vp, i64, vp]
        lib.orc_interval.argtypes = [i64, vp, i64, i64]
        lib.orc_interval.restype = i64
        lib.orc_interval_coords.argtypes = [i32, i64, vp, i64, i64]
        lib.orc_interval_coords.restype = i64
        lib.orc_action_rows.argtypes = [i64, vp, i64, i64, vp, vp, vp, vp, i32]
        lib.orc_finalize.argtypes = [i32, i64, vp, vp, vp]
        lib.orc_action_rows_coords.argtypes = [i32, i64, vp, i64, i64, vp, vp, vp, vp, i32]
        lib.orc_smeared.argtypes = [i64, vp, dbl]
        lib.orc_sprinkle_desitter.argtypes = [i64, dbl, u64, u64, vp]
        lib.orc_sprinkle_desitter.restype = i32
        lib.orc_smeared.restype = dbl
        lib.orc_dalembertian.argtypes = [i64, vp, vp, dbl, vp, vp, i32]
        lib.orc_dalembertian.restype = i32
        for f in (lib.orc_sprinkle, lib.orc_sort, lib.orc_link, lib.orc_link_row,
                  lib.orc_related, lib.orc_pack, lib.orc_action_rows, lib.orc_finalize,
                  lib.orc_action_rows_coords):
            f.restype = i32
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x64_10(ctr, key) -> np.ndarray:
    """One Philox4x64-10 block: 4-word counter, 2-word key -> 4 uint64 words."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint64).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64).reshape(2))
    out = np.zeros(4, dtype=np.uint64)
    _load().orc_philox4x64_10(_p(c), _p(k), _p(out))
    return out


def sprinkle(d: int, N: int, seed: int, seq: int = 0, with_attempts: bool = False):
    """Unsorted sprinkle into the flat causal diamond (Sec. 2.1): coords [4, N]."""
    coords = np.zeros((4, max(N, 0)), dtype=np.float64)
    att = np.zeros(max(N, 0), dtype=np.int32)
    rc = _load().orc_sprinkle(d, N, seed, seq, _p(coords), _p(att))
    if rc != OK:
        raise RuntimeError(f"orc_sprinkle failed: {rc}")
    return (coords, att) if with_attempts else coords


def sprinkle_desitter(N: int, eta0: float, seed: int, seq: int = 0) -> np.ndarray:
    """Unsorted sprinkle into the 1+1 de Sitter slab of Sec. 5.1: rows eta, theta, 0, 0."""
    coords = np.zeros((4, max(N, 0)), dtype=np.float64)
    rc = _load().orc_sprinkle_desitter(N, eta0, seed, seq, _p(coords))
    if rc != OK:
        raise RuntimeError(f"orc_sprinkle_desitter failed: {rc}")
    return coords


def sort(d: int, coords: np.ndarray):
    """Time order (Sec. 2.2): returns (sorted coords [4, N], perm) with perm[p] = sprinkle index."""
    c = np.ascontiguousarray(coords, dtype=np.float64).copy()
    N = c.shape[1]
    perm = np.zeros(N, dtype=np.int64)
    rc = _load().orc_sort(d, N, _p(c), _p(perm))
    if rc != OK:
        raise RuntimeError(f"orc_sort failed: {rc}")
    return c, perm


def sprinkle_sorted(d: int, N: int, seed: int, seq: int = 0) -> np.ndarray:
    return sort(d, sprinkle(d, N, seed, seq))[0]


def link(d: int, coords: np.ndarray, threads: int = 0) -> np.ndarray:
    """Dense symmetric 0/1 adjacency matrix [N, N] of sorted coordinates (Sec. 2.2)."""
    c = np.ascontiguousarray(coords, dtype=np.float64)
    N = c.shape[1]
    rel = np.zeros((N, N), dtype=np.uint8)
    rc = _load().orc_link(d, N, _p(c), _p(rel), threads)
    if rc != OK:
        raise RuntimeError(f"orc_link failed: {rc}")
    return rel


def link_row(d: int, coords: np.ndarray, i: int) -> np.ndarray:
    c = np.ascontiguousarray(coords, dtype=np.float64)
    N = c.shape[1]
    row = np.zeros(N, dtype=np.uint8)
    rc = _load().orc_link_row(d, N, _p(c), i, _p(row))
    if rc != OK:
        raise RuntimeError(f"orc_link_row failed: {rc}")
    return row


def related(d: int, coords: np.ndarray, i: int, j: int) -> bool:
    c = np.ascontiguousarray(coords, dtype=np.float64)
    return bool(_load().orc_related(d, c.shape[1], _p(c), i, j))


def stride_words(N: int) -> int:
    """Row stride of the packed layout: ceil(N/64) words rounded up to 16 words (128 bytes)."""
    w = (N + 63) // 64
    return max(16, (w + 15) // 16 * 16)


def pack(rel: np.ndarray, stride: int | None = None) -> np.ndarray:
    """Pack the 0/1 matrix into uint64 rows, LSB-first, zero padding."""
    r = np.ascontiguousarray(rel, dtype=np.uint8)
    N = r.shape[0]
    s = stride_words(N) if stride is None else stride
    words = np.zeros((N, s), dtype=np.uint64)
    rc = _load().orc_pack(N, _p(r), s, _p(words))
    if rc != OK:
        raise RuntimeError(f"orc_pack failed: {rc}")
    return words


def interval(rel: np.ndarray, i: int, j: int) -> int:
    r = np.ascontiguousarray(rel, dtype=np.uint8)
    return int(_load().orc_interval(r.shape[0], _p(r), i, j))


def interval_coords(d: int, coords: np.ndarray, i: int, j: int) -> int:
    c = np.ascontiguousarray(coords, dtype=np.float64)
    return int(_load().orc_interval_coords(d, c.shape[1], _p(c), i, j))


def action(rel: np.ndarray, threads: int = 0, rows: tuple[int, int] | None = None) -> dict:
    """Interval abundances by the triple loop (Secs. 4.1-4.2).

    Returns dict(hist=uint64[max(N,1)], Nk=uint64[4], R, sum_m, W)."""
    r = np.ascontiguousarray(rel, dtype=np.uint8)
    N = r.shape[0]
    lo, hi = (0, N) if rows is None else rows
    hist = np.zeros(max(N, 1), dtype=np.uint64)
    R = np.zeros(1, np.uint64)
    S = np.zeros(1, np.uint64)
    W = np.zeros(1, np.uint64)
    rc = _load().orc_action_rows(N, _p(r), lo, hi, _p(hist), _p(R), _p(S), _p(W), threads)
    if rc != OK:
        raise RuntimeError(f"orc_action_rows failed: {rc}")
    Nk = np.zeros(4, np.uint64)
    n = min(4, hist.shape[0])
    Nk[:n] = hist[:n]
    return dict(hist=hist, Nk=Nk, R=int(R[0]), sum_m=int(S[0]), W=int(W[0]))


def action_rows_coords(d: int, coords: np.ndarray, lo: int, hi: int, threads: int = 0) -> dict:
    """Abundances of rows [lo, hi) straight from sorted coordinates (no N x N matrix)."""
    c = np.ascontiguousarray(coords, dtype=np.float64)
    N = c.shape[1]
    hist = np.zeros(max(N, 1), dtype=np.uint64)
    R = np.zeros(1, np.uint64)
    S = np.zeros(1, np.uint64)
    W = np.zeros(1, np.uint64)
    rc = _load().orc_action_rows_coords(d, N, _p(c), lo, hi, _p(hist), _p(R), _p(S), _p(W), threads)
    if rc != OK:
        raise RuntimeError(f"orc_action_rows_coords failed: {rc}")
    Nk = np.zeros(4, np.uint64)
    n = min(4, hist.shape[0])
    Nk[:n] = hist[:n]
    return dict(hist=hist, Nk=Nk, R=int(R[0]), sum_m=int(S[0]), W=int(W[0]))


def finalize(d: int, N: int, Nk) -> tuple[int, float]:
    """(combo, S): S2 = 2(N-2N0+4N1-2N2) (Eq. s_local); S4 = (4/sqrt6)(N-N0+9N1-16N2+8N3)."""
    nk = np.ascontiguousarray(np.asarray(Nk, dtype=np.uint64).reshape(4))
    combo = np.zeros(1, np.int64)
    S = np.zeros(1, np.float64)
    rc = _load().orc_finalize(d, N, _p(nk), _p(combo), _p(S))
    if rc != OK:
        raise RuntimeError(f"orc_finalize failed: {rc}")
    return int(combo[0]), float(S[0])


def smeared(N: int, hist: np.ndarray, eps: float) -> float:
    """Smeared action S_eps of Eq. s_smeared from the 0-based histogram (hist[m], m <= N-2)."""
    h = np.zeros(max(N, 1), dtype=np.uint64)
    src = np.asarray(hist, dtype=np.uint64)
    h[:min(len(src), len(h))] = src[:len(h)]
    return float(_load().orc_smeared(N, _p(h), float(eps)))


def dalembertian(rel: np.ndarray, phi, l: float = 1.0, threads: int = 0):
    """Discrete d'Alembertian of Eq. b_local for every element of the time-ordered set
    with relation matrix rel.  Returns (Bphi, L) with L[x] = (|L_1|, |L_2|, |L_3|)."""
    rel = np.ascontiguousarray(rel, dtype=np.uint8)
    N = rel.shape[0]
    ph = np.ascontiguousarray(phi, dtype=np.float64)
    if ph.shape != (N,):
        raise ValueError("phi must have one value per element")
    out = np.zeros(N, dtype=np.float64)
    L = np.zeros((N, 3), dtype=np.int64)
    rc = _load().orc_dalembertian(N, _p(rel), _p(ph), float(l), _p(out), _p(L), threads)
    if rc != 0:
        raise ValueError(f"orc_dalembertian failed ({rc})")
    return out, L


def run(d: int, N: int, seed: int, seq: int = 0, threads: int = 0) -> dict:
    """The whole path on the CPU: sprinkle, sort, link, action, finalize."""
    coords = sprinkle_sorted(d, N, seed, seq)
    rel = link(d, coords, threads)
    out = action(rel, threads)
    combo, S = finalize(d, N, out["Nk"])
    out.update(coords=coords, rel=rel, combo=combo, S=S, d=d, N=N)
    return out
