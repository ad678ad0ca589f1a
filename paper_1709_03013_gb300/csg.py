"""Thin ctypes binding of the C ABI in include/csg.h (argument marshalling only).

Every step of the path runs in the CUDA library ``libcsg.so``; this module only
loads it, converts arguments and results, and raises on error codes.  There is
no CPU fallback: importing the binding fails loudly when the library is missing.
Streams are taken from PyTorch when it is available (``torch.cuda.current_stream``),
which is the only role PyTorch plays here besides device memory.
"""
from __future__ import annotations

import ctypes
from typing import NamedTuple
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcsg.so")

OK, PENDING = 0, 1
E_INVAL, E_NOMEM, E_CUDA, E_TIMEOUT, E_BUSY, E_REJECT, E_NOTFOUND, E_CANCELLED = range(-1, -9, -1)
POPC, TC = 0, 1
TC_FP8, TC_FP4 = 2, 3  # explicit operand formats of the tensor method
MAX_N = 1 << 18


class CsgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class _Result(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("status", ctypes.c_int32), ("N", ctypes.c_int64),
                ("R", ctypes.c_uint64), ("Nk", ctypes.c_uint64 * 4), ("sum_m", ctypes.c_uint64),
                ("W", ctypes.c_uint64), ("combo", ctypes.c_int64), ("S", ctypes.c_double)]


class Result(NamedTuple):
    """One set's counts and action (a csg_result)."""
    d: int
    N: int
    R: int
    Nk: tuple
    sum_m: int
    W: int
    combo: int
    S: float
    status: int = 0

    @staticmethod
    def of(r: _Result) -> "Result":
        return Result(d=r.d, N=r.N, R=r.R, Nk=tuple(int(x) for x in r.Nk), sum_m=r.sum_m, W=r.W,
                      combo=r.combo, S=r.S, status=r.status)


# numpy view of a csg_result array (field offsets as laid out by ctypes)
_RESULT_DTYPE = np.dtype({
    "names": ["d", "status", "N", "R", "Nk", "sum_m", "W", "combo", "S"],
    "formats": [np.int32, np.int32, np.int64, np.uint64, (np.uint64, 4), np.uint64, np.uint64, np.int64,
                np.float64],
    "offsets": [_Result.d.offset, _Result.status.offset, _Result.N.offset, _Result.R.offset,
                _Result.Nk.offset, _Result.sum_m.offset, _Result.W.offset, _Result.combo.offset,
                _Result.S.offset],
    "itemsize": ctypes.sizeof(_Result)})


def _results(buf, n: int) -> list:
    """Result objects of the first n entries of a ctypes csg_result array, converted column
    by column (one Python object per set, no per-field ctypes access)."""
    if n == 0:
        return []
    a = np.frombuffer(buf, dtype=_RESULT_DTYPE, count=n)
    k = a["Nk"]
    nk = list(zip(k[:, 0].tolist(), k[:, 1].tolist(), k[:, 2].tolist(), k[:, 3].tolist()))
    make = tuple.__new__
    return [make(Result, t) for t in zip(a["d"].tolist(), a["N"].tolist(), a["R"].tolist(), nk,
                                         a["sum_m"].tolist(), a["W"].tolist(), a["combo"].tolist(),
                                         a["S"].tolist(), a["status"].tolist())]


EXPORTS = [
    "csg_init", "csg_finalize", "csg_strerror", "csg_last_error", "csg_sprinkle",
    "csg_set_from_coords", "csg_link", "csg_set_from_bitmap", "csg_action", "csg_action_rows",
    "csg_action_hist", "csg_action_batch", "csg_run_batch", "csg_serve_submit", "csg_serve_poll",
    "csg_serve_cancel", "csg_export_coords", "csg_export_bitmap", "csg_set_info", "csg_set_free",
    "csg_action_noalloc", "csg_set_timing", "csg_stage_times", "csg_action_smeared",
    "csg_sprinkle_desitter", "csg_dalembertian", "csg_test_wait_expiry", "csg_test_fail_alloc",
    "csg_measure_popc_rate", "csg_measure_l2_feed", "csg_measure_mma_rate", "csg_check_words",
]

_lib = None


def load(path: str = LIB_PATH):
    """Load libcsg.so and declare its signatures.  Raises if the library is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -c \"import __graft_entry__ as g; "
                          f"g.build()\"` (there is no CPU fallback)")
    L = ctypes.CDLL(path)
    vp, i32, i64, u64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
    pp = ctypes.POINTER(ctypes.c_void_p)
    R = ctypes.POINTER(_Result)
    sig = {
        "csg_init": (i32, [i32, sz, pp]),
        "csg_finalize": (None, [vp]),
        "csg_strerror": (ctypes.c_char_p, [i32]),
        "csg_last_error": (ctypes.c_char_p, []),
        "csg_sprinkle": (i32, [vp, i32, i64, u64, u64, vp, pp]),
        "csg_set_from_coords": (i32, [vp, i32, i64, vp, vp, pp]),
        "csg_link": (i32, [vp, vp, vp]),
        "csg_set_from_bitmap": (i32, [vp, i32, i64, vp, i64, vp, pp]),
        "csg_action": (i32, [vp, vp, i32, R, vp]),
        "csg_action_rows": (i32, [vp, vp, i32, i64, i64, R, vp]),
        "csg_action_hist": (i32, [vp, vp, i32, vp, i64, R, vp]),
        "csg_action_batch": (i32, [vp, pp, i32, i32, R, vp]),
        "csg_run_batch": (i32, [vp, i32, vp, vp, vp, vp, i32, R, vp]),
        "csg_serve_submit": (i32, [vp, i32, i64, u64, u64, ctypes.POINTER(u64)]),
        "csg_serve_poll": (i32, [vp, u64, R, i32]),
        "csg_serve_cancel": (i32, [vp, u64]),
        "csg_export_coords": (i32, [vp, vp, sz]),
        "csg_export_bitmap": (i32, [vp, vp, sz]),
        "csg_set_info": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i64), pp, pp]),
        "csg_set_free": (None, [vp]),
        "csg_action_noalloc": (i32, [i32, i64, vp, i64, vp, vp]),
        "csg_set_timing": (i32, [vp, i32]),
        "csg_sprinkle_desitter": (i32, [vp, i64, ctypes.c_double, u64, u64, vp, pp]),
        "csg_action_smeared": (i32, [vp, vp, i32, ctypes.c_double, ctypes.POINTER(ctypes.c_double), R, vp]),
        "csg_dalembertian": (i32, [vp, vp, i32, vp, ctypes.c_double, vp, R, vp]),
        "csg_stage_times": (i32, [vp, ctypes.POINTER(ctypes.c_double), i32]),
        "csg_test_wait_expiry": (i32, [u64, i32]),
        "csg_test_fail_alloc": (i32, [i32]),
        "csg_measure_popc_rate": (i32, [i32, ctypes.POINTER(ctypes.c_double)]),
        "csg_measure_l2_feed": (i32, [i32, ctypes.POINTER(ctypes.c_double)]),
        "csg_measure_mma_rate": (i32, [i32, i32, ctypes.POINTER(ctypes.c_double)]),
        "csg_check_words": (i32, [vp, i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(rc: int, what: str):
    if rc < 0:
        msg = load().csg_last_error().decode(errors="replace")
        raise CsgError(rc, f"{what}: {load().csg_strerror(rc).decode()}: {msg}")
    return rc


def current_stream() -> int:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return 0


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(current_stream())
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


NOALLOC_MAX_N = 65536
RESULT_BYTES = 88


def action_noalloc(d: int, N: int, dev_rows_ptr: int, stride_words: int, dev_out_ptr: int,
                   stream=None) -> None:
    """Popcount action that allocates nothing (see csg_action_noalloc in include/csg.h).

    For callers that cannot let a library allocate device memory.  The result (a
    csg_result, RESULT_BYTES bytes) is written to dev_out_ptr in stream order; read it
    after synchronising the stream, e.g. with result_from_bytes()."""
    _check(load().csg_action_noalloc(d, N, ctypes.c_void_p(dev_rows_ptr), stride_words,
                                     ctypes.c_void_p(dev_out_ptr), _stream(stream)), "csg_action_noalloc")


def inject_wait_expiry(limit_ns: int, starve: bool) -> None:
    """Failure injection (tests only): every bounded device wait of the interval-count kernels
    gives up after limit_ns (0: built-in limits); with starve, each CTA's first stage gets no
    copies, so its wait runs out and the call returns E_TIMEOUT.  See include/csg.h."""
    _check(load().csg_test_wait_expiry(limit_ns, int(bool(starve))), "csg_test_wait_expiry")


def inject_alloc_failures(n: int) -> None:
    """Failure injection (tests only): the next n device allocations of the library fail."""
    _check(load().csg_test_fail_alloc(n), "csg_test_fail_alloc")


def check_words() -> list:
    """The bounds-check words of a library built with CSG_CHECKED (read and cleared; all 0 when no
    access left its buffer); an empty list for the normal build."""
    arr = (ctypes.c_uint64 * 8)()
    n = _check(load().csg_check_words(ctypes.cast(arr, ctypes.c_void_p), 8), "csg_check_words")
    return [int(arr[k]) for k in range(n)]


def measure_popc_rate(device: int = 0) -> float:
    """Sustained 32-bit popcounts per second of the whole GPU (csg_measure_popc_rate)."""
    v = ctypes.c_double()
    _check(load().csg_measure_popc_rate(device, ctypes.byref(v)), "csg_measure_popc_rate")
    return v.value


def measure_mma_rate(method: int = TC, device: int = 0) -> float:
    """Flops per second of the pair MMA the tensor method issues, on resident operands
    (csg_measure_mma_rate)."""
    v = ctypes.c_double()
    _check(load().csg_measure_mma_rate(device, method, ctypes.byref(v)), "csg_measure_mma_rate")
    return v.value


def measure_l2_feed(device: int = 0) -> float:
    """Bytes per second one SM receives from L2 into shared memory (csg_measure_l2_feed)."""
    v = ctypes.c_double()
    _check(load().csg_measure_l2_feed(device, ctypes.byref(v)), "csg_measure_l2_feed")
    return v.value


def result_from_bytes(buf: bytes) -> Result:
    return Result.of(_Result.from_buffer_copy(bytes(buf)[:RESULT_BYTES]))


class CausalSet:
    """A set handle owned by a Context (coordinates and bitmap live on the device)."""

    def __init__(self, ctx: "Context", handle: int):
        self.ctx = ctx
        self.handle = ctypes.c_void_p(handle)

    def info(self):
        d, N, stride = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
        rows, coords = ctypes.c_void_p(), ctypes.c_void_p()
        _check(load().csg_set_info(self.handle, ctypes.byref(d), ctypes.byref(N), ctypes.byref(stride),
                                   ctypes.byref(rows), ctypes.byref(coords)), "csg_set_info")
        return dict(d=d.value, N=N.value, stride=stride.value, rows_ptr=rows.value,
                    coords_ptr=coords.value)

    @property
    def N(self):
        return self.info()["N"]

    def link(self, stream=None):
        _check(load().csg_link(self.ctx.handle, self.handle, _stream(stream)), "csg_link")
        return self

    def action(self, method: int = POPC, stream=None) -> Result:
        r = _Result()
        _check(load().csg_action(self.ctx.handle, self.handle, method, ctypes.byref(r), _stream(stream)),
               "csg_action")
        return Result.of(r)

    def action_rows(self, lo: int, hi: int, method: int = POPC, stream=None) -> Result:
        r = _Result()
        _check(load().csg_action_rows(self.ctx.handle, self.handle, method, lo, hi, ctypes.byref(r),
                                      _stream(stream)), "csg_action_rows")
        return Result.of(r)

    def action_hist(self, dev_hist_ptr: int, nbins: int, method: int = POPC, stream=None) -> Result:
        r = _Result()
        _check(load().csg_action_hist(self.ctx.handle, self.handle, method, ctypes.c_void_p(dev_hist_ptr),
                                      nbins, ctypes.byref(r), _stream(stream)), "csg_action_hist")
        return Result.of(r)

    def action_smeared(self, eps: float, method: int = POPC, stream=None):
        """(S_eps, Result): the smeared 1+1 action of Eq. s_smeared and the local counts."""
        S = ctypes.c_double()
        r = _Result()
        _check(load().csg_action_smeared(self.ctx.handle, self.handle, method, eps, ctypes.byref(S),
                                         ctypes.byref(r), _stream(stream)), "csg_action_smeared")
        return S.value, Result.of(r)

    def dalembertian(self, dev_phi_ptr: int, dev_Bphi_ptr: int, l: float = 1.0, method: int = POPC,
                     stream=None) -> Result:
        """Discrete d'Alembertian of Eq. b_local: reads N doubles at dev_phi_ptr, writes N
        doubles at dev_Bphi_ptr (device memory, element order of the set); returns the
        action counts of the same pass."""
        r = _Result()
        _check(load().csg_dalembertian(self.ctx.handle, self.handle, method, ctypes.c_void_p(dev_phi_ptr), l,
                                       ctypes.c_void_p(dev_Bphi_ptr), ctypes.byref(r), _stream(stream)),
               "csg_dalembertian")
        return Result.of(r)

    def coords(self) -> np.ndarray:
        N = self.N
        out = np.zeros((4, N), dtype=np.float64)
        _check(load().csg_export_coords(self.handle, out.ctypes.data_as(ctypes.c_void_p), out.size),
               "csg_export_coords")
        return out

    def bitmap(self) -> np.ndarray:
        inf = self.info()
        out = np.zeros((inf["N"], inf["stride"]), dtype=np.uint64)
        _check(load().csg_export_bitmap(self.handle, out.ctypes.data_as(ctypes.c_void_p), out.size),
               "csg_export_bitmap")
        return out

    def free(self):
        if self.handle.value:
            load().csg_set_free(self.handle)
            self.handle = ctypes.c_void_p(0)


class Context:
    """A device context with an optional HBM budget for set memory (0 = unlimited)."""

    def __init__(self, device: int = 0, budget_bytes: int = 0):
        h = ctypes.c_void_p()
        _check(load().csg_init(device, budget_bytes, ctypes.byref(h)), "csg_init")
        self.handle = h

    def close(self):
        if self.handle.value:
            load().csg_finalize(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def sprinkle(self, d: int, N: int, seed: int, seq: int = 0, stream=None) -> CausalSet:
        h = ctypes.c_void_p()
        _check(load().csg_sprinkle(self.handle, d, N, seed, seq, _stream(stream), ctypes.byref(h)),
               "csg_sprinkle")
        return CausalSet(self, h.value)

    def sprinkle_desitter(self, N: int, eta0: float, seed: int, seq: int = 0, stream=None) -> CausalSet:
        """Sprinkle into the 1+1 de Sitter slab |eta| <= eta0 (the paper's benchmark manifold)."""
        h = ctypes.c_void_p()
        _check(load().csg_sprinkle_desitter(self.handle, N, eta0, seed, seq, _stream(stream), ctypes.byref(h)),
               "csg_sprinkle_desitter")
        return CausalSet(self, h.value)

    def set_from_coords(self, d: int, coords: np.ndarray, stream=None) -> CausalSet:
        c = np.ascontiguousarray(coords, dtype=np.float64)
        if c.ndim != 2 or c.shape[0] != 4:
            raise ValueError("coords must be [4, N]")
        h = ctypes.c_void_p()
        _check(load().csg_set_from_coords(self.handle, d, c.shape[1], c.ctypes.data_as(ctypes.c_void_p),
                                          _stream(stream), ctypes.byref(h)), "csg_set_from_coords")
        return CausalSet(self, h.value)

    def set_from_bitmap(self, d: int, N: int, dev_rows_ptr: int, stride_words: int,
                        stream=None) -> CausalSet:
        h = ctypes.c_void_p()
        _check(load().csg_set_from_bitmap(self.handle, d, N, ctypes.c_void_p(dev_rows_ptr), stride_words,
                                          _stream(stream), ctypes.byref(h)), "csg_set_from_bitmap")
        return CausalSet(self, h.value)

    def action_batch(self, sets, method: int = POPC, stream=None) -> list[Result]:
        n = len(sets)
        arr = (ctypes.c_void_p * max(n, 1))(*[s.handle.value for s in sets])
        res = (_Result * max(n, 1))()
        _check(load().csg_action_batch(self.handle, arr, n, method, res, _stream(stream)),
               "csg_action_batch")
        return _results(res, n)

    def run_batch(self, specs, method: int = POPC, stream=None) -> list[Result]:
        """specs: iterable of (d, N, seed, seq)."""
        specs = list(specs)
        n = len(specs)
        d = np.array([s[0] for s in specs], dtype=np.int32)
        N = np.array([s[1] for s in specs], dtype=np.int64)
        seed = np.array([s[2] for s in specs], dtype=np.uint64)
        seq = np.array([s[3] for s in specs], dtype=np.uint64)
        res = (_Result * max(n, 1))()
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(load().csg_run_batch(self.handle, n, p(d), p(N), p(seed), p(seq), method, res,
                                    _stream(stream)), "csg_run_batch")
        return _results(res, n)

    def serve_submit(self, d: int, N: int, seed: int, seq: int = 0) -> int:
        t = ctypes.c_uint64()
        _check(load().csg_serve_submit(self.handle, d, N, seed, seq, ctypes.byref(t)), "csg_serve_submit")
        return t.value

    def serve_poll(self, ticket: int, timeout_ms: int = -1):
        """Returns a Result, or None while the request is pending."""
        r = _Result()
        rc = load().csg_serve_poll(self.handle, ticket, ctypes.byref(r), timeout_ms)
        if rc == PENDING:
            return None
        _check(rc, "csg_serve_poll")
        return Result.of(r)

    STAGES = ("sprinkle", "link", "expand", "action", "finalize")

    def set_timing(self, enable: bool = True):
        _check(load().csg_set_timing(self.handle, int(enable)), "csg_set_timing")

    def stage_times(self) -> dict:
        """Device milliseconds of each stage's last recorded run (None if not run)."""
        arr = (ctypes.c_double * len(self.STAGES))()
        _check(load().csg_stage_times(self.handle, arr, len(self.STAGES)), "csg_stage_times")
        return {k: (arr[i] if arr[i] >= 0 else None) for i, k in enumerate(self.STAGES)}

    def serve_cancel(self, ticket: int) -> int:
        return load().csg_serve_cancel(self.handle, ticket)
