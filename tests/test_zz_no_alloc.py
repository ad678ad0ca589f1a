"""The allocation-free action entry point (csg_action_noalloc).

It serves callers that cannot let a library allocate device memory (graph capture,
applications that own all of HBM, servers that cannot absorb cudaFree's device-wide
synchronisation).  Here it must give the same result as csg_action with the popcount
method, through the C ABI, on two calls in a row -- the second call reuses the
scratch array the first one left behind.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1709_03013_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_S = 1e-12


@pytest.fixture(scope="module")
def csg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_03013_gb300 import csg as m
    m.load()
    return m


def _same(a, b):
    assert (a.d, a.N, a.R, tuple(a.Nk), a.sum_m, a.W, a.combo, a.status) == \
        (b.d, b.N, b.R, tuple(b.Nk), b.sum_m, b.W, b.combo, b.status)
    assert abs(a.S - b.S) <= TOL_S * max(abs(b.S), 1.0)


def _noalloc_twice(csg, d, s):
    import torch
    info = s.info()
    out = torch.zeros(csg.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    got = []
    for _ in range(2):
        out.fill_(0xAB)  # stale bytes must not survive
        csg.action_noalloc(d, info["N"], info["rows_ptr"], info["stride"], out.data_ptr())
        torch.cuda.synchronize()
        got.append(csg.result_from_bytes(out.cpu().numpy().tobytes()))
    return got


@pytest.mark.parametrize("d,N,seed", [(2, 3001, 5), (4, 4097, 6), (4, 65536, 1), (2, 17, 2), (4, 1, 3)])
def test_noalloc_matches_action_twice(csg, d, N, seed):
    with csg.Context(0) as ctx:
        s = ctx.sprinkle(d, N, seed, 0).link()
        want = s.action(csg.POPC)
        first, second = _noalloc_twice(csg, d, s)
        _same(first, want)
        _same(second, want)
        s.free()


def test_noalloc_after_a_larger_call(csg):
    # a small set right after a large one: slots of the larger call must not leak in
    with csg.Context(0) as ctx:
        big = ctx.sprinkle(4, 20000, 9, 0).link()
        small = ctx.sprinkle(2, 700, 9, 1).link()
        for s, d in ((big, 4), (small, 2), (small, 2)):
            want = s.action(csg.POPC)
            first, second = _noalloc_twice(csg, d, s)
            _same(first, want)
            _same(second, want)
        big.free()
        small.free()


def test_noalloc_on_caller_bitmap(csg):
    import torch
    rel = inputs.layered_order_rel(900, 4)
    stride = 16
    dev = torch.from_numpy(inputs.pack_rows(rel, stride).view(np.int64)).cuda()
    with csg.Context(0) as ctx:
        s = ctx.set_from_bitmap(4, 900, dev.data_ptr(), stride)
        want = s.action(csg.POPC)
        s.free()
    out = torch.zeros(csg.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    for _ in range(2):
        csg.action_noalloc(4, 900, dev.data_ptr(), stride, out.data_ptr())
        torch.cuda.synchronize()
        _same(csg.result_from_bytes(out.cpu().numpy().tobytes()), want)


def test_noalloc_rejects_sizes_beyond_its_scratch(csg):
    import torch
    buf = torch.zeros(8, dtype=torch.int64, device="cuda")
    out = torch.zeros(csg.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    with pytest.raises(csg.CsgError) as e:
        csg.action_noalloc(2, csg.NOALLOC_MAX_N + 1, buf.data_ptr(), 2048, out.data_ptr())
    assert e.value.code == csg.E_INVAL
    assert "65536" in str(e.value)
    with pytest.raises(csg.CsgError):
        csg.action_noalloc(3, 10, buf.data_ptr(), 2, out.data_ptr())
