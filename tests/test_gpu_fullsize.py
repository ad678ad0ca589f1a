"""Parity at the full sizes of the benchmark workloads, in the launch configuration the
benchmark times (whole-set csg_action with the tensor and popcount methods).

The oracle cannot run the full O(N^3) count in seconds at these sizes, so each check is
one of: the oracle's own sprinkle (bit-exact coordinates), the oracle's link on sampled
rows (bit-exact bitmap rows), the oracle's matrix-free count on sampled rows, exact
identities that hold at any size and are computed from the downloaded bitmap
(R = half its popcount, sum m = sum_x indeg(x) outdeg(x), W = sum_j j indeg(j) -
sum_i (i+1) outdeg(i)), agreement of the two independent kernels on the full launch,
batch == single, served == alone, and the oracle on sampled sets of the batch.
"""
import numpy as np
import pytest

import oracle
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


@pytest.fixture(scope="module")
def ctx(csg):
    c = csg.Context(0)
    yield c
    c.close()


def _popcount(a):
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(a)
    lut = np.array([bin(x).count("1") for x in range(256)], dtype=np.uint8)
    return lut[a.view(np.uint8)].reshape(a.shape + (8,)).sum(-1).astype(np.uint8)


def _identities(words, N):
    """R, sum m and W of the whole set from the symmetric bitmap alone."""
    pc = _popcount(words)
    rows = np.arange(N, dtype=np.int64)
    wx, bx = rows // 64, (rows % 64).astype(np.uint64)
    indeg = np.zeros(N, dtype=np.int64)
    block = 4096
    for lo in range(0, N, block):
        hi = min(N, lo + block)
        cum = np.cumsum(pc[lo:hi], axis=1, dtype=np.int64)
        r = rows[lo:hi] - lo
        w = wx[lo:hi]
        before = np.where(w > 0, cum[r, np.maximum(w - 1, 0)], 0)
        low = words[lo:hi][r, w] & ((np.uint64(1) << bx[lo:hi]) - np.uint64(1))
        indeg[lo:hi] = before + _popcount(low).astype(np.int64)
    deg = pc.sum(axis=1, dtype=np.int64)
    outdeg = deg - indeg
    R = int(deg.sum()) // 2
    sum_m = int((indeg * outdeg).sum())
    W = int((rows * indeg).sum() - ((rows + 1) * outdeg).sum())
    return R, sum_m, W, int(indeg.sum()), int(outdeg.sum())


def _pack_row(row, stride):
    bits = np.zeros(stride * 64, dtype=np.uint8)
    bits[:row.shape[0]] = row
    return np.packbits(bits, bitorder="little").view(np.uint64)


def _same(a, b):
    assert (a.d, a.N, a.R, tuple(a.Nk), a.sum_m, a.W, a.combo, a.status) == \
        (b.d, b.N, b.R, tuple(b.Nk), b.sum_m, b.W, b.combo, b.status)
    assert abs(a.S - b.S) <= TOL_S * max(abs(b.S), 1.0)


def _check_rows(s, d, coords, rows, csg):
    for i in rows:
        want = oracle.action_rows_coords(d, coords, i, i + 1)
        for method in (csg.TC, csg.POPC):
            got = s.action_rows(i, i + 1, method)
            assert (got.R, list(got.Nk), got.sum_m, got.W) == \
                (want["R"], [int(x) for x in want["Nk"]], want["sum_m"], want["W"]), (i, method)


def test_d2_n2048_full_oracle(ctx, csg):
    d, N, seed = 2, 2048, 0
    s = ctx.sprinkle(d, N, seed).link()
    want = oracle.run(d, N, seed)
    assert np.array_equal(s.coords(), want["coords"])
    assert np.array_equal(s.bitmap(), oracle.pack(want["rel"], s.info()["stride"]))
    for method in (csg.TC, csg.POPC):
        r = s.action(method)
        assert (r.R, list(r.Nk), r.sum_m, r.W, r.combo) == \
            (want["R"], [int(x) for x in want["Nk"]], want["sum_m"], want["W"], want["combo"])
        assert abs(r.S - want["S"]) <= TOL_S * max(abs(want["S"]), 1.0)
    s.free()


@pytest.mark.parametrize("d,N,seed,rows", [
    (4, 65536, 1, (3, 20000, 32768, 65000)),
    (2, 131072, 2, (65536, 131000)),
])
def test_full_size_set(ctx, csg, d, N, seed, rows):
    s = ctx.sprinkle(d, N, seed).link()
    coords = oracle.sprinkle_sorted(d, N, seed)
    assert np.array_equal(s.coords(), coords)                      # bit-exact sprinkle + order
    words = s.bitmap()
    for i in (0, 1, N // 3, N // 2, N - 2, N - 1):                 # sampled bitmap rows
        row = oracle.link_row(d, coords, i)
        assert np.array_equal(words[i], _pack_row(row, words.shape[1])), i
        col = ((words[:, i // 64] >> np.uint64(i % 64)) & np.uint64(1)).astype(np.uint8)
        assert np.array_equal(col, row), i                         # symmetric
    R, sum_m, W, ins, outs = _identities(words, N)
    assert ins == outs == R
    tc = s.action(csg.TC)                                          # the benchmark's launch
    assert (tc.R, tc.sum_m, tc.W) == (R, sum_m, W)
    assert tc.N == N and tc.d == d and tc.status == 0
    pc = s.action(csg.POPC)                                        # independent kernel
    _same(pc, tc)
    for fmt in (csg.TC_FP8, csg.TC_FP4):                           # both tensor operand formats
        _same(s.action(fmt), tc)
    combo, S = oracle.finalize(d, N, tc.Nk)
    assert tc.combo == combo and abs(tc.S - S) <= TOL_S * max(abs(S), 1.0)
    _check_rows(s, d, coords, rows, csg)                           # sampled N_k against the oracle
    s.free()


@pytest.mark.parametrize("d,seed", [(2, 11), (4, 12)])
def test_max_size_set(ctx, csg, d, seed):
    """N = CSG_MAX_N (2^18): 8 GiB bitmap, 64 GiB of fp4 operands.  Bit-exact coordinates
    and sampled bitmap rows and columns, the exact identities for R, sum m and W from the
    whole downloaded bitmap, the oracle's matrix-free counts on late rows, and both tensor
    formats equal (d=2 also against the popcount kernel)."""
    N = csg.MAX_N
    s = ctx.sprinkle(d, N, seed).link()
    coords = oracle.sprinkle_sorted(d, N, seed)
    assert np.array_equal(s.coords(), coords)
    words = s.bitmap()
    for i in (0, 7, N // 2 + 5, N - 1):
        row = oracle.link_row(d, coords, i)
        assert np.array_equal(words[i], _pack_row(row, words.shape[1])), i
        col = ((words[:, i // 64] >> np.uint64(i % 64)) & np.uint64(1)).astype(np.uint8)
        assert np.array_equal(col, row), i
    R, sum_m, W, ins, outs = _identities(words, N)
    del words
    assert ins == outs == R
    tc = s.action(csg.TC)
    assert (tc.R, tc.sum_m, tc.W, tc.N, tc.status) == (R, sum_m, W, N, 0)
    _same(s.action(csg.TC_FP8), tc)
    if d == 2:
        _same(s.action(csg.POPC), tc)
    combo, S = oracle.finalize(d, N, tc.Nk)
    assert tc.combo == combo and abs(tc.S - S) <= TOL_S * max(abs(S), 1.0)
    _check_rows(s, d, coords, (N - 3000, N - 700, N - 2), csg)
    s.free()


def test_batch_4096_sets(ctx, csg):
    specs = inputs.batch_workload()                                # 4096 diamonds, seed 3
    assert len(specs) == 4096
    tup = [(sp.d, sp.N, sp.seed, sp.seq) for sp in specs]
    tc = ctx.run_batch(tup, csg.TC)
    pc = ctx.run_batch(tup, csg.POPC)
    for a, b in zip(tc, pc):
        _same(a, b)
    other = csg.TC_FP4 if csg.TC != csg.TC_FP4 else csg.TC_FP8
    for a, b in zip(ctx.run_batch(tup, other), tc):                # the other tensor operand format
        _same(a, b)
    rng = np.random.default_rng(7)
    sample = sorted(set(rng.choice(4096, 10, replace=False).tolist()) |
                    {int(np.argmax([sp.N for sp in specs]))})
    for k in sample:                                               # batch == single == oracle
        sp = specs[k]
        s = ctx.sprinkle(sp.d, sp.N, sp.seed, sp.seq).link()
        _same(s.action(csg.TC), tc[k])
        s.free()
        if sp.N <= 6000 or sp.d == 4:
            want = oracle.run(sp.d, sp.N, sp.seed, sp.seq)
            assert (tc[k].R, list(tc[k].Nk), tc[k].sum_m, tc[k].W, tc[k].combo) == \
                (want["R"], [int(x) for x in want["Nk"]], want["sum_m"], want["W"], want["combo"]), k


def test_served_requests_equal_alone(ctx, csg):
    reqs = inputs.serve_workload(n_req=48)                         # seed 4, N in [1024, 65536]
    tickets = [ctx.serve_submit(r.spec.d, r.spec.N, r.spec.seed, r.spec.seq) for r in reqs]
    served = [ctx.serve_poll(t, timeout_ms=300000) for t in tickets]
    for r, got in zip(reqs, served):
        alone = ctx.run_batch([(r.spec.d, r.spec.N, r.spec.seed, r.spec.seq)], csg.TC)[0]
        _same(got, alone)
        if r.spec.N <= 2500:
            want = oracle.run(r.spec.d, r.spec.N, r.spec.seed, r.spec.seq)
            assert (got.R, list(got.Nk), got.sum_m, got.W) == \
                (want["R"], [int(x) for x in want["Nk"]], want["sum_m"], want["W"])
