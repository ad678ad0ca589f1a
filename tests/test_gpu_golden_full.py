"""Parity at the full sizes of every workload, against complete oracle runs.

The expected values under tests/golden/ were written by tests/golden/make_fullsize.py,
which calls only the oracle (its sprinkle, time order, unpacked link and triple loop over
every related pair, Secs. 2.1-2.2 and 4.1-4.2; its finalize, Eq. s_local and the 3+1
combination).  Here the GPU path runs in the launch configuration the benchmark times and
is compared with them field by field:

* the single sets d=2 N=2048, d=4 N=65536 and d=2 N=131072: the whole bitmap (SHA-256 of
  every block of 4096 packed rows), R, N_0..N_3, sum m, W, combo and S from every method
  (popcount, tensor in fp4 and fp8), and for d=4 N=65536 the whole interval-size histogram;
* every one of the 4096 sets of the mixed batch: the batched counts from every method and
  each set's whole bitmap (a 64-bit prefix of its SHA-256);
* the served stream: every request with N <= 4096 and 64 larger ones drawn by the script,
  submitted together to the service under its 160 GB budget.
"""
import hashlib

import numpy as np
import pytest

import oracle
from golden_io import read_full, read_table
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


def _same_counts(r, want, what):
    assert (r.R, list(r.Nk), r.sum_m, r.W, r.combo, r.status) == \
        (want["R"], list(want["Nk"]), want["sum_m"], want["W"], want["combo"], 0), what
    assert abs(r.S - want["S"]) <= TOL_S * max(abs(want["S"]), 1.0), what


def _row_fields(row):
    return {"R": int(row["R"]), "Nk": [int(row[f"N{k}"]) for k in range(4)], "sum_m": int(row["sum_m"]),
            "W": int(row["W"]), "combo": int(row["combo"]), "S": float(row["S"])}


def _block_digests(words, rows_per):
    out = []
    for lo in range(0, words.shape[0], rows_per):
        blk = np.ascontiguousarray(words[lo:lo + rows_per]).astype("<u8", copy=False)
        out.append((lo, hashlib.sha256(blk.tobytes()).hexdigest()))
    return out


@pytest.mark.parametrize("name", ["full_d2_n2048_seed0.txt", "full_d4_n65536_seed1.txt",
                                  "full_d2_n131072_seed2.txt"])
def test_single_set_against_full_oracle_run(csg, name):
    import torch
    g = read_full(name)
    d, N, seed = g["d"], g["N"], g["seed"]
    with csg.Context(0) as ctx:
        s = ctx.sprinkle(d, N, seed, g["seq"]).link()
        words = s.bitmap()
        assert words.shape == (N, g["stride"])
        got = _block_digests(words, g["rows_per_digest"])
        del words
        bad = [lo for (lo, h), (_, w) in zip(got, g["digests"]) if h != w]
        assert len(got) == len(g["digests"]) and not bad, f"bitmap row blocks differ: {bad}"
        for method in (csg.TC, csg.POPC, csg.TC_FP8, csg.TC_FP4):
            _same_counts(s.action(method), g, (name, method))
        combo, S = oracle.finalize(d, N, g["Nk"])
        assert combo == g["combo"] and S == g["S"]  # the stored action is the oracle's finalize
        if g["hist"]:
            want = np.zeros(N, dtype=np.uint64)
            for m, c in g["hist"].items():
                want[m] = c
            assert int(want.sum()) == g["R"]
            dev = torch.zeros(N, dtype=torch.int64, device="cuda")
            for method in (csg.TC, csg.POPC):
                _same_counts(s.action_hist(dev.data_ptr(), N, method), g, (name, "hist", method))
                torch.cuda.synchronize()
                got_h = dev.cpu().numpy().view(np.uint64)
                diff = np.nonzero(got_h != want)[0]
                assert diff.size == 0, f"histogram bins differ, first {diff[:8]}"
        s.free()


def test_batch_of_4096_against_full_oracle_runs(csg):
    rows = read_table("batch_4096_seed3.txt")
    specs = inputs.batch_workload()
    assert len(rows) == len(specs) == 4096
    for row, sp in zip(rows, specs):
        assert (int(row["d"]), int(row["N"]), int(row["seed"]), int(row["seq"])) == (sp.d, sp.N, sp.seed, sp.seq)
    tup = [(sp.d, sp.N, sp.seed, sp.seq) for sp in specs]
    with csg.Context(0) as ctx:
        for method in (csg.TC, csg.POPC, csg.TC_FP8, csg.TC_FP4):
            res = ctx.run_batch(tup, method)
            for k, (row, r) in enumerate(zip(rows, res)):
                assert r.d == int(row["d"]) and r.N == int(row["N"])
                _same_counts(r, _row_fields(row), (k, method))
        bad = []
        for k, (row, sp) in enumerate(zip(rows, specs)):  # every set's whole bitmap
            s = ctx.sprinkle(sp.d, sp.N, sp.seed, sp.seq).link()
            w = np.ascontiguousarray(s.bitmap()).astype("<u8", copy=False)
            s.free()
            if hashlib.sha256(w.tobytes()).hexdigest()[:16] != row["bitmap_sha256_16"]:
                bad.append(k)
        assert not bad, f"bitmaps of sets {bad[:16]} differ"


def test_served_sample_against_full_oracle_runs(csg):
    rows = read_table("serve_20000_seed4_sample.txt")
    reqs = inputs.serve_workload(n_req=20000)
    assert len(rows) > 6000 and sum(int(r["N"]) > 4096 for r in rows) == 64
    with csg.Context(0, budget_bytes=160 * 10 ** 9) as ctx:
        tickets = []
        for row in rows:
            sp = reqs[int(row["key"])].spec
            assert (sp.d, sp.N, sp.seed, sp.seq) == (int(row["d"]), int(row["N"]), int(row["seed"]), int(row["seq"]))
            tickets.append(ctx.serve_submit(sp.d, sp.N, sp.seed, sp.seq))
        for row, t in zip(rows, tickets):
            r = ctx.serve_poll(t, timeout_ms=600000)
            assert r.d == int(row["d"]) and r.N == int(row["N"])
            _same_counts(r, _row_fields(row), ("request", row["key"]))
