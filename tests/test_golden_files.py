"""The stored full-size oracle results under tests/golden/ are the oracle's (CPU only).

tests/golden/make_fullsize.py writes them from complete oracle runs, which take hours for
the largest sets; here every file is checked for internal consistency (the histogram
sums to R and to sum m, N_0..N_3 are its first bins, combo and S are the oracle's finalize
of N_0..N_3, one digest per 4096 rows), its workload against the seeded recipes, and the
sets that the oracle finishes in seconds are recomputed from scratch and compared in full.
"""
import hashlib
import importlib.util
import os

import numpy as np
import pytest

import oracle
from golden_io import read_full, read_table
from paper_1709_03013_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    spec = importlib.util.spec_from_file_location(name, os.path.join(GOLDEN, name + ".py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _read_full(name):
    return read_full(name)


def _read_table(name):
    return read_table(name)


def _check_finalize(d, N, fields):
    combo, S = oracle.finalize(d, N, fields["Nk"])
    assert combo == fields["combo"] and S == fields["S"]


SINGLES = ["full_d2_n2048_seed0.txt", "full_d4_n65536_seed1.txt", "full_d2_n131072_seed2.txt"]


@pytest.mark.parametrize("name", SINGLES)
def test_single_set_files_are_consistent(name):
    g = _read_full(name)
    d, N = g["d"], g["N"]
    assert name == f"full_d{d}_n{N}_seed{g['seed']}.txt"
    assert g["stride"] == oracle.stride_words(N) and g["rows_per_digest"] == 4096
    assert [lo for lo, _ in g["digests"]] == list(range(0, N, 4096))
    assert len(g["Nk"]) == 4 and sum(g["Nk"]) <= g["R"] and g["W"] >= g["sum_m"]
    _check_finalize(d, N, g)
    if g["hist"]:
        assert sum(g["hist"].values()) == g["R"]
        assert sum(m * c for m, c in g["hist"].items()) == g["sum_m"]
        assert [g["hist"].get(k, 0) for k in range(4)] == g["Nk"]
        assert max(g["hist"]) <= N - 2


def test_small_single_set_file_equals_a_fresh_oracle_run():
    g = _read_full("full_d2_n2048_seed0.txt")
    want = oracle.run(2, 2048, 0)
    assert (want["R"], [int(x) for x in want["Nk"]], want["sum_m"], want["W"], want["combo"], want["S"]) == \
        (g["R"], g["Nk"], g["sum_m"], g["W"], g["combo"], g["S"])
    words = oracle.pack(want["rel"])
    h = hashlib.sha256(np.ascontiguousarray(words).astype("<u8").tobytes()).hexdigest()
    assert g["digests"] == [(0, h)]


def _fields(row):
    return {"R": int(row["R"]), "Nk": [int(row[f"N{k}"]) for k in range(4)], "sum_m": int(row["sum_m"]),
            "W": int(row["W"]), "combo": int(row["combo"]), "S": float(row["S"])}


def test_batch_file_matches_its_workload_and_fresh_oracle_runs():
    rows = _read_table("batch_4096_seed3.txt")
    specs = inputs.batch_workload()
    assert len(rows) == len(specs) == 4096
    for k, (row, sp) in enumerate(zip(rows, specs)):
        assert (int(row["key"]), int(row["d"]), int(row["N"]), int(row["seed"]), int(row["seq"])) == \
            (k, sp.d, sp.N, sp.seed, sp.seq)
        f = _fields(row)
        _check_finalize(sp.d, sp.N, f)
        assert sum(f["Nk"]) <= f["R"] and len(row["bitmap_sha256_16"]) == 16
    small = [k for k, sp in enumerate(specs) if sp.N <= 1200]
    for k in np.random.default_rng(11).choice(small, 8, replace=False):
        sp, row = specs[k], rows[k]
        want = oracle.run(sp.d, sp.N, sp.seed, sp.seq)
        assert (want["R"], [int(x) for x in want["Nk"]], want["sum_m"], want["W"], want["combo"]) == \
            tuple(_fields(row)[x] for x in ("R", "Nk", "sum_m", "W", "combo"))
        words = np.ascontiguousarray(oracle.pack(want["rel"])).astype("<u8")
        assert hashlib.sha256(words.tobytes()).hexdigest()[:16] == row["bitmap_sha256_16"]


def test_serve_file_matches_its_sample_and_fresh_oracle_runs():
    mk = _load("make_fullsize")
    rows = _read_table("serve_20000_seed4_sample.txt")
    reqs = inputs.serve_workload(n_req=20000)
    keys = [int(r["key"]) for r in rows]
    assert keys == mk.serve_sample(reqs)
    assert sum(reqs[k].spec.N > 4096 for k in keys) == 64
    kset = set(keys)
    assert all(k in kset for k in range(20000) if reqs[k].spec.N <= 4096)
    for row in rows:
        sp = reqs[int(row["key"])].spec
        assert (int(row["d"]), int(row["N"]), int(row["seed"]), int(row["seq"])) == (sp.d, sp.N, sp.seed, sp.seq)
        _check_finalize(sp.d, sp.N, _fields(row))
    for k in np.random.default_rng(12).choice(len(rows), 4, replace=False):
        row = rows[k]
        if int(row["N"]) > 1500:
            continue
        sp = reqs[int(row["key"])].spec
        want = oracle.run(sp.d, sp.N, sp.seed, sp.seq)
        assert (want["R"], [int(x) for x in want["Nk"]], want["sum_m"], want["W"], want["combo"]) == \
            tuple(_fields(row)[x] for x in ("R", "Nk", "sum_m", "W", "combo"))
