#!/usr/bin/env python3
"""Writes the oracle's results for the full benchmark workloads into tests/golden/.

Only the oracle (``oracle/``) computes anything here; the seeded recipes of
``paper_1709_03013_gb300/inputs.py`` only say which (d, N, seed, seq) each set has.
Every value written is the oracle's: its sprinkle and time order (Secs. 2.1-2.2), its
unpacked link (Sec. 2.2), its triple loop over every related pair (Secs. 4.1-4.2) and
its finalize (Eq. s_local; the 3+1 combination for d=4).

Files (plain text, '#' comments):
  full_d2_n2048_seed0.txt, full_d4_n65536_seed1.txt, full_d2_n131072_seed2.txt
      one set each: R, N_0..N_3, sum m, W, combo, S; a SHA-256 digest of every block of
      4096 rows of the packed bitmap in the library's layout (row stride ceil(N/64)
      rounded up to 16 words, little-endian words, zero padding); for d=4 N=65536 also
      the whole interval-size histogram
  batch_4096_seed3.txt
      every set of the 4096-diamond batch: its counts and the first 16 hex digits of the
      SHA-256 of its packed bitmap
  serve_20000_seed4_sample.txt
      the requests of the 20000-request stream with N <= 4096, and 64 of the larger ones
      drawn with numpy.random.default_rng(40): their counts

The run is long (the d=2 N=131072 set is about 2.6e14 bit tests), so results are kept
per block of rows (single sets) or per set (batch, serve) in a checkpoint directory and
a rerun resumes there.  Timings of the oracle (link and interval counts, threads, CPU)
go into each file's header.

  python tests/golden/make_fullsize.py [--only single1,single2,single3,batch,serve]
                                       [--threads T] [--ckpt DIR]
  python tests/golden/make_fullsize.py --verify single1,single2,batch [--threads T]

--verify reruns the named parts with the oracle, compares every value with the stored files
(writing nothing) and prints one JSON line of timings per part: how long the oracle takes on
this machine's cores, and that it gives the same results here as where the files were written.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import subprocess
import sys
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1709_03013_gb300 import inputs  # noqa: E402

ROWS_PER_DIGEST = 4096
SERVE_SMALL_N = 4096
SERVE_LARGE_SAMPLE = 64
SERVE_SAMPLE_SEED = 40
SINGLES = {"single1": (2, 2048, 0), "single2": (4, 65536, 1), "single3": (2, 131072, 2)}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


def bitmap_digests(words: np.ndarray, rows_per: int = ROWS_PER_DIGEST) -> list[tuple[int, str]]:
    """SHA-256 of the little-endian bytes of every block of rows of the packed bitmap."""
    out = []
    for lo in range(0, words.shape[0], rows_per):
        blk = np.ascontiguousarray(words[lo:lo + rows_per]).astype("<u8", copy=False)
        out.append((lo, hashlib.sha256(blk.tobytes()).hexdigest()))
    return out


def set_digest16(words: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(words).astype("<u8", copy=False).tobytes()).hexdigest()[:16]


def counts_fields(d: int, N: int, out: dict) -> list:
    combo, S = oracle.finalize(d, N, out["Nk"])
    return [out["R"], *[int(x) for x in out["Nk"]], out["sum_m"], out["W"], combo, repr(S)]


def run_single(name: str, threads: int, ckpt: str) -> None:
    d, N, seed = SINGLES[name]
    tag = f"full_d{d}_n{N}_seed{seed}"
    path = os.path.join(HERE, tag + ".txt")
    blocks_file = os.path.join(ckpt, tag + ".blocks.jsonl")
    t0 = time.perf_counter()
    coords = oracle.sprinkle_sorted(d, N, seed, 0)
    rel = oracle.link(d, coords, threads)
    t_link = time.perf_counter() - t0
    print(f"{tag}: link {t_link:.1f} s", flush=True)
    words = oracle.pack(rel)
    digests = bitmap_digests(words)
    stride = words.shape[1]
    del words
    done = {}
    if os.path.exists(blocks_file):
        with open(blocks_file) as fh:
            for ln in fh:
                b = json.loads(ln)
                done[b["lo"]] = b
    hist = np.zeros(max(N, 1), dtype=np.uint64)
    R = sum_m = W = 0
    t_count = 0.0
    block = max(1, min(N, 4096))
    for lo in range(0, N, block):
        hi = min(N, lo + block)
        if lo in done:
            b = done[lo]
        else:
            t1 = time.perf_counter()
            out = oracle.action(rel, threads, rows=(lo, hi))
            dt = time.perf_counter() - t1
            nz = np.nonzero(out["hist"])[0]
            b = {"lo": lo, "hi": hi, "R": out["R"], "sum_m": out["sum_m"], "W": out["W"], "s": dt,
                 "hist": [[int(m), int(out["hist"][m])] for m in nz]}
            with open(blocks_file, "a") as fh:
                fh.write(json.dumps(b) + "\n")
            print(f"{tag}: rows [{lo}, {hi}) {dt:.1f} s", flush=True)
        for m, c in b["hist"]:
            hist[m] += np.uint64(c)
        R += b["R"]
        sum_m += b["sum_m"]
        W += b["W"]
        t_count += b["s"]
    Nk = [int(hist[k]) if k < hist.shape[0] else 0 for k in range(4)]
    out = dict(R=R, Nk=np.array(Nk, dtype=np.uint64), sum_m=sum_m, W=W)
    assert int(hist.sum()) == R and int((hist * np.arange(hist.shape[0], dtype=np.uint64)).sum()) == sum_m
    combo, S = oracle.finalize(d, N, out["Nk"])
    T = threads or os.cpu_count()
    extra = ""
    if name == "single1":  # the small set is also timed on one thread
        t1 = time.perf_counter()
        oracle.action(rel, 1)
        extra = f"; counts on 1 thread {time.perf_counter() - t1:.3f} s"
    with open(path, "w") as fh:
        fh.write(f"# Oracle results for the whole d={d} N={N} flat diamond (seed {seed}, seq 0): its sprinkle,\n"
                 f"# time order, unpacked link and triple loop over every related pair (Secs. 2.1-2.2, 4.1-4.2).\n"
                 f"# Written by tests/golden/make_fullsize.py {name}.\n"
                 f"# oracle timing: {T} threads on {cpu_model()}; link {t_link:.1f} s; interval counts "
                 f"{t_count:.1f} s ({R / max(t_count, 1e-9):.4g} pairs/s, {W / max(t_count, 1e-9):.4g} bit tests/s)"
                 f"{extra}\n")
        fh.write(f"d: {d}\nN: {N}\nseed: {seed}\nseq: 0\nR: {R}\nNk: {' '.join(str(x) for x in Nk)}\n"
                 f"sum_m: {sum_m}\nW: {W}\ncombo: {combo}\nS: {S!r}\n")
        fh.write(f"# bitmap digests: SHA-256 of rows [lo, lo+{ROWS_PER_DIGEST}) of the packed rows, "
                 f"{stride} little-endian uint64 words per row\nstride: {stride}\nrows_per_digest: {ROWS_PER_DIGEST}\n")
        for lo, h in digests:
            fh.write(f"digest: {lo} {h}\n")
        if name == "single2":
            top = int(np.nonzero(hist)[0].max()) if R else 0
            fh.write(f"# interval-size histogram: 'hist: m0 c(m0) c(m0+1) ...', 32 bins per line, bins 0..{top}\n")
            for m0 in range(0, top + 1, 32):
                fh.write("hist: " + str(m0) + " " + " ".join(str(int(x)) for x in hist[m0:min(top + 1, m0 + 32)]) + "\n")
    print(f"{tag}: wrote {path}", flush=True)


def _run_list(tag: str, items: list, header: str, path: str, threads: int, ckpt: str, with_digest: bool) -> None:
    """items: (key, SetSpec).  One checkpoint line per set; the golden file is written in key order."""
    cfile = os.path.join(ckpt, tag + ".jsonl")
    done = {}
    if os.path.exists(cfile):
        with open(cfile) as fh:
            for ln in fh:
                r = json.loads(ln)
                done[r["key"]] = r
    t_link = t_count = 0.0
    for n, (key, sp) in enumerate(items):
        if key in done:
            continue
        t0 = time.perf_counter()
        coords = oracle.sprinkle_sorted(sp.d, sp.N, sp.seed, sp.seq)
        rel = oracle.link(sp.d, coords, threads)
        t1 = time.perf_counter()
        out = oracle.action(rel, threads)
        t2 = time.perf_counter()
        rec = {"key": key, "d": sp.d, "N": sp.N, "seed": sp.seed, "seq": sp.seq,
               "fields": counts_fields(sp.d, sp.N, out), "link_s": t1 - t0, "count_s": t2 - t1}
        if with_digest:
            rec["digest"] = set_digest16(oracle.pack(rel))
        with open(cfile, "a") as fh:
            fh.write(json.dumps(rec) + "\n")
        done[key] = rec
        if n % 200 == 0 or sp.N > 16384:
            print(f"{tag}: {n + 1}/{len(items)} N={sp.N} d={sp.d} {t2 - t1:.2f} s", flush=True)
    R = sum(done[k]["fields"][0] for k, _ in items)
    W = sum(done[k]["fields"][6] for k, _ in items)
    t_link = sum(done[k]["link_s"] for k, _ in items)
    t_count = sum(done[k]["count_s"] for k, _ in items)
    T = threads or os.cpu_count()
    with open(path, "w") as fh:
        fh.write(header)
        fh.write(f"# oracle timing: {T} threads on {cpu_model()}; links {t_link:.1f} s; interval counts "
                 f"{t_count:.1f} s ({R / max(t_count, 1e-9):.4g} pairs/s, {W / max(t_count, 1e-9):.4g} bit tests/s)\n")
        cols = "key d N seed seq R N0 N1 N2 N3 sum_m W combo S" + (" bitmap_sha256_16" if with_digest else "")
        fh.write(f"# columns: {cols}\n")
        for key, _ in items:
            r = done[key]
            row = [r["key"], r["d"], r["N"], r["seed"], r["seq"], *r["fields"]]
            if with_digest:
                row.append(r["digest"])
            fh.write(" ".join(str(x) for x in row) + "\n")
    print(f"{tag}: wrote {path}", flush=True)


def serve_sample(reqs) -> list[int]:
    """Indices of the checked requests: every N <= 4096, and 64 larger ones drawn with
    default_rng(40) (sorted)."""
    small = [r for r, q in enumerate(reqs) if q.spec.N <= SERVE_SMALL_N]
    large = [r for r, q in enumerate(reqs) if q.spec.N > SERVE_SMALL_N]
    pick = np.random.default_rng(SERVE_SAMPLE_SEED).choice(len(large), SERVE_LARGE_SAMPLE, replace=False)
    return sorted(small + [large[int(k)] for k in pick])


def run_batch(threads: int, ckpt: str) -> None:
    specs = inputs.batch_workload()
    header = ("# Oracle results for every set of the 4096-diamond batch (d alternating 2/4, N log-uniform in\n"
              "# [256, 8192] from seed 3, set s sprinkled with (3, s)): sprinkle, time order, link, triple loop,\n"
              "# finalize.  key = set index.  Written by tests/golden/make_fullsize.py batch.\n")
    _run_list("batch_4096_seed3", list(enumerate(specs)), header,
              os.path.join(HERE, "batch_4096_seed3.txt"), threads, ckpt, with_digest=True)


def run_serve(threads: int, ckpt: str) -> None:
    reqs = inputs.serve_workload(n_req=20000)
    idx = serve_sample(reqs)
    header = ("# Oracle results for the checked requests of the 20000-request stream (seed 4; d in {2,4} 50/50,\n"
              "# N log-uniform in [1024, 65536]; request r sprinkled with (4, r)): every request with N <= 4096\n"
              "# and 64 of the larger ones drawn with numpy.random.default_rng(40).  key = request index.\n"
              "# Written by tests/golden/make_fullsize.py serve.\n")
    # the large requests first, so that a long run reports its slow part early
    items = sorted(((r, reqs[r].spec) for r in idx), key=lambda kv: -kv[1].N)
    _run_list("serve_20000_seed4_sample", items, header, os.path.join(HERE, "serve_20000_seed4_sample.txt"),
              threads, ckpt, with_digest=False)
    # keep the file in request order
    path = os.path.join(HERE, "serve_20000_seed4_sample.txt")
    with open(path) as fh:
        lines = fh.readlines()
    head = [ln for ln in lines if ln.startswith("#")]
    body = sorted((ln for ln in lines if not ln.startswith("#")), key=lambda ln: int(ln.split()[0]))
    with open(path, "w") as fh:
        fh.writelines(head + body)


def _stored_single(name: str) -> dict:
    g = {"digests": []}
    with open(os.path.join(HERE, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, val = (x.strip() for x in line.split(":", 1))
            if key == "digest":
                g["digests"].append(tuple(val.split()))
            elif key == "Nk":
                g["Nk"] = [int(x) for x in val.split()]
            elif key == "S":
                g["S"] = float(val)
            elif key != "hist":
                g[key] = int(val)
    return g


def verify(parts: list, threads: int) -> int:
    """Reruns the named parts with the oracle and compares them with the stored files."""
    T = threads or os.cpu_count()
    ok = True
    for name in parts:
        if name in SINGLES:
            d, N, seed = SINGLES[name]
            g = _stored_single(f"full_d{d}_n{N}_seed{seed}.txt")
            t0 = time.perf_counter()
            coords = oracle.sprinkle_sorted(d, N, seed, 0)
            rel = oracle.link(d, coords, threads)
            t1 = time.perf_counter()
            out = oracle.action(rel, threads)
            t2 = time.perf_counter()
            f = counts_fields(d, N, out)
            same = (f[:8] == [g["R"], *g["Nk"], g["sum_m"], g["W"], g["combo"]] and float(f[8]) == g["S"] and
                    [(str(lo), h) for lo, h in bitmap_digests(oracle.pack(rel))] == g["digests"])
            rec = {"part": name, "workload": f"d={d} N={N} seed {seed}", "threads": T, "cpu": cpu_model(),
                   "link_s": t1 - t0, "count_s": t2 - t1, "pairs_per_s": out["R"] / (t2 - t1),
                   "bit_tests_per_s": out["W"] / (t2 - t1), "equal_to_stored": bool(same)}
            if name == "single1":
                t3 = time.perf_counter()
                oracle.action(rel, 1)
                rec["count_s_1_thread"] = time.perf_counter() - t3
            print(json.dumps(rec), flush=True)
            ok = ok and same
        elif name == "batch":
            rows = {}
            with open(os.path.join(HERE, "batch_4096_seed3.txt")) as fh:
                for ln in fh:
                    if not ln.startswith("#") and ln.strip():
                        v = ln.split()
                        rows[int(v[0])] = v
            t_link = t_count = 0.0
            R = W = 0
            bad = []
            for k, sp in enumerate(inputs.batch_workload()):
                t0 = time.perf_counter()
                rel = oracle.link(sp.d, oracle.sprinkle_sorted(sp.d, sp.N, sp.seed, sp.seq), threads)
                t1 = time.perf_counter()
                out = oracle.action(rel, threads)
                t2 = time.perf_counter()
                t_link += t1 - t0
                t_count += t2 - t1
                R += out["R"]
                W += out["W"]
                f = [str(x) for x in counts_fields(sp.d, sp.N, out)] + [set_digest16(oracle.pack(rel))]
                if f != rows[k][5:]:
                    bad.append(k)
            print(json.dumps({"part": "batch", "workload": "4096 diamonds, seed 3", "threads": T,
                              "cpu": cpu_model(), "link_s": t_link, "count_s": t_count, "pairs_per_s": R / t_count,
                              "bit_tests_per_s": W / t_count, "equal_to_stored": not bad,
                              "differing_sets": bad[:16]}), flush=True)
            ok = ok and not bad
        else:
            raise SystemExit(f"--verify: unknown part {name}")
    return 0 if ok else 1


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default="single1,single2,batch,serve,single3")
    ap.add_argument("--verify", default=None)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--ckpt", default=os.path.join(tempfile.gettempdir(), "csg_golden_ckpt"))
    args = ap.parse_args()
    if args.verify:
        return verify(args.verify.split(","), args.threads)
    os.makedirs(args.ckpt, exist_ok=True)
    for name in args.only.split(","):
        if name in SINGLES:
            run_single(name, args.threads, args.ckpt)
        elif name == "batch":
            run_batch(args.threads, args.ckpt)
        elif name == "serve":
            run_serve(args.threads, args.ckpt)
        else:
            raise SystemExit(f"unknown part {name}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
