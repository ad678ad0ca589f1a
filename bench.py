#!/usr/bin/env python3
"""Benchmark of the causal-set action path on GB300.

One step is one pass of the whole path over one synthetic set: sprinkle N elements
into the flat causal diamond, sort them by time, link them into the bit-packed
causal matrix, count every related pair's interval (N_0..N_3, R, sum m, W) and form
the action.  The default workload is the d=4 diamond with N=65536 (seed 1): its
bitmap is 512 MiB, larger than the 129 MB L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0).  `value` is related-pair interval counts per second
(R / step time) with the set generated on the device; `e2e` is the same metric
through the public API from host coordinates (copied in every step) to the host
result.  `roofline` is the action kernel of the chosen method (default: the tensor-core
form with fp4 operands, against the fp4 tensor peak; the popcount form against the
integer-pipe popcount peak is reported beside it, the tensor form's operand feed against
the per-SM L2-to-shared-memory rate a probe measures in the run (`roofline_tc_feed`), the
tensor rate also against the pair MMA's own rate on resident operands (`mma_probe_tflops`), and
the link kernel against the fp32 pipe for d=4 and HBM write bandwidth for d=2);
`cpu_baseline` is the CPU oracle on a
bounded, stratified sample of the same workload (the same measurement as
`--impl reference`).  `batch` compares the batched (CUDA-graph) path with
one-set-at-a-time calls on 4096 mixed diamonds, and `serve` gives p50/p99 latency of the
20000-request Poisson stream through the service (--no-workloads skips both).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "related-pair interval counts/s + p99 latency, served vs plain, bit-exact N_k"
UNIT = "pairs/s"
WORKLOAD = dict(d=4, N=65536, seed=1)
# interval-count methods of the C ABI (CSG_POPC, CSG_TC, CSG_TC_FP8, CSG_TC_FP4)
METHODS = {"popc": 0, "tc": 1, "tc8": 2, "tc4": 3}
WORKLOAD_NAME = "d=4 flat causal diamond, N=65536, seed 1 (sprinkle+sort+link+action)"


def arm_config(method: str, world: int) -> dict:
    """The default line's config (both arms report the same one)."""
    fp4 = method in ("tc", "tc4")
    return {"workload": WORKLOAD_NAME, "d": WORKLOAD["d"], "N": WORKLOAD["N"], "seed": WORKLOAD["seed"],
            "method": method,
            "l2": ("inputs larger than L2 (512 MiB bitmap, "
                   f"{'4 GiB fp4' if fp4 else '8 GiB fp8'} operands per step)"),
            "parallelism": "replicas" if world > 1 else "single"}

# Popcount peak: 16 32-bit POPC results per SM per clock (the CUDA programming guide's
# throughput table; csg_measure_popc_rate's loop of independent popcounts sustains 15.2 on
# this GB300, measured live in every run), 32 bit-ops each.
POPC_PER_SM_CLK = 16
SMS = 152


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh)
    except OSError:
        return {}


class NvmlClockSampler:
    """Samples the SM clock and the clock-event (throttle) reasons through NVML every few
    milliseconds while running (read-only queries; nothing is set).  Raises OSError when
    NVML cannot be used, so the caller can fall back to nvidia-smi."""

    # nvmlClocksEventReasons bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, cuda_index: int, period_s: float = 0.002):
        import ctypes
        self.period = period_s
        try:
            self.nv = ctypes.CDLL("libnvidia-ml.so.1")
        except OSError as e:
            raise OSError(f"NVML unavailable: {e}")
        if self.nv.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.handle = ctypes.c_void_p()
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
        target = vis[cuda_index].strip() if cuda_index < len(vis) and vis[cuda_index].strip() else str(cuda_index)
        if target.startswith("GPU-"):
            rc = self.nv.nvmlDeviceGetHandleByUUID(target.encode(), ctypes.byref(self.handle))
        else:
            rc = self.nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(int(target)), ctypes.byref(self.handle))
        if rc != 0:
            self.nv.nvmlShutdown()
            raise OSError("no NVML handle for the device")
        mx = ctypes.c_uint()
        self.max_mhz = float(mx.value) if self.nv.nvmlDeviceGetMaxClockInfo(self.handle, 1, ctypes.byref(mx)) == 0 else None
        self.fn_reasons = getattr(self.nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(self.nv, "nvmlDeviceGetCurrentClocksThrottleReasons")
        self.sm, self.masks = [], []
        self._stop = threading.Event()

    def _run(self):
        import ctypes
        mhz, mask = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            if self.nv.nvmlDeviceGetClockInfo(self.handle, 1, ctypes.byref(mhz)) == 0:
                self.sm.append(float(mhz.value))
                self.masks.append(mask.value if self.fn_reasons(self.handle, ctypes.byref(mask)) == 0 else 0)
            time.sleep(self.period)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        self._t.join(timeout=2)
        self.nv.nvmlShutdown()

    def summary(self):
        if not self.sm:
            return None
        reasons = sorted({nm for m in self.masks for bit, nm in self.REASONS.items() if m & bit})
        return {"sm_mhz": statistics.median(self.sm), "sm_max_mhz": self.max_mhz or max(self.sm),
                "reasons": reasons, "samples": len(self.sm), "source": "nvml, 2 ms period"}


def clock_sampler(cuda_index: int):
    """NVML sampling when the library can be loaded, else nvidia-smi."""
    try:
        return NvmlClockSampler(cuda_index)
    except (OSError, AttributeError, ValueError):
        return ClockSampler(cuda_index)


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


TRAFFIC_BASIS = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch on this workload, recorded in "
                 "profiles/traffic.json for this exact kernel source (hash of the whole file); null once it changed")


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu record, or None when the kernel's
    source has changed since the counters were taken (or no record exists)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            rec = json.load(fh).get(kernel)
        if not rec or rec.get("workload") != workload:
            return None
        with open(os.path.join(ROOT, rec["source"]), "rb") as fh:
            text = fh.read()
        # the whole source file (kernels and the host code that orders their work), with
        # comments and whitespace removed (a comment edit does not change the kernel)
        code = re.sub(r"/\*.*?\*/", "", text.decode(), flags=re.S)
        code = re.sub(r"//[^\n]*", "", code)
        code = re.sub(r"\s+", " ", code)
        sha = hashlib.sha256(code.encode()).hexdigest()[:16]
        return rec["dram_bytes_per_launch"] if sha == rec["code_sha256_16"] else None
    except (OSError, ValueError, KeyError):
        return None


def reduce_over_ranks(dist, ms: float, units: float, device) -> tuple[float, float]:
    """Replicas: the job's time is the slowest rank's, its work the sum over ranks."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def launches_per_step(N: int, tc: bool) -> int:
    # sprinkle+keys, chunk sort, merge passes, gather; link screen values, link; [expand];
    # action; finalize
    passes, w = 0, 1024
    while w < N:
        passes += 1
        w *= 2
    return 3 + passes + 2 + (1 if tc else 0) + 2


STRATA = 16  # equal row strata of the bench set; one block of rows is drawn from each in turn


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def oracle_sample(steps: int, warmup: int):
    """The oracle as it stands on a bounded, stratified sample of the bench set (d=4,
    N=65536, seed 1): its link of the whole set (built once, not timed), then, per step,
    its triple loop over one block of 16 rows per thread (so every thread gets several
    dynamic chunks), centred in stratum k mod 16 of 16 equal row strata (strata visited in
    an interleaved order).  Returns the timed steps' pairs, bit tests and seconds."""
    import oracle
    d, N, seed = WORKLOAD["d"], WORKLOAD["N"], WORKLOAD["seed"]
    threads = os.cpu_count() or 1
    rows = 16 * threads
    c = oracle.sprinkle_sorted(d, N, seed, 0)
    rel = oracle.link(d, c, threads)
    order = [0, 8, 4, 12, 2, 10, 6, 14, 1, 9, 5, 13, 3, 11, 7, 15]
    per = {}  # stratum -> [(pairs, bit tests, seconds)] of its timed blocks
    for k in range(warmup + steps):
        st = order[k % STRATA]
        mid = (2 * st + 1) * N // (2 * STRATA)
        lo = max(0, min(N - rows, mid - rows // 2))
        t0 = time.perf_counter()
        out = oracle.action(rel, threads, rows=(lo, lo + rows))
        dt = time.perf_counter() - t0
        if k >= warmup:
            per.setdefault(st, []).append((out["R"], out["W"], dt))
    # stratified estimate of the whole set's rates: each visited stratum's mean block counts
    mean = lambda v, i: sum(x[i] for x in v) / len(v)
    P = sum(mean(v, 0) for v in per.values())
    B = sum(mean(v, 1) for v in per.values())
    T = sum(mean(v, 2) for v in per.values())
    allb = [x for v in per.values() for x in v]
    return {"pairs_per_s": P / T, "bits_per_s": B / T, "pairs": sum(x[0] for x in allb),
            "bits": sum(x[1] for x in allb), "seconds": sum(x[2] for x in allb), "threads": threads,
            "rows": rows, "steps": steps, "strata": len(per)}


def sample_description(m: dict) -> str:
    return (f"{m['steps']} blocks of {m['rows']} consecutive first elements (16 per thread), each centred in "
            f"one of 16 equal row strata in turn ({m['strata']} strata visited), of the d=4 N=65536 set "
            f"(seed 1); the oracle's own link of the whole set built first (not timed); {m['pairs']} related "
            f"pairs and {m['bits']:.3e} bit tests in {m['seconds']:.2f} s; value = the strata's summed mean "
            f"pairs per block over their summed mean seconds per block")


def cpu_baseline():
    """One stratum each: the same measurement as the reference arm with 16 steps."""
    m = oracle_sample(steps=STRATA, warmup=1)
    return {"value": m["pairs_per_s"], "unit": UNIT, "cores": m["threads"], "kind": "oracle",
            "cpu": cpu_model(), "bit_tests_per_s": m["bits_per_s"], "sample": sample_description(m)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    m = oracle_sample(steps=args.steps, warmup=args.warmup)
    value = m["pairs_per_s"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * m["seconds"] / m["steps"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": arm_config(args.method, int(os.environ.get("WORLD_SIZE", "1"))),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": m["threads"], "kind": "oracle",
                             "cpu": cpu_model(), "bit_tests_per_s": m["bits_per_s"],
                             "sample": sample_description(m)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def profile_action(args):
    """A small fixed workload for ncu captures: sprinkle (seed 1), link, then
    --reps action launches of the chosen method (the first one warms up)."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_1709_03013_gb300 import csg
    method = METHODS[args.method]
    with csg.Context(0) as ctx:
        s = ctx.sprinkle(args.d, args.n, 1, 0).link()
        for r in range(args.reps):
            t0 = time.perf_counter()
            res = s.action(method)
            print(r, res.R, res.Nk, res.W, f"{(time.perf_counter() - t0) * 1e3:.2f} ms", flush=True)
        s.free()
    return 0


def profile_batch(args):
    """A fixed workload for ncu launch lists of the batch: the 4096-set batch (seed 3) built
    into its CUDA graph with the default tuning (autotuning off, so no candidate runs), then
    --reps replays."""
    os.environ["CSG_AUTOTUNE"] = "0"
    import __graft_entry__
    __graft_entry__.build()
    from paper_1709_03013_gb300 import csg, inputs
    method = METHODS[args.method]
    specs = [(s.d, s.N, s.seed, s.seq) for s in inputs.batch_workload(n_sets=args.n_sets)]
    with csg.Context(0) as ctx:
        for r in range(args.reps + 1):
            t0 = time.perf_counter()
            res = ctx.run_batch(specs, method)
            print("build" if r == 0 else f"replay {r}", sum(x.R for x in res),
                  f"{(time.perf_counter() - t0) * 1e3:.2f} ms", flush=True)
    return 0


def bench_batch(args, emit=True):
    """Plain (one set at a time, each call synchronised) vs batched (one call for all
    sets, every step batched) on the mixed-size workload: 4096 diamonds, d alternating
    2/4, N log-uniform in [256, 8192], seed 3."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1709_03013_gb300 import csg, inputs
    method = METHODS[args.method]
    specs = [(s.d, s.N, s.seed, s.seq) for s in inputs.batch_workload(n_sets=args.n_sets)]
    ctx = csg.Context(0)
    stream = torch.cuda.current_stream()

    def plain():
        out = []
        for d, N, seed, seq in specs:
            st = ctx.sprinkle(d, N, seed, seq)
            st.link()
            out.append(st.action(method))
            st.free()
        return out

    def batched():
        return ctx.run_batch(specs, method)

    res_b = batched()
    res_p = plain()
    assert [(r.R, r.Nk, r.W) for r in res_b] == [(r.R, r.Nk, r.W) for r in res_p]
    for _ in range(max(0, args.warmup - 1)):
        batched()
    times = {}
    for name, fn in (("batched", batched), ("plain", plain)):
        reps = args.steps if name == "batched" else max(1, args.steps // 2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        times[name] = e0.elapsed_time(e1) / reps
    R = sum(r.R for r in res_b)
    W = sum(r.W for r in res_b)
    line = {"metric": METRIC, "value": R / (times["batched"] / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": times["batched"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {0: "u64", 2: "fp8"}.get(method, "fp4"), "data": "synthetic",
            "config": {"workload": f"batch: {len(specs)} flat diamonds, d alternating 2/4, N log-uniform "
                                   f"in [256, 8192], seed 3 (sprinkle+sort+link+action per set)",
                       "method": args.method, "sets": len(specs), "sum_R": R, "sum_W": W},
            "plain": {"value": R / (times["plain"] / 1e3), "ms": times["plain"]},
            "batched_over_plain": times["plain"] / times["batched"]}
    ctx.close()
    if emit:
        print(json.dumps(line), flush=True)
    return line


def bench_desitter(args):
    """The paper's convergence experiment (Sec. 5.2, Fig. action): smeared action
    (Eq. s_smeared, eps = 2^-6) of sprinkles into the 1+1 de Sitter slab with eta0 = 0.5,
    ten sets per size for N = 2^10 .. 2^17; the mean should approach the Einstein-Hilbert
    value 4 pi tan(eta0) ~ 6.865 from N ~ 2^14 on, with a spread growing like sqrt(N)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1709_03013_gb300 import csg
    eta0, eps, graphs = 0.5, 2.0 ** -6, 10
    S_EH = 4 * math.pi * math.tan(eta0)
    rows = []
    hists = []  # interval abundances of the N = 2^15 slabs (the left panel of the paper's figure)
    with csg.Context(0) as ctx:
        for p in range(10, 18):
            N = 1 << p
            vals, t0 = [], time.perf_counter()
            for g in range(graphs):
                s = ctx.sprinkle_desitter(N, eta0, seed=5, seq=g)
                s.link()
                S, _ = s.action_smeared(eps, csg.TC)
                vals.append(S)
                if p == 15:
                    dev = torch.zeros(N, dtype=torch.int64, device="cuda")
                    s.action_hist(dev.data_ptr(), N, csg.TC)
                    torch.cuda.synchronize()
                    hists.append(dev.cpu().numpy().astype(np.float64))
                s.free()
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1e3 / graphs
            v = np.array(vals)
            rows.append({"N": N, "mean": float(v.mean()), "std": float(v.std(ddof=1)),
                         "sem": float(v.std(ddof=1) / math.sqrt(graphs)), "ms_per_set": ms})
    # n_i (1-based: pairs whose interval holds i - 1 elements) of the paper's figure: every i up
    # to 64, then sums over octaves [2^k, 2^(k+1)) of i
    H = np.array(hists)
    top = int(np.nonzero(H.sum(axis=0))[0].max()) + 1
    single = [{"i": m + 1, "mean": float(H[:, m].mean()), "std": float(H[:, m].std(ddof=1))} for m in range(min(64, top))]
    octaves = []
    lo = 64
    while lo < top:
        hi = min(top, 2 * lo)
        blk = H[:, lo:hi].sum(axis=1)
        octaves.append({"i_from": lo + 1, "i_to": hi, "mean": float(blk.mean()), "std": float(blk.std(ddof=1))})
        lo = hi
    abundance = {"N": 1 << 15, "sets": len(hists), "largest_i": top, "mean_pairs": float(H.sum(axis=1).mean()),
                 "n_i": single, "octaves": octaves}
    print(json.dumps({"experiment": "smeared action in the 1+1 de Sitter slab (Sec. 5.2)", "eta0": eta0,
                      "eps": eps, "sets_per_size": graphs, "S_EH": S_EH, "sizes": rows,
                      "interval_abundances": abundance}), flush=True)
    return 0


def bench_sizes(args):
    """Interval-count throughput against set size: K linked d=4/d=2 diamonds of one size
    (K N^3 fixed near 2.7e11 for N <= 8192), counted in one batch launch; the stage time of the
    counting kernel alone (operand expansion reported beside it), in algorithmic tensor
    flops 2 C(N,3) per set.  Small sets show the per-tile cost of the tensor form: each
    256 x 256 tile drains its accumulator and books its pairs however short its K range."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1709_03013_gb300 import csg
    rows = []
    with csg.Context(0) as ctx:
        for N, K in ((512, 2048), (1024, 1024), (2048, 512), (4096, 128), (8192, 32), (16384, 8), (32768, 2)):
            sets = [ctx.sprinkle(2 + 2 * (k % 2), N, 99, k).link() for k in range(K)]
            torch.cuda.synchronize()
            flops = K * 2.0 * math.comb(N, 3)
            row = {"N": N, "sets": K}
            for name, m in (("tc4", csg.TC_FP4), ("tc8", csg.TC_FP8), ("popc", csg.POPC)):
                ctx.action_batch(sets, m)
                ctx.set_timing(True)
                ctx.action_batch(sets, m)
                st = ctx.stage_times()
                ctx.set_timing(False)
                a = st.get("action") or float("nan")
                row[name] = {"action_ms": a, "expand_ms": st.get("expand"), "tflops": flops / (a * 1e-3) / 1e12}
            rows.append(row)
            for x in sets:
                x.free()
    print(json.dumps({"experiment": "interval counts against set size (batch launches of equal sets)",
                      "unit": "algorithmic TFLOP/s (2 C(N,3) per set)", "sizes": rows}), flush=True)
    return 0


def bench_dalembertian(args):
    """Cost of the discrete d'Alembertian (Eq. b_local) beside the plain interval counts on
    the d=2 N=131072 set (seed 2): the layer sums ride on the counting pass, so the extra
    time is the atomics of the pairs with m <= 2 and one elementwise pass."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1709_03013_gb300 import csg
    d, N, seed = 2, 131072, 2
    out = {"experiment": "discrete d'Alembertian (Eq. b_local) beside the action",
           "workload": f"d={d} N={N} seed {seed}", "phi": "t^2 - x^2 at the sprinkled coordinates", "l": 1.0}
    with csg.Context(0) as ctx:
        s = ctx.sprinkle(d, N, seed, 0).link()
        c = torch.from_numpy(s.coords()).cuda()
        phi = (c[0] * c[0] - c[1] * c[1]).contiguous()
        B = torch.empty_like(phi)
        stream = torch.cuda.current_stream()
        for name, method, reps in (("tc", csg.TC, 3), ("popc", csg.POPC, 1)):
            times = {}
            for label, fn in (("action", lambda: s.action(method)),
                              ("action+dalembertian", lambda: s.dalembertian(phi.data_ptr(), B.data_ptr(), 1.0, method))):
                fn()  # warm-up
                ms = []
                for _ in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    fn()
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms.append(e0.elapsed_time(e1))
                times[label] = min(ms)
            res = s.action(method)
            out[name] = {"ms": times, "L123_pairs": [int(v) for v in res.Nk[:3]],
                         "overhead": times["action+dalembertian"] / times["action"] - 1.0}
        s.free()
    print(json.dumps(out), flush=True)
    return 0


def bench_serve(args, emit=True):
    """Requests arrive as a Poisson stream (d in {2,4} 50/50, N log-uniform in
    [1024, 65536], seed 4) and go through the continuous-batching service; latency is
    arrival -> result ready.  Capacity is the service's own throughput with every request
    submitted at once (admission by the 160 GB budget keeps the resident sets bounded, so
    any number of requests works); the rate is swept as fractions of it.  Every served
    result must equal the result of the same request computed alone."""
    import threading as th
    import __graft_entry__
    __graft_entry__.build()
    from paper_1709_03013_gb300 import csg, inputs
    reqs = inputs.serve_workload(n_req=args.n_req)
    specs = [(r.spec.d, r.spec.N, r.spec.seed, r.spec.seq) for r in reqs]
    ctx = csg.Context(0, budget_bytes=160 * 10 ** 9)

    def run_stream(arrive):
        """Submits request k at arrive[k] seconds; returns (results, completion times)."""
        n = len(specs)
        done = [0.0] * n
        results = [None] * n
        tickets = [None] * n
        submitted = [0]
        start = time.perf_counter()

        def collect():
            # poll the submitted, unfinished tickets without blocking, so that out-of-order
            # completions are timed when they happen
            pending, seen = [], 0
            while seen < n or pending:
                upto = submitted[0]
                while seen < upto:
                    pending.append(seen)
                    seen += 1
                still = []
                for k in pending:
                    r = ctx.serve_poll(tickets[k], timeout_ms=0)
                    if r is None:
                        still.append(k)
                    else:
                        results[k] = r
                        done[k] = time.perf_counter() - start
                pending = still
                time.sleep(0.0002)

        poller = th.Thread(target=collect)
        poller.start()
        for k, (d, N, seed, seq) in enumerate(specs):
            delay = arrive[k] - (time.perf_counter() - start)
            if delay > 0:
                time.sleep(delay)
            tickets[k] = ctx.serve_submit(d, N, seed, seq)
            submitted[0] = k + 1
        poller.join()
        return results, done

    # warm the service and the single-set path
    warm = specs[:16]
    for d, N, seed, seq in warm:
        st = ctx.sprinkle(d, N, seed, seq)
        st.link()
        st.action(csg.TC)
        st.free()
    # plain: the requests one at a time through the single-set calls (also the reference
    # results the served ones are checked against)
    res_b = []
    t0 = time.perf_counter()
    for d, N, seed, seq in specs:
        st = ctx.sprinkle(d, N, seed, seq)
        st.link()
        res_b.append(st.action(csg.TC))
        st.free()
    plain_rate = len(specs) / (time.perf_counter() - t0)
    # capacity: everything submitted at once
    res_cap, done_cap = run_stream(np.zeros(len(specs)))
    capacity = len(specs) / max(done_cap)
    cap_ok = all(r is not None and (r.R, r.Nk, r.W) == (b.R, b.Nk, b.W) for r, b in zip(res_cap, res_b))
    cap_s = max(done_cap)
    sweeps = []
    for frac in [float(x) for x in args.rates.split(",")]:
        rate = frac * capacity
        gaps = np.random.default_rng(4).exponential(1.0 / rate, size=len(specs))
        arrive = np.cumsum(gaps) - gaps[0]
        results, done = run_stream(arrive)
        lat = np.array(done) - arrive
        span = max(done)
        ok = all(r is not None and (r.R, r.Nk, r.W) == (b.R, b.Nk, b.W) for r, b in zip(results, res_b))
        sweeps.append({"rate_frac": frac, "rate_req_s": rate, "throughput_req_s": len(specs) / span,
                       "pairs_per_s": sum(r.R for r in results) / span,
                       "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                       "results_equal_alone": ok})
    R = sum(r.R for r in res_b)
    line = {"metric": METRIC, "value": R / cap_s, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": cap_s * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "fp4", "data": "synthetic",
            "config": {"workload": f"serve: {len(specs)} requests, d in {{2,4}} 50/50, N log-uniform in "
                                   f"[1024, 65536], Poisson arrivals, seed 4, 160 GB admission budget",
                       "method": "tc"},
            "capacity_req_s": capacity, "capacity_results_equal_alone": cap_ok, "plain_req_s": plain_rate,
            "served_capacity_over_plain": capacity / plain_rate, "sweep": sweeps}
    ctx.close()
    if emit:
        print(json.dumps(line), flush=True)
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--method", default="tc4", choices=list(METHODS),
                    help="popc, or the tensor form: tc (library default format), tc8 (fp8), tc4 (fp4)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the batch and serve summaries of the default line")
    ap.add_argument("--profile-batch", action="store_true",
                    help="profiling mode: the 4096-set batch graph, then --reps replays")
    ap.add_argument("--profile-action", action="store_true",
                    help="profiling mode: one sprinkled set, then --reps action launches")
    ap.add_argument("--d", type=int, default=4)
    ap.add_argument("--n", type=int, default=40000)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--workload", default="single", choices=["single", "batch", "serve", "desitter", "dalembertian", "sizes"],
                    help="single: the d=4 N=65536 set; batch: 4096 mixed diamonds, plain vs batched; "
                         "serve: Poisson request stream through the service, p50/p99 latency")
    ap.add_argument("--n-sets", type=int, default=4096)
    ap.add_argument("--n-req", type=int, default=20000,
                    help="serve: number of requests (the default is the full 20000-request stream)")
    ap.add_argument("--rates", default="0.25,0.5,0.75,0.9,1.1",
                    help="serve: arrival rates as fractions of the measured batched capacity")
    args = ap.parse_args()
    if args.profile_action:
        return profile_action(args)
    if args.profile_batch:
        return profile_batch(args)
    if args.workload == "batch":
        bench_batch(args)
        return 0
    if args.workload == "serve":
        bench_serve(args)
        return 0
    if args.workload == "desitter":
        bench_desitter(args)
        return 0
    if args.workload == "dalembertian":
        bench_dalembertian(args)
        return 0
    if args.workload == "sizes":
        bench_sizes(args)
        return 0
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    __graft_entry__.build()
    from paper_1709_03013_gb300 import csg

    method = METHODS[args.method]
    is_tc = method != csg.POPC
    d, N, seed = WORKLOAD["d"], WORKLOAD["N"], WORKLOAD["seed"]
    seq = rank  # replicas: each rank runs its own independent set
    ctx = csg.Context(local)
    ctx.set_timing(True)
    stream = torch.cuda.current_stream()

    def step(m=method):
        s = ctx.sprinkle(d, N, seed, seq)
        s.link()
        r = s.action(m)
        s.free()
        return r

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()

    # ---- device-resident timing: the inputs are (d, N, seed); the set is generated on the GPU
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stage_ms = {k: 0.0 for k in csg.Context.STAGES}
    results = []
    step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with clock_sampler(local) as clk:
        ev0.record(stream)
        step_ev[0].record(stream)
        for k_step in range(args.steps):
            results.append(step())
            step_ev[k_step + 1].record(stream)
            for k, v in ctx.stage_times().items():
                stage_ms[k] += v or 0.0
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    step_times = [step_ev[k].elapsed_time(step_ev[k + 1]) for k in range(args.steps)]
    R_total = sum(r.R for r in results)
    if dist is not None:
        ms, R_total = reduce_over_ranks(dist, ms, R_total, torch.device("cuda", local))
    value = R_total / (ms / 1e3)
    res = results[-1]
    stage_avg = {k: v / args.steps for k, v in stage_ms.items()}
    act_ms = stage_avg["action"]

    # ---- the other method's action kernel on the same set (reported beside the main one)
    other = csg.TC_FP8 if method == csg.POPC else csg.POPC
    s = ctx.sprinkle(d, N, seed, seq).link()
    s.action(other)
    ro = s.action(other)
    other_ms = ctx.stage_times()["action"]
    assert (ro.R, tuple(ro.Nk), ro.sum_m, ro.W) == (res.R, tuple(res.Nk), res.sum_m, res.W)
    coords_host = s.coords()
    s.free()

    # ---- the link kernel of the d=2 N=131072 set (seed 2), whose 2 GiB bitmap write is its bound
    s2 = ctx.sprinkle(2, 131072, 2, seq)
    s2.link()
    s2.link()
    link2_ms = ctx.stage_times()["link"]
    link2_bytes = 131072 * s2.info()["stride"] * 8
    s2.free()

    # ---- end to end through the public API from pinned host coordinates to the host result
    pinned = torch.from_numpy(coords_host).pin_memory()
    host_np = pinned.numpy()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    e_pairs = 0
    for _ in range(args.steps):
        se = ctx.set_from_coords(d, host_np)
        se.link()
        re_ = se.action(method)
        se.free()
        e_pairs += re_.R
    e1.record(stream)
    barrier()
    e_ms = e0.elapsed_time(e1)

    if rank != 0:
        ctx.close()
        if dist is not None:
            dist.destroy_process_group()
        return 0

    pk = peaks()
    clocks = clk.summary()
    popc_rate = csg.measure_popc_rate(local)  # popcounts per second, measured live
    sm_max = (clocks or {}).get("sm_max_mhz") or pk.get("sm_max_mhz") or 2070.0
    popc_peak = SMS * POPC_PER_SM_CLK * 32 * sm_max * 1e6          # bit-ops/s
    fp4 = method in (csg.TC, csg.TC_FP4)  # the tensor form's default format is fp4
    # the contraction's own dtype: measured bf16 dense burst x the nominal ratio (fp8 2, fp4 6)
    tc_peak = (6.0 if fp4 else 2.0) * pk.get("bf16_tflops", 1900.0)
    tc_flops = 2.0 * math.comb(N, 3)                                # triangle-restricted contraction
    popc_ms = act_ms if method == csg.POPC else other_ms
    tc_ms = act_ms if is_tc else other_ms
    popc_roof = {"bound": "alu", "achieved": res.W / (popc_ms / 1e3), "peak": popc_peak,
                 "unit": "bit-ops/s", "frac": res.W / (popc_ms / 1e3) / popc_peak,
                 "traffic": recorded_traffic("action_popc_kernel<16, 0>", f"d={d} N={N} seed {seed}"),
                 "traffic_basis": TRAFFIC_BASIS,
                 "kernel_ms": popc_ms,
                 "peak_basis": (f"{SMS} SMs x {POPC_PER_SM_CLK} POPC/clk (CUDA guide throughput table) x 32 bits x "
                                f"{sm_max:.0f} MHz"),
                 "popc_probe_per_sm_clk": popc_rate / SMS / (sm_max * 1e6)}
    tc_ach = tc_flops / (tc_ms / 1e3) / 1e12
    try:  # the pair MMA itself on resident operands, measured live (beside the contract's peak)
        mma_probe = csg.measure_mma_rate(csg.TC_FP4 if fp4 else csg.TC_FP8, local) / 1e12
    except csg.CsgError:
        mma_probe = None
    tc_roof = {"bound": "tensor", "achieved": tc_ach, "peak": tc_peak, "unit": "TFLOP/s",
               "frac": tc_ach / tc_peak,
               "mma_probe_tflops": mma_probe, "frac_of_mma_probe": tc_ach / mma_probe if mma_probe else None,
               "traffic": recorded_traffic(f"action_tc_kernel<{1 if fp4 else 0}>", f"d={d} N={N} seed {seed}"),
               "traffic_basis": TRAFFIC_BASIS,
               "kernel_ms": tc_ms,
               "peak_basis": (f"{'fp4 = 6' if fp4 else 'fp8 = 2'} x measured bf16 dense burst "
                              "(MEASURED_PEAKS.json; nominal dense ratio), of measured")}
    # the tensor form's second bound: the operand feed from L2 into shared memory, against
    # the per-SM rate a bulk-copy probe sustains (measured live).  Tile (I, J) of the pair
    # streams K = [256 I, 256 (J + 1)) in 32 KB stages per CTA (256 elements of K in fp4, 128
    # in fp8) and one 4 KB slot of relation words per CTA.
    try:
        feed_rate = csg.measure_l2_feed(local)                      # bytes per SM per second
    except csg.CsgError as exc:
        feed_rate, feed_err = None, str(exc)
    nb = (N + 255) // 256
    pair_stages = (256 // (256 if fp4 else 128)) * nb * (nb + 1) * (nb + 2) // 6
    feed_bytes = pair_stages * 2 * 32768 + nb * (nb + 1) // 2 * 2 * 4096
    feed_ach = feed_bytes / SMS / (tc_ms / 1e3)
    feed_roof = {"bound": "l2_to_smem", "achieved": feed_ach / 1e9,
                 "peak": feed_rate / 1e9 if feed_rate else None,
                 "unit": "GB/s per SM", "frac": feed_ach / feed_rate if feed_rate else None, "kernel_ms": tc_ms,
                 "bytes_per_launch": feed_bytes,
                 "peak_basis": "csg_measure_l2_feed: the kernel's copies (2D tensor-map loads, 128 rows x "
                               "128 B, 128-byte swizzle), six 32 KB stages in flight per SM, all SMs pulling "
                               "from an L2-resident matrix, measured in this run"}
    if feed_rate is None:
        feed_roof["probe_error"] = feed_err
    # link: d=4 against the fp32 pipe its screen runs on (the expanded interval of each pair
    # i < k as one add and four fused multiply-adds, and the margin's second sign: 10 flops a
    # pair), d=2 against HBM bandwidth for the bitmap it writes (every word once)
    fp32_peak = SMS * 128 * 2 * sm_max * 1e6 / 1e12                # TFLOP/s, non-tensor
    link4_ms = stage_avg["link"]
    link4_flops = 10.0 * N * (N - 1) / 2
    hbm = pk.get("hbm_gbs", 6687.1)
    link_roof = {
        "d4": {"bound": "fp32", "achieved": link4_flops / (link4_ms / 1e3) / 1e12, "peak": fp32_peak,
               "unit": "TFLOP/s", "frac": link4_flops / (link4_ms / 1e3) / 1e12 / fp32_peak, "kernel_ms": link4_ms,
               "workload": f"d=4 N={N} seed {seed}",
               "peak_basis": f"{SMS} SMs x 128 fp32 lanes x 2 flops x {sm_max:.0f} MHz (nominal)"},
        "d2": {"bound": "hbm", "achieved": link2_bytes / (link2_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
               "frac": link2_bytes / (link2_ms / 1e3) / 1e9 / hbm, "kernel_ms": link2_ms,
               "workload": "d=2 N=131072 seed 2 (2 GiB bitmap written)",
               "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs), of measured"},
    }
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "step_ms": {"min": min(step_times), "median": statistics.median(step_times), "max": max(step_times)},
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ("fp4" if fp4 else "fp8") if is_tc else "u64",
        "data": "synthetic",
        "config": arm_config(args.method, world),
        "gpu_launches": launches_per_step(N, is_tc) * args.steps,
        "result": {"R": res.R, "Nk": list(res.Nk), "sum_m": res.sum_m, "W": res.W, "combo": res.combo,
                   "S": res.S},
        "stage_ms": stage_avg,
        "bitops_per_s": res.W / (act_ms / 1e3),
        "roofline": tc_roof if is_tc else popc_roof,
        "roofline_other_method": popc_roof if is_tc else tc_roof,
        "roofline_tc_feed": feed_roof,
        "roofline_link": link_roof,
        "e2e": {"value": e_pairs / (e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(host_np.nbytes),
                "d2h_bytes_per_step": 88},
    }
    if clocks:
        line["clocks"] = clocks
    if not args.no_workloads and world == 1:
        # the metric's other halves: batched vs plain on the 4096-set mixed workload, and
        # served p50/p99 latency on the whole 20000-request Poisson stream at half and 0.9 of
        # the service's capacity
        ctx.close()
        ctx = None
        ns = argparse.Namespace(**vars(args))
        ns.n_sets, ns.steps, ns.warmup = 4096, 2, 1
        b = bench_batch(ns, emit=False)
        line["batch"] = {"workload": b["config"]["workload"], "value": b["value"], "unit": UNIT,
                         "batched_ms": b["ms_per_step"], "plain_ms": b["plain"]["ms"],
                         "batched_over_plain": b["batched_over_plain"]}
        ns.n_req, ns.rates = 20000, "0.5,0.9"
        v = bench_serve(ns, emit=False)
        line["serve"] = {"workload": v["config"]["workload"], "capacity_req_s": v["capacity_req_s"],
                         "plain_req_s": v["plain_req_s"],
                         "served_capacity_over_plain": v["served_capacity_over_plain"],
                         "capacity_results_equal_alone": v["capacity_results_equal_alone"],
                         "sweep": [{k: x[k] for k in ("rate_frac", "throughput_req_s", "pairs_per_s", "p50_ms",
                                                      "p99_ms", "results_equal_alone")} for x in v["sweep"]]}
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    if ctx is not None:
        ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
