"""Runs the library's calls on small and odd-sized sets, a mixed batch, caller bitmaps, the
allocation-free call, the service and the bench-size set, through the library given on the
command line (the bounds-checked build), compares every result with the oracle, then requires
every bounds-check word to be zero.  Started by tests/test_gpu_zy_checked.py in a fresh
process, so the checked library is the one the binding loads."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import oracle  # noqa: E402
from golden_io import read_full  # noqa: E402
from paper_1709_03013_gb300 import csg, inputs  # noqa: E402


def same(r, want, what):
    got = (r.R, list(r.Nk), r.sum_m, r.W, r.combo, r.status)
    exp = (want["R"], [int(x) for x in want["Nk"]], want["sum_m"], want["W"], want["combo"], 0)
    assert got == exp, (what, got, exp)
    assert abs(r.S - want["S"]) <= 1e-12 * max(1.0, abs(want["S"])), what


def main(lib_path):
    import torch
    csg.load(lib_path)
    methods = (csg.POPC, csg.TC_FP4, csg.TC_FP8)
    with csg.Context(0) as ctx:
        for d, N, seed in ((2, 1, 1), (2, 2, 2), (4, 3, 3), (2, 5, 4), (4, 127, 5), (2, 1000, 6), (4, 2048, 7),
                           (2, 3001, 8), (4, 4097, 9)):
            s = ctx.sprinkle(d, N, seed).link()
            want = oracle.run(d, N, seed)
            assert np.array_equal(s.bitmap(), oracle.pack(want["rel"], s.info()["stride"])), (d, N)
            for m in methods:
                same(s.action(m), want, (d, N, m))
            if d == 2 and N >= 1000:
                dev = torch.zeros(N, dtype=torch.int64, device="cuda")
                for m in (csg.POPC, csg.TC):
                    s.action_hist(dev.data_ptr(), N, m)
                    torch.cuda.synchronize()
                    assert np.array_equal(dev.cpu().numpy().view(np.uint64), want["hist"]), (d, N, m)
                phi = torch.from_numpy(np.arange(N, dtype=np.float64) % 7 - 3).cuda()
                B = torch.empty_like(phi)
                want_b, _ = oracle.dalembertian(want["rel"], phi.cpu().numpy(), 1.0)
                for m in (csg.POPC, csg.TC):
                    s.dalembertian(phi.data_ptr(), B.data_ptr(), 1.0, m)
                    torch.cuda.synchronize()
                    assert np.array_equal(B.cpu().numpy(), want_b), (d, N, m)  # integer phi: exact
                S_eps, _ = s.action_smeared(0.25, csg.POPC)
                ref = oracle.smeared(N, want["hist"], 0.25)
                assert abs(S_eps - ref) <= 1e-9 * max(1.0, abs(ref)), (S_eps, ref)
            info = s.info()
            out = torch.zeros(csg.RESULT_BYTES, dtype=torch.uint8, device="cuda")
            csg.action_noalloc(d, N, info["rows_ptr"], info["stride"], out.data_ptr())
            torch.cuda.synchronize()
            same(csg.result_from_bytes(out.cpu().numpy().tobytes()), want, (d, N, "noalloc"))
            s.free()
        specs = [(2 if k % 2 == 0 else 4, int(n), 31, k)
                 for k, n in enumerate(np.random.default_rng(31).integers(1, 3000, 24))]
        for m in methods:
            for sp, r in zip(specs, ctx.run_batch(specs, m)):
                same(r, oracle.run(*sp), (sp, m))
        rel = inputs.layered_order_rel(900, 4)
        dev = torch.from_numpy(inputs.pack_rows(rel, 16).view(np.int64)).cuda()
        s = ctx.set_from_bitmap(4, 900, dev.data_ptr(), 16)
        want = oracle.action(rel)
        want["combo"], want["S"] = oracle.finalize(4, 900, want["Nk"])
        for m in methods:
            same(s.action(m), want, ("bitmap", m))
        s.free()
        tickets = [(sp, ctx.serve_submit(*sp)) for sp in specs[:10]]
        for sp, t in tickets:
            same(ctx.serve_poll(t, timeout_ms=120000), oracle.run(*sp), ("served", sp))
        g = read_full("full_d4_n65536_seed1.txt")
        s = ctx.sprinkle(4, 65536, 1).link()
        for m in (csg.TC, csg.POPC):
            same(s.action(m), g, ("d=4 N=65536", m))
        s.free()
    words = csg.check_words()
    assert len(words) == 6, words
    assert all(w == 0 for w in words), [hex(w) for w in words]
    print("checked build clean:", [hex(w) for w in words])


if __name__ == "__main__":
    main(sys.argv[1])
