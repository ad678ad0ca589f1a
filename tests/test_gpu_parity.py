"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Sprinkled coordinates, the bitmap C, R, N_0..N_3, sum m, W and the full
histogram must match bit for bit; the actions are exact integer combinations
scaled once in double, so they must match to 1e-12 relative (they are in fact
identical).  Sizes span several 256-element link tiles, several 16-row action
groups and ragged tails; the degenerate sizes N = 1, 2, 3 are included.
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


def _dev_words(words):
    import torch
    return torch.from_numpy(np.ascontiguousarray(words).view(np.int64)).cuda()


def _check_result(res, want, d, N):
    assert res.d == d and res.N == N and res.status == 0
    assert res.R == want["R"]
    assert list(res.Nk) == [int(x) for x in want["Nk"]]
    assert res.sum_m == want["sum_m"]
    assert res.W == want["W"]
    combo, S = oracle.finalize(d, N, want["Nk"])
    assert res.combo == combo
    assert abs(res.S - S) <= TOL_S * max(abs(S), 1.0)


SIZES = [(2, 1), (2, 2), (2, 3), (4, 3), (2, 64), (4, 65), (2, 255), (4, 257), (2, 1000),
         (4, 1000), (2, 2048), (4, 2500), (2, 4099), (4, 5000)]


@pytest.mark.parametrize("d,N", SIZES)
def test_sprinkle_link_action_match_oracle(ctx, csg, d, N):
    seed, seq = 1000 + N, d
    s = ctx.sprinkle(d, N, seed, seq)
    want_c = oracle.sprinkle_sorted(d, N, seed, seq)
    assert np.array_equal(s.coords(), want_c)           # bit-exact coordinates and order
    s.link()
    rel = oracle.link(d, want_c)
    got = s.bitmap()
    assert np.array_equal(got, oracle.pack(rel, got.shape[1]))  # every word, padding included
    want = oracle.action(rel)
    _check_result(s.action(csg.POPC), want, d, N)
    _check_result(s.action(csg.TC), want, d, N)
    s.free()


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("d,N", [(2, 700), (4, 1500), (2, 3000)])
def test_full_histogram(ctx, d, N, method):
    import torch
    s = ctx.sprinkle(d, N, 7, 0).link()
    want = oracle.action(oracle.link(d, oracle.sprinkle_sorted(d, N, 7, 0)))
    h = torch.full((N,), 7, dtype=torch.int64, device="cuda")  # the call zeroes it
    res = s.action_hist(h.data_ptr(), N, method)
    assert np.array_equal(h.cpu().numpy().astype(np.uint64), want["hist"])
    _check_result(res, want, d, N)
    # a short histogram keeps the low bins only
    h4 = torch.zeros(3, dtype=torch.int64, device="cuda")
    s.action_hist(h4.data_ptr(), 3, method)
    assert np.array_equal(h4.cpu().numpy().astype(np.uint64), want["hist"][:3])
    s.free()


@pytest.mark.parametrize("name,rel", [
    ("chain1", inputs.chain_rel(1)), ("chain5", inputs.chain_rel(5)), ("chain200", inputs.chain_rel(200)),
    ("chain1030", inputs.chain_rel(1030)), ("antichain77", inputs.antichain_rel(77)),
    ("random300", inputs.random_upper_rel(300, 0.3, 1)), ("random2000", inputs.random_upper_rel(2000, 0.05, 2)),
    ("layered1200", inputs.layered_order_rel(1200, 3)),
])
def test_action_from_bitmap(ctx, csg, name, rel):
    N = rel.shape[0]
    stride = max(1, (N + 63) // 64) + 3  # a caller stride unlike the library's
    dev = _dev_words(inputs.pack_rows(rel, stride))
    want = oracle.action(rel)
    for d in (2, 4):
        s = ctx.set_from_bitmap(d, N, dev.data_ptr(), stride)
        _check_result(s.action(csg.POPC), want, d, N)
        _check_result(s.action(csg.TC), want, d, N)
        s.free()


@pytest.mark.parametrize("name", ["diamond4.txt", "npos6.txt"])
def test_golden_fixtures_on_gpu(ctx, csg, golden, name):
    g = golden(name)
    rel = inputs.rel_from_edges(g["N"], g["rel"])
    dev = _dev_words(inputs.pack_rows(rel, 16))
    for d, key in ((2, "S2"), (4, "S4")):
        s = ctx.set_from_bitmap(d, g["N"], dev.data_ptr(), 16)
        for method in (csg.POPC, csg.TC, csg.TC_FP8, csg.TC_FP4):
            r = s.action(method)
            assert list(r.Nk) == g["Nk"] and r.R == g["R"] and r.sum_m == g["sum_m"]
            assert r.combo == g["combo2" if d == 2 else "combo4"]
            assert abs(r.S - g[key]) <= TOL_S * abs(g[key])
        s.free()


@pytest.mark.parametrize("d", [2, 4])
def test_set_from_host_coords(ctx, d):
    N = 1777
    c = oracle.sprinkle(d, N, 31, 5)            # unsorted, as sprinkled
    scale = 1000.0                              # exact power-free scale keeps order; margins scale
    cs = c * scale
    s = ctx.set_from_coords(d, cs)
    sorted_c, _ = oracle.sort(d, cs)
    assert np.array_equal(s.coords(), sorted_c)
    s.link()
    rel = oracle.link(d, sorted_c)
    assert np.array_equal(s.bitmap(), oracle.pack(rel, s.info()["stride"]))
    _check_result(s.action(), oracle.action(rel), d, N)
    s.free()


@pytest.mark.parametrize("d,scale", [(4, 1.0), (4, 1000.0), (2, 1.0), (2, 1000.0)])
def test_link_on_and_near_light_cones(ctx, d, scale):
    """Exactly null pairs, pairs one ulp off the cone, float ties, duplicates and signed
    zeros: every pair the float screens cannot settle must still get the double decision."""
    N = 1500
    c = inputs.light_cone_coords(d, N, 77, scale)
    s = ctx.set_from_coords(d, c)
    sorted_c, _ = oracle.sort(d, c)
    assert np.array_equal(s.coords(), sorted_c)
    s.link()
    rel = oracle.link(d, sorted_c)
    assert np.array_equal(s.bitmap(), oracle.pack(rel, s.info()["stride"]))
    _check_result(s.action(), oracle.action(rel), d, N)
    s.free()


@pytest.mark.parametrize("N", [2305, 300])
def test_d2_link_on_few_distinct_values(ctx, N):
    """The d=2 link sorts each row block by u and v and searches column keys: u and v drawn
    from eleven values (signed zeros, the smallest subnormals, negatives, 1e15) give ties
    between rows, between columns and across blocks, and a ragged last block."""
    rng = np.random.default_rng(123)
    vals = np.array([-1e15, -2.0, -5e-324, -0.0, 0.0, 5e-324, 1e-300, 0.25, 0.5, 3.0, 1e15])
    u, v = rng.choice(vals, N), rng.choice(vals, N)
    c = np.stack([(u + v) / 2, (v - u) / 2, u, v])
    s = ctx.set_from_coords(2, c)
    sorted_c, _ = oracle.sort(2, c)
    assert np.array_equal(s.coords(), sorted_c)
    s.link()
    rel = oracle.link(2, sorted_c)
    assert np.array_equal(s.bitmap(), oracle.pack(rel, s.info()["stride"]))
    _check_result(s.action(), oracle.action(rel), 2, N)
    s.free()


def test_d2_link_with_a_caller_time_order(ctx):
    """A caller's d=2 set whose t is not (u + v) / 2: the elements are ordered by that t, and
    the matrix, like the oracle's, relates each pair by u and v in that order only (i before
    k and u_i < u_k, v_i < v_k), inside the diagonal blocks as everywhere else."""
    rng = np.random.default_rng(321)
    N = 1300
    u, v = rng.random(N), rng.random(N)
    c = np.stack([rng.random(N), (v - u) / 2, u, v])
    s = ctx.set_from_coords(2, c)
    sorted_c, _ = oracle.sort(2, c)
    assert np.array_equal(s.coords(), sorted_c)
    s.link()
    rel = oracle.link(2, sorted_c)
    assert np.array_equal(s.bitmap(), oracle.pack(rel, s.info()["stride"]))
    s.free()


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("d,N", [(2, 3000), (4, 4100)])
def test_action_rows(ctx, d, N, method):
    s = ctx.sprinkle(d, N, 99, 1).link()
    rel = oracle.link(d, oracle.sprinkle_sorted(d, N, 99, 1))
    for lo, hi in [(0, 1), (5, 40), (1000, 1017), (N - 70, N), (N - 1, N)]:
        _check_result(s.action_rows(lo, hi, method), oracle.action(rel, rows=(lo, hi)), d, N)
    s.free()


def test_batch_equals_single(ctx, csg):
    specs = inputs.batch_workload(n_sets=24, seed=3, lo=64, hi=3000)
    sets = [ctx.sprinkle(sp.d, sp.N, sp.seed, sp.seq).link() for sp in specs]
    single = [s.action() for s in sets]
    batch = ctx.action_batch(sets)
    assert batch == single
    run = ctx.run_batch([(sp.d, sp.N, sp.seed, sp.seq) for sp in specs])
    assert run == single
    assert ctx.action_batch(sets, csg.TC) == single
    for sp, r in list(zip(specs, single))[:6]:
        want = oracle.run(sp.d, sp.N, sp.seed, sp.seq)
        _check_result(r, want, sp.d, sp.N)
    for s in sets:
        s.free()


def test_batch_degenerate_and_empty(ctx, csg):
    """Empty batches, and batches of the degenerate sizes N = 1, 2, 3 mixed with sets that
    span several tiles and ragged tails, in every method: each result equals the set alone
    and the oracle."""
    assert ctx.run_batch([], csg.TC) == [] and ctx.action_batch([], csg.POPC) == []
    specs = [(2, 1, 7, 0), (4, 1, 7, 1), (2, 2, 7, 2), (4, 3, 7, 3), (2, 257, 7, 4), (4, 700, 7, 5),
             (2, 3, 7, 6), (4, 2, 7, 7), (2, 1500, 7, 8)]
    for method in (csg.POPC, csg.TC, csg.TC_FP8):
        got = ctx.run_batch(specs, method)
        for (d, N, seed, seq), r in zip(specs, got):
            want = oracle.run(d, N, seed, seq)
            _check_result(r, want, d, N)
    sets = [ctx.sprinkle(d, N, seed, seq).link() for d, N, seed, seq in specs]
    for method in (csg.POPC, csg.TC_FP4):
        assert ctx.action_batch(sets, method) == [x.action(method) for x in sets]
    for x in sets:
        x.free()


def test_serve_alone_equals_in_mix(ctx, csg):
    specs = inputs.batch_workload(n_sets=40, seed=11, lo=32, hi=2500)
    alone = [ctx.run_batch([(sp.d, sp.N, sp.seed, sp.seq)])[0] for sp in specs]
    tickets = [ctx.serve_submit(sp.d, sp.N, sp.seed, sp.seq) for sp in specs]
    mixed = [ctx.serve_poll(t, timeout_ms=60000) for t in tickets]
    assert mixed == alone
    for sp, r in list(zip(specs, alone))[:4]:
        _check_result(r, oracle.run(sp.d, sp.N, sp.seed, sp.seq), sp.d, sp.N)


def test_errors(ctx, csg):
    with pytest.raises(csg.CsgError) as e:
        ctx.sprinkle(3, 10, 0)
    assert e.value.code == csg.E_INVAL
    with pytest.raises(csg.CsgError):
        ctx.sprinkle(2, 0, 0)
    with pytest.raises(csg.CsgError):
        ctx.sprinkle(2, csg.MAX_N + 1, 0)
    s = ctx.sprinkle(2, 100, 0)
    with pytest.raises(csg.CsgError):
        s.action()                     # not linked yet
    s.free()
    small = csg.Context(0, budget_bytes=1 << 20)
    try:
        with pytest.raises(csg.CsgError) as e:
            small.sprinkle(2, 8192, 0)     # 8 MiB bitmap over a 1 MiB budget
        assert e.value.code == csg.E_NOMEM
        with pytest.raises(csg.CsgError) as e:
            small.serve_submit(2, 8192, 0)
        assert e.value.code == csg.E_NOMEM
    finally:
        small.close()


def test_cancel_and_unknown_ticket(ctx, csg):
    with pytest.raises(csg.CsgError) as e:
        ctx.serve_poll(987654321, 0)
    assert e.value.code == csg.E_NOTFOUND
    big = [ctx.serve_submit(4, 12000, 5, q) for q in range(4)]
    t = ctx.serve_submit(2, 500, 1, 1)
    rc = ctx.serve_cancel(t)
    if rc == 0:
        with pytest.raises(csg.CsgError) as e:
            ctx.serve_poll(t, 0)
        assert e.value.code == csg.E_CANCELLED
    else:
        assert rc == csg.E_BUSY  # already admitted
        assert ctx.serve_poll(t, 60000) is not None
    for b in big:
        assert ctx.serve_poll(b, 120000) is not None


def test_serve_calls_on_a_fresh_context(csg):
    # polls and cancels before any submission find no ticket (and start no service);
    # the first submission then starts it
    with csg.Context(0) as c:
        with pytest.raises(csg.CsgError) as e:
            c.serve_poll(1, 0)
        assert e.value.code == csg.E_NOTFOUND
        assert c.serve_cancel(1) == csg.E_NOTFOUND
        t = c.serve_submit(2, 300, 7, 0)
        r = c.serve_poll(t, 60000)
        want = oracle.run(2, 300, 7, 0)
        _check_result(r, want, 2, 300)
        with pytest.raises(csg.CsgError) as e:
            c.serve_poll(t, 0)
        assert e.value.code == csg.E_NOTFOUND


def test_batch_autotune_records_choice(csg, tmp_path, monkeypatch):
    # the first batch of a shape times candidate tunings and records the winner; every
    # candidate gives the same counts, so the results stay exact whichever wins
    cache = tmp_path / "autotune.jsonl"
    monkeypatch.setenv("CSG_AUTOTUNE_CACHE", str(cache))
    specs = inputs.batch_workload(n_sets=30, seed=5, lo=300, hi=2600)
    tup = [(sp.d, sp.N, sp.seed, sp.seq) for sp in specs]
    with csg.Context(0) as c:
        got = c.run_batch(tup, csg.TC)
        again = c.run_batch(tup, csg.TC)          # replay of the captured graph
    assert got == again
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == 1 and '"popc_below"' in lines[0] and '"super"' in lines[0]
    for sp, r in list(zip(specs, got))[:5]:
        _check_result(r, oracle.run(sp.d, sp.N, sp.seed, sp.seq), sp.d, sp.N)


@pytest.mark.parametrize("N", [1, 2, 3, 700, 3000])
@pytest.mark.parametrize("eps", [2 ** -6, 0.3])
def test_smeared_action(ctx, csg, N, eps):
    # Eq. s_smeared from the GPU's full histogram against the oracle's; the sum is
    # reduced in a different order, so the bound is relative to the sum of |terms|
    s = ctx.sprinkle(2, N, 77, 0).link()
    want = oracle.action(oracle.link(2, oracle.sprinkle_sorted(2, N, 77, 0)))
    S_ref = oracle.smeared(N, want["hist"], eps)
    scale = 2 * eps * N + 8 * eps * eps * want["R"]
    for method in (csg.POPC, csg.TC):
        S, res = s.action_smeared(eps, method)
        assert abs(S - S_ref) <= 1e-12 * max(scale, 1.0), (method, S, S_ref)
        _check_result(res, want, 2, N)
    s.free()


def test_smeared_rejects_bad_arguments(ctx, csg):
    s4 = ctx.sprinkle(4, 100, 1, 0).link()
    with pytest.raises(csg.CsgError) as e:
        s4.action_smeared(0.1)
    assert e.value.code == csg.E_INVAL
    s2 = ctx.sprinkle(2, 100, 1, 0).link()
    for bad in (0.0, 1.0, -0.5, 2.0):
        with pytest.raises(csg.CsgError):
            s2.action_smeared(bad)
    s4.free()
    s2.free()


@pytest.mark.parametrize("N", [1, 2, 700, 3001])
def test_desitter_slab(ctx, csg, N):
    # Sec. 5.1 slab: theta is the same IEEE product on both sides (bit-exact); eta goes
    # through each side's own atan (CUDA's and the C library's differ by an ulp or two),
    # so coordinates match to 4e-16 and the link is checked on the GPU's own coordinates
    eta0 = 0.5
    s = ctx.sprinkle_desitter(N, eta0, 11, 2)
    got_c = s.coords()
    want_c, _ = oracle.sort(oracle.DS2, oracle.sprinkle_desitter(N, eta0, 11, 2))
    assert np.array_equal(got_c[1], want_c[1])
    assert np.max(np.abs(got_c[0] - want_c[0]), initial=0.0) <= 4e-16
    assert np.all(np.diff(got_c[0]) >= 0)
    s.link()
    rel = oracle.link(oracle.DS2, got_c)
    assert np.array_equal(s.bitmap(), oracle.pack(rel, s.info()["stride"]))
    want = oracle.action(rel)
    for method in (csg.POPC, csg.TC):
        _check_result(s.action(method), want, 2, N)
        S, _ = s.action_smeared(2 ** -6, method)
        S_ref = oracle.smeared(N, want["hist"], 2 ** -6)
        assert abs(S - S_ref) <= 1e-12 * max(2 * 2 ** -6 * N + 8 * 2 ** -12 * want["R"], 1.0)
    s.free()


def test_desitter_slab_at_the_distribution_size(ctx, csg):
    """The slab of the interval-abundance experiment (Sec. 5.2, N = 2^15, eta0 = 0.5): the
    whole bitmap (128 row blocks, many CTAs of the chunked tile kernel) equals the oracle's
    link of the GPU's coordinates, and both interval-count kernels agree on every count."""
    N, eta0 = 2 ** 15, 0.5
    s = ctx.sprinkle_desitter(N, eta0, 5, 0).link()
    got_c = s.coords()
    rel = oracle.link(oracle.DS2, got_c)
    assert np.array_equal(s.bitmap(), oracle.pack(rel, s.info()["stride"]))
    R = int(rel.sum(dtype=np.int64)) // 2  # symmetric, zero diagonal
    del rel
    a, b = s.action(csg.POPC), s.action(csg.TC)
    assert (a.R, list(a.Nk), a.sum_m, a.W) == (b.R, list(b.Nk), b.sum_m, b.W)
    assert a.R == R and a.status == 0 and b.status == 0
    s.free()


# ------------------------------------------------------------ d'Alembertian (Eq. b_local)

def _dalembert_tol(phi, L, l):
    # Both sides sum at most n_x = |L1|+|L2|+|L3| terms c_m phi(y) in some order, then form
    # (2/l^2)(2A - phi): each is within gamma_{n_x + 3} (2/l^2) T(x) of the exact value, with
    # T(x) = |phi(x)| + 2 sum |c_m phi(y)| <= |phi(x)| + 2 (|L1| + 2|L2| + |L3|) max|phi|.
    n = L.sum(axis=1)
    T = np.abs(phi) + 2.0 * (L[:, 0] + 2 * L[:, 1] + L[:, 2]) * np.abs(phi).max(initial=0.0)
    return 2.0 * (n + 4) * 2.0 ** -53 * (2.0 / l ** 2) * T * 1.01


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("N", [1, 2, 3, 700, 3001])
def test_dalembertian_matches_oracle(ctx, csg, N, method):
    import torch
    s = ctx.sprinkle(2, N, 21, 1).link()
    rel = oracle.link(2, oracle.sprinkle_sorted(2, N, 21, 1))
    phi = np.random.default_rng(N).uniform(-1.0, 1.0, size=N)
    l = 0.3
    want, L = oracle.dalembertian(rel, phi, l)
    phi_d = torch.from_numpy(phi).cuda()
    B_d = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")  # every entry is written
    res = s.dalembertian(phi_d.data_ptr(), B_d.data_ptr(), l, method)
    got = B_d.cpu().numpy()
    assert np.all(np.abs(got - want) <= _dalembert_tol(phi, L, l))
    _check_result(res, oracle.action(rel), 2, N)
    # phi = 1, l = 1: integer arithmetic throughout, so the values are exact and sum to -S_BD
    one = torch.ones(N, dtype=torch.float64, device="cuda")
    res = s.dalembertian(one.data_ptr(), B_d.data_ptr(), 1.0, method)
    want1, _ = oracle.dalembertian(rel, np.ones(N), 1.0)
    got1 = B_d.cpu().numpy()
    assert np.array_equal(got1, want1)
    assert float(got1.sum()) == -res.S
    s.free()


@pytest.mark.parametrize("name", ["diamond4.txt", "npos6.txt"])
def test_dalembertian_golden_on_gpu(ctx, csg, golden, name):
    import torch
    g = golden(name)
    rel = inputs.rel_from_edges(g["N"], g["rel"])
    dev = _dev_words(inputs.pack_rows(rel, 16))
    s = ctx.set_from_bitmap(2, g["N"], dev.data_ptr(), 16)
    phi = torch.tensor(g["phi"], dtype=torch.float64, device="cuda")
    B = torch.empty_like(phi)
    for method in (csg.POPC, csg.TC):
        s.dalembertian(phi.data_ptr(), B.data_ptr(), 1.0, method)
        assert B.cpu().tolist() == g["Bphi"]
    s.free()


def test_dalembertian_desitter_and_bitmap_orders(ctx, csg):
    import torch
    # a de Sitter slab (Sec. 5.1) and caller-made orders through the bitmap entry point
    s = ctx.sprinkle_desitter(2500, 0.5, 3, 0).link()
    cases = [(s, oracle.link(oracle.DS2, s.coords()), None)]
    for r in (inputs.chain_rel(300), inputs.layered_order_rel(900, 5), inputs.random_upper_rel(600, 0.2, 6)):
        N = r.shape[0]
        stride = (N + 63) // 64 + 1  # a caller stride unlike the library's
        dev = _dev_words(inputs.pack_rows(r, stride))
        cases.append((ctx.set_from_bitmap(2, N, dev.data_ptr(), stride), r, dev))
    for st, r, _keep in cases:
        N = r.shape[0]
        phi = np.random.default_rng(N).normal(size=N)
        want, L = oracle.dalembertian(r, phi, 0.5)
        phi_d = torch.from_numpy(phi).cuda()
        B = torch.empty_like(phi_d)
        for method in (csg.POPC, csg.TC):
            st.dalembertian(phi_d.data_ptr(), B.data_ptr(), 0.5, method)
            assert np.all(np.abs(B.cpu().numpy() - want) <= _dalembert_tol(phi, L, 0.5))
        st.free()


def test_dalembertian_rejects_bad_arguments(ctx, csg):
    import torch
    s4 = ctx.sprinkle(4, 100, 1, 0).link()
    s2 = ctx.sprinkle(2, 100, 1, 0)
    buf = torch.zeros(300, dtype=torch.float64, device="cuda")
    p, q = buf.data_ptr(), buf.data_ptr() + 100 * 8
    with pytest.raises(csg.CsgError) as e:
        s4.dalembertian(p, q)                     # 3+1: not given by the paper
    assert e.value.code == csg.E_INVAL
    with pytest.raises(csg.CsgError):
        s2.dalembertian(p, q)                     # not linked yet
    s2.link()
    for l in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(csg.CsgError):
            s2.dalembertian(p, q, l)
    with pytest.raises(csg.CsgError):
        s2.dalembertian(p, p + 50 * 8)            # phi and Bphi overlap
    with pytest.raises(csg.CsgError):
        s2.dalembertian(0, q)
    s2.dalembertian(p, q, 1.0, csg.TC)            # still usable afterwards
    s4.free()
    s2.free()


# ------------------------------------------------------------ tensor operand formats

FORMATS = [2, 3]  # CSG_TC_FP8 (e4m3, kind::f8f6f4) and CSG_TC_FP4 (packed e2m1, kind::mxf4)


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("d,N", [(2, 1), (2, 2), (4, 3), (2, 129), (4, 257), (2, 1000), (4, 2500),
                                 (2, 4099), (4, 5000)])
def test_tensor_formats_match_oracle(ctx, csg, fmt, d, N):
    seed, seq = 1000 + N, d
    s = ctx.sprinkle(d, N, seed, seq).link()
    want = oracle.action(oracle.link(d, oracle.sprinkle_sorted(d, N, seed, seq)))
    _check_result(s.action(fmt), want, d, N)
    s.free()


@pytest.mark.parametrize("fmt", FORMATS)
def test_tensor_formats_hist_bitmaps_batch_rows(ctx, csg, fmt):
    import torch
    # full histogram
    N = 3000
    s = ctx.sprinkle(2, N, 7, 0).link()
    want = oracle.action(oracle.link(2, oracle.sprinkle_sorted(2, N, 7, 0)))
    h = torch.full((N,), 7, dtype=torch.int64, device="cuda")
    _check_result(s.action_hist(h.data_ptr(), N, fmt), want, 2, N)
    assert np.array_equal(h.cpu().numpy().astype(np.uint64), want["hist"][:N])
    # a row range
    res = s.action_rows(300, 2100, fmt)
    rr = oracle.action(oracle.link(2, oracle.sprinkle_sorted(2, N, 7, 0)), rows=(300, 2100))
    assert res.R == rr["R"] and list(res.Nk) == [int(x) for x in rr["Nk"]] and res.W == rr["W"]
    s.free()
    # caller bitmaps, including orders no sprinkle produces
    for rel in (inputs.random_upper_rel(700, 0.3, 1), inputs.layered_order_rel(1200, 3), inputs.chain_rel(1030)):
        n = rel.shape[0]
        stride = (n + 63) // 64 + 3
        dev = _dev_words(inputs.pack_rows(rel, stride))
        b = ctx.set_from_bitmap(2, n, dev.data_ptr(), stride)
        _check_result(b.action(fmt), oracle.action(rel), 2, n)
        b.free()
    # several sets in one launch
    sets = [ctx.sprinkle(d, n, 40 + k, 1).link() for k, (d, n) in enumerate([(2, 500), (4, 1700), (2, 2600), (4, 90)])]
    got = ctx.action_batch(sets, fmt)
    for st, r, (d, n, k) in zip(sets, got, [(2, 500, 0), (4, 1700, 1), (2, 2600, 2), (4, 90, 3)]):
        _check_result(r, oracle.action(oracle.link(d, oracle.sprinkle_sorted(d, n, 40 + k, 1))), d, n)
        st.free()


# ------------------------------------------------------------ stream-ordered sets

def test_sets_on_side_streams(ctx, csg):
    # sprinkle enqueues and returns; set memory is allocated and freed in stream order on the
    # creating stream.  Sets made, used and freed back to back on two side streams, with
    # their memory recycled between rounds, must give the oracle's counts every time.
    import torch
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    cases = [(4, 3000, 5), (2, 5000, 6), (4, 1200, 7), (2, 700, 8)]
    wants = {k: oracle.action(oracle.link(d, oracle.sprinkle_sorted(d, N, seed, 0))) for k, (d, N, seed) in enumerate(cases)}
    for rnd in range(3):
        for k, (d, N, seed) in enumerate(cases):
            st = streams[(k + rnd) % 2]
            s = ctx.sprinkle(d, N, seed, 0, stream=st)
            s.link(stream=st)
            for method in (csg.POPC, csg.TC):
                _check_result(s.action(method, stream=st), wants[k], d, N)
            s.free()
    # a set made on one stream and read on another after an explicit wait
    s = ctx.sprinkle(4, 2000, 9, 0, stream=streams[0])
    s.link(stream=streams[0])
    streams[1].wait_stream(streams[0])
    _check_result(s.action(csg.TC, stream=streams[1]),
                  oracle.action(oracle.link(4, oracle.sprinkle_sorted(4, 2000, 9, 0))), 4, 2000)
    torch.cuda.synchronize()
    s.free()


def test_popc_pipe_probe_rate(csg):
    """The roofline of the popcount method takes 16 32-bit popcounts per SM per clock (the
    CUDA guide's throughput table); the probe's sustained rate must agree with it."""
    import torch
    rate = csg.measure_popc_rate(0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    per_sm = rate / sms
    # 12 to 17 results per SM per clock at a clock between 1.4 and 2.1 GHz
    assert 12 * 1.4e9 < per_sm < 17 * 2.1e9, per_sm


def test_mma_probe_rate(csg):
    """The pair MMA on resident operands: fp4 (kind::mxf4) at about twice the fp8 rate
    (kind::f8f6f4; on this GPU it reaches about 4.85 PFLOP/s at 2.07 GHz, a little above the
    nominal dense 4.5), below the nominal dense fp4 peak of 13.5 PFLOP/s; a non-tensor
    method is rejected."""
    f4, f8 = csg.measure_mma_rate(csg.TC_FP4, 0), csg.measure_mma_rate(csg.TC_FP8, 0)
    assert 4e15 < f4 < 13.5e15 and 2e15 < f8 < 6e15, (f4, f8)
    assert 1.6 < f4 / f8 < 2.4
    with pytest.raises(csg.CsgError):
        csg.measure_mma_rate(csg.POPC, 0)


def test_l2_feed_probe_rate(csg):
    """The tensor form's second roofline: bytes per SM per second from L2 into shared memory
    through swizzled 2D tensor-map loads with six 32 KB stages in flight on every SM (about
    68 bytes per clock on this GPU)."""
    rate = csg.measure_l2_feed(0)
    # 40 to 80 bytes per SM per clock at a clock between 1.4 and 2.1 GHz
    assert 40 * 1.4e9 < rate < 80 * 2.1e9, rate
