"""Error paths on the GPU, made without a fault, a trap or a hang.

* Bounded device waits: csg_test_wait_expiry shortens every wait of the interval-count
  kernels and makes each CTA's producer skip the copies of its first stage, so that
  stage's barrier never completes and nothing is in flight.  The first wait on it must run
  out after the short limit, the kernel must record the expiry and return, the call must
  return CSG_E_TIMEOUT well before the built-in 2-4 s limits, and the same context must
  then give the oracle's counts.
* Device allocations: csg_test_fail_alloc makes the library's next allocations fail as
  if the allocator were out of memory; each call that needed one returns CSG_E_NOMEM,
  frees what it had taken, and the context keeps working.
"""
import time

import pytest

import oracle

pytestmark = pytest.mark.gpu

TOL_S = 1e-12


@pytest.fixture(scope="module")
def csg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_03013_gb300 import csg as m
    m.load()
    yield m
    m.inject_wait_expiry(0, False)
    m.inject_alloc_failures(0)


def _assert_counts(r, want):
    assert (r.R, list(r.Nk), r.sum_m, r.W, r.combo, r.status) == \
        (want["R"], [int(x) for x in want["Nk"]], want["sum_m"], want["W"], want["combo"], 0)
    assert abs(r.S - want["S"]) <= TOL_S * max(abs(want["S"]), 1.0)


@pytest.mark.parametrize("method", ["POPC", "TC_FP4", "TC_FP8"])
def test_starved_wait_times_out_and_context_recovers(csg, method):
    m = getattr(csg, method)
    d, N, seed = 4, 3000, 21  # 188 row groups and 78 pair tiles: every CTA gets a first item
    want = oracle.run(d, N, seed)
    with csg.Context(0) as ctx:
        s = ctx.sprinkle(d, N, seed).link()
        _assert_counts(s.action(m), want)
        csg.inject_wait_expiry(20_000_000, True)  # 20 ms; every CTA's first stage gets no copies
        try:
            t0 = time.perf_counter()
            with pytest.raises(csg.CsgError) as e:
                s.action(m)
            elapsed = time.perf_counter() - t0
        finally:
            csg.inject_wait_expiry(0, False)
        assert e.value.code == csg.E_TIMEOUT
        assert elapsed < 1.5, elapsed  # wound down after the short limit, not the built-in one
        for _ in range(2):  # the same context and set afterwards
            _assert_counts(s.action(m), want)
        s.free()


def test_starve_needs_a_limit(csg):
    with pytest.raises(csg.CsgError) as e:
        csg.inject_wait_expiry(0, True)
    assert e.value.code == csg.E_INVAL


def test_injected_allocation_failures(csg):
    d, N, seed = 2, 1500, 22
    want = oracle.run(d, N, seed)
    with csg.Context(0) as ctx:
        csg.inject_alloc_failures(1)  # the set's coordinates
        with pytest.raises(csg.CsgError) as e:
            ctx.sprinkle(d, N, seed)
        assert e.value.code == csg.E_NOMEM
        s = ctx.sprinkle(d, N, seed).link()  # the count is used up
        for m in (csg.POPC, csg.TC_FP4, csg.TC_FP8):
            csg.inject_alloc_failures(1)  # the call's scratch arena
            with pytest.raises(csg.CsgError) as e:
                s.action(m)
            assert e.value.code == csg.E_NOMEM
            _assert_counts(s.action(m), want)
        S_ref, _ = s.action_smeared(0.25, csg.POPC)
        csg.inject_alloc_failures(1)  # the smeared action's histogram
        with pytest.raises(csg.CsgError) as e:
            s.action_smeared(0.25, csg.POPC)
        assert e.value.code == csg.E_NOMEM
        S_eps, r = s.action_smeared(0.25, csg.POPC)
        _assert_counts(r, want)
        assert S_eps == S_ref  # fixed-order reduction: the same value as before the failure
        s.free()
        specs = [(2, 700, 23, k) for k in range(3)] + [(4, 900, 23, 3)]
        csg.inject_alloc_failures(2)  # the batch's sets
        with pytest.raises(csg.CsgError) as e:
            ctx.run_batch(specs, csg.TC)
        assert e.value.code == csg.E_NOMEM
        got = ctx.run_batch(specs, csg.TC)
        for (dd, NN, sd, sq), r in zip(specs, got):
            _assert_counts(r, oracle.run(dd, NN, sd, sq))
        csg.inject_alloc_failures(1)  # a served request's set
        t = ctx.serve_submit(d, N, seed, 0)
        with pytest.raises(csg.CsgError) as e:
            ctx.serve_poll(t, timeout_ms=60000)
        assert e.value.code == csg.E_NOMEM
        t = ctx.serve_submit(d, N, seed, 0)
        _assert_counts(ctx.serve_poll(t, timeout_ms=60000), want)
    csg.inject_alloc_failures(0)
