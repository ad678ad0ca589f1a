"""The seeded input recipes (CPU): the workload generators are deterministic, and the
light-cone stress sets really contain the cases the link's float screens must hand to the
double decision (so the GPU parity tests on them exercise those paths)."""
import numpy as np

from paper_1709_03013_gb300 import inputs


def test_workloads_are_deterministic():
    a, b = inputs.batch_workload(n_sets=64), inputs.batch_workload(n_sets=64)
    assert a == b and all(256 <= s.N <= 8192 for s in a)
    assert [s.d for s in a[:4]] == [2, 4, 2, 4]
    r1, r2 = inputs.serve_workload(n_req=50), inputs.serve_workload(n_req=50)
    assert r1 == r2 and all(1024 <= r.spec.N <= 65536 for r in r1)
    t = [r.arrival_s for r in r1]
    assert t == sorted(t) and t[0] == 0.0


def test_light_cone_stress_d4_contains_nulls_and_near_nulls():
    c = inputs.light_cone_coords(4, 600, 77)
    assert np.array_equal(c, inputs.light_cone_coords(4, 600, 77))
    t, x, y, z = c
    dt = t[None, :] - t[:, None]
    s2 = dt * dt - (((x[None, :] - x[:, None]) ** 2 + (y[None, :] - y[:, None]) ** 2) + (z[None, :] - z[:, None]) ** 2)
    off = ~np.eye(600, dtype=bool)
    exact_null = (s2 == 0) & off & (dt != 0)
    near = (np.abs(s2) < 1e-5) & (s2 != 0) & off          # inside the float screen's margin
    dup = (dt == 0) & (s2 == 0) & off                      # identical elements
    assert exact_null.sum() >= 100 and near.sum() >= 50 and dup.sum() >= 2
    scaled = inputs.light_cone_coords(4, 600, 77, 1000.0)
    assert np.array_equal(scaled, c * 1000.0)


def test_light_cone_stress_d2_contains_float_ties_and_signed_zeros():
    c = inputs.light_cone_coords(2, 1500, 77)
    u, v = c[2], c[3]
    uf = u.astype(np.float32)
    same_float = (uf[None, :] == uf[:, None]) & (u[None, :] != u[:, None])
    same_double = (u[None, :] == u[:, None]) & ~np.eye(1500, dtype=bool)
    assert same_float.sum() >= 10 and same_double.sum() >= 10
    assert np.any((u == 0) & np.signbit(u)) and np.any((u == 0) & ~np.signbit(u))
    assert np.allclose(c[0], (u + v) / 2) and np.allclose(c[1], (v - u) / 2)


def test_workload_distributions():
    # the batch and serve recipes draw what they state: N log-uniform on [lo, hi], d 50/50
    # (alternating in a batch, Bernoulli(1/2) in the stream), exponential gaps at the rate
    from scipy import stats
    b = inputs.batch_workload()
    lnN = np.log([s.N for s in b])
    assert stats.kstest(lnN, "uniform", args=(np.log(256), np.log(8192) - np.log(256))).pvalue > 1e-4
    reqs = inputs.serve_workload(n_req=20000, rate_per_s=90.0)
    lnN = np.log([r.spec.N for r in reqs])
    assert stats.kstest(lnN, "uniform", args=(np.log(1024), np.log(65536) - np.log(1024))).pvalue > 1e-4
    d4 = np.mean([r.spec.d == 4 for r in reqs])
    assert abs(d4 - 0.5) < 5 * np.sqrt(0.25 / len(reqs))
    gaps = np.diff([r.arrival_s for r in reqs])
    assert stats.kstest(gaps, "expon", args=(0, 1 / 90.0)).pvalue > 1e-4
    assert len({(r.spec.seed, r.spec.seq) for r in reqs}) == len(reqs)   # every request its own stream
