"""Pins for the CPU oracle against facts fixed outside the oracle itself.

Each test checks the oracle against something it does not compute the same way:
a library generator (numpy's Philox), a library sort, exact rational arithmetic,
a graph library's reachability sets, a 2D dominance count, closed forms for
chains and antichains, hand-worked fixtures under tests/golden, exact identities,
the Myrheim-Meyer ordering fraction of a flat diamond, and the exact expected
interval abundances of a sprinkled diamond (from the volume of k-chains).
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1709_03013_gb300 import inputs

SQ6 = math.sqrt(6.0)


# ----------------------------------------------------------------- RNG pins

@pytest.mark.parametrize("key", [0, 1, 12345, (7 << 64) | 99, (1 << 128) - 1])
@pytest.mark.parametrize("ctr", [1, 6, (3 << 64) | 17, (5 << 192) | (9 << 128) | (1 << 64) | 3])
def test_philox_matches_numpy(key, ctr):
    # numpy's Philox (4x64, 10 rounds) emits block(counter + 1) first.
    bg = np.random.Philox(key=key, counter=ctr - 1)
    want = [int(bg.random_raw()) for _ in range(4)]
    words = [(ctr >> (64 * w)) & ((1 << 64) - 1) for w in range(4)]
    kwords = [key & ((1 << 64) - 1), key >> 64]
    got = [int(x) for x in oracle.philox4x64_10(words, kwords)]
    assert got == want


def test_sprinkle_uses_philox_words_d2():
    # u, v are the top 53 bits of the first two words of block (e, 0, 0, 0).
    coords = oracle.sprinkle(2, 5, seed=11, seq=3)
    for e in range(5):
        bg = np.random.Philox(key=11 | (3 << 64), counter=e - 1 if e > 0 else (1 << 256) - 1)
        r = [int(bg.random_raw()) for _ in range(2)]
        assert coords[2, e] == (r[0] >> 11) / 2.0 ** 53
        assert coords[3, e] == (r[1] >> 11) / 2.0 ** 53


# ------------------------------------------------------------ sprinkle pins

def test_sprinkle_d2_uniform_and_light_cone_coords():
    from scipy import stats
    c = oracle.sprinkle(2, 20000, seed=5)
    t, x, u, v = c
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    assert stats.kstest(v, "uniform").pvalue > 1e-4
    assert np.all((u >= 0) & (u < 1) & (v >= 0) & (v < 1))
    # t and x are the diamond coordinates: |x| <= t <= 1 - |x|
    assert np.all(np.abs(x) <= t) and np.all(t <= 1 - np.abs(x) + 1e-15)


def test_sprinkle_d4_acceptance_and_marginal():
    from scipy import stats
    n = 20000
    c, att = oracle.sprinkle(4, n, seed=6, with_attempts=True)
    t, x, y, z = c
    r = np.sqrt(x * x + y * y + z * z)
    assert np.all(np.abs(t) + r <= 1.0)
    # acceptance = vol(diamond) / vol([-1,1]^4) = (2 * pi/3 * 1/4 ... ) = 2*(4pi/3)/4 / 16 = pi/24
    p = math.pi / 24.0
    tries = int((att + 1).sum())
    mean, sd = tries * p, math.sqrt(tries * p * (1 - p))
    assert abs(n - mean) < 5 * sd
    # time marginal of a uniform point in |t| + r <= 1: density (3/2)(1-|t|)^3 ... cdf of |t| is 1-(1-a)^4
    a = np.abs(t)
    assert stats.kstest(a, lambda q: 1 - (1 - q) ** 4).pvalue > 1e-4
    # isotropy: the direction of (x,y,z) is uniform, so each component/r is U[-1,1]
    assert stats.kstest(z / r, "uniform", args=(-1, 2)).pvalue > 1e-4


def test_sprinkle_deterministic_and_seq_independent():
    a = oracle.sprinkle(4, 100, seed=1, seq=0)
    b = oracle.sprinkle(4, 100, seed=1, seq=0)
    c = oracle.sprinkle(4, 100, seed=1, seq=1)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    # element e does not depend on N (counter-based)
    d = oracle.sprinkle(4, 37, seed=1, seq=0)
    assert np.array_equal(a[:, :37], d)


# ---------------------------------------------------------------- sort pins

def test_sort_matches_library_sort_with_ties():
    rng = np.random.default_rng(0)
    N = 300
    coords = np.zeros((4, N))
    coords[0] = rng.integers(0, 20, N) / 8.0  # many equal times
    coords[2] = rng.integers(0, 5, N) / 4.0   # and equal u
    coords[1] = rng.random(N)
    coords[3] = rng.random(N)
    for d in (2, 4):
        _, perm = oracle.sort(d, coords)
        if d == 2:
            want = sorted(range(N), key=lambda e: (coords[0, e], coords[2, e], e))
        else:
            want = sorted(range(N), key=lambda e: (coords[0, e], e))
        assert list(perm) == want


def test_sort_permutes_all_rows():
    c = oracle.sprinkle(4, 500, seed=2)
    s, perm = oracle.sort(4, c)
    assert np.array_equal(s, c[:, perm])
    assert np.all(np.diff(s[0]) >= 0)


# ---------------------------------------------------------------- link pins

def _exact_related(d, c, i, j):
    """Exact real-number light-cone test on the stored coordinates (rationals)."""
    if d == 2:
        ti, tj = Fraction(c[0, i]), Fraction(c[0, j])
        xi, xj = Fraction(c[1, i]), Fraction(c[1, j])
        dt = tj - ti
        return dt > 0 and dt * dt > (xj - xi) ** 2
    dt = Fraction(c[0, j]) - Fraction(c[0, i])
    s = sum((Fraction(c[r, j]) - Fraction(c[r, i])) ** 2 for r in (1, 2, 3))
    return dt > 0 and dt * dt > s


@pytest.mark.parametrize("d", [2, 4])
def test_link_matches_exact_light_cone(d):
    c = oracle.sprinkle_sorted(d, 120, seed=7)
    rel = oracle.link(d, c)
    for i, j in itertools.combinations(range(120), 2):
        assert rel[i, j] == _exact_related(d, c, i, j)


def test_link_light_cone_stress_set():
    """On a set crowded onto light cones (exact nulls, one-ulp nudges, duplicates), the
    oracle's double decision agrees with the exact rational one wherever the exact
    interval is clearly away from zero, and exactly null pairs are unrelated (Sec. 2.2:
    related means strictly inside the light cone)."""
    from paper_1709_03013_gb300 import inputs
    N = 300
    c, _ = oracle.sort(4, inputs.light_cone_coords(4, N, 5))
    rel = oracle.link(4, c)
    F = [[Fraction(float(v)) for v in row] for row in c]
    nulls = clear = 0
    for i, j in itertools.combinations(range(N), 2):
        dt = F[0][j] - F[0][i]
        s2 = dt * dt - sum((F[r][j] - F[r][i]) ** 2 for r in (1, 2, 3))
        if s2 == 0:
            nulls += 1
            assert rel[i, j] == 0
        elif abs(s2) > Fraction(1, 10 ** 12):
            clear += 1
            assert rel[i, j] == (dt > 0 and s2 > 0)
    assert nulls >= 50 and clear > N * (N - 1) // 2 - 2 * N


@pytest.mark.parametrize("d", [2, 4])
def test_link_symmetric_zero_diagonal_row_and_pair(d):
    c = oracle.sprinkle_sorted(d, 200, seed=8)
    rel = oracle.link(d, c)
    assert np.array_equal(rel, rel.T) and not rel.diagonal().any()
    for i in (0, 17, 199):
        assert np.array_equal(oracle.link_row(d, c, i), rel[i])
    # time order: a later label never precedes an earlier one (Sec. 2.2)
    for i, j in itertools.combinations(range(200), 2):
        if rel[i, j]:
            assert c[0, i] <= c[0, j]


@pytest.mark.parametrize("d,frac", [(2, 0.5), (4, 0.1)])
def test_ordering_fraction_myrheim_meyer(d, frac):
    # For iid uniform points in a flat diamond each pair is related with probability
    # f(d) = Gamma(d+1) Gamma(d/2) / (2 Gamma(3d/2)): 1/2 in 1+1, 1/10 in 3+1.
    f = math.gamma(d + 1) * math.gamma(d / 2) / (2 * math.gamma(3 * d / 2))
    assert abs(f - frac) < 1e-12
    N, seeds = 600, range(6)
    Rs = [oracle.link(d, oracle.sprinkle_sorted(d, N, s)).sum() // 2 for s in seeds]
    pairs = N * (N - 1) // 2
    mean = np.mean(Rs) / pairs
    # pair indicators are positively correlated; 5 binomial sigmas of the mean over
    # 6 sets times a generous factor 8 for the correlation
    sd = math.sqrt(frac * (1 - frac) / pairs / len(Rs)) * 8
    assert abs(mean - frac) < 5 * sd


# -------------------------------------------------------------- action pins

def _nx_intervals(rel):
    import networkx as nx
    N = rel.shape[0]
    g = nx.DiGraph()
    g.add_nodes_from(range(N))
    for i, j in zip(*np.nonzero(np.triu(rel, 1))):
        g.add_edge(int(i), int(j))
    desc = {v: nx.descendants(g, v) for v in range(N)}
    anc = {v: nx.ancestors(g, v) for v in range(N)}
    return g, desc, anc


@pytest.mark.parametrize("d,N,seed", [(2, 48, 1), (4, 64, 2), (2, 64, 3), (4, 40, 4)])
def test_action_matches_graph_library_brute_force(d, N, seed):
    pytest.importorskip("networkx")
    c = oracle.sprinkle_sorted(d, N, seed)
    rel = oracle.link(d, c)
    g, desc, anc = _nx_intervals(rel)
    hist = np.zeros(max(N, 1), dtype=np.int64)
    for i, j in g.edges():
        hist[len(desc[i] & anc[j])] += 1
    out = oracle.action(rel)
    assert np.array_equal(out["hist"].astype(np.int64), hist)
    assert out["R"] == g.number_of_edges()
    # pair-by-pair entry points agree with the histogram
    for i, j in list(g.edges())[:50]:
        m = len(desc[i] & anc[j])
        assert oracle.interval(rel, i, j) == m
        assert oracle.interval_coords(d, c, i, j) == m


def test_links_equal_transitive_reduction():
    nx = pytest.importorskip("networkx")
    for d, seed in ((2, 5), (4, 6)):
        rel = oracle.link(d, oracle.sprinkle_sorted(d, 150, seed))
        g, _, _ = _nx_intervals(rel)
        assert oracle.action(rel)["Nk"][0] == nx.transitive_reduction(g).number_of_edges()


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 9, 64, 65, 130])
def test_chain_closed_form(N):
    out = oracle.action(inputs.chain_rel(N))
    want = np.zeros(max(N, 1), dtype=np.uint64)
    for k in range(N - 1):
        want[k] = N - 1 - k  # pairs at distance k+1 along the chain
    assert np.array_equal(out["hist"], want)
    assert out["R"] == N * (N - 1) // 2
    combo2, S2 = oracle.finalize(2, N, out["Nk"])
    combo4, S4 = oracle.finalize(4, N, out["Nk"])
    if N >= 4:
        assert combo2 == N and S2 == 2.0 * N
    if N >= 5:
        assert combo4 == N - 1 and abs(S4 - 4 / SQ6 * (N - 1)) <= 1e-12 * abs(S4)


@pytest.mark.parametrize("N", [0, 1, 7, 100])
def test_antichain_closed_form(N):
    out = oracle.action(inputs.antichain_rel(N))
    assert out["R"] == 0 and not out["hist"].any()
    assert oracle.finalize(2, N, out["Nk"]) == (N, 2.0 * N)
    combo4, S4 = oracle.finalize(4, N, out["Nk"])
    assert combo4 == N and abs(S4 - 4 / SQ6 * N) <= 1e-12 * max(abs(S4), 1)


@pytest.mark.parametrize("name", ["diamond4.txt", "npos6.txt"])
def test_golden_hand_worked(golden, name):
    g = golden(name)
    rel = inputs.rel_from_edges(g["N"], g["rel"])
    out = oracle.action(rel)
    assert list(out["Nk"]) == g["Nk"]
    assert out["R"] == g["R"] and out["sum_m"] == g["sum_m"]
    combo2, S2 = oracle.finalize(2, g["N"], out["Nk"])
    combo4, S4 = oracle.finalize(4, g["N"], out["Nk"])
    assert combo2 == g["combo2"] and combo4 == g["combo4"]
    assert abs(S2 - g["S2"]) <= 1e-12 * abs(g["S2"])
    assert abs(S4 - g["S4"]) <= 1e-12 * abs(g["S4"])


@pytest.mark.parametrize("d,N,seed", [(2, 300, 1), (4, 400, 2)])
def test_identities(d, N, seed):
    rel = oracle.link(d, oracle.sprinkle_sorted(d, N, seed))
    out = oracle.action(rel)
    up = np.triu(rel, 1).astype(np.int64)
    outdeg, indeg = up.sum(1), up.sum(0)
    ks = np.arange(out["hist"].shape[0], dtype=np.int64)
    assert int(out["hist"].sum()) == out["R"] == int(up.sum())
    # sum_k k N_k counts 3-chains i<k<j, i.e. sum over middles of indeg * outdeg
    assert int((ks * out["hist"].astype(np.int64)).sum()) == out["sum_m"] == int((indeg * outdeg).sum())
    ii, jj = np.nonzero(up)
    assert out["W"] == int((jj - ii - 1).sum())


def test_2d_dominance_count():
    # In 1+1 the light-cone sprinkle is a 2D order: m(i,j) is the number of points in
    # the open rectangle (u_i,u_j) x (v_i,v_j), counted here with a prefix-sum table.
    d, N = 2, 700
    c = oracle.sprinkle_sorted(d, N, 9)
    u, v = c[2], c[3]
    ru = np.argsort(np.argsort(u))
    rv = np.argsort(np.argsort(v))
    grid = np.zeros((N + 1, N + 1), dtype=np.int64)
    grid[ru + 1, rv + 1] = 1
    P = grid.cumsum(0).cumsum(1)
    rel = oracle.link(d, c)
    hist = np.zeros(N, dtype=np.int64)
    ii, jj = np.nonzero(np.triu(rel, 1))
    a0, b0, a1, b1 = ru[ii] + 1, rv[ii] + 1, ru[jj], rv[jj]
    m = P[a1, b1] - P[a0, b1] - P[a1, b0] + P[a0, b0]
    np.add.at(hist, m, 1)
    assert np.array_equal(oracle.action(rel)["hist"].astype(np.int64), hist)


def test_2d_three_chain_expectation():
    # E[# 3-chains] in a random 2D order is C(N,3)/6
    N, Ns = 400, []
    for s in range(8):
        Ns.append(oracle.action(oracle.link(2, oracle.sprinkle_sorted(2, N, 100 + s)))["sum_m"])
    want = math.comb(N, 3) / 6
    assert abs(np.mean(Ns) / want - 1) < 0.05


def _chain_volume(k, d):
    """chi_k of a flat Alexandrov interval: the volume of ordered k-chains x1 < ... < xk inside
    an interval of volume V is chi_k V^k, with (Meyer's closed form)
    chi_k = (Gamma(d+1)/2)^(k-1) Gamma(d/2) Gamma(d) / (k Gamma(kd/2) Gamma((k+1)d/2)),
    chi_0 = 1.  Exact rational for even d (every Gamma argument is an integer)."""
    if k == 0:
        return Fraction(1)
    h, fac = d // 2, math.factorial
    return (Fraction(fac(d), 2) ** (k - 1)
            * Fraction(fac(h - 1) * fac(d - 1), k * fac(k * h - 1) * fac((k + 1) * h - 1)))


def _expected_abundance(d, N, m):
    """<N_m> for N iid uniform points in a flat d-dimensional diamond (N fixed).

    An ordered pair x < y holds exactly m of the other N-2 points with probability
    C(N-2, m) E[1(x<y) p^m (1-p)^(N-2-m)], p = V(x, y)/V the fraction of the diamond inside
    their interval.  Splitting a (j+2)-chain at its ends gives E[1(x<y) p^j] = chi_{j+2}/chi_j,
    so the binomial expansion of (1-p)^(N-2-m) makes <N_m> an exact finite sum."""
    n = N - 2 - m
    s = sum(Fraction(math.comb(n, i) * (-1) ** i) * _chain_volume(m + i + 2, d) / _chain_volume(m + i, d)
            for i in range(n + 1))
    return N * (N - 1) * math.comb(N - 2, m) * s


def test_chain_volume_closed_form():
    # chi_k: 1/(k!)^2 in 1+1 (two random orders agree), the ordering probability f(d)/2 for k = 2,
    # and in 3+1 the recursion chi_{k+1} V^{k+1} = chi_k int_I V(x, top)^k dx over the diamond
    # (every chain's later part lies in the interval from its first element to the top vertex),
    # integrated numerically with V(x, top) = (pi/24) tau^4.
    from scipy import integrate
    for k in range(1, 7):
        assert _chain_volume(k, 2) == Fraction(1, math.factorial(k) ** 2)
    assert _chain_volume(2, 4) == Fraction(1, 20) and _chain_volume(3, 4) == Fraction(1, 2100)
    V = math.pi / 24    # unit-height diamond: bottom (-1/2, 0), top (1/2, 0)

    def tau_moment(a):
        f = lambda r, t: 4 * math.pi * r * r * ((0.5 - t) ** 2 - r * r) ** (a / 2)
        return integrate.dblquad(f, -0.5, 0.5, lambda t: 0.0, lambda t: 0.5 - abs(t),
                                 epsabs=1e-15, epsrel=1e-11)[0]

    assert abs(tau_moment(0) / V - 1) < 1e-10
    for k in (1, 2, 3):
        lhs = float(_chain_volume(k + 1, 4)) * V ** (k + 1)
        rhs = float(_chain_volume(k, 4)) * (math.pi / 24) ** k * tau_moment(4 * k)
        assert abs(lhs / rhs - 1) < 1e-9


@pytest.mark.parametrize("d,N", [(2, 24), (2, 40), (4, 24), (4, 40)])
def test_mean_abundances_and_action_exact(d, N):
    # Means over 20000 sprinkled sets against the exact expectations of N_0..N_3, of the related
    # pairs R = sum_m N_m, of the 3-chains sum_m m N_m, and of the action (linear in the N_k).
    E = [_expected_abundance(d, N, m) for m in range(N - 1)]
    assert sum(E) == Fraction(N * (N - 1), 2) * 2 * _chain_volume(2, d)
    assert sum(m * e for m, e in enumerate(E)) == N * (N - 1) * (N - 2) * _chain_volume(3, d)
    if d == 2:
        ES = 2 * (N - 2 * E[0] + 4 * E[1] - 2 * E[2])
        assert ES == 2    # the mean 1+1 action of a flat diamond is 2 at every N
    else:
        ES = (N - E[0] + 9 * E[1] - 16 * E[2] + 8 * E[3]) * 4 / SQ6
    want = np.array([float(x) for x in E[:4]] + [float(sum(E)),
                    float(sum(m * e for m, e in enumerate(E))), float(ES)])
    T = 20000
    X = np.empty((T, 7))
    for s in range(T):
        r = oracle.run(d, N, seed=s, seq=7, threads=1)
        X[s, :4] = r["Nk"]
        X[s, 4:] = r["R"], r["sum_m"], r["S"]
    z = (X.mean(0) - want) / (X.std(0, ddof=1) / math.sqrt(T))
    assert np.all(np.abs(z) < 5), z


def test_rows_partition():
    rel = oracle.link(4, oracle.sprinkle_sorted(4, 300, 3))
    full = oracle.action(rel)
    a = oracle.action(rel, rows=(0, 120))
    b = oracle.action(rel, rows=(120, 300))
    assert np.array_equal(a["hist"] + b["hist"], full["hist"])
    assert a["R"] + b["R"] == full["R"] and a["W"] + b["W"] == full["W"]


@pytest.mark.parametrize("d,N,rows", [(2, 300, (0, 300)), (4, 500, (7, 60)), (2, 257, (250, 257))])
def test_rows_from_coords_match_matrix(d, N, rows):
    # the matrix-free row count agrees with the graph-library-pinned matrix count
    c = oracle.sprinkle_sorted(d, N, 21)
    a = oracle.action(oracle.link(d, c), rows=rows)
    b = oracle.action_rows_coords(d, c, *rows)
    assert np.array_equal(a["hist"], b["hist"])
    assert (a["R"], a["sum_m"], a["W"]) == (b["R"], b["sum_m"], b["W"])


# ------------------------------------------------------------ smeared action

def test_smeared_golden(golden):
    g = golden("diamond4.txt")
    h = oracle.action(inputs.rel_from_edges(g["N"], g["rel"]))["hist"]
    assert abs(oracle.smeared(g["N"], h, 0.5) - g["Seps_half"]) <= 1e-14
    assert abs(oracle.smeared(g["N"], h, 0.25) - g["Seps_quarter"]) <= 1e-14


@pytest.mark.parametrize("eps", [0.01, 2 ** -6, 0.3, 0.7])
def test_smeared_weights_are_binomial(eps):
    # f2(m, e) = P(B=0) - 2 P(B=1) + P(B=2) for B ~ Binomial(m, e): the sum in Eq.
    # s_smeared evaluated with the library binomial pmf
    from scipy import stats
    d, N = 2, 400
    h = oracle.action(oracle.link(d, oracle.sprinkle_sorted(d, N, 33)))["hist"]
    m = np.arange(N)
    w = stats.binom.pmf(0, m, eps) - 2 * stats.binom.pmf(1, m, eps) + stats.binom.pmf(2, m, eps)
    want = 2 * eps * (N - 2 * eps * float((h.astype(np.float64) * w).sum()))
    got = oracle.smeared(N, h, eps)
    scale = 2 * eps * (N + 2 * eps * float((h.astype(np.float64) * np.abs(w)).sum()))
    assert abs(got - want) <= 1e-12 * scale


def test_smeared_tends_to_local_action():
    # as e -> 1 only f2(0)=1, f2(1)=-2, f2(2)=1 survive, giving Eq. s_local
    for d, N, seed in ((2, 300, 4), (4, 250, 5)):
        out = oracle.action(oracle.link(d, oracle.sprinkle_sorted(d, N, seed)))
        _, S2 = oracle.finalize(2, N, out["Nk"])
        S = oracle.smeared(N, out["hist"], 1 - 1e-9)
        assert abs(S - S2) <= 1e-5 * max(abs(S2), N)


@pytest.mark.parametrize("d,N,seed", [(2, 11, 21), (4, 12, 22), (2, 12, 23)])
def test_smeared_is_mean_local_action_of_thinnings(d, N, seed):
    # Keeping each element independently with probability e, a pair with m elements between
    # them survives as a pair with k between with probability e^2 P(Binomial(m, e) = k), so the
    # mean local 1+1 action (Eq. s_local) of the kept subset is the smeared action S_e.  Brute
    # force over all 2^N subsets of a small sprinkled set, each subset counted by the pinned
    # interval counter and action.
    rel = oracle.link(d, oracle.sprinkle_sorted(d, N, seed))
    hist = oracle.action(rel)["hist"]
    S_sub = {}
    for mask in range(1 << N):
        keep = [e for e in range(N) if mask >> e & 1]
        if keep:
            sub = rel[np.ix_(keep, keep)]
            S_sub[mask] = (len(keep), oracle.finalize(2, len(keep), oracle.action(sub)["Nk"])[1])
        else:
            S_sub[mask] = (0, 0.0)
    for eps in (0.5, 0.25, 0.1, 0.9):
        want = math.fsum(eps ** n * (1 - eps) ** (N - n) * S for n, S in S_sub.values())
        got = oracle.smeared(N, hist, eps)
        assert abs(got - want) <= 1e-12 * max(1.0, math.fsum(
            eps ** n * (1 - eps) ** (N - n) * abs(S) for n, S in S_sub.values())), (eps, got, want)


@pytest.mark.parametrize("N", [24, 40])
def test_mean_smeared_action_2d_exact(N):
    # With the thinning reading above, a thinned uniform sprinkle of N elements is a uniform
    # sprinkle of Binomial(N, e) elements, whose mean 1+1 action is 2 at every size >= 1 (and
    # 0 for the empty set): E[S_e] = 2 (1 - (1 - e)^N).  Checked exactly against the expected
    # abundances, then against the oracle's mean over 20000 sets.
    E = [_expected_abundance(2, N, m) for m in range(N - 1)]
    for e in (Fraction(1, 2), Fraction(1, 4), Fraction(1, 10)):
        w = [sum(c * math.comb(m, k) * e ** k * (1 - e) ** (m - k) for k, c in ((0, 1), (1, -2), (2, 1)) if k <= m)
             for m in range(N - 1)]
        assert 2 * e * (N - 2 * e * sum(a * b for a, b in zip(E, w))) == 2 * (1 - (1 - e) ** N)
    T = 20000
    X = np.empty((T, 3))
    for s in range(T):
        h = oracle.run(2, N, seed=s, seq=9, threads=1)["hist"]
        X[s] = [oracle.smeared(N, h, eps) for eps in (0.5, 0.25, 0.1)]
    want = np.array([2 * (1 - (1 - eps) ** N) for eps in (0.5, 0.25, 0.1)])
    z = (X.mean(0) - want) / (X.std(0, ddof=1) / math.sqrt(T))
    assert np.all(np.abs(z) < 5), z


@pytest.mark.parametrize("N", [1, 50])
def test_smeared_antichain(N):
    assert oracle.smeared(N, np.zeros(N, np.uint64), 0.2) == 2 * 0.2 * N


# ------------------------------------------------------ 1+1 de Sitter slab

def test_desitter_sampler_distribution():
    # Sec. 5.1: eta has density sec^2(eta) / (2 tan eta0) on [-eta0, eta0], theta is uniform
    from scipy import stats
    eta0 = 0.5
    c = oracle.sprinkle_desitter(20000, eta0, seed=3)
    eta, theta = c[0], c[1]
    assert np.all(np.abs(eta) <= eta0) and np.all((theta >= 0) & (theta < 2 * math.pi))
    cdf = lambda x: (np.tan(x) + math.tan(eta0)) / (2 * math.tan(eta0))
    assert stats.kstest(eta, cdf).pvalue > 1e-4
    assert stats.kstest(theta, "uniform", args=(0, 2 * math.pi)).pvalue > 1e-4


@pytest.mark.parametrize("eta0", [0.5, 1.2])
def test_desitter_ordering_fraction(eta0):
    # For two iid elements of the slab the shorter arc between their angles is uniform on
    # [0, pi], so they are related with probability P = E|eta_1 - eta_2| / pi (|d eta| < pi),
    # eta with density sec^2(eta) / (2 tan eta0).  The related fraction of a set is a
    # U-statistic: variance 4 var(g)/N + 2 P(1-P)/N^2 with g(a) = E|a - eta| / pi.
    from scipy import integrate
    f = lambda a: 1.0 / (math.cos(a) ** 2 * 2.0 * math.tan(eta0))
    g = lambda a: integrate.quad(lambda b: abs(a - b) * f(b), -eta0, eta0, points=[a])[0] / math.pi
    P = integrate.quad(lambda a: g(a) * f(a), -eta0, eta0)[0]
    var_g = integrate.quad(lambda a: g(a) ** 2 * f(a), -eta0, eta0)[0] - P * P
    N, sets = 3000, 6
    frac = [oracle.link(oracle.DS2, oracle.sprinkle_desitter(N, eta0, s)).sum() / (N * (N - 1)) for s in range(sets)]
    sd = math.sqrt((4 * var_g / N + 2 * P * (1 - P) / N ** 2) / sets)
    assert abs(np.mean(frac) - P) < 5 * sd


def test_desitter_relation_is_cylinder_light_cone():
    # timelike iff the shorter arc between the angles is below |d eta| (Eq. ds_metric),
    # decided here in exact rationals with the min(|dth|, 2 pi - |dth|) form of the arc
    c, _ = oracle.sort(oracle.DS2, oracle.sprinkle_desitter(150, 0.5, seed=4))
    rel = oracle.link(oracle.DS2, c)
    pi = Fraction(math.pi)
    for i, j in itertools.combinations(range(150), 2):
        dth = abs(Fraction(c[1, j]) - Fraction(c[1, i]))
        arc = min(dth, 2 * pi - dth)
        assert rel[i, j] == (arc < abs(Fraction(c[0, j]) - Fraction(c[0, i])))
    assert np.all(np.diff(c[0]) >= 0)


def test_pack_layout():
    rel = inputs.random_upper_rel(130, 0.3, 1)
    w = oracle.pack(rel)
    assert w.shape == (130, 16)
    for i in (0, 63, 64, 129):
        for k in range(130):
            assert ((int(w[i, k // 64]) >> (k % 64)) & 1) == rel[i, k]
    assert np.array_equal(w, inputs.pack_rows(rel, 16))


def test_finalize_rejects_bad_dimension():
    with pytest.raises(RuntimeError):
        oracle.finalize(3, 5, [0, 0, 0, 0])


# ------------------------------------------------------- d'Alembertian pins

@pytest.mark.parametrize("name", ["diamond4.txt", "npos6.txt"])
def test_dalembertian_golden(golden, name):
    g = golden(name)
    rel = inputs.rel_from_edges(g["N"], g["rel"])
    B, L = oracle.dalembertian(rel, g["phi"], 1.0)
    assert B.tolist() == g["Bphi"]
    assert L.reshape(-1).tolist() == g["L123"]
    # B scales as 1/l^2 (Eq. b_local); powers of two scale exactly
    B2, _ = oracle.dalembertian(rel, g["phi"], 0.5)
    assert B2.tolist() == [4.0 * b for b in g["Bphi"]]


@pytest.mark.parametrize("N", [1, 2, 3, 4, 12, 70])
def test_dalembertian_chain(N):
    # In a chain the element k steps before x has k-1 elements between it and x, so
    # L_1, L_2, L_3 of x are x-1, x-2, x-3 (those that exist).
    phi = np.random.default_rng(N).normal(size=N)
    B, L = oracle.dalembertian(inputs.chain_rel(N), phi, 0.75)
    for x in range(N):
        terms = [(1.0, x - 1), (-2.0, x - 2), (1.0, x - 3)]
        inner = sum(c * phi[y] for c, y in terms if y >= 0)
        want = 2.0 / 0.75 ** 2 * (-phi[x] + 2.0 * inner)
        assert abs(B[x] - want) <= 1e-13 * (1.0 + abs(want))
        assert L[x].tolist() == [int(x >= 1), int(x >= 2), int(x >= 3)]


@pytest.mark.parametrize("N", [0, 1, 9])
def test_dalembertian_antichain(N):
    phi = np.arange(N, dtype=np.float64) - 3.5
    B, L = oracle.dalembertian(inputs.antichain_rel(N), phi, 2.0)
    assert B.tolist() == (-0.5 * phi).tolist()  # 2/l^2 = 1/2, no past
    assert not L.any()


@pytest.mark.parametrize("d,N,seed", [(2, 40, 5), (2, 64, 6)])
def test_dalembertian_matches_graph_library(d, N, seed):
    pytest.importorskip("networkx")
    rel = oracle.link(d, oracle.sprinkle_sorted(d, N, seed))
    g, desc, anc = _nx_intervals(rel)
    phi = np.random.default_rng(seed).uniform(-1, 1, size=N)
    B, L = oracle.dalembertian(rel, phi, 1.0)
    for x in range(N):
        layers = [[], [], []]
        for y in sorted(anc[x]):
            m = len(desc[y] & anc[x])
            if m <= 2:
                layers[m].append(y)
        assert L[x].tolist() == [len(v) for v in layers]
        inner = math.fsum(phi[y] for y in layers[0]) - 2 * math.fsum(phi[y] for y in layers[1]) \
            + math.fsum(phi[y] for y in layers[2])
        want = 2.0 * (-phi[x] + 2.0 * inner)
        bound = 2.0 * (abs(phi[x]) + 2.0 * sum(abs(phi[y]) * (2 if k == 1 else 1)
                                               for k in range(3) for y in layers[k]))
        assert abs(B[x] - want) <= 8 * (N + 4) * 2.0 ** -53 * bound


@pytest.mark.parametrize("d,N,seed", [(2, 300, 7), (2, 700, 8)])
def test_dalembertian_of_one_sums_to_minus_action(d, N, seed):
    # With phi = 1 and l = 1, sum_x B1(x) = 2(-N + 2 n_1 - 4 n_2 + 2 n_3) = -S_BD (Eq. s_local),
    # and every partial sum is a small integer, so the identity is exact.
    rel = oracle.link(d, oracle.sprinkle_sorted(d, N, seed))
    B, L = oracle.dalembertian(rel, np.ones(N), 1.0)
    _, S2 = oracle.finalize(2, N, oracle.action(rel)["Nk"])
    assert float(B.sum()) == -S2
    assert L.sum(axis=0).tolist() == [int(v) for v in oracle.action(rel)["Nk"][:3]]
