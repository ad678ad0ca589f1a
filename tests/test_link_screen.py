"""The link kernel's float screens, checked on the CPU against their error analysis.

The d=4 link settles each pair by the sign of the expanded interval
    e = t_k t_i - x_k x_i - y_k y_i - z_k z_i - h_k - h_i = -s^2 / 2,   h = (t^2 - |x|^2) / 2,
evaluated in float (one add, then four fused multiply-adds) with the margin m = 4e-6 S^2
folded into the row value: a set sign bit of e' = fl(e + m) means certainly related, a clear
sign bit of fl(e' - 2m) certainly unrelated, and the pairs in between are decided in double.
The argument rests on |e' - (e + m)| <= 37.5 u S^2 (u = 2^-24, S = max(1, max |coordinate|)).

These tests replay that arithmetic operation by operation in numpy float32 (a fused
multiply-add as the exact double product plus the addend, rounded to float) and check, on
sprinkles, boxes and light-cone stress sets at scales 1 to 1e15, that no certain bit
contradicts the double predicate (the oracle's link), that the error stays inside the bound,
and that the pairs left to double are few.  The de Sitter slab's screen (arc against
|d eta|, margin 1e-5) is checked the same way, and the d=2 link, which has no float screen
(integer keys that order as the doubles do, sorted per row block, searched as trees, with
prefix row sets), is replayed step by step against the oracle's link.  No GPU is involved:
the kernel itself is compared with the oracle bit for bit by the GPU tests.
"""
import numpy as np
import pytest

import oracle
from paper_1709_03013_gb300 import inputs

f32 = np.float32
U = 2.0 ** -24


def _fma(a, b, c):
    # float32 fused multiply-add: the product of two floats is exact in double
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def _screen_d4(c, S):
    """Certain-related bits A, not-certainly-unrelated bits B (upper triangle, k > i) and the
    largest |e' - (e + m)| / (u S^2) over the pairs."""
    t, x, y, z = c
    T, X, Y, Z = (v.astype(f32) for v in (t, x, y, z))
    Hn = (-(0.5 * (t * t - ((x * x + y * y) + z * z)))).astype(f32)   # -h, formed in double
    m = f32(4e-6) * f32(S * S)
    aH = (Hn + m).astype(f32)                                          # row value fl(-h_i + m)
    m2 = -(m + m)
    N = t.shape[0]
    A = np.zeros((N, N), bool)
    B = np.zeros((N, N), bool)
    worst = 0.0
    for i in range(N - 1):
        k = np.arange(i + 1, N)
        e = (Hn[k] + aH[i]).astype(f32)
        e = _fma(T[k], np.full(k.size, T[i]), e)
        e = _fma(X[k], np.full(k.size, -X[i]), e)
        e = _fma(Y[k], np.full(k.size, -Y[i]), e)
        e = _fma(Z[k], np.full(k.size, -Z[i]), e)
        A[i, k] = np.signbit(e)
        B[i, k] = np.signbit((e + m2).astype(f32))
        dt = t[k] - t[i]
        s2 = dt * dt - ((x[k] - x[i]) ** 2 + (y[k] - y[i]) ** 2 + (z[k] - z[i]) ** 2)
        worst = max(worst, float(np.max(np.abs(e.astype(np.float64) - (-0.5 * s2 + float(m))))))
    return A, B, worst / (S * S * U)


def _box(N, seed, scale):
    # coordinates anywhere in [-scale, scale]^4 (the bound assumes only |coordinate| <= S)
    rng = np.random.default_rng(seed)
    c = rng.uniform(-scale, scale, size=(4, N))
    return oracle.sort(4, c)[0]


def _cases():
    out = []
    for sc in (1.0, 1e3, 1e15):
        out.append((f"sprinkle x{sc:g}", lambda sc=sc: oracle.sprinkle_sorted(4, 1200, 3) * sc))
        out.append((f"light cones x{sc:g}", lambda sc=sc: oracle.sort(4, inputs.light_cone_coords(4, 1200, 5, scale=sc))[0]))
        out.append((f"box x{sc:g}", lambda sc=sc: _box(1200, 7, sc)))
    return out


@pytest.mark.parametrize("name,make", _cases(), ids=[n for n, _ in _cases()])
def test_d4_screen_never_contradicts_double_predicate(name, make):
    c = np.ascontiguousarray(make())
    S = max(1.0, float(np.abs(c).max()))
    rel = oracle.link(4, c).astype(bool)
    A, B, worst = _screen_d4(c, S)
    iu = np.triu_indices(c.shape[1], 1)
    a, b, r = A[iu], B[iu], rel[iu]
    assert not (a & ~r).any()          # certainly related => related in double
    assert not (~b & r).any()          # certainly unrelated => unrelated in double
    assert not (a & ~b).any()          # the two sign words are nested
    assert worst <= 37.5, worst        # the error bound the margin is built on
    assert (b & ~a).sum() <= max(8, 0.01 * r.size)   # few pairs go to double


def _order_key(x):
    # the 64-bit integer with the order of the doubles: -0 folded onto +0, negative values'
    # magnitude bits flipped
    b = np.ascontiguousarray(x, dtype=np.float64).view(np.int64).copy()
    b[b == np.iinfo(np.int64).min] = 0
    return b ^ ((b >> 63) & np.int64(0x7FFFFFFFFFFFFFFF))


def _tree_rank(j):
    d = int(j).bit_length() - 1
    return ((2 * (j - (1 << d)) + 1) << (7 - d)) - 1


def _dominance_bitmap(c, rng):
    """The d=2 link as the dominance tiles compute it: per 256-row block, the rows sorted by
    the u and v keys (ties in any order), each order's first 255 keys as a breadth-first
    search tree plus the largest key, the prefix row sets, and for every column k of the
    block's tiles (k >= the block's first row) the row set Pu[#u below] & Pv[#v below];
    the same bits are stored for row i (future) and, mirrored, for row k (past)."""
    N = c.shape[1]
    ku, kv = _order_key(c[2]), _order_key(c[3])
    pad = np.iinfo(np.int64).max
    C = np.zeros((N, N), dtype=bool)
    for R in range(0, N, 256):
        cols = np.arange(R, N)
        masks = []
        for key in (ku, kv):
            rk = np.full(256, pad, dtype=np.int64)
            rk[:min(256, N - R)] = key[R:R + 256]
            order = np.lexsort((rng.random(256), rk))        # ascending, ties in random order
            srt = rk[order]
            tree = np.zeros(256, dtype=np.int64)
            for j in range(1, 256):
                tree[j] = srt[_tree_rank(j)]
            x = key[cols]
            j = np.ones(cols.size, dtype=np.int64)
            for _ in range(8):
                j = 2 * j + (tree[j] < x)
            cnt = j - 256
            cnt = cnt + ((cnt == 255) & (srt[255] < x))
            pre = np.zeros((257, 256), dtype=bool)            # pre[p]: the first p rows in order
            for p in range(1, 257):
                pre[p] = pre[p - 1]
                pre[p, order[p - 1]] = True
            masks.append(pre[cnt])
        m = masks[0] & masks[1]                               # (column, row of the block)
        rows = np.arange(R, min(R + 256, N))
        sub = m[:, :rows.size].T                              # (row, column)
        C[np.ix_(rows, cols)] |= sub
        C[np.ix_(cols, rows)] |= sub.T
    return C


@pytest.mark.parametrize("scale", [1.0, 1e3, 1e15])
def test_d2_dominance_tiles_match_double_predicate(scale):
    # d=2: related iff u_i < u_k and v_i < v_k in double.  The link kernel compares integer
    # keys that order as the doubles do; on light-cone stress sets (steps in u or v only,
    # one-ulp nudges, duplicates, signed zeros) its arithmetic must give the oracle's bitmap.
    N = 1500
    c = oracle.sort(2, inputs.light_cone_coords(2, N, 4, scale=scale))[0]
    rel = oracle.link(2, c).astype(bool)
    got = _dominance_bitmap(c, np.random.default_rng(7))
    assert np.array_equal(got, rel | rel.T)
    assert (np.diff(np.sort(c[2])) == 0).any() or (c[2] == 0).any()  # the set holds ties or zeros


def test_order_key_orders_as_doubles():
    x = np.array([-np.inf, -1e300, -2.0, -1.0, -5e-324, -0.0, 0.0, 5e-324, 1e-300, 0.5, 1.0, 2.0, 1e15, np.inf])
    k = _order_key(x)
    assert (np.diff(k[:5]) > 0).all() and k[5] == k[6] and (np.diff(k[6:]) > 0).all()
    rng = np.random.default_rng(3)
    y = np.concatenate([rng.normal(size=4000) * 10.0 ** rng.integers(-300, 300, 4000), [0.0, -0.0]])
    a, b = rng.choice(y, 20000), rng.choice(y, 20000)
    assert np.array_equal(a < b, _order_key(a) < _order_key(b))


@pytest.mark.parametrize("eta0,seed", [(0.5, 1), (1.2, 2), (1.5, 3)])
def test_desitter_screen_margin(eta0, seed):
    # 1+1 de Sitter slab: related iff the shorter arc pi - |pi - |d theta|| is below |d eta|
    # (in double).  The float form diff = |d eta| - arc (pi rounded to float) is within
    # 2.6e-6 of the real value, so diff > 1e-5 must mean related and diff < -1e-5 unrelated.
    N = 1500
    c = oracle.sprinkle_desitter(N, eta0, seed)
    rel = oracle.link(oracle.DS2, c).astype(bool)
    eta, th = c[0].astype(f32), c[1].astype(f32)
    pi_f, m = f32(3.14159265), f32(1e-5)
    i, k = np.triu_indices(N, 1)
    deta = np.abs((eta[k] - eta[i]).astype(f32))
    dth = np.abs((th[k] - th[i]).astype(f32))
    ang = (pi_f - np.abs((pi_f - dth).astype(f32))).astype(f32)
    diff = (deta - ang).astype(f32)
    r = rel[i, k]
    assert not ((diff > m) & ~r).any()
    assert not ((diff < -m) & r).any()
    assert (np.abs(diff) <= m).sum() <= 0.01 * r.size


@pytest.mark.parametrize("C", [4, 16])
def test_link_work_items_cover_the_upper_triangle_once(C):
    # A link CTA takes up to C consecutive column blocks of one row block (C = 4 for the
    # d=4 and de Sitter tile kernel, 16 for d=2): CTA t of a set is decoded with the closed
    # form sum_{n=1}^{M} ceil(n / C) = C a (a + 1) / 2 + r (a + 1), M = a C + r.  Every tile
    # bi <= bj < nbc must be visited exactly once, for row blocks nb <= nbc.
    def ceil_sum(M):
        a, r = divmod(M, C)
        return C * a * (a + 1) // 2 + r * (a + 1)

    def items_before(b, nbc):
        return ceil_sum(nbc) - ceil_sum(nbc - b)

    for nbc in list(range(1, 40)) + [160, 512]:
        for nb in sorted({0, 1, nbc // 3, nbc - 1, nbc}):
            seen = set()
            for t in range(items_before(nb, nbc)):
                lo, hi = 0, nb - 1
                while lo < hi:
                    mid = (lo + hi + 1) >> 1
                    if items_before(mid, nbc) <= t:
                        lo = mid
                    else:
                        hi = mid - 1
                bj0 = lo + (t - items_before(lo, nbc)) * C
                for bj in range(bj0, min(bj0 + C, nbc)):
                    assert (lo, bj) not in seen
                    seen.add((lo, bj))
            assert seen == {(a, b) for a in range(nb) for b in range(a, nbc)}
