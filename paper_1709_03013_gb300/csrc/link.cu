// Linking: the symmetric bit-packed causal matrix of sorted coordinates (Sec. 2.2,
// "Optimized GPU Linking Algorithm": tiles of the adjacency matrix, coordinates
// staged in shared memory, dense output).
//
// d=4 and the de Sitter slab: a CTA takes up to kTileChunk 256 x 256 tiles (row block
// bi <= column block bj) of one row block of the upper triangle, setting up the rows once
// and staging each next column block by asynchronous copies while the current one is
// screened.  Warp w computes the 64-column word q = w / 2 of the tile for 4 x 32 rows (rows
// 32 (w & 1) + 64 s + lane, s = 0..3), so the column coordinates it reads from shared memory
// are the same for all of its lanes (broadcast 16-byte loads, one load per coordinate for
// four columns, used for four rows).  Row words are staged in shared memory and written as
// 32-byte row segments, one store each.  The lower triangle is the same tile transposed: a
// five-step warp-shuffle transpose per 32 x 32 block, staged in shared memory and written
// the same way.  Column blocks run to the row stride, so every word of every row --
// padding included -- is written exactly once and no memset is needed.
//
// Each pair is settled by a float screen, and the few pairs the screen cannot settle are
// decided exactly in double, so the bitmap equals the one of the exact (IEEE double)
// predicate:
//
// d=4 (flat diamond): related iff t_k > t_i and dt*dt > (dx*dx + dy*dy) + dz*dz in
// double, the elements time-sorted so that k > i.  The screen evaluates the interval in
// its expanded form,
//     e = p - h_k - h_i = -s^2 / 2,   p = t_k t_i - x_k x_i - y_k y_i - z_k z_i,
//     h = (t^2 - x^2 - y^2 - z^2) / 2 (formed in double, rounded once to float),
// as one float add and four fused multiply-adds on packed pairs of columns (f32x2).
// Error bound, with every |coordinate| <= S (S >= 1) and u = 2^-24: rounding the
// coordinates to float moves the four products by at most 2u * 4 S^2; |h| <= 1.5 S^2, so
// rounding the two h moves e by at most 3u S^2; the first add (|sum| <= 3 S^2) rounds by at
// most 3u S^2 and the four fused multiply-adds (partial sums below 4, 5, 6, 7 S^2) by 22u S^2.
// So |fl(e) + s^2/2| <= 36u S^2 < 2.2e-6 S^2 (plus terms of order u^2), while the double
// predicate is within 1e-14 S^2 of the real one.  With the margin m = 4e-6 S^2 (every word
// of a d=4 tile, words on the diagonal and ragged words included, under a column mask):
//   * the rows carry fl(-h_i + m), so the chain gives e' ~ e + m within
//     37.5u S^2 < 2.3e-6 S^2 (one more rounding).  A sign bit of e' (e' <= 0) means
//     s^2 / 2 >= m - 2.3e-6 S^2 > 0: certainly related.  A clear sign bit of
//     fl(e' - 2m) means e' >= 2m - 7u S^2, hence -s^2 / 2 >= m - 2.7e-6 S^2 > 0:
//     certainly unrelated.  The funnel-shifted sign words give both per pair, and only the
//     pairs between them are evaluated in double (from shared memory).
//
// d=2 (flat diamond): related iff u_i < u_k and v_i < v_k (light-cone coordinates) in
// double; this product order is settled without a pair-by-pair test (link_d2_kernel below).
//
// 1+1 de Sitter slab (Sec. 5.1): related when the shorter arc between the angles is below
// |d eta|, i.e. pi - |pi - |d theta|| < |d eta| in double.  With |eta| < pi/2 and theta in
// [0, 2 pi), the float form of |d eta| minus that arc is within 2.6e-6 of the real value,
// so a float difference beyond +-1e-5 fixes the decision; this geometry is evaluated
// pair by pair.
//
// Coordinates are limited to 1e15 in magnitude (checked where sets are made), far below
// float overflow of every product and sum above.
#include <cuda_runtime.h>
#include <stdint.h>

#include "csg_internal.cuh"

namespace csg {
namespace {

constexpr int kTile = 256;      // rows and columns per tile
constexpr int kTileWords = 4;   // 64-bit words per tile row
constexpr int kRowsPer = 4;     // rows per thread (one 64-column word each)
constexpr int kLinkMinBlocks = 3;  // resident CTAs per SM of the tile kernel (80 registers)
constexpr int kTileChunk = 4;      // column blocks per CTA of the tile kernel (d=4, de Sitter)
constexpr int kD2Chunk = 16;       // column blocks per CTA of the d=2 kernel

struct LinkRow {
    int32_t d;  // 2, 4 or GEOM_DS2
    int32_t pad;
    int64_t N, stride;
    const double *coords;
    uint64_t *rows;
    int64_t tile_off;  // first CTA of the set (d=4, de Sitter: one per tile; d=2: per row-block chunk)
    int64_t nb, nbc;   // row blocks, column blocks
    int64_t eoff;     // first element of the set within its geometry's elements
    int64_t foff;     // first float of the set's screen values (screen_floats(d) rows of N)
    float margin;     // float-screen margin: d=4 4e-6 S^2 on e, de Sitter 1e-5
    float pad2;
    int64_t rboff;    // d=2: the set's first row block in the sorted-block scratch
};

// float screen values per element: d=4 T, X, Y, Z, -H; de Sitter eta, theta
__host__ __device__ constexpr int screen_floats(int d) { return d == 4 ? 5 : 2; }

__device__ __forceinline__ int find_set(const int64_t *__restrict__ starts, int n, int64_t g) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (starts[mid] <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// A CTA takes up to C consecutive column blocks bj of one row block bi (bi <= bj < nbc).
// sum_{n=1}^{M} ceil(n / C) = C a (a + 1) / 2 + r (a + 1) with M = a C + r.
template <int C>
__host__ __device__ __forceinline__ int64_t ceil_sum(int64_t M) {
    const int64_t a = M / C, r = M % C;
    return C * a * (a + 1) / 2 + r * (a + 1);
}
// CTAs before row block b: sum_{q<b} ceil((nbc - q) / C)
template <int C>
__host__ __device__ __forceinline__ int64_t items_before(int64_t b, int64_t nbc) {
    return ceil_sum<C>(nbc) - ceil_sum<C>(nbc - b);
}
// The row block bi and column blocks [bj0, bj1) of the set's CTA t.
template <int C>
__device__ __forceinline__ void item_blocks(int64_t t, int64_t nb, int64_t nbc, int64_t &bi, int64_t &bj0,
                                            int64_t &bj1) {
    int64_t lo = 0, hi = nb - 1;  // largest b with items_before(b) <= t
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (items_before<C>(mid, nbc) <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    bi = lo;
    bj0 = bi + (t - items_before<C>(bi, nbc)) * C;
    bj1 = bj0 + C < nbc ? bj0 + C : nbc;
}

// 32 bytes to global memory in one store (dst 32-byte aligned)
__device__ __forceinline__ void st_global_32B(uint64_t *dst, uint64_t a, uint64_t b, uint64_t c, uint64_t d) {
    asm volatile("st.global.v4.u64 [%0], {%1, %2, %3, %4};" ::"l"(dst), "l"(a), "l"(b), "l"(c), "l"(d) : "memory");
}

// Asynchronous copies of 4 or 8 bytes from global to shared memory (cp.async): `ok` false
// copies nothing and zero-fills the destination.
__device__ __forceinline__ void cp_async4(void *dst, const void *src, bool ok) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src, bool ok) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(ok ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

// packed pairs of floats (f32x2): low half = first column, high half = second
__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(uint64_t v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t fadd2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// shift the sign bit of e in at the bottom of acc
__device__ __forceinline__ uint32_t push_sign(float e, uint32_t acc) {
    return __funnelshift_l(__float_as_uint(e), acc, 1);
}

// 1+1 de Sitter slab (Sec. 5.1): related iff pi - |pi - |d theta|| < |d eta| in double
__device__ __forceinline__ bool exact_ds(double ei, double thi, double ek, double thk) {
    const double pi = 3.141592653589793;
    const double ang = __dsub_rn(pi, fabs(__dsub_rn(pi, fabs(__dsub_rn(thk, thi)))));
    return ang < fabs(__dsub_rn(ek, ei));
}

__device__ __forceinline__ bool exact4(double ti, double xi, double yi, double zi, double tk,
                                       double xk, double yk, double zk) {
    if (!(tk > ti)) return false;
    double dt = __dsub_rn(tk, ti);
    double dx = __dsub_rn(xk, xi), dy = __dsub_rn(yk, yi), dz = __dsub_rn(zk, zi);
    double s = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return __dmul_rn(dt, dt) > s;
}

// 32x32 bit transpose across a warp: lane r holds row r's bits (bit c = column c) and
// ends holding column r's bits (bit k = row k).  Five butterfly stages, each swapping
// the off-diagonal s x s blocks between lanes r and r ^ s.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const uint32_t m = s == 16 ? 0x0000FFFFu : s == 8 ? 0x00FF00FFu : s == 4 ? 0x0F0F0F0Fu : s == 2 ? 0x33333333u : 0x55555555u;
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, s);
        x = (lane & s) ? ((x & ~m) | ((y & ~m) >> s)) : ((x & m) | ((y & m) << s));
    }
    return x;
}

// Screen values of one element from its double coordinates (rounded once to float):
// d=4 T, X, Y, Z, -H with H = fl(h), h = (t^2 - x^2 - y^2 - z^2) / 2 formed in double;
// de Sitter eta, theta.
template <int D>
__device__ __forceinline__ void screen_values(const double *v, float *f) {
    if (D == 4) {
#pragma unroll
        for (int a = 0; a < 4; ++a) f[a] = __double2float_rn(v[a]);
        f[4] = -__double2float_rn(0.5 * (v[0] * v[0] - ((v[1] * v[1] + v[2] * v[2]) + v[3] * v[3])));
    } else {
        f[0] = __double2float_rn(v[0]);
        f[1] = __double2float_rn(v[1]);
    }
}

// Writes every element's screen values once per set (the tiles then read floats only):
// F[foff + a N + e] = value a of element e.
template <int D>
__global__ void __launch_bounds__(256)
link_screen_kernel(const LinkRow *__restrict__ sets, const int64_t *__restrict__ estarts, int n, int64_t E,
                   float *__restrict__ F) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= E) return;
    const LinkRow &S = sets[find_set(estarts, n, g)];
    const int64_t e = g - S.eoff, N = S.N;
    double v[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) v[a] = S.coords[a * N + e];
    float f[5];
    screen_values<D>(v, f);
#pragma unroll
    for (int a = 0; a < screen_floats(D); ++a) F[S.foff + a * N + e] = f[a];
}

// The double decision for tile row rt and tile column c (Sec. 2.2; d=4 in the time order of
// the set, de Sitter on the cylinder).  rd, cd: the tile's row and column coordinates in
// double (d=4 t, x, y, z; de Sitter eta, theta).
template <int D>
__device__ __forceinline__ bool exact_pair(const double (*rd)[kTile], const double (*cd)[kTile], int rt, int c) {
    if (D == 4) return exact4(rd[0][rt], rd[1][rt], rd[2][rt], rd[3][rt], cd[0][c], cd[1][c], cd[2][c], cd[3][c]);
    return exact_ds(rd[0][rt], rd[1][rt], cd[0][c], cd[1][c]);
}

// One 64-column word of tile row rt of the 1+1 de Sitter slab evaluated pair by pair: bit b
// set iff the row and column 64 q + b are related; columns outside [c0, ncol) stay 0.  The
// float screen (|d eta| minus the shorter arc, beyond the margin m) settles almost every pair
// and the rest are decided in double.  cf: the tile's column screen values (eta, theta); Fs:
// the set's screen values (row i's read).
__device__ __noinline__ uint64_t word_by_pair_ds(int q, int c0, int ncol, const float (*cf)[kTile],
                                                 const double (*rd)[kTile], const double (*cd)[kTile], int rt,
                                                 const float *__restrict__ Fs, int64_t N, int64_t i, float m) {
    const float eta = Fs[i], theta = Fs[N + i];
    uint64_t acc = 0;
    for (int b = 0; b < 64; ++b) {
        const int c = q * 64 + b;
        if (c < c0 || c >= ncol) continue;
        // cylinder light cone: shorter arc below |d eta|
        const float deta = fabsf(__fsub_rn(cf[0][c], eta));
        const float dth = fabsf(__fsub_rn(cf[1][c], theta));
        const float ang = __fsub_rn(3.14159265f, fabsf(__fsub_rn(3.14159265f, dth)));
        const float diff = __fsub_rn(deta, ang);
        if (diff > m || (diff >= -m && exact_pair<GEOM_DS2>(rd, cd, rt, c))) acc |= 1ull << b;
    }
    return acc;
}

// The packed d=4 screen over one full 64-column word for the thread's four rows.
// a[s][0..4]: row s's screen values, each duplicated into both halves of a packed pair;
// a[s][4] is fl(-H_i + m), so the chain gives e' ~ e + m.  A[s] holds the sign bits of e'
// (certainly related) and B[s] those of e' - 2m (related, or inside the margin): B & ~A are
// the pairs to decide in double.  Bit b of a word stands for column 64 q + b.
__device__ __forceinline__ void word_packed(int q, const float (*cf)[kTile], const uint64_t (*a)[5],
                                            uint64_t m2n, uint64_t *A, uint64_t *B) {
#pragma unroll
    for (int s = 0; s < kRowsPer; ++s) {
        A[s] = 0;
        B[s] = 0;
    }
    // columns from the top of the word down, so that column 64 q + b ends at bit b
#pragma unroll 1
    for (int h = 1; h >= 0; --h) {
        uint32_t acc[kRowsPer] = {0, 0, 0, 0}, bcc[kRowsPer] = {0, 0, 0, 0};
#pragma unroll 1
        for (int j = 7; j >= 0; --j) {
            const int c = 64 * q + 32 * h + 4 * j;
            const ulonglong2 cT = *reinterpret_cast<const ulonglong2 *>(&cf[0][c]);
            const ulonglong2 cX = *reinterpret_cast<const ulonglong2 *>(&cf[1][c]);
            const ulonglong2 cY = *reinterpret_cast<const ulonglong2 *>(&cf[2][c]);
            const ulonglong2 cZ = *reinterpret_cast<const ulonglong2 *>(&cf[3][c]);
            const ulonglong2 cH = *reinterpret_cast<const ulonglong2 *>(&cf[4][c]);
#pragma unroll
            for (int s = 0; s < kRowsPer; ++s) {
                uint64_t e01 = fadd2(cH.x, a[s][4]);
                uint64_t e23 = fadd2(cH.y, a[s][4]);
                e01 = ffma2(cT.x, a[s][0], e01);
                e23 = ffma2(cT.y, a[s][0], e23);
                e01 = ffma2(cX.x, a[s][1], e01);
                e23 = ffma2(cX.y, a[s][1], e23);
                e01 = ffma2(cY.x, a[s][2], e01);
                e23 = ffma2(cY.y, a[s][2], e23);
                e01 = ffma2(cZ.x, a[s][3], e01);
                e23 = ffma2(cZ.y, a[s][3], e23);
                float e0, e1, e2, e3, f0, f1, f2, f3;
                unpack2(e01, e0, e1);
                unpack2(e23, e2, e3);
                unpack2(fadd2(e01, m2n), f0, f1);
                unpack2(fadd2(e23, m2n), f2, f3);
                acc[s] = push_sign(e0, push_sign(e1, push_sign(e2, push_sign(e3, acc[s]))));
                bcc[s] = push_sign(f0, push_sign(f1, push_sign(f2, push_sign(f3, bcc[s]))));
            }
        }
#pragma unroll
        for (int s = 0; s < kRowsPer; ++s) {
            A[s] |= (uint64_t)acc[s] << (32 * h);
            B[s] |= (uint64_t)bcc[s] << (32 * h);
        }
    }
}

template <int D>
__global__ void __launch_bounds__(kTile, kLinkMinBlocks)
link_kernel(const LinkRow *__restrict__ sets, const int64_t *__restrict__ starts, int n,
            const float *__restrict__ F) {
    constexpr int ND = D == 4 ? 4 : 2;             // double coordinates the exact test reads
    __shared__ __align__(16) float cf[2][5][kTile];  // column screen values (two buffers)
    __shared__ double cd[ND][kTile];              // column coordinates in double
    __shared__ double rd[ND][kTile];              // row coordinates in double
    __shared__ uint64_t ow[kTileWords][kTile];    // row words: ow[q][r] = word q of tile row r
    __shared__ uint32_t tb[kTile][9];             // mirrored bits: tb[c][g] = rows 32g..32g+31 of column c

    const LinkRow S = sets[find_set(starts, n, blockIdx.x)];
    int64_t bi, bj0, bj1;
    item_blocks<kTileChunk>(blockIdx.x - S.tile_off, S.nb, S.nbc, bi, bj0, bj1);
    const int64_t R = bi * kTile;
    const int64_t N = S.N;
    const int r = threadIdx.x;
    const int lane = r & 31, warp = r >> 5;
    const float *__restrict__ Fs = F + S.foff;
    const double *__restrict__ co = S.coords;
    const int q = warp >> 1;                       // this warp's 64-column word
    const int rfirst = 32 * (warp & 1);            // tile rows rfirst + 64 s + lane
    const float m = S.margin;

    // the row block: row R + r in double (beyond N: zeros; no word reads them), and the
    // rows' screen values, each duplicated into a packed pair; d=4 rows carry the signs of
    // the space products and the margin: T, -X, -Y, -Z, fl(-H + m)
    {
        const int64_t i = R + r;
#pragma unroll
        for (int a = 0; a < ND; ++a) rd[a][r] = i < N ? co[a * N + i] : 0.0;
    }
    uint64_t a[kRowsPer][5];
#pragma unroll
    for (int s = 0; s < kRowsPer; ++s) {
        const int64_t i = R + rfirst + 64 * s + lane;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            float x = 0.f;
            if (c < screen_floats(D) && i < N) x = Fs[c * N + i];
            if (D == 4 && c >= 1 && c <= 3) x = -x;
            if (D == 4 && c == 4) x = __fadd_rn(x, m);
            a[s][c] = pack2(x, x);
        }
    }

    uint64_t *rows = S.rows;
    const int64_t stride = S.stride;
    // Column K + r is staged by asynchronous copies (beyond N: zeros; no word reads them):
    // the screen values of the next column block while this one is screened, the doubles
    // (read only for the pairs inside the margin) while the screen runs.
    auto stage_cf = [&](int64_t K, int buf) {
        const int64_t kc = K + r;
#pragma unroll
        for (int a = 0; a < screen_floats(D); ++a) cp_async4(&cf[buf][a][r], Fs + a * N + (kc < N ? kc : 0), kc < N);
        cp_async_commit();
    };
    stage_cf(bj0 * kTile, 0);
    int buf = 0;
    for (int64_t bj = bj0; bj < bj1; ++bj) {
        const int64_t K = bj * kTile;
        const bool diag = (bi == bj);
        {
            const int64_t kc = K + r;
#pragma unroll
            for (int a = 0; a < ND; ++a) cp_async8(&cd[a][r], co + a * N + (kc < N ? kc : 0), kc < N);
            cp_async_commit();
        }
        if (bj + 1 < bj1)
            stage_cf(K + kTile, buf ^ 1);
        else
            cp_async_commit();  // an empty group keeps the count of groups in flight fixed
        cp_async_wait<2>();     // this block's screen values have landed
        __syncthreads();

        const int ncol = N - K <= 0 ? 0 : (N - K >= kTile ? kTile : (int)(N - K));
        // Rows of this slot with any column of the word after them and before N (the same
        // for all lanes of the warp: slots start at multiples of 32, words at multiples of 64).
        bool any = false;
        bool live[kRowsPer];
#pragma unroll
        for (int s = 0; s < kRowsPer; ++s) {
            const int rlo = rfirst + 64 * s;
            live[s] = 64 * q < ncol && !(diag && rlo >= 64 * q + 64);
            any |= live[s];
        }

        uint64_t A[kRowsPer] = {0, 0, 0, 0}, B[kRowsPer] = {0, 0, 0, 0};
        if constexpr (D == 4) {
            if (any) {
                const float m2 = -(m + m);
                word_packed(q, cf[buf], a, pack2(m2, m2), A, B);
            }
        }
        cp_async_wait<1>();  // and this block's doubles
        __syncthreads();
#pragma unroll
        for (int s = 0; s < kRowsPer; ++s) {
            const int rt = rfirst + 64 * s + lane;     // tile row
            const int64_t i = R + rt;
            uint64_t wd = 0;
            if (i < N && live[s]) {
                // the word's columns after the row (diagonal tile) and before N
                const int lo = diag ? max(rt + 1 - 64 * q, 0) : 0;
                const int hi = min(ncol - 64 * q, 64);
                const uint64_t mask =
                    lo >= hi ? 0ull : ((hi == 64 ? ~0ull : (1ull << hi) - 1) & ~((1ull << lo) - 1));
                if constexpr (D == 4) {
                    // pairs the screen left open: decide them in double
                    wd = A[s] & mask;
                    uint64_t amb = B[s] & ~A[s] & mask;
                    while (amb) {
                        const int b = __ffsll((long long)amb) - 1;
                        amb &= amb - 1;
                        if (exact_pair<D>(rd, cd, rt, 64 * q + b))
                            wd |= 1ull << b;
                        else
                            wd &= ~(1ull << b);
                    }
                } else {
                    wd = word_by_pair_ds(q, lo + 64 * q, ncol, cf[buf], rd, cd, rt, Fs, N, i, m);
                }
            }
            ow[q][rt] = wd;
            // mirrored half: columns 64 q + 32 h + lane get the bits of rows 32 g .. 32 g + 31
#pragma unroll
            for (int h = 0; h < 2; ++h)
                tb[64 * q + 32 * h + lane][(warp & 1) + 2 * s] = warp_transpose32((uint32_t)(wd >> (32 * h)), lane);
        }
        __syncthreads();

        const int64_t i = R + r;
        const int64_t kc = K + r;
        uint64_t mw[kTileWords];
#pragma unroll
        for (int w = 0; w < kTileWords; ++w) mw[w] = (uint64_t)tb[r][2 * w] | ((uint64_t)tb[r][2 * w + 1] << 32);
        if (diag) {
            // both halves land in the same words: OR them
            if (i < N && CSG_IN_BOUNDS(K / 64 + kTileWords <= stride, 0x30, i))
                st_global_32B(rows + i * stride + K / 64, ow[0][r] | mw[0], ow[1][r] | mw[1], ow[2][r] | mw[2],
                              ow[3][r] | mw[3]);
        } else {
            if (i < N && CSG_IN_BOUNDS(K / 64 + kTileWords <= stride, 0x30, i))
                st_global_32B(rows + i * stride + K / 64, ow[0][r], ow[1][r], ow[2][r], ow[3][r]);
            if (kc < N && CSG_IN_BOUNDS(R / 64 + kTileWords <= stride, 0x31, kc))
                st_global_32B(rows + kc * stride + R / 64, mw[0], mw[1], mw[2], mw[3]);
        }
        // No barrier here: the next block's copies into cd and into this cf buffer, and its
        // writes of ow and tb, all come after a barrier that every thread reaches only once
        // its reads of this block are done.
        buf ^= 1;
    }
    cp_async_wait<0>();
}


// ------------------------------------------------------------------ d=2: dominance tiles
//
// In light-cone coordinates the d=2 relation is a product order: i < k iff u_i < u_k and
// v_i < v_k.  For the rows of one row block sorted by u, the rows with u_i < u_k are the first
// p_u(k) of them, p_u(k) = #{i : u_i < u_k}, found by a binary search of u_k in the sorted u;
// so with Pu[p] (Pv[p]) the set of the first p rows in u (v) order, column k's row set is
// Pu[p_u(k)] & Pv[p_v(k)].  A pre-pass sorts every row block once (a CTA per block: bitonic
// networks in shared memory, u and v side by side) and stores each sorted order as an
// implicit search tree (breadth-first, so that the first levels of every search read a few
// shared words that the lanes share) with the rows in that order.  A link CTA loads its row
// block's trees, builds the 257 prefix sets of each order (a warp per 64-row word: per-lane
// ORs, then a shuffle OR scan), and then runs kD2Chunk column blocks: one thread per column,
// two tree searches and four ANDs give the column's 256 row bits (the mirrored half), and a
// warp-shuffle transpose gives the row words; each thread writes its 32 bytes of a row with
// one 32-byte store.  Coordinates are compared as 64-bit integer keys that order exactly as
// the doubles do (-0 folded onto +0, negative values' magnitude bits flipped), so every
// decision is the exact double one, on the integer pipe rather than the few FP64 units; ties
// are no special case (equal values are not less), and padding rows carry the largest key,
// which no finite coordinate reaches.  A pair i < k always has i earlier in the time order
// (t is (u + v) / 2, its ties broken by u); the diagonal block, whose row words and mirrored
// words are ORed, still keeps only rows before each column, as the tile kernel does, so a
// caller's set with some other t gets the same matrix from both.
// One row block in u (g = 0) and v (g = 1) order: tree[g][j], j = 1..255, the search tree
// of the first 255 sorted keys (node j holds the key of in-order rank tree_rank(j)),
// tree[g][0] the largest key; idx[g][q] the tile row of sorted position q.
struct SortedBlock {
    long long tree[2][kTile];
    uint16_t idx[2][kTile];
};

// A 64-bit integer with the order of the double x: a < b as doubles iff key(a) < key(b)
// (finite values; -0 and +0 get the same key).
__device__ __forceinline__ long long order_key(double x) {
    long long b = __double_as_longlong(x);
    if (b == (long long)0x8000000000000000ull) b = 0;
    return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}
constexpr long long kKeyPad = 0x7fffffffffffffffll;  // above every finite coordinate's key

// In-order rank of node j (1..255) of the complete search tree of 255 keys whose node j has
// children 2j and 2j + 1 (depth d = floor(log2 j)).
__device__ __forceinline__ int tree_rank(int j) {
    const int d = 31 - __clz(j);
    return ((2 * (j - (1 << d)) + 1) << (7 - d)) - 1;
}

// #{q : sorted[q] < x} for 256 ascending keys held as the tree tree[1..255] of the first 255
// and `last`: eight steps down the tree leave j - 256 = the count among the 255.
__device__ __forceinline__ int count_below(const long long *tree, long long last, long long x) {
    int j = 1;
#pragma unroll
    for (int l = 0; l < 8; ++l) j = 2 * j + (tree[j] < x);
    const int c = j - kTile;
    return c + (c == kTile - 1 && last < x);
}

// Pre-pass: one CTA per d=2 row block (numbered across the sets, rbstarts[s] = first row
// block of set s) sorts the block's u and v keys with their rows and stores the result as
// one SortedBlock.
__global__ void __launch_bounds__(kTile)
link_d2_sort_kernel(const LinkRow *__restrict__ sets, const int64_t *__restrict__ rbstarts, int n,
                    SortedBlock *__restrict__ out) {
    __shared__ long long key[2][kTile];
    __shared__ uint16_t idx[2][kTile];
    const int sidx = find_set(rbstarts, n, blockIdx.x);
    const LinkRow &S = sets[sidx];
    const int64_t R = (blockIdx.x - rbstarts[sidx]) * kTile, N = S.N;
    const int r = threadIdx.x;
    {
        const int64_t i = R + r;
        key[0][r] = i < N ? order_key(S.coords[2 * N + i]) : kKeyPad;  // u
        key[1][r] = i < N ? order_key(S.coords[3 * N + i]) : kKeyPad;  // v
        idx[0][r] = idx[1][r] = (uint16_t)r;
    }
    __syncthreads();
    {
        const int g = r >> 7, q = r & 127;  // threads 0-127 sort u, 128-255 sort v
        for (int k = 2; k <= kTile; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                const int a = 2 * q - (q & (j - 1)), b = a + j;
                const long long ka = key[g][a], kb = key[g][b];
                if ((ka > kb) == ((a & k) == 0)) {
                    key[g][a] = kb;
                    key[g][b] = ka;
                    const uint16_t ia = idx[g][a];
                    idx[g][a] = idx[g][b];
                    idx[g][b] = ia;
                }
                __syncthreads();
            }
    }
    SortedBlock &o = out[blockIdx.x];
    const int g = r >> 7, j = r & 127;
    o.tree[g][j] = j > 0 ? key[g][tree_rank(j)] : key[g][kTile - 1];
    o.tree[g][j + 128] = key[g][tree_rank(j + 128)];
    o.idx[0][r] = idx[0][r];
    o.idx[1][r] = idx[1][r];
}

__global__ void __launch_bounds__(kTile, 5)
link_d2_kernel(const LinkRow *__restrict__ sets, const int64_t *__restrict__ starts, int n,
               const SortedBlock *__restrict__ sorted) {
    __shared__ __align__(16) SortedBlock blk;           // the row block's trees and orders
    __shared__ uint64_t pre[2][kTileWords][kTile + 1];  // pre[g][w][p]: word w of prefix set p
    __shared__ uint32_t tb[2][kTile][9];                // tb[b][r][g]: row r, columns 32g..32g+31 (two buffers)

    const LinkRow S = sets[find_set(starts, n, blockIdx.x)];
    int64_t bi, bj0, bj1;
    item_blocks<kD2Chunk>(blockIdx.x - S.tile_off, S.nb, S.nbc, bi, bj0, bj1);
    const int64_t R = bi * kTile, N = S.N, stride = S.stride;
    const double *__restrict__ cu = S.coords + 2 * N;  // u, then v
    const double *__restrict__ cv = S.coords + 3 * N;
    const int r = threadIdx.x, lane = r & 31, warp = r >> 5;

    {
        // the row block's SortedBlock, 16 bytes per thread and step
        const uint4 *src = reinterpret_cast<const uint4 *>(sorted + S.rboff + bi);
        uint4 *dst = reinterpret_cast<uint4 *>(&blk);
        for (int q = r; q < (int)(sizeof(SortedBlock) / 16); q += kTile) dst[q] = src[q];
    }
    // the first column block's coordinates
    int64_t kc = bj0 * kTile + r;
    long long xu = kc < N ? order_key(cu[kc]) : 0, xv = kc < N ? order_key(cv[kc]) : 0;
    __syncthreads();
    {
        // warps 0-3: u order, 64-row word `warp`; warps 4-7: v order
        const int g = warp >> 2, w = warp & 3;
        uint64_t loc[8], x = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int rr = blk.idx[g][8 * lane + j];
            if ((rr >> 6) == w) x |= 1ull << (rr & 63);
            loc[j] = x;
        }
        uint64_t inc = x;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc |= y;
        }
        uint64_t exc = __shfl_up_sync(0xffffffffu, inc, 1);
        if (lane == 0) exc = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) pre[g][w][8 * lane + j + 1] = exc | loc[j];
        if (lane == 0) pre[g][w][0] = 0;
    }
    __syncthreads();
    const long long lastu = blk.tree[0][0], lastv = blk.tree[1][0];

    uint64_t *rows = S.rows;
    const int64_t i = R + r;
    int buf = 0;
    for (int64_t bj = bj0; bj < bj1; ++bj) {
        const int64_t K = bj * kTile;
        uint64_t cm[kTileWords] = {0, 0, 0, 0};  // column K + r: its rows i < (K + r)
        const bool live = kc < N;
        if (live) {
            const int pu = count_below(blk.tree[0], lastu, xu), pv = count_below(blk.tree[1], lastv, xv);
#pragma unroll
            for (int w = 0; w < kTileWords; ++w) cm[w] = pre[0][w][pu] & pre[1][w][pv];
            if (bj == bi) {
                // within the diagonal block only the rows before the column count, as the
                // other tiles see only later columns (for coordinates whose t is (u + v) / 2
                // this removes nothing)
#pragma unroll
                for (int w = 0; w < kTileWords; ++w)
                    cm[w] &= r >= 64 * w + 64 ? ~0ull : (r <= 64 * w ? 0ull : (1ull << (r - 64 * w)) - 1ull);
            }
        }
        const int64_t kcur = kc;
        kc += kTile;  // the next column block's coordinates, loaded during the transpose
        if (bj + 1 < bj1) {
            xu = kc < N ? order_key(cu[kc]) : 0;
            xv = kc < N ? order_key(cv[kc]) : 0;
        }
        // lanes hold columns 32 warp + lane; after the transpose lane l holds row 32 c + l
#pragma unroll
        for (int c = 0; c < 8; ++c)
            tb[buf][32 * c + lane][warp] = warp_transpose32((uint32_t)(cm[c >> 1] >> (32 * (c & 1))), lane);
        __syncthreads();
        uint64_t rw[kTileWords];
#pragma unroll
        for (int w = 0; w < kTileWords; ++w)
            rw[w] = (uint64_t)tb[buf][r][2 * w] | ((uint64_t)tb[buf][r][2 * w + 1] << 32);
        if (bj == bi) {
            if (i < N && CSG_IN_BOUNDS(K / 64 + kTileWords <= stride, 0x30, i))
                st_global_32B(rows + i * stride + K / 64, rw[0] | cm[0], rw[1] | cm[1], rw[2] | cm[2], rw[3] | cm[3]);
        } else {
            if (i < N && CSG_IN_BOUNDS(K / 64 + kTileWords <= stride, 0x30, i))
                st_global_32B(rows + i * stride + K / 64, rw[0], rw[1], rw[2], rw[3]);
            if (live && CSG_IN_BOUNDS(R / 64 + kTileWords <= stride, 0x31, kcur))
                st_global_32B(rows + kcur * stride + R / 64, cm[0], cm[1], cm[2], cm[3]);
        }
        // No second barrier: the next block writes the other buffer, and this one is written
        // again only after the next block's barrier, which every thread reaches after its reads.
        buf ^= 1;
    }
}

}  // namespace

unsigned long long check_word_link() { return take_check_word(); }

LinkPlan link_plan(const LinkSpec *specs, int n, Arena &a, int *rc) {
    LinkPlan p;
    *rc = CSG_OK;
    int64_t nf = 0;  // floats of screen values over all sets
    // one tile space per geometry: each launch runs one instantiation of the kernel
    for (int part = 0; part < 3; ++part) {
        const int d = part == 0 ? 2 : (part == 1 ? 4 : GEOM_DS2);
        std::vector<LinkRow> rows;
        std::vector<int64_t> starts, estarts, rbstarts;
        int64_t T = 0, E = 0, RB = 0;
        for (int s = 0; s < n; ++s) {
            if (specs[s].d != d) continue;
            LinkRow L;
            L.d = d;
            L.pad = 0;
            L.N = specs[s].N;
            L.stride = specs[s].stride;
            L.coords = specs[s].coords;
            L.rows = specs[s].rows;
            L.nb = (L.N + kTile - 1) / kTile;
            L.nbc = L.stride / kTileWords;
            L.tile_off = T;
            L.eoff = E;
            L.foff = nf;
            L.margin = d == GEOM_DS2 ? 1e-5f
                       : d == 4     ? 4e-6f * (float)(specs[s].coord_scale * specs[s].coord_scale)
                                    : 0.f;
            L.pad2 = 0.f;
            L.rboff = RB;
            if (L.stride % 16 != 0 || L.nbc < L.nb || ((uintptr_t)L.rows & 31) != 0) {
                set_error("link: stride %lld does not cover N=%lld, or the rows are not 32-byte aligned",
                          (long long)L.stride, (long long)L.N);
                *rc = CSG_E_INVAL;
                return p;
            }
            starts.push_back(T);
            estarts.push_back(E);
            rows.push_back(L);
            if (d == 2) {
                T += items_before<kD2Chunk>(L.nb, L.nbc);  // no screen values
                rbstarts.push_back(RB);
                RB += L.nb;                      // row blocks the pre-pass sorts
            } else {
                T += items_before<kTileChunk>(L.nb, L.nbc);
                nf += (int64_t)screen_floats(d) * L.N;
            }
            E += L.N;
        }
        if (T > 0x7fffffffLL || (E + 255) / 256 > 0x7fffffffLL || RB > 0x7fffffffLL) {
            set_error("link: %lld tiles exceed one launch", (long long)T);
            *rc = CSG_E_INVAL;
            return p;
        }
        LinkPlan::Part &P = p.part[part];
        P.n = (int)rows.size();
        P.T = T;
        P.E = E;
        P.RB = RB;
        if (P.n) {
            P.t_rows = a.put(rows.data(), rows.size() * sizeof(LinkRow));
            P.t_starts = a.put(starts.data(), starts.size() * sizeof(int64_t));
            P.t_estarts = a.put(estarts.data(), estarts.size() * sizeof(int64_t));
            if (!rbstarts.empty()) P.t_rbstarts = a.put(rbstarts.data(), rbstarts.size() * sizeof(int64_t));
        }
        p.T += T;
    }
    p.s_screen = a.reserve((size_t)nf * sizeof(float));
    p.s_sorted = a.reserve((size_t)p.part[0].RB * sizeof(SortedBlock));
    return p;
}

template <int D>
static void link_part_launch(const LinkPlan::Part &P, const Arena &a, float *F, SortedBlock *sorted,
                             cudaStream_t st) {
    if (P.T == 0) return;
    if constexpr (D == 2) {
        link_d2_sort_kernel<<<(unsigned)P.RB, kTile, 0, st>>>(a.tab<LinkRow>(P.t_rows), a.tab<int64_t>(P.t_rbstarts),
                                                              P.n, sorted);
        link_d2_kernel<<<(unsigned)P.T, kTile, 0, st>>>(a.tab<LinkRow>(P.t_rows), a.tab<int64_t>(P.t_starts), P.n,
                                                        sorted);
    } else {
        link_screen_kernel<D><<<(unsigned)((P.E + 255) / 256), 256, 0, st>>>(
            a.tab<LinkRow>(P.t_rows), a.tab<int64_t>(P.t_estarts), P.n, P.E, F);
        link_kernel<D><<<(unsigned)P.T, kTile, 0, st>>>(a.tab<LinkRow>(P.t_rows), a.tab<int64_t>(P.t_starts), P.n, F);
    }
}

void link_launch(const LinkPlan &p, const Arena &a, cudaStream_t st) {
    if (p.T == 0) return;
    stage_begin(CSG_STAGE_LINK, st);
    float *F = a.scr<float>(p.s_screen);
    SortedBlock *sorted = a.scr<SortedBlock>(p.s_sorted);
    link_part_launch<2>(p.part[0], a, F, sorted, st);
    link_part_launch<4>(p.part[1], a, F, sorted, st);
    link_part_launch<GEOM_DS2>(p.part[2], a, F, sorted, st);
    stage_end(CSG_STAGE_LINK, st);
}

int link_batch(const LinkSpec *specs, int n, cudaStream_t st) {
    if (n <= 0) return CSG_OK;
    Arena a;
    int rc;
    LinkPlan p = link_plan(specs, n, a, &rc);
    if (rc != CSG_OK || p.T == 0) return rc;
    rc = arena_alloc(a, st);
    if (rc != CSG_OK) return rc;
    arena_upload(a, st);
    link_launch(p, a, st);
    cudaError_t le = cudaGetLastError();
    arena_free(a, st);
    if (le != cudaSuccess) {
        set_error("link launch: %s", cudaGetErrorString(le));
        return CSG_E_CUDA;
    }
    return CSG_OK;
}

}  // namespace csg
