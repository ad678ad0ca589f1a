// Linking: the symmetric bit-packed causal matrix of sorted coordinates (Sec. 2.2,
// "Optimized GPU Linking Algorithm": tiles of the adjacency matrix, coordinates
// staged in shared memory, dense output).
//
// A CTA owns a 256 x 256 tile (row block bi <= column block bj) of the upper
// triangle.  Thread r evaluates the 256 pairs (R+r, K+c) with column coordinates
// read from shared memory (broadcast) and keeps the four row words in registers.
// The lower triangle is the same tile transposed: a warp ballot over its 32 rows
// per column gives 32 bits of the mirrored row, staged in shared memory and
// written as 32-byte row segments.  Column blocks run to the row stride, so every
// word of every row -- padding included -- is written exactly once and no memset
// is needed.
//
// d=4 decisions are the exact IEEE double ones (t_k > t_i and dt*dt > (dx*dx +
// dy*dy) + dz*dz, separately rounded).  A float screen settles almost every pair
// first: with coordinates in [-1, 1], rounding them to float moves each difference
// by at most 4.0001 * 2^-24 and each square by at most 16.004 * 2^-24; the four
// fused multiply-adds that form dt^2 - ((dx^2 + dy^2) + dz^2) add at most
// 4 * 4.01 * 2^-24, so the float value is within 80.1 * 2^-24 (< 4.8e-6) of the real
// one, and the double expression within 40 * 2^-53 of it.  A float difference
// beyond +-1e-5 therefore fixes the double decision.
// Pairs inside the margin are decided in double.
//
// The 1+1 de Sitter slab (Sec. 5.1) relates two elements when the shorter arc between
// their angles is below |d eta|, i.e. pi - |pi - |d theta|| < |d eta| in double.  With
// |eta| < pi/2 and theta in [0, 2 pi), the float form of |d eta| minus that arc is within
// 2.6e-6 of the real value, so the same 1e-5 screen applies.  Every error term scales with the
// square of the coordinate range, so sets whose coordinates exceed 1 in magnitude
// use the margin 1e-5 * max|coordinate|^2 (coordinates are limited to 1e15, far
// below float overflow of the squares).
#include <cuda_runtime.h>
#include <stdint.h>

#include "csg_internal.cuh"

namespace csg {
namespace {

constexpr int kTile = 256;      // rows and columns per tile
constexpr int kTileWords = 4;   // 64-bit words per tile row

struct LinkRow {
    int32_t d;  // 2 or 4
    int32_t pad;
    int64_t N, stride;
    const double *coords;
    uint64_t *rows;
    int64_t tile_off;
    int64_t nb, nbc;  // row blocks, column blocks
    float screen;     // d=4 float-screen margin: 1e-5 * max(1, max |coordinate|)^2
    float pad2;
};

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

// tiles before row block b: sum_{q<b} (nbc - q)
__device__ __forceinline__ int64_t tiles_before(int64_t b, int64_t nbc) {
    return b * nbc - b * (b - 1) / 2;
}

// order-preserving encoding of a double (no NaN); -0 is folded onto +0, so that
// integer order equals IEEE order
__device__ __forceinline__ uint64_t order_key(double x) {
    if (x == 0.0) x = 0.0;
    uint64_t b = (uint64_t)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
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

// One 64-column word of row i: bit b set iff i and column K + q*64 + b are related.
// FULL: every column of the word is a valid later column (no bounds checks).
template <int D, bool FULL>
__device__ __forceinline__ uint64_t link_word(int q, int c0, int ncol, const uint64_t (*ck)[kTile],
                                              const float4 *cf4, const double (*cd)[kTile], uint64_t ui,
                                              uint64_t vi, float tf, float xf, float yf, float zf,
                                              double ti, double xi, double yi, double zi, float screen) {
    uint64_t acc = 0, amb = 0;
#pragma unroll
    for (int b = 0; b < 64; ++b) {
        const int c = q * 64 + b;
        if (!FULL && (c < c0 || c >= ncol)) continue;
        if (D == 2) {
            if ((ui < ck[0][c]) & (vi < ck[1][c])) acc |= 1ull << b;
        } else if (D == GEOM_DS2) {
            // cylinder light cone: shorter arc below |d eta|
            const float4 k4 = cf4[c];
            const float deta = fabsf(__fsub_rn(k4.x, tf));
            const float dth = fabsf(__fsub_rn(k4.y, xf));
            const float ang = __fsub_rn(3.14159265f, fabsf(__fsub_rn(3.14159265f, dth)));
            const float diff = __fsub_rn(deta, ang);
            if (diff > screen) acc |= 1ull << b;
            if (fabsf(diff) <= screen) amb |= 1ull << b;
        } else {
            const float4 k4 = cf4[c];
            const float dt = __fsub_rn(k4.x, tf);
            const float dx = __fsub_rn(k4.y, xf);
            const float dy = __fsub_rn(k4.z, yf);
            const float dz = __fsub_rn(k4.w, zf);
            const float sp = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
            const float diff = __fmaf_rn(dt, dt, -sp);
            if (diff > screen) acc |= 1ull << b;
            if (fabsf(diff) <= screen) amb |= 1ull << b;
        }
    }
    if (D != 2) {
        // pairs inside the screen's margin: decide in double (rare)
        while (amb) {
            const int b = __ffsll((long long)amb) - 1;
            amb &= amb - 1;
            const int c = q * 64 + b;
            if (D == GEOM_DS2 ? exact_ds(ti, xi, cd[0][c], cd[1][c])
                              : exact4(ti, xi, yi, zi, cd[0][c], cd[1][c], cd[2][c], cd[3][c]))
                acc |= 1ull << b;
            else
                acc &= ~(1ull << b);
        }
    }
    return acc;
}

template <int D>
__global__ void __launch_bounds__(kTile)
link_kernel(const LinkRow *__restrict__ sets, const int64_t *__restrict__ starts, int n) {
    __shared__ double cd[4][kTile];       // column coordinates (d=4: t,x,y,z)
    __shared__ uint64_t ck[2][kTile];     // column order keys of u and v (d=2)
    __shared__ float4 cf4[kTile];         // column coordinates in float (d=4): t, x, y, z
    __shared__ uint32_t tb[kTile][9];     // mirrored bits: tb[c][w] = rows 32w..32w+31 of column c

    const int s = find_set(starts, n, blockIdx.x);
    const LinkRow S = sets[s];
    const int64_t t = blockIdx.x - S.tile_off;
    // row block: largest b with tiles_before(b) <= t
    int64_t lo = 0, hi = S.nb - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (tiles_before(mid, S.nbc) <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    const int64_t bi = lo;
    const int64_t bj = bi + (t - tiles_before(bi, S.nbc));
    const int64_t R = bi * kTile, K = bj * kTile;
    const int64_t N = S.N;
    const bool diag = (bi == bj);
    const int r = threadIdx.x;
    const int lane = r & 31, warp = r >> 5;
    const int64_t i = R + r;
    const int64_t kc = K + r;  // column staged by this thread

    if (kc < N) {
        if (D == 2) {
            ck[0][r] = order_key(S.coords[2 * N + kc]);
            ck[1][r] = order_key(S.coords[3 * N + kc]);
        } else {  // d=4: t, x, y, z; de Sitter: eta, theta, 0, 0
            double v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                v[q] = S.coords[q * N + kc];
                cd[q][r] = v[q];
            }
            cf4[r] = make_float4(__double2float_rn(v[0]), __double2float_rn(v[1]), __double2float_rn(v[2]),
                                 __double2float_rn(v[3]));
        }
    }
    __syncthreads();

    uint64_t w[kTileWords] = {0, 0, 0, 0};
    const int64_t ncol_l = N - K;
    const int ncol = ncol_l <= 0 ? 0 : (ncol_l >= kTile ? kTile : (int)ncol_l);
    if (i < N) {
        const int c0 = diag ? r + 1 : 0;   // first column strictly after row i
        uint64_t ui = 0, vi = 0;
        double ti = 0, xi = 0, yi = 0, zi = 0;
        float tf = 0, xf = 0, yf = 0, zf = 0;
        if (D == 2) {
            ui = order_key(S.coords[2 * N + i]);
            vi = order_key(S.coords[3 * N + i]);
        } else {  // d=4 and de Sitter read the same rows
            ti = S.coords[i];
            xi = S.coords[N + i];
            yi = S.coords[2 * N + i];
            zi = S.coords[3 * N + i];
            tf = __double2float_rn(ti);
            xf = __double2float_rn(xi);
            yf = __double2float_rn(yi);
            zf = __double2float_rn(zi);
        }
        const bool full = !diag && ncol == kTile;
#pragma unroll 1
        for (int q = 0; q < kTileWords; ++q) {
            const uint64_t word =
                full ? link_word<D, true>(q, c0, ncol, ck, cf4, cd, ui, vi, tf, xf, yf, zf, ti, xi, yi, zi, S.screen)
                     : link_word<D, false>(q, c0, ncol, ck, cf4, cd, ui, vi, tf, xf, yf, zf, ti, xi, yi, zi, S.screen);
            if (q == 0) w[0] = word;
            else if (q == 1) w[1] = word;
            else if (q == 2) w[2] = word;
            else w[3] = word;
        }
    }

    // mirrored half: transpose each 32 x 32 block of this warp's rows
#pragma unroll
    for (int g = 0; g < kTile / 32; ++g) {
        const uint64_t word = w[g >> 1];
        const uint32_t x = (uint32_t)(word >> (32 * (g & 1)));
        tb[32 * g + lane][warp] = warp_transpose32(x, lane);
    }
    __syncthreads();

    uint64_t *rows = S.rows;
    const int64_t stride = S.stride;
    if (diag) {
        // both halves land in the same words: OR them
        if (i < N) {
            uint64_t *dst = rows + i * stride + K / 64;
#pragma unroll
            for (int q = 0; q < kTileWords; ++q) {
                uint64_t m = (uint64_t)tb[r][2 * q] | ((uint64_t)tb[r][2 * q + 1] << 32);
                dst[q] = w[q] | m;
            }
        }
    } else {
        if (i < N) {
            uint64_t *dst = rows + i * stride + K / 64;
            reinterpret_cast<ulonglong2 *>(dst)[0] = make_ulonglong2(w[0], w[1]);
            reinterpret_cast<ulonglong2 *>(dst)[1] = make_ulonglong2(w[2], w[3]);
        }
        if (kc < N) {
            uint64_t m[kTileWords];
#pragma unroll
            for (int q = 0; q < kTileWords; ++q)
                m[q] = (uint64_t)tb[r][2 * q] | ((uint64_t)tb[r][2 * q + 1] << 32);
            uint64_t *dst = rows + kc * stride + R / 64;
            reinterpret_cast<ulonglong2 *>(dst)[0] = make_ulonglong2(m[0], m[1]);
            reinterpret_cast<ulonglong2 *>(dst)[1] = make_ulonglong2(m[2], m[3]);
        }
    }
}

}  // namespace

LinkPlan link_plan(const LinkSpec *specs, int n, Arena &a, int *rc) {
    LinkPlan p;
    *rc = CSG_OK;
    // one tile space per geometry: each launch runs one instantiation of the kernel
    for (int part = 0; part < 3; ++part) {
        const int d = part == 0 ? 2 : (part == 1 ? 4 : GEOM_DS2);
        std::vector<LinkRow> rows;
        std::vector<int64_t> starts;
        int64_t T = 0;
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
            L.screen = d == GEOM_DS2 ? 1e-5f : 1e-5f * (float)(specs[s].coord_scale * specs[s].coord_scale);
            L.pad2 = 0.f;
            if (L.stride % 16 != 0 || L.nbc < L.nb) {
                set_error("link: stride %lld does not cover N=%lld", (long long)L.stride, (long long)L.N);
                *rc = CSG_E_INVAL;
                return p;
            }
            starts.push_back(T);
            rows.push_back(L);
            T += L.nb * L.nbc - L.nb * (L.nb - 1) / 2;
        }
        if (T > 0x7fffffffLL) {
            set_error("link: %lld tiles exceed one launch", (long long)T);
            *rc = CSG_E_INVAL;
            return p;
        }
        LinkPlan::Part &P = p.part[part];
        P.n = (int)rows.size();
        P.T = T;
        if (P.n) {
            P.t_rows = a.put(rows.data(), rows.size() * sizeof(LinkRow));
            P.t_starts = a.put(starts.data(), starts.size() * sizeof(int64_t));
        }
        p.T += T;
    }
    return p;
}

void link_launch(const LinkPlan &p, const Arena &a, cudaStream_t st) {
    if (p.T == 0) return;
    stage_begin(CSG_STAGE_LINK, st);
    const LinkPlan::Part &p2 = p.part[0], &p4 = p.part[1], &p3 = p.part[2];
    if (p2.T) link_kernel<2><<<(unsigned)p2.T, kTile, 0, st>>>(a.tab<LinkRow>(p2.t_rows), a.tab<int64_t>(p2.t_starts), p2.n);
    if (p4.T) link_kernel<4><<<(unsigned)p4.T, kTile, 0, st>>>(a.tab<LinkRow>(p4.t_rows), a.tab<int64_t>(p4.t_starts), p4.n);
    if (p3.T)
        link_kernel<GEOM_DS2><<<(unsigned)p3.T, kTile, 0, st>>>(a.tab<LinkRow>(p3.t_rows), a.tab<int64_t>(p3.t_starts), p3.n);
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
