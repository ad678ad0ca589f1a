// Sprinkling into a flat causal diamond (Sec. 2.1) and time ordering (Sec. 2.2),
// batched over many sets: every kernel walks a flattened element space with a
// small per-set table, so one launch sequence serves one set or thousands.
//
// Sort: composite keys (t, u, e) for d=2 and (t, e) for d=4 are encoded as two
// order-preserving uint64 words plus the element index, so every key is unique
// and the order is total.  Chunks of 1024 keys are ranked in shared memory, then
// sorted runs are merged pairwise: an element's place in the merged run is its
// rank in its own run plus the number of smaller keys in the sibling run (a
// binary search).  All of it is exact integer work.
#include <cuda_runtime.h>
#include <stdint.h>

#include "arena.h"
#include "csg_internal.cuh"

namespace csg {
namespace {

constexpr int kChunk = 1024;
constexpr int kSortThreads = 256;

// ------------------------------------------------------------ Philox4x64-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): ten rounds, each two 64x64->128 products, keys bumped by Weyl constants.
struct U64x4 {
    uint64_t w[4];
};

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                uint64_t k0, uint64_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t m0 = 0xD2E7470EE14C6C93ULL, m1 = 0xCA5A826395121157ULL;
        uint64_t hi0 = __umul64hi(m0, c0), lo0 = m0 * c0;
        uint64_t hi1 = __umul64hi(m1, c2), lo1 = m1 * c2;
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B97F4A7C15ULL;
        k1 += 0xBB67AE8584CAA73BULL;
    }
    U64x4 out;
    out.w[0] = c0;
    out.w[1] = c1;
    out.w[2] = c2;
    out.w[3] = c3;
    return out;
}

// top 53 bits scaled into [0, 1): exact conversion and power-of-two scaling
__device__ __forceinline__ double unit53(uint64_t x) {
    return __dmul_rn(__ull2double_rn(x >> 11), 0x1.0p-53);
}

// order-preserving encoding of a double (no NaN); -0 is folded onto +0
__device__ __forceinline__ uint64_t order_key(double x) {
    if (x == 0.0) x = 0.0;
    uint64_t b = (uint64_t)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}

// ------------------------------------------------------------ batch tables

struct SetRow {
    int32_t d;     // geometry: 2, 4 or GEOM_DS2
    int64_t N;
    uint64_t seed, seq;
    double *coords;      // sorted output [4][N]
    int64_t off;         // element offset in the flattened batch
    int64_t chunk_off;   // first chunk index of the set
    unsigned long long *err;  // set to CNT_ERR_REJECT when an element hits the attempt cap
    double param;             // GEOM_DS2: tan(eta0)
};

__device__ __forceinline__ int find_set(const int64_t *__restrict__ starts, int n, int64_t g) {
    // largest s with starts[s] <= g
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

struct Keys {
    uint64_t *k1, *k2;
    uint32_t *idx;
};

// One attempt of element e of set S (Sec. 2.1): returns true when the element is settled
// (accepted, a single-draw geometry, or out of attempts) with its coordinates in c.
__device__ __forceinline__ bool sprinkle_attempt(const SetRow &S, int64_t e, int a, double (&c)[4]) {
    if (S.d == GEOM_DS2) {
        // 1+1 de Sitter slab (Sec. 5.1): eta by inverting the sec^2 distribution,
        // theta uniform on the circle; rows eta, theta, 0, 0
        U64x4 r = philox4x64_10((uint64_t)e, 0, 0, 0, S.seed, S.seq);
        c[0] = atan(__dmul_rn(S.param, __dsub_rn(__dmul_rn(2.0, unit53(r.w[0])), 1.0)));
        c[1] = __dmul_rn(6.283185307179586, unit53(r.w[1]));
        c[2] = 0.0;
        c[3] = 0.0;
        return true;
    }
    if (S.d == 2) {
        U64x4 r = philox4x64_10((uint64_t)e, 0, 0, 0, S.seed, S.seq);
        double u = unit53(r.w[0]), v = unit53(r.w[1]);
        c[0] = __dmul_rn(__dadd_rn(u, v), 0.5);
        c[1] = __dmul_rn(__dsub_rn(v, u), 0.5);
        c[2] = u;
        c[3] = v;
        return true;
    }
    U64x4 r = philox4x64_10((uint64_t)e, (uint64_t)a, 0, 0, S.seed, S.seq);
    // fp32 screen: the top 24 bits of each word give the coordinate within 2^-23, and the
    // screened sum is within 2e-6 of the fp64 one; attempts closer than 4e-6 to the
    // boundary take the exact fp64 test (the decision is the fp64 one)
    const float tf = __fmaf_rn((float)(uint32_t)(r.w[0] >> 40), 0x1.0p-23f, -1.0f);
    const float xf = __fmaf_rn((float)(uint32_t)(r.w[1] >> 40), 0x1.0p-23f, -1.0f);
    const float yf = __fmaf_rn((float)(uint32_t)(r.w[2] >> 40), 0x1.0p-23f, -1.0f);
    const float zf = __fmaf_rn((float)(uint32_t)(r.w[3] >> 40), 0x1.0p-23f, -1.0f);
    const float sf = fabsf(tf) + sqrtf(__fmaf_rn(xf, xf, __fmaf_rn(yf, yf, zf * zf)));
    bool accept = false;
    if (sf <= 1.0f + 4e-6f) {
        const double t = __dsub_rn(__dmul_rn(2.0, unit53(r.w[0])), 1.0);
        const double x = __dsub_rn(__dmul_rn(2.0, unit53(r.w[1])), 1.0);
        const double y = __dsub_rn(__dmul_rn(2.0, unit53(r.w[2])), 1.0);
        const double z = __dsub_rn(__dmul_rn(2.0, unit53(r.w[3])), 1.0);
        accept = sf < 1.0f - 4e-6f;
        if (!accept) {
            const double rr = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
            accept = __dadd_rn(fabs(t), rr) <= 1.0;
        }
        if (accept) {
            c[0] = t;
            c[1] = x;
            c[2] = y;
            c[3] = z;
            return true;
        }
    }
    if (a + 1 >= 256) {  // out of attempts: the set reports CSG_E_REJECT
        atomicExch(S.err, (unsigned long long)CNT_ERR_REJECT);
        c[0] = c[1] = c[2] = c[3] = 0.0;
        return true;
    }
    return false;
}

// Sprinkle (or take host coordinates) into the unsorted buffer and emit sort keys.
// tmp is [4][E] (row r of set s at tmp + r*E + off).
// Each warp takes runs of `run` elements; a lane works on one element at a time, attempt
// after attempt (d=4 rejection sampling accepts 13 % of draws), and a lane whose element is
// settled takes the run's next element, so the warp's lanes stay busy instead of all waiting
// for the element that needs the most draws.  Attempt a of element e always uses the
// same counter (e, a), so the coordinates do not depend on which lane draws them.
__global__ void sprinkle_keys_kernel(const SetRow *__restrict__ sets, const int64_t *__restrict__ starts,
                                     int n, int64_t E, double *__restrict__ tmp, Keys keys,
                                     int from_coords, int64_t run) {
    const int lane = threadIdx.x & 31;
    const uint32_t below = (1u << lane) - 1u;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r0 = warp * run; r0 < E; r0 += warps * run) {
        const int64_t r1 = r0 + run < E ? r0 + run : E;
        int64_t g = r0 + lane;   // this lane's element (>= r1: idle)
        int64_t next = r0 + 32;  // the run's next unassigned element
        int a = 0;
        int s = g < r1 ? find_set(starts, n, g) : 0;
        SetRow S = sets[s];
        while (__any_sync(0xffffffffu, g < r1)) {
            bool done = false;
            if (g < r1) {
                const int64_t e = g - S.off;
                double c[4];
                if (from_coords) {
                    c[0] = tmp[g];
                    c[1] = tmp[E + g];
                    c[2] = tmp[2 * E + g];
                    c[3] = tmp[3 * E + g];
                    done = true;
                } else {
                    done = sprinkle_attempt(S, e, a, c);
                    if (done) {
                        tmp[g] = c[0];
                        tmp[E + g] = c[1];
                        tmp[2 * E + g] = c[2];
                        tmp[3 * E + g] = c[3];
                    }
                }
                if (done) {
                    keys.k1[g] = order_key(c[0]);
                    keys.k2[g] = (S.d == 2) ? order_key(c[2]) : 0ULL;
                    keys.idx[g] = (uint32_t)e;
                } else {
                    ++a;
                }
            }
            const uint32_t dm = __ballot_sync(0xffffffffu, done);
            if (done) {
                g = next + __popc(dm & below);
                a = 0;
                if (g < r1) {
                    // a lane's elements only move forward: step over at most four set
                    // boundaries, else search
                    int s2 = s;
                    for (int k = 0; k < 4 && s2 + 1 < n && starts[s2 + 1] <= g; ++k) ++s2;
                    if (s2 + 1 < n && starts[s2 + 1] <= g) s2 = find_set(starts, n, g);
                    if (s2 != s) {
                        s = s2;
                        S = sets[s];
                    }
                }
            }
            next += __popc(dm);
        }
    }
}

__device__ __forceinline__ bool key_less(uint64_t a1, uint64_t a2, uint32_t ai, uint64_t b1,
                                         uint64_t b2, uint32_t bi) {
    if (a1 != b1) return a1 < b1;
    if (a2 != b2) return a2 < b2;
    return ai < bi;
}

// Sort each chunk of kChunk keys in shared memory with a bitonic network (the keys of a
// set are all distinct, so the order is the same total order the rank would give); a
// partial last chunk is padded with keys above every real one.
__global__ void __launch_bounds__(kSortThreads)
chunk_sort_kernel(const SetRow *__restrict__ sets, const int64_t *__restrict__ chunk_starts, int n,
                  Keys in, Keys out) {
    __shared__ uint64_t s1[kChunk], s2[kChunk];
    __shared__ uint32_t si[kChunk];
    const int s = find_set(chunk_starts, n, blockIdx.x);
    const SetRow S = sets[s];
    const int64_t c = blockIdx.x - S.chunk_off;
    const int64_t base = S.off + c * kChunk;
    const int64_t rem = S.N - c * kChunk;
    const int len = rem < kChunk ? (int)rem : kChunk;
    for (int t = threadIdx.x; t < kChunk; t += kSortThreads) {
        const bool real = t < len;
        s1[t] = real ? in.k1[base + t] : ~0ull;
        s2[t] = real ? in.k2[base + t] : ~0ull;
        si[t] = real ? in.idx[base + t] : 0xFFFFFFFFu;
    }
    __syncthreads();
    for (int k = 2; k <= kChunk; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < kChunk; t += kSortThreads) {
                const int u = t ^ j;
                if (u > t) {
                    const bool up = (t & k) == 0;  // this pair's half of the network sorts ascending
                    const bool gt = key_less(s1[u], s2[u], si[u], s1[t], s2[t], si[t]);
                    if (gt == up) {
                        const uint64_t a1 = s1[t], a2 = s2[t];
                        const uint32_t ai = si[t];
                        s1[t] = s1[u];
                        s2[t] = s2[u];
                        si[t] = si[u];
                        s1[u] = a1;
                        s2[u] = a2;
                        si[u] = ai;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < len; t += kSortThreads) {
        if (!CSG_IN_BOUNDS(c * kChunk + t < S.N, 0x42, base + t)) continue;
        out.k1[base + t] = s1[t];
        out.k2[base + t] = s2[t];
        out.idx[base + t] = si[t];
    }
}

// One merge pass with run width w: runs [2q w, (2q+1) w) and [(2q+1) w, (2q+2) w).
__global__ void merge_pass_kernel(const SetRow *__restrict__ sets, const int64_t *__restrict__ starts,
                                  int n, int64_t E, int64_t w, Keys in, Keys out) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < E;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int s = find_set(starts, n, g);
        const SetRow S = sets[s];
        const int64_t p = g - S.off;
        const uint64_t a1 = in.k1[g], a2 = in.k2[g];
        const uint32_t ai = in.idx[g];
        int64_t dst = p;
        if (S.N > w) {
            const int64_t run = p / w;
            const int64_t sib = run ^ 1;
            const int64_t sib_lo = sib * w;
            if (sib_lo < S.N) {
                const int64_t sib_hi = (sib_lo + w < S.N) ? sib_lo + w : S.N;
                // number of sibling keys below a (keys distinct)
                int64_t lo = sib_lo, hi = sib_hi;
                while (lo < hi) {
                    int64_t mid = (lo + hi) >> 1;
                    const int64_t gm = S.off + mid;
                    if (key_less(in.k1[gm], in.k2[gm], in.idx[gm], a1, a2, ai))
                        lo = mid + 1;
                    else
                        hi = mid;
                }
                const int64_t pair_lo = (run < sib ? run : sib) * w;
                dst = pair_lo + (p - run * w) + (lo - sib_lo);
            }
        }
        if (!CSG_IN_BOUNDS(dst >= 0 && dst < S.N, 0x40, g)) continue;
        out.k1[S.off + dst] = a1;
        out.k2[S.off + dst] = a2;
        out.idx[S.off + dst] = ai;
    }
}

// coords_sorted[r][p] = tmp[r][idx[p]]
__global__ void gather_kernel(const SetRow *__restrict__ sets, const int64_t *__restrict__ starts,
                              int n, int64_t E, const double *__restrict__ tmp,
                              const uint32_t *__restrict__ idx) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < E;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int s = find_set(starts, n, g);
        const SetRow S = sets[s];
        const int64_t p = g - S.off;
        const int64_t src = S.off + idx[g];
        if (!CSG_IN_BOUNDS(idx[g] < (uint64_t)S.N && p < S.N, 0x41, g)) continue;
#pragma unroll
        for (int r = 0; r < 4; ++r) S.coords[r * S.N + p] = tmp[r * E + src];
    }
}

int grid_for(int64_t E, int threads) {
    int64_t b = (E + threads - 1) / threads;
    if (b > 152 * 64) b = 152 * 64;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

unsigned long long check_word_sprinkle() { return take_check_word(); }

SprinklePlan sprinkle_plan(const SprinkleSpec *specs, int n, Arena &a, bool from_coords,
                           size_t s_counters) {
    SprinklePlan p;
    p.n = n;
    p.from_coords = from_coords;
    p.s_counters = s_counters;
    std::vector<SetRow> rows(n);
    std::vector<int64_t> starts(n), cstarts(n);
    bool shared_err = false;
    for (int s = 0; s < n; ++s) {
        rows[s].d = specs[s].geom ? specs[s].geom : specs[s].d;
        rows[s].param = specs[s].param;
        rows[s].N = specs[s].N;
        rows[s].seed = specs[s].seed;
        rows[s].seq = specs[s].seq;
        rows[s].coords = specs[s].coords;
        rows[s].off = p.E;
        rows[s].chunk_off = p.C;
        rows[s].err = specs[s].err;
        if (!specs[s].err && s_counters == (size_t)-1) shared_err = true;
        starts[s] = p.E;
        cstarts[s] = p.C;
        p.E += specs[s].N;
        p.C += (specs[s].N + kChunk - 1) / kChunk;
        if (specs[s].N > p.maxN) p.maxN = specs[s].N;
    }
    p.t_rows = a.put(rows.data(), n * sizeof(SetRow));
    p.t_starts = a.put(starts.data(), n * sizeof(int64_t));
    p.t_cstarts = a.put(cstarts.data(), n * sizeof(int64_t));
    p.s_tmp = a.reserve(4 * p.E * sizeof(double));
    p.s_keys = a.reserve(4 * p.E * sizeof(uint64_t));
    p.s_idx = a.reserve(2 * p.E * sizeof(uint32_t));
    p.s_err = shared_err ? a.reserve(sizeof(unsigned long long)) : (size_t)-1;
    return p;
}

void sprinkle_patch(const SprinklePlan &p, Arena &a) {
    SetRow *rows = a.host<SetRow>(p.t_rows);
    for (int s = 0; s < p.n; ++s) {
        if (rows[s].err) continue;
        if (p.s_counters != (size_t)-1)
            rows[s].err = a.scr<unsigned long long>(p.s_counters) + (size_t)s * CNT_WORDS + CNT_ERR;
        else
            rows[s].err = a.scr<unsigned long long>(p.s_err);
    }
}

void sprinkle_launch(const SprinklePlan &p, const Arena &a, cudaStream_t st) {
    if (p.E == 0) return;
    const int64_t E = p.E;
    SetRow *d_rows = a.tab<SetRow>(p.t_rows);
    int64_t *d_starts = a.tab<int64_t>(p.t_starts);
    int64_t *d_cstarts = a.tab<int64_t>(p.t_cstarts);
    double *tmp = a.scr<double>(p.s_tmp);
    uint64_t *kb = a.scr<uint64_t>(p.s_keys);
    uint32_t *ib = a.scr<uint32_t>(p.s_idx);
    if (p.s_err != (size_t)-1) cudaMemsetAsync(a.scr<unsigned long long>(p.s_err), 0, sizeof(unsigned long long), st);
    Keys ka{kb, kb + E, ib}, kb2{kb + 2 * E, kb + 3 * E, ib + E};
    const int T = 256;
    stage_begin(CSG_STAGE_SPRINKLE, st);
    // runs of 32 .. 1024 elements per warp: long runs keep the lanes busy through the d=4
    // rejection draws, and about 4864 warps (32 per SM) keep the SMs busy
    int64_t run = (E / 4864 + 31) / 32 * 32;
    run = run < 32 ? 32 : (run > 1024 ? 1024 : run);
    const int64_t nwarp = (E + run - 1) / run;
    sprinkle_keys_kernel<<<(unsigned)((nwarp + T / 32 - 1) / (T / 32)), T, 0, st>>>(d_rows, d_starts, p.n, E, tmp,
                                                                                ka, p.from_coords ? 1 : 0, run);
    chunk_sort_kernel<<<(unsigned)p.C, kSortThreads, 0, st>>>(d_rows, d_cstarts, p.n, ka, kb2);
    Keys cur = kb2, nxt = ka;
    for (int64_t w = kChunk; w < p.maxN; w *= 2) {
        merge_pass_kernel<<<grid_for(E, T), T, 0, st>>>(d_rows, d_starts, p.n, E, w, cur, nxt);
        Keys t = cur;
        cur = nxt;
        nxt = t;
    }
    gather_kernel<<<grid_for(E, T), T, 0, st>>>(d_rows, d_starts, p.n, E, tmp, cur.idx);
    stage_end(CSG_STAGE_SPRINKLE, st);
}

int sprinkle_sort_batch(const SprinkleSpec *specs, int n, cudaStream_t st,
                        const double *const *host_coords, bool sync) {
    if (n <= 0) return CSG_OK;
    Arena a;
    SprinklePlan p = sprinkle_plan(specs, n, a, host_coords != nullptr);
    if (p.E == 0) return CSG_OK;
    int rc = arena_alloc(a, st);
    if (rc != CSG_OK) return rc;
    sprinkle_patch(p, a);
    arena_upload(a, st);
    if (host_coords) {
        const SetRow *rows = a.host<SetRow>(p.t_rows);
        double *tmp = a.scr<double>(p.s_tmp);
        for (int s = 0; s < n; ++s)
            for (int r = 0; r < 4; ++r)
                cudaMemcpyAsync(tmp + r * p.E + rows[s].off, host_coords[s] + r * rows[s].N,
                                rows[s].N * sizeof(double), cudaMemcpyHostToDevice, st);
    }
    sprinkle_launch(p, a, st);
    rc = CSG_OK;
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) {
        set_error("sprinkle/sort launch: %s", cudaGetErrorString(le));
        rc = CSG_E_CUDA;
    }
    // collect the rejection flags of sets that had no error slot of their own
    unsigned long long err_host = 0;
    if (rc == CSG_OK && p.s_err != (size_t)-1)
        cudaMemcpyAsync(&err_host, a.scr<unsigned long long>(p.s_err), sizeof err_host,
                        cudaMemcpyDeviceToHost, st);
    arena_free(a, st);
    if (!sync) return rc;  // stream-ordered; each set's own error word carries a rejection
    cudaError_t se = cudaStreamSynchronize(st);
    if (rc == CSG_OK && se != cudaSuccess) {
        set_error("sprinkle/sort: %s", cudaGetErrorString(se));
        rc = CSG_E_CUDA;
    }
    if (rc == CSG_OK && err_host != 0) {
        set_error("sprinkle: an element hit the 256-attempt rejection cap");
        rc = CSG_E_REJECT;
    }
    return rc;
}

}  // namespace csg
