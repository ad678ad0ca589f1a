// Interval abundances by AND + popcount of packed row words (Sec. 4.3, Alg. 5,
// restated for the GPU).
//
// For a related pair i < j of time-ordered elements, the elements strictly between
// them are the k with i < k < j set in both row i (future of i) and row j (past of
// j), so m(i,j) = popcount(row_i AND row_j) over bits i < k < j (Fig. 2).
//
// Work decomposition: a work item is a group of G consecutive rows I = [i0, i0+G)
// (G divides 64, so the group sits inside one 64-bit word of every row).  The CTA
// bulk-copies the group's rows, from the group's word to the end, into shared
// memory with TMA and clears every bit k <= i of row i, so each staged row holds
// only the future of its element.  Warps then sweep the later elements j in runs
// of 32: one load of word w0 of each row j gives the G-bit mask of group rows
// related to j, unrelated j are skipped at once (Alg. 5 skips unrelated pairs),
// and for every j with a nonempty mask the warp streams row j's words up to j
// (coalesced) and ANDs each with the staged row of every related i in the mask.
// One read of a word of row j thus serves all related rows of the group.
//
// The popcount pipe (16 results per SM per clock) bounds the AND + popcount loop, so each lane
// takes two word pairs per step and sends three of the four ANDed words through a full adder
// (their sum and majority words, counted once and twice): three 64-bit popcounts per four
// words instead of four (Sec. 3.3 cites Mula's table-driven popcount for the same purpose).
//
// The lanes' partial counts of a pair are summed with one warp reduction (redux); the
// pair's m goes into per-warp counters (N_0..N_3, R, sum m, W) flushed with 64-bit atomics,
// optionally into a full histogram in global memory and, for pairs with m <= 2, into
// the per-element sums of the discrete d'Alembertian (Eq. b_local).  Work items come from an
// atomic queue (persistent CTAs), in ascending i0, which is roughly longest first.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "arena.h"
#include "csg_internal.cuh"
#include "ptx.cuh"

namespace csg {
namespace {

constexpr int kWarps = 32;
constexpr int kThreads = kWarps * 32;
constexpr int kMaxK = 4;  // group rows per pass over row j (1024 threads leave 64 registers a thread)
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s for a bulk copy to land

struct Smem {
    uint64_t bar;
    int item;
    int stop;
    const double *phi;  // the current item's d'Alembertian field and sums (or null)
    double *acc;
};

// Per-warp totals of one work item.  Every lane holds the same R, M and W; lane k < 4
// holds N_k in nk (the lane whose index equals m counts the pair).
struct Counters {
    unsigned long long nk = 0, R = 0, M = 0, W = 0;
};

// The cnt <= K group rows related to j (the set bits of mask) against row j: each lane
// takes word pairs (2 lane, 2 lane + 1) + 64 t, so every load is 16 bytes, and the K
// staged rows are compile-time slots (no per-row branches in the loop); slots beyond
// cnt read the all-zero row at zoff.  K is 1, 2, 4 or 8, which keeps the code small
// enough for the instruction cache.  Lane 0 books the pairs' interval sizes after a
// warp reduction.
template <int K, bool PHI>
__device__ __forceinline__ void sweep_rows(uint32_t mask, int cnt, int zoff, const uint64_t *__restrict__ A,
                                           int pitch,
                                           const uint64_t *__restrict__ bj, int wj, uint64_t lastmask,
                                           int lane, int64_t j, int64_t i0, Counters &c,
                                           unsigned long long *__restrict__ hist, long long nbins,
                                           const Smem *ctl, int blim, int alim, int64_t N) {
    int off[K];
    uint32_t m = mask;
    int rsum = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int r = __ffs(m) - 1;
        m &= m - 1;
        off[k] = k < cnt ? r * pitch : zoff;
        rsum += k < cnt ? r : 0;
    }
    uint32_t acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0;
    // two word pairs per lane and step (w and w + 64): of the four ANDed words, three go
    // through a full adder (sum and majority words) and one is counted directly, so four words
    // cost three 64-bit popcounts instead of four
    int w = 2 * lane;
    const ulonglong2 z2 = make_ulonglong2(0ull, 0ull);
    for (; w + 65 < wj; w += 128) {  // all four words lie before row j's last word
        const ulonglong2 b0 = CSG_IN_BOUNDS(w + 65 < blim, 0x11, j) ? __ldg(reinterpret_cast<const ulonglong2 *>(bj + w)) : z2;
        const ulonglong2 b1 = CSG_IN_BOUNDS(w + 65 < blim, 0x11, j) ? __ldg(reinterpret_cast<const ulonglong2 *>(bj + w + 64)) : z2;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const bool ain = CSG_IN_BOUNDS(off[k] + w + 65 < alim, 0x12, off[k] + w);
            const ulonglong2 a0 = ain ? *reinterpret_cast<const ulonglong2 *>(A + off[k] + w) : z2;
            const ulonglong2 a1 = ain ? *reinterpret_cast<const ulonglong2 *>(A + off[k] + w + 64) : z2;
            const uint64_t x = a0.x & b0.x, y = a0.y & b0.y, z = a1.x & b1.x;
            const uint64_t sum = x ^ y ^ z, carry = (x & y) | (x & z) | (y & z);
            acc[k] += __popcll(sum) + 2 * __popcll(carry) + __popcll(a1.y & b1.y);
        }
    }
    for (; w <= wj; w += 64) {  // the rest, one pair per lane, the last word masked
        ulonglong2 b = CSG_IN_BOUNDS(w + 1 < blim, 0x11, j) ? __ldg(reinterpret_cast<const ulonglong2 *>(bj + w)) : z2;
        if (w + 1 >= wj) {
            if (w == wj) {
                b.x &= lastmask;
                b.y = 0;
            } else {
                b.y &= lastmask;
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const ulonglong2 a = CSG_IN_BOUNDS(off[k] + w + 1 < alim, 0x12, off[k] + w)
                                     ? *reinterpret_cast<const ulonglong2 *>(A + off[k] + w)
                                     : z2;
            acc[k] += __popcll(a.x & b.x) + __popcll(a.y & b.y);
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (k >= cnt) break;
        const uint32_t v = __reduce_add_sync(0xffffffffu, acc[k]);  // m of the pair, on every lane
        c.nk += (uint32_t)lane == v;
        c.M += v;
        if (hist != nullptr && lane == 0 && (long long)v < nbins) atomicAdd(&hist[v], 1ull);
        // Eq. b_local: i = i0 + r is in L_{v+1} of j, r the k-th set bit of mask
        if (PHI && lane == 0 && v < 3u) {
            double *acc_phi = ctl->acc;
            uint32_t mm = mask;  // k < cnt = popc(mask), so mm keeps a set bit
            for (int t = 0; t < k; ++t) mm &= mm - 1;
            const int r = __ffs(mm) - 1;
            if (CSG_IN_BOUNDS(j < N && i0 + r < N, 0x13, j))
                atomicAdd(&acc_phi[j], (v == 1u ? -2.0 : 1.0) * ctl->phi[i0 + r]);
        }
    }
    c.R += (unsigned long long)cnt;
    // sum over the cnt rows r of (j - (i0 + r) - 1)
    c.W += (unsigned long long)cnt * (unsigned long long)(j - i0 - 1) - (unsigned long long)rsum;
}

template <int G, bool PHI>
__device__ __forceinline__ void dispatch_rows(int cnt, uint32_t mask, const uint64_t *__restrict__ A,
                                              int pitch, const uint64_t *__restrict__ bj, int wj,
                                              uint64_t lastmask, int lane, int64_t j, int64_t i0,
                                              Counters &c, unsigned long long *__restrict__ hist,
                                              long long nbins, const Smem *ctl, int blim, int64_t N) {
    const int alim = (G + 1) * pitch;  // the staged rows and the zero row after them
    const int zoff = G * pitch;  // the zero row after the G staged rows
    if (cnt <= 1)
        sweep_rows<1, PHI>(mask, cnt, zoff, A, pitch, bj, wj, lastmask, lane, j, i0, c, hist, nbins, ctl, blim, alim, N);
    else if (cnt <= 2)
        sweep_rows<2, PHI>(mask, cnt, zoff, A, pitch, bj, wj, lastmask, lane, j, i0, c, hist, nbins, ctl, blim, alim, N);
    else if (cnt <= 4 || G <= 4 || kMaxK <= 4) {
        if constexpr (G >= 4)
            sweep_rows<4, PHI>(mask, cnt, zoff, A, pitch, bj, wj, lastmask, lane, j, i0, c, hist, nbins, ctl, blim, alim, N);
    } else {
        if constexpr (G >= 8 && kMaxK >= 8)
            sweep_rows<8, PHI>(mask, cnt, zoff, A, pitch, bj, wj, lastmask, lane, j, i0, c, hist, nbins, ctl, blim, alim, N);
    }
}

template <int G, bool PHI>
__global__ void __launch_bounds__(kThreads, 1)
action_popc_kernel(const SetDesc *__restrict__ sets, const WorkItem *__restrict__ items,
                   int n_items, int pitch, unsigned int *__restrict__ queue,
                   unsigned long long *__restrict__ hist, long long nbins, unsigned long long wait_ns,
                   int starve) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem *ctl = reinterpret_cast<Smem *>(smem_raw);
    uint64_t *A = reinterpret_cast<uint64_t *>(smem_raw + 128);  // G rows x pitch words, then a zero row

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&ctl->bar, 1);
        ptx::fence_mbar_init();
    }
    for (int w = threadIdx.x; w < pitch; w += blockDim.x) A[(size_t)G * pitch + w] = 0;  // zero row
    __syncthreads();

    uint32_t phase = 0;
    bool first = true;  // this CTA's first item (the one a failure-handling test starves)
    for (;;) {
        if (threadIdx.x == 0) ctl->item = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int k = ctl->item;
        if (k >= n_items) break;
        const WorkItem it = items[k];
        const SetDesc S = sets[it.set];
        const int64_t N = S.N, stride = S.stride, i0 = it.i0;
        const uint64_t *__restrict__ rows = S.rows;
        const int64_t w0 = i0 >> 6;
        const int64_t w0a = w0 & ~int64_t(1);
        const int64_t wN = (N + 63) >> 6;
        const int nwa = (int)(((wN - w0a) + 1) & ~int64_t(1));
        // rows of the group that are counted
        uint32_t gmask = 0;
#pragma unroll
        for (int r = 0; r < G; ++r) {
            const int64_t i = i0 + r;
            if (i < N && i >= S.row_lo && i < S.row_hi) gmask |= 1u << r;
        }
        if (gmask == 0) {
            __syncthreads();
            continue;
        }

        // ---- stage the group's rows with bulk copies (a failure-handling test starves the
        // first item: its barrier then gets no arrival and nothing is in flight)
        if (threadIdx.x == 0) {
            if (PHI) {
                ctl->phi = S.phi;
                ctl->acc = S.acc;
            }
            if (!(starve && first)) {
                ptx::fence_proxy_async_smem();
                const uint32_t bytes = (uint32_t)nwa * 8u;
                ptx::mbar_arrive_expect_tx(&ctl->bar, bytes * (uint32_t)__popc(gmask));
                for (int r = 0; r < G; ++r)
                    if ((gmask >> r & 1u) &&
                        CSG_IN_BOUNDS(nwa <= pitch && i0 + r < N && w0a + nwa <= stride, 0x10, i0 + r))
                        ptx::bulk_g2s(A + (size_t)r * pitch, rows + (i0 + r) * stride + w0a, bytes,
                                      &ctl->bar);
            }
        }
        first = false;
        const bool landed = ptx::mbar_wait_bounded(&ctl->bar, phase, wait_ns);
        if (__syncthreads_or(!landed)) {
            // a copy did not land in time: record it, keep the CTA alive until the
            // copy lands (bounded again), then stop
            if (threadIdx.x == 0) {
                atomicExch(&S.counters[CNT_ERR], 1ull);
                ptx::mbar_wait_bounded(&ctl->bar, phase, wait_ns);
            }
            __syncthreads();
            break;
        }
        phase ^= 1u;
        // keep only the future of each row: clear bits k <= i
        const int lead = (int)(w0 - w0a);  // 0 or 1 words before the group's word
        if (threadIdx.x < G && (gmask >> threadIdx.x & 1u)) {
            const int r = threadIdx.x;
            const int b = (int)((i0 + r) & 63);
            uint64_t *a = A + (size_t)r * pitch;
            if (lead) a[0] = 0;
            a[lead] &= ~((2ull << b) - 1ull);  // b == 63 clears the whole word
        }
        __syncthreads();

        // ---- sweep later elements j in runs of 32 per warp
        Counters cnt;
        const int gshift = (int)(i0 & 63);
        const uint32_t Gbits = (G == 32) ? 0xffffffffu : ((1u << G) - 1u);
        for (int64_t jb = i0 + 1 + 32 * (int64_t)warp; jb < N; jb += 32 * kWarps) {
            const int64_t jl = jb + lane;
            uint32_t my = 0;
            if (jl < N) {
                const uint64_t word = CSG_IN_BOUNDS(w0 < stride, 0x14, jl) ? __ldg(rows + jl * stride + w0) : 0ull;
                my = (uint32_t)(word >> gshift) & Gbits & gmask;
                const int64_t off = jl - i0;  // elements of the group after j do not precede it
                if (off < G) my &= (1u << off) - 1u;
            }
            uint32_t todo = __ballot_sync(0xffffffffu, my != 0);
            while (todo) {
                const int src = __ffs(todo) - 1;
                todo &= todo - 1;
                const uint32_t mask = __shfl_sync(0xffffffffu, my, src);
                const int64_t j = jb + src;
                const int wj = (int)((j >> 6) - w0a);                 // last word, relative
                const uint64_t lastmask = (1ull << (j & 63)) - 1ull;  // bits k < j
                const uint64_t *__restrict__ bj = rows + j * stride + w0a;
                const int blim = (int)(stride - w0a);  // words of row j from w0a on
                // at most kMaxK rows per pass keeps the row slots and sums in registers
                uint32_t rest = mask;
                while (rest) {
                    uint32_t part = rest;
                    if (__popc(rest) > kMaxK) {
                        uint32_t t = rest;
#pragma unroll
                        for (int k = 0; k < kMaxK; ++k) t &= t - 1;
                        part = rest & ~t;  // the lowest kMaxK rows
                    }
                    rest &= ~part;
                    dispatch_rows<G, PHI>(__popc(part), part, A, pitch, bj, wj, lastmask, lane, j, i0, cnt, hist, nbins,
                                          ctl, blim, N);
                }
            }
        }
        if (cnt.R != 0) {
            unsigned long long *g = S.counters;
            if (lane < 4 && cnt.nk) atomicAdd(&g[CNT_N0 + lane], cnt.nk);
            if (lane == 0) {
                atomicAdd(&g[CNT_R], cnt.R);
                atomicAdd(&g[CNT_SUM_M], cnt.M);
                atomicAdd(&g[CNT_W], cnt.W);
            }
        }
        __syncthreads();  // the staged rows are reused by the next item
    }
}

template <int G, bool PHI>
int launch_g(const PopcPlan &p, const Arena &a, cudaStream_t st) {
    const size_t smem = 128 + (size_t)(G + 1) * p.pitch * sizeof(uint64_t);
    auto kern = action_popc_kernel<G, PHI>;
    CSG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0, per_sm = 0;
    CSG_CUDA_TRY(cudaGetDevice(&dev));
    CSG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CSG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    if (per_sm < 1) {
        set_error("action_popc: %zu bytes of shared memory per CTA do not fit", smem);
        return CSG_E_INVAL;
    }
    int grid = sms * per_sm;
    if (grid > p.n_items) grid = p.n_items;
    unsigned int *queue = a.scr<unsigned int>(p.s_queue);
    CSG_CUDA_TRY(cudaMemsetAsync(queue, 0, sizeof(unsigned int), st));
    stage_begin(CSG_STAGE_ACTION, st);
    kern<<<grid, kThreads, smem, st>>>(a.tab<SetDesc>(p.t_sets), a.tab<WorkItem>(p.t_items), p.n_items,
                                       p.pitch, queue, p.hist, (long long)p.nbins, wait_limit_ns(kWaitLimitNs),
                                       starve_first_stage());
    stage_end(CSG_STAGE_ACTION, st);
    CSG_CUDA_TRY(cudaGetLastError());
    return CSG_OK;
}

}  // namespace

unsigned long long check_word_popc() { return take_check_word(); }

// Shared-memory budget for the staged rows of one CTA.
static constexpr size_t kRowBudget = 200 * 1024;

PopcPlan popc_plan(const SetDesc *sets, int n, Arena &a, size_t s_counters, unsigned long long *hist,
                   int64_t nbins, int *rc, const int *slots) {
    PopcPlan p;
    *rc = CSG_OK;
    if (slots) p.slot.assign(slots, slots + n);
    p.n_sets = n;
    p.s_counters = s_counters;
    p.hist = hist;
    p.nbins = nbins;
    for (int s = 0; s < n; ++s) p.phi = p.phi || sets[s].acc != nullptr;
    int64_t maxw = 0;
    for (int s = 0; s < n; ++s) maxw = std::max<int64_t>(maxw, (sets[s].N + 63) / 64 + 2);
    p.pitch = (int)((maxw + 1) & ~int64_t(1));
    int G = 16;
    while (G > 1 && (size_t)(G + 1) * p.pitch * 8 > kRowBudget) G >>= 1;
    if ((size_t)(G + 1) * p.pitch * 8 > kRowBudget) {
        set_error("action_popc: rows of %lld words do not fit shared memory", (long long)maxw);
        *rc = CSG_E_INVAL;
        return p;
    }
    p.G = G;
    // work items: groups of G rows over each set's row range
    std::vector<WorkItem> items;
    for (int s = 0; s < n; ++s) {
        int64_t lo = std::max<int64_t>(0, sets[s].row_lo), hi = std::min<int64_t>(sets[s].N, sets[s].row_hi);
        for (int64_t i0 = lo / G * G; i0 < hi; i0 += G) items.push_back(WorkItem{s, 0, i0});
    }
    if (items.size() > 0x7fffffff) {
        set_error("action_popc: too many work items");
        *rc = CSG_E_INVAL;
        return p;
    }
    // longest first: an item's work grows with the number of later rows
    std::stable_sort(items.begin(), items.end(), [&](const WorkItem &x, const WorkItem &y) {
        const int64_t rx = sets[x.set].N - x.i0, ry = sets[y.set].N - y.i0;
        return rx * sets[x.set].N > ry * sets[y.set].N;
    });
    p.n_items = (int)items.size();
    p.t_sets = a.put(sets, n * sizeof(SetDesc));
    p.t_items = a.put(items.data(), items.size() * sizeof(WorkItem));
    p.s_queue = a.reserve(sizeof(unsigned int));
    return p;
}

void popc_patch(const PopcPlan &p, Arena &a) {
    SetDesc *d = a.host<SetDesc>(p.t_sets);
    for (int s = 0; s < p.n_sets; ++s)
        d[s].counters = a.scr<unsigned long long>(p.s_counters) +
                        (size_t)(p.slot.empty() ? s : p.slot[s]) * CNT_WORDS;
}

int popc_launch(const PopcPlan &p, const Arena &a, cudaStream_t st) {
    if (p.n_items == 0) return CSG_OK;
    if (p.phi) {
        switch (p.G) {
            case 16: return launch_g<16, true>(p, a, st);
            case 8: return launch_g<8, true>(p, a, st);
            case 4: return launch_g<4, true>(p, a, st);
            case 2: return launch_g<2, true>(p, a, st);
            default: return launch_g<1, true>(p, a, st);
        }
    }
    switch (p.G) {
        case 16: return launch_g<16, false>(p, a, st);
        case 8: return launch_g<8, false>(p, a, st);
        case 4: return launch_g<4, false>(p, a, st);
        case 2: return launch_g<2, false>(p, a, st);
        default: return launch_g<1, false>(p, a, st);
    }
}

}  // namespace csg
