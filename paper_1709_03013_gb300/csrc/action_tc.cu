// Interval counts as a masked 0/1 matrix product on the tcgen05 tensor cores.
//
// With elements in time order, the interval size of a related pair i < j is
//   m(i,j) = sum_k U[i][k] * P[j][k],   U[i][k] = S[i][k] [k > i],  P[j][k] = S[j][k] [k < j]
// where S is the symmetric causal matrix: U holds each element's future, P its past
// (Fig. 2: the inner product of rows i and j between columns i and j).  X = U P^T is
// a dense contraction, so it runs on the tensor cores; only the entries with
// S[i][j] = 1, i < j, are histogrammed (Alg. 5 counts related pairs only).
//
// Exactness: the operands are 0 and 1, either in fp8 e4m3 (0x00, 0x38; kind::f8f6f4) or
// in packed fp4 e2m1 (nibbles 0x0, 0x2; kind::mxf4 with every block scale factor 1.0);
// products are exact and the fp32 accumulator holds integers up to 2^24 exactly, far
// above the largest interval (N - 2 <= 2^18).  The result is converted back to an
// integer before it is used, so the counts are bit-exact in either format.
//
// Pass 1 (expand): one warp per operand row (per group of four consecutive rows in a batch
// of many sets), one lane per packed word, writes the operand bytes of U and of P the word
// covers (64 fp8 bytes or 32 fp4 bytes each); only the column ranges the product reads are
// written.
// Pass 2 (product): persistent CTA pairs (clusters of two CTAs, one per SM) take pair tiles
// (256 rows i x 256 columns j, upper triangle only, K from the first row of the tile to its
// last column) from a global work queue: the leader CTA claims each tile with an atomic
// counter over a tile list ordered set by set, longest first, block-rasterised (one step ahead
// of the tile it is loading), and mails the tile itself (set, row and column tile, K range) to
// the other CTA; claiming in list order keeps the tiles running at once on the same set's
// operands, which then stay in L2.  The pair runs 2-SM MMAs (cta_group::2): each CTA
// stages its own 128 rows of U and 128 of the tile's 256 rows of P, the leader issues the
// MMAs, and each CTA's TMEM receives the accumulator of its own 128 rows, so each SM loads
// 32 KB per stage instead of the 48 KB a one-SM 128 x 256 tile needs.
// Warp roles per CTA:
//   warp 0     the tile queue (leader) or its mailbox (other CTA), handed to warps 1-9
//              through a 4-slot shared-memory ring together with the tile's relation words
//              for this CTA's 128 rows (staged by TMA into the slot); TMA producer:
//              128-byte-swizzled K stages of 128 rows of U and 128 rows of P (16 KB each)
//              into a 6-stage ring whose transaction bytes are counted on the leader's barrier
//   warp 1     allocates 512 TMEM columns together with the other CTA; in the leader one
//              lane issues the MMAs (M=256, N=256, 32 bytes of K each: 32 fp8 or 64 fp4
//              elements) and commits each stage back to both producers and each finished
//              tile to both epilogues
//   warps 2-9  epilogue: tcgen05.ld of the CTA's 128 rows from TMEM (each thread owns one
//              row and half of the columns); the S bits of the row (from the ring slot) select
//              the related pairs, whose counts update the counters, the optional full
//              histogram and the optional d'Alembertian sums (Eq. b_local).  The fp8 form keeps two accumulators (columns 0
//              and 256) so the epilogue of one tile overlaps the product of the next; the
//              fp4 form keeps one accumulator at column 0 and its scale factors in columns
//              256..511, and releases the accumulator as soon as the last columns are in
//              registers.  Both CTAs' epilogues release an accumulator to the leader.
// Every wait is bounded (globaltimer); on expiry the kernel records an error in the
// set's counters and winds down instead of spinning.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "arena.h"
#include "csg_internal.cuh"
#include "ptx.cuh"

namespace csg {
namespace {

constexpr int BM = 128;          // rows i per CTA; a pair tile of the two CTAs of a cluster has 2 * BM
constexpr int BN = 256;          // columns j per tile
constexpr int BKB = 128;         // bytes of each operand row per stage (one 128-byte swizzle row)
constexpr int STAGES = 6;
constexpr int A_BYTES = BM * BKB;        // this CTA's 128 rows of U
constexpr int B_BYTES = (BN / 2) * BKB;  // this CTA's 128 of the tile's 256 rows of P
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int EPI_WARPS = 8;  // two per TMEM lane quarter, one for each half of the tile's columns
constexpr int THREADS = (2 + EPI_WARPS) * 32;
constexpr uint32_t TMEM_COLS = 2 * BN;
constexpr uint64_t kWaitNs = 4000000000ull;
constexpr uint8_t kOne = 0x38;   // 1.0 in fp8 e4m3

struct __align__(16) TcTile {
    int32_t set;     // index into the launch's set table (-1: no more tiles)
    int32_t ti, tj;  // rows [BM ti, BM ti + BM), columns [BN tj, BN tj + BN)
    int32_t kk;      // K stages [kk & 0xFFFF, kk >> 16): the tile's first row to its last column
};

struct TcArgs {
    const TcSetDesc *sets;
    const CUtensorMap *maps;  // 3 per set: U, P, relation bits (global memory, 128-byte aligned)
    const TcTile *tiles;
    int n_tiles;
    unsigned int *queue;       // tile counter (zeroed before the launch)
    unsigned long long *hist;  // optional full histogram (single-set launches)
    long long nbins;
    unsigned long long wait_ns;  // limit of every bounded wait (kWaitNs unless a test shortens it)
    int starve;                  // test only: the producers skip the loads of their first stage
};

constexpr int RING = 4;  // tiles handed from the producer to the MMA and epilogue warps
// Per ring slot, the tile's relation words for this CTA's 128 rows (4 words of 64 columns
// each), staged by TMA so the epilogue reads them from shared memory.
constexpr int BITS_BYTES = BM * (BN / 64) * 8;

// ------------------------------------------------------------------ expand

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

// Four relation bits -> four fp8 bytes (0x00 or 0x38): multiplying by 1 + 2^7 + 2^14 +
// 2^21 places bit b of the nibble at bit 8b, the mask keeps exactly those, and the
// second multiply turns each 0/1 byte into 0x00/0x38 (no carries between bytes).
__device__ __forceinline__ uint32_t nibble_fp8(uint32_t nib) {
    return ((nib * 0x00204081u) & 0x01010101u) * (uint32_t)kOne;
}

// Eight relation bits -> four bytes of packed fp4 e2m1 (1.0 = 0x2): byte k holds elements
// 2k (low nibble) and 2k+1 (high nibble).  Each multiply moves the even (odd) bits to bit
// 8k+1 (8k+5) of byte k; the other partial products land on bits the mask drops.
__device__ __forceinline__ uint32_t octet_fp4(uint32_t o) {
    return (((o & 0x55u) * 0x00082082u) & 0x02020202u) | (((o & 0xAAu) * 0x00410410u) & 0x20202020u);
}

__device__ __forceinline__ void put64_fp4(uint8_t *dst, uint64_t m) {
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    const uint32_t lo = (uint32_t)m, hi = (uint32_t)(m >> 32);
    d4[0] = make_uint4(octet_fp4(lo & 0xFFu), octet_fp4((lo >> 8) & 0xFFu), octet_fp4((lo >> 16) & 0xFFu),
                       octet_fp4(lo >> 24));
    d4[1] = make_uint4(octet_fp4(hi & 0xFFu), octet_fp4((hi >> 8) & 0xFFu), octet_fp4((hi >> 16) & 0xFFu),
                       octet_fp4(hi >> 24));
}

__device__ __forceinline__ void put64(uint8_t *dst, uint64_t m) {
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    const uint32_t lo = (uint32_t)m, hi = (uint32_t)(m >> 32);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t h = q < 2 ? lo >> (16 * q) : hi >> (16 * (q - 2));
        d4[q] = make_uint4(nibble_fp8(h & 0xFu), nibble_fp8((h >> 4) & 0xFu), nibble_fp8((h >> 8) & 0xFu),
                           nibble_fp8((h >> 12) & 0xFu));
    }
}

// Warps take groups of `group` consecutive operand rows of the sets [set_lo, set_lo + nset)
// (rows numbered across the sets, rstarts[s] = first row of set s; a set lookup per group,
// then a step forward at set boundaries; groups of four pay off for batches of many sets):
// the lanes walk the row's words and write the
// operand bytes (64 fp8 bytes or 32 packed fp4 bytes per word) where the product reads them:
// U row i from the first column of its pair tile, 2*BM*floor(i/(2*BM)) (a whole number of
// stages in either format), P row i up to column BN*(floor(i/BN)+1).
// FMT 0: fp8 e4m3, 128 elements per stage; FMT 1: fp4 e2m1, 256.
template <int FMT>
__global__ void expand_kernel(const TcSetDesc *__restrict__ sets, const int64_t *__restrict__ rstarts,
                              int set_lo, int nset, int64_t total_rows, int group) {
    const int lane = threadIdx.x & 31;
    const int64_t step = (int64_t)gridDim.x * (blockDim.x >> 5) * group;
    for (int64_t g0 = (blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5)) * group; g0 < total_rows;
         g0 += step) {
        int ls = find_set(rstarts, nset, g0);  // warp-uniform
        const int64_t g1 = min(g0 + group, total_rows);
        for (int64_t gr = g0; gr < g1; ++gr) {
            while (ls + 1 < nset && rstarts[ls + 1] <= gr) ++ls;  // sets without rows are stepped over
            const TcSetDesc &S = sets[set_lo + ls];
            const int64_t i = gr - rstarts[ls];
            const int64_t wpr = (FMT ? 2 * S.kp : S.kp) / 64;  // words per operand row
            const uint64_t *__restrict__ row = S.rows + i * S.stride;
            uint8_t *__restrict__ urow = S.U + i * S.kp;
            uint8_t *__restrict__ prow = S.P + i * S.kp;
            const int64_t u0 = (i / (2 * BM)) * (2 * BM) / 64;                  // first U word read
            const int64_t p1 = min(wpr, (i / BN + 1) * BN / 64);                // P words read: [0, p1)
            for (int64_t w = u0 + lane; w < wpr; w += 32) {
                const int64_t k0 = w * 64;
                uint64_t m = CSG_IN_BOUNDS(w < S.stride, 0x20, w) ? __ldg(row + w) : 0ull;
                if (k0 + 63 <= i)
                    m = 0;
                else if (k0 <= i)
                    m &= ~((2ull << (i - k0)) - 1ull);  // keep k > i
                if (!CSG_IN_BOUNDS(i < S.N && (FMT ? k0 / 2 + 32 : k0 + 64) <= S.kp, 0x21, w)) continue;
                if (FMT)
                    put64_fp4(urow + k0 / 2, m);
                else
                    put64(urow + k0, m);
            }
            for (int64_t w = lane; w < p1; w += 32) {
                const int64_t k0 = w * 64;
                uint64_t m = CSG_IN_BOUNDS(w < S.stride, 0x20, w) ? __ldg(row + w) : 0ull;
                if (k0 >= i)
                    m = 0;
                else if (k0 + 63 >= i)
                    m &= (1ull << (i - k0)) - 1ull;  // keep k < i
                if (!CSG_IN_BOUNDS(i < S.N && (FMT ? k0 / 2 + 32 : k0 + 64) <= S.kp, 0x21, w)) continue;
                if (FMT)
                    put64_fp4(prow + k0 / 2, m);
                else
                    put64(prow + k0, m);
            }
        }
    }
}

// ------------------------------------------------------------------ product

__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);   // start address
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused, K-major SW128)
    d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                     // descriptor version
    d |= (uint64_t)2 << 61;                     // 128-byte swizzle
    return d;
}

// kind::f8f6f4, A = B = e4m3, D = f32, K-major A and B, M = 256 (two CTAs), N = 256
constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)((2 * BM) >> 4) << 24);
// kind::mxf4 with block scaling: A = B = e2m1 (1), scale factors ue8m0 (bit 23), scale
// factor ids 0, D = f32, K-major A and B, M = 256 (two CTAs), N = 256
constexpr uint32_t kIdescF4 = (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | (1u << 23) |
                              ((uint32_t)((2 * BM) >> 4) << 24);
// TMEM columns of the fp4 form: accumulator 0..255, scale factors of A at 256 and of B at
// 384 (every scale factor is 1.0, so columns 256..511 are filled with the byte 0x7F)
constexpr uint32_t kSfA = 256, kSfB = 384;

// TMA tile load into this CTA's shared memory whose bytes are counted on the pair's
// barrier `bar` (a shared::cluster address: the leader CTA's barrier)
__device__ __forceinline__ void tma_load_2d_pair(void *dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cta.global.tile.mbarrier::complete_tx::bytes.cta_group::2"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(ptx::smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// TMA tile load into this CTA's shared memory completing on this CTA's barrier `bar`.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(ptx::smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(ptx::smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// shared::cluster address of this CTA's shared variable at `p` as seen in CTA `rank`
__device__ __forceinline__ uint32_t cluster_addr(const void *p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(ptx::smem_addr(p)), "r"(rank));
    return r;
}

// All threads of both CTAs of the cluster (release / acquire at cluster scope).
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Bounded wait with cluster-scope acquire (the barriers of this kernel are completed by
// the other CTA of the pair as well).
__device__ __forceinline__ bool mbar_wait_cl(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    auto try_wait = [&]() {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(ptx::smem_addr(bar)), "r"(parity)
            : "memory");
        return ok != 0;
    };
    if (try_wait()) return true;
    const uint64_t t0 = ptx::globaltimer_ns();
    while (!try_wait()) {
        if (ptx::globaltimer_ns() - t0 > limit_ns) return false;
    }
    return true;
}

// One MMA of the CTA pair (issued by the leader): A rows 0..127 from the leader's shared
// memory and 128..255 from the other CTA's, B rows split the same way, D into both TMEMs.
__device__ __forceinline__ void mma_f8(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_f4(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t sfa, uint32_t sfb,
                                       uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %6, 0;\n"
        "tcgen05.mma.cta_group::2.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], p;\n}\n" ::"r"(
            dtmem),
        "l"(ad), "l"(bd), "r"(kIdescF4), "r"(sfa), "r"(sfb), "r"(acc)
        : "memory");
}

// Arrive on the barrier at the same offset in both CTAs of the pair once the leader's
// issued MMAs have completed.
__device__ __forceinline__ void mma_commit_pair(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            ptx::smem_addr(bar)),
        "h"((uint16_t)0x3)
        : "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(ptx::smem_addr(bar)) : "memory");
}

#define TMEM_LD16(addr, v)                                                                          \
    asm volatile(                                                                                   \
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];" \
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),       \
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), \
          "=r"(v[14]), "=r"(v[15])                                                                  \
        : "r"(addr))

#define TMEM_LD32(addr, v)                                                                          \
    asm volatile(                                                                                   \
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17," \
        "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                        \
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),       \
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), \
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),            \
          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),            \
          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])             \
        : "r"(addr))

// The value of the 16-column chunk at runtime column u (0..15), by a select tree: registers
// cannot be indexed at run time without going through local memory.
__device__ __forceinline__ uint32_t pick16(const uint32_t (&v)[16], int u) {
    const bool s1 = u & 1, s2 = u & 2, s4 = u & 4, s8 = u & 8;
    const uint32_t a0 = s1 ? v[1] : v[0], a1 = s1 ? v[3] : v[2], a2 = s1 ? v[5] : v[4], a3 = s1 ? v[7] : v[6];
    const uint32_t a4 = s1 ? v[9] : v[8], a5 = s1 ? v[11] : v[10], a6 = s1 ? v[13] : v[12], a7 = s1 ? v[15] : v[14];
    const uint32_t b0 = s2 ? a1 : a0, b1 = s2 ? a3 : a2, b2 = s2 ? a5 : a4, b3 = s2 ? a7 : a6;
    const uint32_t c0 = s4 ? b1 : b0, c1 = s4 ? b3 : b2;
    return s8 ? c1 : c0;
}

// Books the pair (i, jbase + u) whose accumulator value (an exact integer in fp32) is x.
template <bool PHI>
__device__ __forceinline__ void book1(uint32_t x, int64_t j, unsigned long long &packed, unsigned long long &cM,
                                      unsigned long long *__restrict__ hist, long long nbins, double phi_i,
                                      double *__restrict__ acc_phi) {
    const uint32_t m = __float2uint_rn(__uint_as_float(x));
    cM += m;
    if (m < 4u) packed += 1ull << (16u * m);
    if (hist != nullptr && (long long)m < nbins) atomicAdd(&hist[m], 1ull);
    if (PHI && m < 3u) atomicAdd(&acc_phi[j], (m == 1u ? -2.0 : 1.0) * phi_i);
}

// Books the pairs (i, j) of one 16-column chunk whose relation bits are set in `bits`
// (column u of the chunk is element jbase + u).  Without a full histogram the sum of m over
// the chunk is taken in fp32 (exact: at most 16 integers below 2^18) and only the pairs with
// m < 4, found by a compare on the fp32 value, go through the counters one by one; with a
// histogram every pair does.  PHI adds, for pairs with m <= 2, c_m phi[i] to the
// d'Alembertian sums of element j (Eq. b_local).
template <bool PHI>
__device__ __forceinline__ void book16(const uint32_t (&v)[16], uint32_t bits, int64_t jbase, int64_t i,
                                       unsigned long long &packed, unsigned long long &cR,
                                       unsigned long long &cM, unsigned long long &cW,
                                       unsigned long long *__restrict__ hist, long long nbins, double phi_i,
                                       double *__restrict__ acc_phi) {
    if (!__any_sync(0xffffffffu, bits != 0u)) return;
    // R and W of the chunk from bit counts: sum over set bits u of (jbase + u - i - 1)
    const unsigned pc = __popc(bits);
    const unsigned su = __popc(bits & 0xAAAAu) + 2u * __popc(bits & 0xCCCCu) + 4u * __popc(bits & 0xF0F0u) +
                        8u * __popc(bits & 0xFF00u);
    cR += pc;
    cW += (unsigned long long)pc * (unsigned long long)(jbase - i - 1) + su;
    if (hist != nullptr) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
            if (bits >> u & 1u) book1<PHI>(v[u], jbase + u, packed, cM, hist, nbins, phi_i, acc_phi);
        return;
    }
    float sum = 0.f;
    uint32_t small = 0;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        if (bits >> u & 1u) {
            const float x = __uint_as_float(v[u]);
            sum += x;
            if (x < 4.0f) small |= 1u << u;
        }
    }
    cM += (unsigned long long)__float2uint_rn(sum);
    while (small) {
        const int u = __ffs(small) - 1;
        small &= small - 1;
        const uint32_t m = __float2uint_rn(__uint_as_float(pick16(v, u)));
        packed += 1ull << (16u * m);
        if (PHI && m < 3u) atomicAdd(&acc_phi[jbase + u], (m == 1u ? -2.0 : 1.0) * phi_i);
    }
}

// Epilogue of one tile for the thread owning row i and columns [cb, ce) of it (half the
// tile: two warps share each TMEM lane quarter): reads the accumulator 64 columns at a
// time (four loads, one wait, so the TMEM latency is paid four times per tile instead of
// sixteen) and books the pairs (i, j) whose relation bit is set in w4.  The accumulator is
// released (an arrival on the leader CTA's barrier `release`, a shared::cluster address)
// as soon as its last columns are in registers, before they are booked.  PHI is a template argument so the plain epilogue carries none of the
// d'Alembertian code.
template <bool PHI>
__device__ __forceinline__ unsigned long long epi_tile(uint32_t tbase, const uint64_t (&w4)[4], int64_t i,
                                                       int64_t J0, unsigned long long &cR,
                                                       unsigned long long &cM, unsigned long long &cW,
                                                       unsigned long long *__restrict__ hist, long long nbins,
                                                       double phi_i, double *__restrict__ acc_phi,
                                                       uint32_t release, int cb, int ce) {
    unsigned long long packed = 0;  // N0..N3 of this thread's columns [cb, ce), 16 bits each
#pragma unroll 1
    for (int c = cb; c < ce; c += 64) {
        uint32_t v0[16], v1[16], v2[16], v3[16];
        TMEM_LD16(tbase + (uint32_t)c, v0);
        TMEM_LD16(tbase + (uint32_t)c + 16u, v1);
        TMEM_LD16(tbase + (uint32_t)c + 32u, v2);
        TMEM_LD16(tbase + (uint32_t)c + 48u, v3);
        const uint64_t w = c < 64 ? w4[0] : (c < 128 ? w4[1] : (c < 192 ? w4[2] : w4[3]));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (c + 64 == ce) {
            // the warp's reads of the accumulator are done: one arrival of 32 on the leader's barrier
            tc_fence_before();
            __syncwarp();
            if ((threadIdx.x & 31) == 0) mbar_arrive_cluster(release, 32);
        }
        book16<PHI>(v0, (uint32_t)w & 0xFFFFu, J0 + c, i, packed, cR, cM, cW, hist, nbins, phi_i, acc_phi);
        book16<PHI>(v1, (uint32_t)(w >> 16) & 0xFFFFu, J0 + c + 16, i, packed, cR, cM, cW, hist, nbins, phi_i,
                    acc_phi);
        book16<PHI>(v2, (uint32_t)(w >> 32) & 0xFFFFu, J0 + c + 32, i, packed, cR, cM, cW, hist, nbins, phi_i,
                    acc_phi);
        book16<PHI>(v3, (uint32_t)(w >> 48), J0 + c + 48, i, packed, cR, cM, cW, hist, nbins, phi_i, acc_phi);
    }
    return packed;
}

// The fp4 form's epilogue (one accumulator, so its drain is on the critical path): all 128
// columns of this thread's half row come into registers with eight loads and one wait, the
// accumulator is released at once, and the pairs are booked from registers afterwards.
template <bool PHI>
__device__ __forceinline__ unsigned long long epi_tile_all(uint32_t tbase, const uint64_t (&w4)[4], int64_t i,
                                                           int64_t J0, unsigned long long &cR,
                                                           unsigned long long &cM, unsigned long long &cW,
                                                           unsigned long long *__restrict__ hist, long long nbins,
                                                           double phi_i, double *__restrict__ acc_phi,
                                                           uint32_t release, int cb) {
    uint32_t v0[16], v1[16], v2[16], v3[16], v4[16], v5[16], v6[16], v7[16];
    const uint32_t t = tbase + (uint32_t)cb;
    TMEM_LD16(t, v0);
    TMEM_LD16(t + 16u, v1);
    TMEM_LD16(t + 32u, v2);
    TMEM_LD16(t + 48u, v3);
    TMEM_LD16(t + 64u, v4);
    TMEM_LD16(t + 80u, v5);
    TMEM_LD16(t + 96u, v6);
    TMEM_LD16(t + 112u, v7);
    const uint64_t wl = cb == 0 ? w4[0] : w4[2], wh = cb == 0 ? w4[1] : w4[3];
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    tc_fence_before();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive_cluster(release, 32);
    unsigned long long packed = 0;
    const int64_t j0 = J0 + cb;
    book16<PHI>(v0, (uint32_t)wl & 0xFFFFu, j0, i, packed, cR, cM, cW, hist, nbins, phi_i, acc_phi);
    book16<PHI>(v1, (uint32_t)(wl >> 16) & 0xFFFFu, j0 + 16, i, packed, cR, cM, cW, hist, nbins, phi_i, acc_phi);
    book16<PHI>(v2, (uint32_t)(wl >> 32) & 0xFFFFu, j0 + 32, i, packed, cR, cM, cW, hist, nbins, phi_i, acc_phi);
    book16<PHI>(v3, (uint32_t)(wl >> 48), j0 + 48, i, packed, cR, cM, cW, hist, nbins, phi_i, acc_phi);
    book16<PHI>(v4, (uint32_t)wh & 0xFFFFu, j0 + 64, i, packed, cR, cM, cW, hist, nbins, phi_i, acc_phi);
    book16<PHI>(v5, (uint32_t)(wh >> 16) & 0xFFFFu, j0 + 80, i, packed, cR, cM, cW, hist, nbins, phi_i, acc_phi);
    book16<PHI>(v6, (uint32_t)(wh >> 32) & 0xFFFFu, j0 + 96, i, packed, cR, cM, cW, hist, nbins, phi_i, acc_phi);
    book16<PHI>(v7, (uint32_t)(wh >> 48), j0 + 112, i, packed, cR, cM, cW, hist, nbins, phi_i, acc_phi);
    return packed;
}

// K stages of a tile: from the tile's first row to its last column (or N), in stages of
// 256 fp4 or 128 fp8 elements (at most 2^11 stages for N <= 2^18, so both fit 16 bits)
inline int32_t k_range_packed(int ti, int tj, int64_t N, int fmt) {
    const int64_t KSTAGE = fmt ? 256 : 128;
    const int64_t I0 = (int64_t)ti * BM;
    const int64_t J1 = std::min<int64_t>((int64_t)(tj + 1) * BN, N);
    const int64_t kt0 = I0 / KSTAGE, kt1 = (J1 + KSTAGE - 1) / KSTAGE;
    return (int32_t)(kt0 | (kt1 << 16));
}

template <int FMT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(THREADS, 1)
action_tc_kernel(const TcArgs args) {
    constexpr uint32_t NACC = FMT ? 1u : 2u;  // TMEM accumulators (the fp4 form keeps its scale factors in the rest)
    // The two CTAs of a cluster form a tensor-core pair: each stages its 128 rows of U and
    // 128 of the tile's 256 rows of P, the leader (rank 0) issues the MMAs of the 256 x 256
    // pair tile, and each CTA's TMEM receives the accumulator of its own 128 rows.
    const uint32_t rank = cluster_rank();
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *sbits = reinterpret_cast<uint64_t *>(base + STAGES * STAGE_BYTES);  // [RING][BM][4]
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + STAGES * STAGE_BYTES + RING * BITS_BYTES);
    uint64_t *full = bars, *empty = bars + STAGES, *tfull = bars + 2 * STAGES,
             *tempty = bars + 2 * STAGES + 2;
    uint64_t *rfull = bars + 2 * STAGES + 4, *rempty = rfull + RING;
    // tile indices the leader claims and mails to the other CTA (slots in the other CTA's
    // shared memory): mail_full lives with the reader, mail_empty with the leader
    uint64_t *mail_full = rempty + RING, *mail_empty = mail_full + RING;
    uint64_t *sfull = mail_empty + RING;  // the slot's relation words have landed
    TcTile *ring = reinterpret_cast<TcTile *>(sfull + RING);  // 16-byte aligned (36 barriers before it)
    TcTile *mail = ring + RING;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mail + RING);
    int *bad_flag = reinterpret_cast<int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            ptx::mbar_init(&full[s], 1);   // leader: its own arrival + the bytes of both CTAs' loads
            ptx::mbar_init(&empty[s], 1);  // the leader's commit, multicast to both CTAs
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&tfull[b], 1);                   // the leader's commit, multicast
            ptx::mbar_init(&tempty[b], 2 * EPI_WARPS * 32);  // leader: the epilogue threads of both CTAs
        }
        for (int q = 0; q < RING; ++q) {
            ptx::mbar_init(&rfull[q], 1);
            ptx::mbar_init(&rempty[q], 1 + EPI_WARPS * 32);  // the MMA lane and every epilogue thread
            ptx::mbar_init(&mail_full[q], 1);   // other CTA: the leader's remote arrival
            ptx::mbar_init(&mail_empty[q], 1);  // leader: the other CTA's producer has read the slot
            ptx::mbar_init(&sfull[q], 1);       // this CTA's producer: its arrival + the bits' bytes
        }
        *bad_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 1) {  // one warp of each CTA of the pair allocates together
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         ptx::smem_addr(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool bad = false;
    if (FMT && warp >= 2 && warp < 6) {
        // scale factors 1.0 (ue8m0 0x7F) in columns 256..511 of this warp's lane quarter
        const uint32_t one4 = 0x7F7F7F7Fu;
        for (uint32_t c = 256; c < TMEM_COLS; c += 32) {
            const uint32_t addr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + c;
            asm volatile(
                "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
                "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(addr),
                "r"(one4)
                : "memory");
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();  // both CTAs' barriers and scale factors exist before either uses the other's
    tc_fence_after();

    if (warp == 0) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int cur_set = -1;
            // the leader claims the pair's next tile one step ahead, so the atomic's round
            // trip overlaps the current tile's loads
            int t_next = rank == 0 ? (int)atomicAdd(args.queue, 1u) : 0;
            for (int n = 0; !bad; ++n) {
                // the pair's next tile: the leader claims it from the global queue (in list
                // order, so the tiles running at once stay neighbours in L2) and mails the tile
                // itself to the other CTA; each producer hands it to its own MMA and epilogue
                // warps through the ring
                const int slot = n % RING;
                const uint32_t rph = (uint32_t)(n / RING) & 1u;
                if (!ptx::mbar_wait_bounded(&rempty[slot], rph ^ 1u, args.wait_ns)) {
                    bad = true;
                    break;
                }
                TcTile tile;
                if (rank == 0) {
                    if (!mbar_wait_cl(&mail_empty[slot], rph ^ 1u, args.wait_ns)) {
                        bad = true;
                        break;
                    }
                    const int t = t_next;
                    if (t < args.n_tiles) {
                        tile = args.tiles[t];
                        t_next = (int)atomicAdd(args.queue, 1u);
                    } else {
                        tile.set = -1;
                        tile.ti = tile.tj = tile.kk = 0;
                    }
                    asm volatile("st.shared::cluster.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(cluster_addr(&mail[slot], 1)),
                                 "r"(tile.set), "r"(tile.ti), "r"(tile.tj), "r"(tile.kk)
                                 : "memory");
                    mbar_arrive_cluster(cluster_addr(&mail_full[slot], 1), 1);
                } else {
                    if (!mbar_wait_cl(&mail_full[slot], rph, args.wait_ns)) {
                        bad = true;
                        break;
                    }
                    tile = mail[slot];
                    mbar_arrive_cluster(cluster_addr(&mail_empty[slot], 0), 1);
                }
                const CUtensorMap *mU = args.maps + 3 * (tile.set < 0 ? 0 : tile.set), *mP = mU + 1, *mS = mU + 2;
                if (tile.set >= 0) {
                    if (tile.set != cur_set) {
                        // a new set's maps: fetch the descriptors before the first copy
                        asm volatile("prefetch.tensormap [%0];" ::"l"(mU) : "memory");
                        asm volatile("prefetch.tensormap [%0];" ::"l"(mP) : "memory");
                        asm volatile("prefetch.tensormap [%0];" ::"l"(mS) : "memory");
                        cur_set = tile.set;
                    }
                    // the relation words of this CTA's 128 rows and the tile's 256 columns
                    ptx::mbar_arrive_expect_tx(&sfull[slot], BITS_BYTES);
                    tma_load_2d(sbits + slot * (BITS_BYTES / 8), mS, tile.tj * (BN / 64), (tile.ti + (int)rank) * BM,
                                &sfull[slot]);
                }
                ring[slot] = tile;
                mbar_arrive(&rfull[slot]);
                if (tile.set < 0) break;
                const int kt0 = tile.kk & 0xFFFF, kt1 = tile.kk >> 16;
#ifdef CSG_CHECKED
                {  // the tile lies in its set and its K range in the set's operand rows
                    const TcSetDesc &TS = args.sets[tile.set];
                    CSG_IN_BOUNDS((int64_t)tile.ti * BM < TS.N && (int64_t)tile.tj * BN < TS.N &&
                                      (int64_t)kt1 * BKB <= TS.kp && kt0 <= kt1,
                                  0x22, tile.ti);
                }
#endif
                for (int kt = kt0; kt < kt1; ++kt) {
                    if (!mbar_wait_cl(&empty[s], ph ^ 1u, args.wait_ns)) {
                        bad = true;
                        break;
                    }
                    if (rank == 0) ptx::mbar_arrive_expect_tx(&full[s], 2 * STAGE_BYTES);
                    unsigned char *st = base + s * STAGE_BYTES;
                    const uint32_t lead_full = cluster_addr(&full[s], 0);
                    // (a failure-handling test starves the first stage: its barrier then waits for
                    // bytes that never come, and nothing is in flight when the waits run out)
                    if (!(args.starve && n == 0 && kt == kt0)) {
                        tma_load_2d_pair(st, mU, kt * BKB, (tile.ti + (int)rank) * BM, lead_full);
                        tma_load_2d_pair(st + A_BYTES, mP, kt * BKB, tile.tj * BN + (int)rank * (BN / 2),
                                         lead_full);
                    }
                    if (++s == STAGES) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0, b = 0, bph = 0;
            for (int n = 0; !bad; ++n) {
                const int slot = n % RING;
                if (!ptx::mbar_wait_bounded(&rfull[slot], (uint32_t)(n / RING) & 1u, args.wait_ns)) {
                    bad = true;
                    break;
                }
                const TcTile tile = ring[slot];
                mbar_arrive(&rempty[slot]);
                if (tile.set < 0) break;
                if (rank != 0) continue;  // the leader issues the pair's MMAs
                const int kt0 = tile.kk & 0xFFFF, kt1 = tile.kk >> 16;
                // both CTAs' epilogues have drained accumulator b
                if (!mbar_wait_cl(&tempty[b], bph ^ 1u, args.wait_ns)) {
                    bad = true;
                    break;
                }
                tc_fence_after();
                const uint32_t dt = tmem + b * BN;
                for (int kt = kt0; kt < kt1; ++kt) {
                    if (!mbar_wait_cl(&full[s], ph, args.wait_ns)) {
                        bad = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = ptx::smem_addr(base + s * STAGE_BYTES);
#pragma unroll
                    for (int k = 0; k < BKB / 32; ++k) {  // 32 bytes: K = 32 fp8 or 64 fp4 elements
                        const uint64_t ad = smem_desc_sw128(sa + 32 * k);
                        const uint64_t bd = smem_desc_sw128(sa + A_BYTES + 32 * k);
                        if (FMT)
                            mma_f4(dt, ad, bd, tmem + kSfA, tmem + kSfB, (kt > kt0 || k > 0) ? 1u : 0u);
                        else
                            mma_f8(dt, ad, bd, (kt > kt0 || k > 0) ? 1u : 0u);
                    }
                    mma_commit_pair(&empty[s]);  // frees stage s in both CTAs
                    if (++s == STAGES) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (bad) break;
                mma_commit_pair(&tfull[b]);  // accumulator b complete in both CTAs
                if (NACC == 2) b ^= 1u;
                if (b == 0) bph ^= 1u;
            }
        }
    } else {
        // epilogue: TMEM lane quarter of this warp, and which half of the tile's columns
        const int q = warp & 3;
        const int r = q * 32 + lane;
        const int g = (warp - 2) >> 2;
        const int cb = g * (BN / 2), ce = cb + BN / 2;
        // per-thread counters; N0..N3 are packed 16 bits each and spilled into the
        // 64-bit totals after every tile (a tile holds at most 256 pairs per row)
        unsigned long long c0 = 0, c1 = 0, c2 = 0, c3 = 0, cR = 0, cM = 0, cW = 0;
        int cur = -1;  // set whose counters are being accumulated
        auto flush = [&](int set) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                c0 += __shfl_xor_sync(0xffffffffu, c0, o);
                c1 += __shfl_xor_sync(0xffffffffu, c1, o);
                c2 += __shfl_xor_sync(0xffffffffu, c2, o);
                c3 += __shfl_xor_sync(0xffffffffu, c3, o);
                cR += __shfl_xor_sync(0xffffffffu, cR, o);
                cM += __shfl_xor_sync(0xffffffffu, cM, o);
                cW += __shfl_xor_sync(0xffffffffu, cW, o);
            }
            if (lane == 0 && cR) {
                unsigned long long *cnt = args.sets[set].counters;
                atomicAdd(&cnt[CNT_N0], c0);
                atomicAdd(&cnt[CNT_N1], c1);
                atomicAdd(&cnt[CNT_N2], c2);
                atomicAdd(&cnt[CNT_N3], c3);
                atomicAdd(&cnt[CNT_R], cR);
                atomicAdd(&cnt[CNT_SUM_M], cM);
                atomicAdd(&cnt[CNT_W], cW);
            }
            c0 = c1 = c2 = c3 = cR = cM = cW = 0;
        };
        uint32_t b = 0, bph = 0;
        for (int n = 0;; ++n) {
            const int slot = n % RING;
            const bool got = ptx::mbar_wait_bounded(&rfull[slot], (uint32_t)(n / RING) & 1u, args.wait_ns);
            if (!__all_sync(0xffffffffu, got)) {
                bad = true;
                break;
            }
            const TcTile tile = ring[slot];
            if (tile.set < 0) {
                mbar_arrive(&rempty[slot]);
                break;
            }
            // the row's relation words for this warp's half of the tile's columns, staged in
            // shared memory by the producer
            const bool staged = ptx::mbar_wait_bounded(&sfull[slot], (uint32_t)(n / RING) & 1u, args.wait_ns);
            if (!__all_sync(0xffffffffu, staged)) {
                bad = true;
                break;
            }
            const int bidx = slot * (BITS_BYTES / 8) + r * 4 + 2 * g;
            const ulonglong2 wv = CSG_IN_BOUNDS(bidx + 1 < RING * (BITS_BYTES / 8), 0x23, bidx)
                                      ? *reinterpret_cast<const ulonglong2 *>(sbits + bidx)
                                      : make_ulonglong2(0ull, 0ull);
            mbar_arrive(&rempty[slot]);  // the slot's tile and words are read
            if (tile.set != cur) {
                if (cur >= 0) flush(cur);
                cur = tile.set;
            }
            const TcSetDesc S = args.sets[tile.set];
            const int64_t N = S.N;
            const int64_t i = (int64_t)(tile.ti + (int)rank) * BM + r;
            const int64_t J0 = (int64_t)tile.tj * BN;
            uint64_t w4[4] = {0, 0, 0, 0};
            if (i < N && i >= S.row_lo && i < S.row_hi) {
                w4[0] = g == 0 ? wv.x : 0ull;
                w4[1] = g == 0 ? wv.y : 0ull;
                w4[2] = g == 1 ? wv.x : 0ull;
                w4[3] = g == 1 ? wv.y : 0ull;
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (J0 + 64 * u >= N) w4[u] = 0;
                // only columns j > i
                const int64_t rel = i - J0;  // bit positions k > rel survive
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t lo = rel - 64 * u;
                    if (lo >= 63)
                        w4[u] = 0;
                    else if (lo >= 0)
                        w4[u] &= ~((2ull << lo) - 1ull);
                }
            }
            const double phi_i = (S.acc != nullptr && i < N) ? S.phi[i] : 0.0;
            const bool ok = mbar_wait_cl(&tfull[b], bph, args.wait_ns);
            if (!__all_sync(0xffffffffu, ok)) {
                bad = true;
                break;
            }
            tc_fence_after();
            const uint32_t tbase = tmem + b * BN + ((uint32_t)(q * 32) << 16);
            const uint32_t release = cluster_addr(&tempty[b], 0);
            unsigned long long packed;
            if (FMT)
                packed = S.acc != nullptr ? epi_tile_all<true>(tbase, w4, i, J0, cR, cM, cW, args.hist, args.nbins,
                                                               phi_i, S.acc, release, cb)
                                          : epi_tile_all<false>(tbase, w4, i, J0, cR, cM, cW, args.hist, args.nbins,
                                                                0.0, nullptr, release, cb);
            else
                packed = S.acc != nullptr ? epi_tile<true>(tbase, w4, i, J0, cR, cM, cW, args.hist, args.nbins, phi_i,
                                                           S.acc, release, cb, ce)
                                          : epi_tile<false>(tbase, w4, i, J0, cR, cM, cW, args.hist, args.nbins, 0.0,
                                                            nullptr, release, cb, ce);
            c0 += packed & 0xFFFFull;
            c1 += (packed >> 16) & 0xFFFFull;
            c2 += (packed >> 32) & 0xFFFFull;
            c3 += packed >> 48;
            if (NACC == 2) b ^= 1u;
            if (b == 0) bph ^= 1u;
        }
        if (cur >= 0) flush(cur);
    }
    if (bad) atomicExch(bad_flag, 1);
    tc_fence_before();
    __syncthreads();
    // neither CTA frees TMEM or leaves while the other may still load into it, commit to its
    // barriers or arrive on them
    cluster_sync();
    if (*bad_flag && threadIdx.x == 0 && args.n_tiles > 0)
        atomicExch(&args.sets[args.tiles[0].set].counters[CNT_ERR], CNT_ERR_TIMEOUT);
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                     : "memory");
    }
}

// ------------------------------------------------------------------ MMA rate probe

// Throughput probe of the pair MMA the product issues: the same instruction, instruction
// descriptor, TMEM layout (accumulator at column 0; the fp4 form's unit scale factors at
// columns 256 and 384) and shared-memory descriptors, on one 32 KB stage of zeros resident in
// each CTA's shared memory.  The leader issues `iters` groups of four MMAs (one 128-byte K
// stage) back to back and commits once; both CTAs wait for that commit (bounded) before
// freeing TMEM.  One CTA per SM (the dynamic shared memory is sized for it).
constexpr int PROBE_THREADS = 192;

template <int FMT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(PROBE_THREADS, 1)
mma_probe_kernel(int iters, uint64_t limit, unsigned long long *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *done = reinterpret_cast<uint64_t *>(base + STAGE_BYTES);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    const uint32_t rank = cluster_rank();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = threadIdx.x; q < STAGE_BYTES / 16; q += PROBE_THREADS)
        reinterpret_cast<uint4 *>(base)[q] = make_uint4(0u, 0u, 0u, 0u);
    ptx::fence_proxy_async_smem();  // the zeros are visible to the tensor cores
    if (threadIdx.x == 0) {
        ptx::mbar_init(done, 1);
        ptx::fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         ptx::smem_addr(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (FMT && warp >= 2 && warp < 6) {
        const uint32_t one4 = 0x7F7F7F7Fu;  // scale factors 1.0 in columns 256..511
        for (uint32_t c = 256; c < TMEM_COLS; c += 32) {
            const uint32_t addr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + c;
            asm volatile(
                "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
                "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(addr),
                "r"(one4)
                : "memory");
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();  // both CTAs' operands, barrier and scale factors exist
    tc_fence_after();
    if (rank == 0 && warp == 1 && lane == 0) {
        const uint32_t sa = ptx::smem_addr(base);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < BKB / 32; ++k) {
                const uint64_t ad = smem_desc_sw128(sa + 32 * k);
                const uint64_t bd = smem_desc_sw128(sa + A_BYTES + 32 * k);
                if (FMT)
                    mma_f4(tmem, ad, bd, tmem + kSfA, tmem + kSfB, (it > 0 || k > 0) ? 1u : 0u);
                else
                    mma_f8(tmem, ad, bd, (it > 0 || k > 0) ? 1u : 0u);
            }
        }
        mma_commit_pair(done);  // arrives in both CTAs once every MMA has completed
    }
    if (warp == 1 && lane == 0 && !mbar_wait_cl(done, 0u, limit)) atomicAdd(err, 1ull);
    tc_fence_before();
    __syncthreads();
    cluster_sync();  // neither CTA frees TMEM while the other's MMAs may still write it
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                     : "memory");
    }
}

// ------------------------------------------------------------------ host side

PFN_cuTensorMapEncodeTiled_v12000 get_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}


// Output tiles of the upper triangle of one set in super x super blocks: block rows in
// turn (their U panels stay in L2 while the row's blocks run), each row's blocks from the
// longest K range down, and column-major inside a block, so tiles sharing a P panel run
// together.  The list is generated in that order directly and kept per (N, row range,
// block).  Each entry is a pair tile: 256 rows (row tiles ti and ti + 1, ti even) by 256
// columns.  (Across orders and block sizes the kernel's time moves by under 4 %: it is bound
// by the operand feed from L2 and the MMA issue, not by DRAM.)
struct TileCache {
    std::mutex mu;
    std::map<std::tuple<int64_t, int64_t, int64_t, int>, std::vector<TcTile>> lists;
};
TileCache g_tiles;

std::vector<TcTile> single_set_tiles(int64_t N, int64_t lo, int64_t hi, int super) {
    std::lock_guard<std::mutex> g(g_tiles.mu);
    auto key = std::make_tuple(N, lo, hi, super);
    auto it = g_tiles.lists.find(key);
    if (it != g_tiles.lists.end()) return it->second;
    if (g_tiles.lists.size() >= 256) g_tiles.lists.clear();
    std::vector<TcTile> tiles;
    const int NI = (int)((N + BM - 1) / BM), NJ = (int)((N + BN - 1) / BN);
    const int rows_per_block = super / BM, cols_per_block = super / BN;
    const int NB = (int)((N + super - 1) / super);
    auto block = [&](int bi, int bj) {
        for (int tj = bj * cols_per_block; tj < std::min(NJ, (bj + 1) * cols_per_block); ++tj) {
            for (int ti = bi * rows_per_block; ti < std::min(NI, (bi + 1) * rows_per_block); ++ti) {
                if (tj < ti / 2) continue;
                const int64_t I0 = (int64_t)ti * BM, I1 = I0 + BM;
                if (I1 <= lo || I0 >= hi) continue;
                const int64_t J1 = std::min<int64_t>((int64_t)(tj + 1) * BN, N);
                if (J1 <= I0 + 1) continue;
                // as a pair tile: row tiles ti & ~1 and (ti & ~1) + 1 go to the two CTAs of a pair
                const TcTile pt{0, ti & ~1, tj, 0};  // set and K range filled in per launch
                if (tiles.empty() || tiles.back().ti != pt.ti || tiles.back().tj != pt.tj) tiles.push_back(pt);
            }
        }
    };
    for (int bi = 0; bi < NB; ++bi)
        for (int bj = NB - 1; bj >= bi; --bj) block(bi, bj);
    return g_tiles.lists[key] = std::move(tiles);
}

int encode_map(CUtensorMap *m, void *base, int64_t rows, int64_t kp, int box_rows) {
    auto enc = get_encoder();
    if (!enc) {
        set_error("action_tc: cuTensorMapEncodeTiled is unavailable");
        return CSG_E_CUDA;
    }
    cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kp};
    cuuint32_t box[2] = {(cuuint32_t)BKB, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("action_tc: tensor map encoding failed (%d)", (int)r);
        return CSG_E_CUDA;
    }
    return CSG_OK;
}

// The relation words as a 2D tensor of 64-bit words (stride words x N rows); a box is the
// 4 words of one tile's columns for one CTA's 128 rows (rows past N read as zero).
int encode_bits_map(CUtensorMap *m, const uint64_t *rows, int64_t N, int64_t stride) {
    auto enc = get_encoder();
    if (!enc) {
        set_error("action_tc: cuTensorMapEncodeTiled is unavailable");
        return CSG_E_CUDA;
    }
    if ((reinterpret_cast<uintptr_t>(rows) & 15) != 0 || stride % 2 != 0) {
        set_error("action_tc: relation rows are not 16-byte aligned");
        return CSG_E_INVAL;
    }
    cuuint64_t dims[2] = {(cuuint64_t)stride, (cuuint64_t)N};
    cuuint64_t strides[1] = {(cuuint64_t)stride * 8};
    cuuint32_t box[2] = {(cuuint32_t)(BN / 64), (cuuint32_t)BM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<uint64_t *>(rows), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("action_tc: tensor map encoding failed (%d)", (int)r);
        return CSG_E_CUDA;
    }
    return CSG_OK;
}

}  // namespace

unsigned long long check_word_tc() { return take_check_word(); }

// Largest N the tensor form accepts (every N a set can have): its operands take N^2
// bytes of scratch in fp4 (64 GiB at N = 2^18) and 2 N^2 in fp8 (128 GiB).  The fp32
// accumulator stays exact (m < 2^18, a 16-column sum < 2^22, both below 2^24).
static constexpr int64_t kTcMaxN = CSG_MAX_N;
// Operand scratch shared by the sets of one chunk (a larger single set gets its own).
static constexpr int64_t kChunkBytes = 16ll << 30;

TcPlan tc_plan(const SetDesc *sets, int n, Arena &a, size_t s_counters, unsigned long long *hist,
               int64_t nbins, int *rc, const int *slots, int super, int fmt) {
    TcPlan p;
    *rc = CSG_OK;
    fmt = fmt ? 1 : 0;
    p.fmt = fmt;
    if (slots) p.slot.assign(slots, slots + n);
    if (super < BN) super = BN;
    p.n_sets = n;
    p.s_counters = s_counters;
    p.hist = hist;
    p.nbins = nbins;
    std::vector<TcSetDesc> desc(n);
    int64_t chunk_bytes = 0, max_chunk = 0;
    TcPlan::Chunk cur;
    cur.set_lo = 0;
    for (int s = 0; s < n; ++s) {
        const SetDesc &S = sets[s];
        if (S.N > kTcMaxN) {
            set_error("action_tc: N=%lld exceeds the tensor form's limit %lld", (long long)S.N,
                      (long long)kTcMaxN);
            *rc = CSG_E_INVAL;
            return p;
        }
        TcSetDesc &D = desc[s];
        D.rows = S.rows;
        D.N = S.N;
        D.stride = S.stride;
        D.row_lo = std::max<int64_t>(0, S.row_lo);
        D.row_hi = std::min<int64_t>(S.N, S.row_hi);
        D.counters = nullptr;
        D.phi = S.phi;
        D.acc = S.acc;
        // operand row bytes: N rounded up to a whole stage (128 fp8 or 256 fp4 elements)
        D.kp = fmt ? (S.N + 255) / 256 * 128 : (S.N + 127) / 128 * 128;
        const int64_t ob = 2 * S.N * D.kp;
        if (s > cur.set_lo && chunk_bytes + ob > kChunkBytes) {
            cur.set_hi = s;
            p.chunks.push_back(cur);
            max_chunk = std::max(max_chunk, chunk_bytes);
            cur = TcPlan::Chunk();
            cur.set_lo = s;
            chunk_bytes = 0;
        }
        D.U = reinterpret_cast<uint8_t *>(chunk_bytes);           // offsets, patched later
        D.P = reinterpret_cast<uint8_t *>(chunk_bytes + S.N * D.kp);
        chunk_bytes += ob;
    }
    cur.set_hi = n;
    p.chunks.push_back(cur);
    max_chunk = std::max(max_chunk, chunk_bytes);
    p.t_sets = a.put(desc.data(), n * sizeof(TcSetDesc));
    p.t_maps = a.put(nullptr, 3 * (size_t)n * sizeof(CUtensorMap));
    p.s_ops = a.reserve((size_t)max_chunk);
    p.s_queues = a.reserve(p.chunks.size() * sizeof(unsigned int));
    for (TcPlan::Chunk &c : p.chunks) {
        std::vector<int64_t> rstarts;  // first operand row of each set of the chunk
        int64_t total = 0;
        std::vector<TcTile> tiles;
        for (int s = c.set_lo; s < c.set_hi; ++s) {
            rstarts.push_back(total);
            total += desc[s].N;
        }
        if (c.set_hi - c.set_lo == 1) {
            const TcSetDesc &D = desc[c.set_lo];
            if (D.row_hi > D.row_lo) {
                tiles = single_set_tiles(D.N, D.row_lo, D.row_hi, super);
                for (TcTile &t : tiles) {
                    t.set = c.set_lo;
                    t.kk = k_range_packed(t.ti, t.tj, D.N, fmt);
                }
            }
        } else {
            // set by set, largest first: the CTAs running at any moment then work on one or
            // two sets whose operands stay in L2, and the small sets fill the tail
            std::vector<int> order;
            for (int s = c.set_lo; s < c.set_hi; ++s)
                if (desc[s].row_hi > desc[s].row_lo) order.push_back(s);
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return desc[x].N > desc[y].N; });
            for (int s : order) {
                std::vector<TcTile> ts = single_set_tiles(desc[s].N, desc[s].row_lo, desc[s].row_hi, super);
                for (TcTile &t : ts) {
                    t.set = s;
                    t.kk = k_range_packed(t.ti, t.tj, desc[s].N, fmt);
                }
                tiles.insert(tiles.end(), ts.begin(), ts.end());
            }
        }
        if (tiles.size() > 0x7fffffff) {
            set_error("action_tc: too many tiles");
            *rc = CSG_E_INVAL;
            return p;
        }
        c.rows = total;
        c.t_rstarts = a.put(rstarts.data(), rstarts.size() * sizeof(int64_t));
        c.n_tiles = (int)tiles.size();
        c.t_tiles = a.put(tiles.data(), tiles.size() * sizeof(TcTile));
    }
    return p;
}

int tc_patch(const TcPlan &p, Arena &a) {
    TcSetDesc *desc = a.host<TcSetDesc>(p.t_sets);
    CUtensorMap *maps = a.host<CUtensorMap>(p.t_maps);
    uint8_t *ops = a.scr<uint8_t>(p.s_ops);
    for (int s = 0; s < p.n_sets; ++s) {
        TcSetDesc &D = desc[s];
        D.counters = a.scr<unsigned long long>(p.s_counters) + (size_t)(p.slot.empty() ? s : p.slot[s]) * CNT_WORDS;
        D.U = ops + reinterpret_cast<uintptr_t>(D.U);
        D.P = ops + reinterpret_cast<uintptr_t>(D.P);
        int rc = encode_map(&maps[3 * s], D.U, D.N, D.kp, BM);
        if (rc == CSG_OK) rc = encode_map(&maps[3 * s + 1], D.P, D.N, D.kp, BN / 2);  // each CTA's half
        if (rc == CSG_OK) rc = encode_bits_map(&maps[3 * s + 2], D.rows, D.N, D.stride);
        if (rc != CSG_OK) return rc;
    }
    return CSG_OK;
}

template <int FMT>
static int tc_launch_fmt(const TcPlan &p, const Arena &a, cudaStream_t st) {
    const size_t smem = 1024 + STAGES * STAGE_BYTES + RING * BITS_BYTES + 512;
    CSG_CUDA_TRY(cudaFuncSetAttribute(action_tc_kernel<FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // CTA pairs (clusters of two, one CTA per SM) that can be resident at once
    int clusters = 0;
    {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2, 1, 1);
        cfg.blockDim = dim3(THREADS, 1, 1);
        cfg.dynamicSmemBytes = smem;
        if (cudaOccupancyMaxActiveClusters(&clusters, (const void *)action_tc_kernel<FMT>, &cfg) != cudaSuccess ||
            clusters < 1) {
            cudaGetLastError();
            clusters = 0;
        }
    }
    unsigned int *queues = a.scr<unsigned int>(p.s_queues);
    CSG_CUDA_TRY(cudaMemsetAsync(queues, 0, p.chunks.size() * sizeof(unsigned int), st));
    int dev = 0, sms = 0;
    CSG_CUDA_TRY(cudaGetDevice(&dev));
    CSG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const TcSetDesc *d_sets = a.tab<TcSetDesc>(p.t_sets);
    for (size_t ci = 0; ci < p.chunks.size(); ++ci) {
        const TcPlan::Chunk &c = p.chunks[ci];
        if (c.rows > 0) {
            const int group = c.set_hi - c.set_lo > 1 ? 4 : 1;  // rows per warp and step
            const int64_t groups = (c.rows + group - 1) / group;
            const int blocks = (int)std::min<int64_t>((groups + 7) / 8, (int64_t)sms * 16);
            stage_begin(CSG_STAGE_EXPAND, st);
            expand_kernel<FMT><<<blocks, 256, 0, st>>>(d_sets, a.tab<int64_t>(c.t_rstarts), c.set_lo,
                                                       c.set_hi - c.set_lo, c.rows, group);
            stage_end(CSG_STAGE_EXPAND, st);
        }
        if (c.n_tiles > 0) {
            TcArgs args;
            args.sets = d_sets;
            args.maps = a.tab<CUtensorMap>(p.t_maps);
            args.tiles = a.tab<TcTile>(c.t_tiles);
            args.n_tiles = c.n_tiles;
            args.queue = queues + ci;
            args.hist = p.hist;
            args.nbins = (long long)p.nbins;
            args.wait_ns = wait_limit_ns(kWaitNs);
            args.starve = starve_first_stage();
            stage_begin(CSG_STAGE_ACTION, st);
            const int pairs = std::min(clusters > 0 ? clusters : sms / 2, c.n_tiles);
            action_tc_kernel<FMT><<<2 * pairs, THREADS, smem, st>>>(args);
            stage_end(CSG_STAGE_ACTION, st);
        }
        CSG_CUDA_TRY(cudaGetLastError());
    }
    return CSG_OK;
}

int tc_launch(const TcPlan &p, const Arena &a, cudaStream_t st) {
    return p.fmt ? tc_launch_fmt<1>(p, a, st) : tc_launch_fmt<0>(p, a, st);
}

}  // namespace csg

namespace csg {
namespace {

template <int FMT>
int measure_mma_rate(int device, double *flops_per_second) {
    CSG_CUDA_TRY(cudaSetDevice(device));
    int sms = 0;
    CSG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const int smem = 200 * 1024;  // one CTA per SM, as the product kernel
    CSG_CUDA_TRY(cudaFuncSetAttribute(mma_probe_kernel<FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int pairs = sms / 2;
    {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * pairs);
        cfg.blockDim = dim3(PROBE_THREADS);
        cfg.dynamicSmemBytes = smem;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, (const void *)mma_probe_kernel<FMT>, &cfg) == cudaSuccess &&
            clusters > 0 && clusters < pairs)
            pairs = clusters;
        cudaGetLastError();
    }
    unsigned long long *err = nullptr;
    if (dev_malloc((void **)&err, 8) != cudaSuccess) {
        cudaGetLastError();
        set_error("csg_measure_mma_rate: allocation failed");
        return CSG_E_NOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = CSG_OK;
    float ms = 0.f;
    unsigned long long h_err = 0;
    const int iters = 20000;
    if (cudaMemset(err, 0, 8) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        rc = CSG_E_CUDA;
    if (rc == CSG_OK) {
        const uint64_t limit = wait_limit_ns(kWaitNs);
        mma_probe_kernel<FMT><<<2 * pairs, PROBE_THREADS, smem>>>(200, limit, err);  // warm-up
        cudaEventRecord(e0);
        mma_probe_kernel<FMT><<<2 * pairs, PROBE_THREADS, smem>>>(iters, limit, err);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f ||
            cudaMemcpy(&h_err, err, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = CSG_E_CUDA;
        else if (h_err != 0)
            rc = CSG_E_TIMEOUT;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(err);
    if (rc != CSG_OK) {
        set_error(rc == CSG_E_TIMEOUT ? "csg_measure_mma_rate: a bounded wait expired"
                                      : "csg_measure_mma_rate: the probe failed");
        return rc;
    }
    // each MMA: M = 256 rows x N = 256 columns x K = 64 fp4 or 32 fp8 elements, 2 flops a product
    const double per_mma = 2.0 * (2 * BM) * BN * (FMT ? 64 : 32);
    *flops_per_second = (double)pairs * iters * (BKB / 32) * per_mma / (ms * 1e-3);
    return CSG_OK;
}

}  // namespace
}  // namespace csg

extern "C" int csg_measure_mma_rate(int device, int method, double *flops_per_second) {
    if (device < 0 || !flops_per_second || (method != CSG_TC && method != CSG_TC_FP4 && method != CSG_TC_FP8)) {
        csg::set_error("csg_measure_mma_rate: bad arguments");
        return CSG_E_INVAL;
    }
    return method == CSG_TC_FP8 ? csg::measure_mma_rate<0>(device, flops_per_second)
                                : csg::measure_mma_rate<1>(device, flops_per_second);
}
