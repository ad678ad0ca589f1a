// csg_action_noalloc: the popcount action for callers that must not allocate.
//
// Some callers cannot let a library allocate device memory: code that records its
// work into a CUDA graph, where a cudaMalloc would break the capture; applications
// that hand all of HBM to their own arena and forbid allocations from anyone else;
// and multi-stream servers that cannot afford the device-wide synchronisation a
// cudaFree implies.  This entry point serves them.  It takes the caller's bitmap and
// a caller-owned device result slot, and keeps its own scratch -- the work-queue
// counter and one block of partial counters per group of 16 rows -- in a fixed
// file-scope device array.  The array costs every GPU that loads the library
// kScratchBytes of memory until the process exits.
//
// The kernel is a variant of the popcount action (AND + popcount of packed row
// words, Alg. 5): the same row-group staging and sweep, but each work item writes
// its partial counters to its own scratch slot instead of adding them atomically,
// and a one-block finalize sums the slots in a fixed order, forms the action and
// writes the result.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "csg_internal.cuh"
#include "ptx.cuh"

namespace csg {
namespace {

constexpr int kG = 16;                        // rows per work item
constexpr int64_t kMaxN = 65536;              // largest set this entry point takes
constexpr int kMaxItems = (int)(kMaxN / kG);  // 4096 row groups
constexpr int kSlot = 8;                      // counters per slot (CNT_* layout)
constexpr int kWarps = 16;
constexpr int kThreads = kWarps * 32;
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// [0]: work-queue counter (low 32 bits); [1]: error word; then kMaxItems slots.
constexpr size_t kScratchWords = 2 + (size_t)kMaxItems * kSlot;
constexpr size_t kScratchBytes = kScratchWords * sizeof(unsigned long long);  // 256 KiB + 16 B

static __device__ __align__(256) unsigned long long g_scratch[kScratchWords];

struct NaSet {
    const uint64_t *rows;
    int64_t N, stride;
    int d;
};

__global__ void __launch_bounds__(kThreads, 1)
noalloc_popc_kernel(const NaSet S, int n_items, int pitch, unsigned long long *scratch) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    uint64_t *bar = reinterpret_cast<uint64_t *>(base);
    int *item_slot = reinterpret_cast<int *>(base + 8);
    uint64_t *A = reinterpret_cast<uint64_t *>(base + 128);
    unsigned int *queue = reinterpret_cast<unsigned int *>(&scratch[0]);
    unsigned long long *part = scratch + 2;
    // per-warp partial counters of the current item, reduced across warps in smem
    __shared__ unsigned long long wsum[kWarps][7];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        ptx::mbar_init(bar, 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();
    const int64_t N = S.N, stride = S.stride;
    const uint64_t *__restrict__ rows = S.rows;
    uint32_t phase = 0;
    for (;;) {
        if (threadIdx.x == 0) *item_slot = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int k = *item_slot;
        if (k >= n_items) break;
        const int64_t i0 = (int64_t)k * kG;
        const int64_t w0 = i0 >> 6, w0a = w0 & ~int64_t(1);
        const int64_t wN = (N + 63) >> 6;
        const int nwa = (int)(((wN - w0a) + 1) & ~int64_t(1));
        uint32_t gmask = 0;
#pragma unroll
        for (int r = 0; r < kG; ++r)
            if (i0 + r < N) gmask |= 1u << r;
        if (threadIdx.x == 0) {
            ptx::fence_proxy_async_smem();
            const uint32_t bytes = (uint32_t)nwa * 8u;
            ptx::mbar_arrive_expect_tx(bar, bytes * (uint32_t)__popc(gmask));
            for (int r = 0; r < kG; ++r)
                if ((gmask >> r & 1u) && CSG_IN_BOUNDS(nwa <= pitch && w0a + nwa <= stride, 0x60, i0 + r))
                    ptx::bulk_g2s(A + (size_t)r * pitch, rows + (i0 + r) * stride + w0a, bytes, bar);
        }
        const bool landed = ptx::mbar_wait_bounded(bar, phase, kWaitLimitNs);
        if (__syncthreads_or(!landed)) {
            if (threadIdx.x == 0) {
                atomicExch(&scratch[1], 1ull);
                ptx::mbar_wait_bounded(bar, phase, kWaitLimitNs);
            }
            __syncthreads();
            break;
        }
        phase ^= 1u;
        const int lead = (int)(w0 - w0a);
        if (threadIdx.x < kG && (gmask >> threadIdx.x & 1u)) {
            const int r = threadIdx.x;
            const int b = (int)((i0 + r) & 63);
            uint64_t *a = A + (size_t)r * pitch;
            if (lead) a[0] = 0;
            a[lead] &= ~((2ull << b) - 1ull);
        }
        __syncthreads();

        unsigned long long c0 = 0, c1 = 0, c2 = 0, c3 = 0, cR = 0, cM = 0, cW = 0;
        const int gshift = (int)(i0 & 63);
        for (int64_t jb = i0 + 1 + 32 * (int64_t)warp; jb < N; jb += 32 * kWarps) {
            const int64_t jl = jb + lane;
            uint32_t my = 0;
            if (jl < N) {
                const uint64_t word = __ldg(rows + jl * stride + w0);
                my = (uint32_t)(word >> gshift) & 0xffffu & gmask;
                const int64_t off = jl - i0;
                if (off < kG) my &= (1u << off) - 1u;
            }
            uint32_t todo = __ballot_sync(0xffffffffu, my != 0);
            while (todo) {
                const int src = __ffs(todo) - 1;
                todo &= todo - 1;
                const uint32_t mask = __shfl_sync(0xffffffffu, my, src);
                const int64_t j = jb + src;
                const int wj = (int)((j >> 6) - w0a);
                const uint64_t lastmask = (1ull << (j & 63)) - 1ull;
                const uint64_t *__restrict__ bj = rows + j * stride + w0a;
                uint32_t acc[kG];
#pragma unroll
                for (int r = 0; r < kG; ++r) acc[r] = 0;
                for (int w = lane; w <= wj; w += 32) {
                    uint64_t b = CSG_IN_BOUNDS(w0a + w < stride, 0x61, j) ? __ldg(bj + w) : 0ull;
                    if (w == wj) b &= lastmask;
#pragma unroll
                    for (int r = 0; r < kG; ++r)
                        if ((mask >> r & 1u) && CSG_IN_BOUNDS(w < pitch, 0x62, w))
                            acc[r] += __popcll(A[(size_t)r * pitch + w] & b);
                }
#pragma unroll
                for (int r = 0; r < kG; ++r) {
                    if (mask >> r & 1u) {
                        uint32_t m = acc[r];
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
                        if (lane == 0) {
                            c0 += (m == 0);
                            c1 += (m == 1);
                            c2 += (m == 2);
                            c3 += (m == 3);
                            cR += 1;
                            cM += m;
                            cW += (unsigned long long)(j - (i0 + r) - 1);
                        }
                    }
                }
            }
        }
        if (lane == 0) {
            wsum[warp][0] = c0;
            wsum[warp][1] = c1;
            wsum[warp][2] = c2;
            wsum[warp][3] = c3;
            wsum[warp][4] = cR;
            wsum[warp][5] = cM;
            wsum[warp][6] = cW;
        }
        __syncthreads();
        // every item overwrites its whole slot, so no slot needs clearing between calls
        if (threadIdx.x < 7 && CSG_IN_BOUNDS(k < kMaxItems, 0x63, k)) {
            unsigned long long s = 0;
            for (int w = 0; w < kWarps; ++w) s += wsum[w][threadIdx.x];
            part[(size_t)k * kSlot + threadIdx.x] = s;
        }
        __syncthreads();
    }
}

// Sums the item slots in order, forms the action (Eq. s_local for d=2, the 3+1 BD
// combination for d=4) and writes the caller's result.
__global__ void noalloc_finalize_kernel(int d, int64_t N, int n_items,
                                        const unsigned long long *__restrict__ scratch,
                                        csg_result *__restrict__ out) {
    __shared__ unsigned long long tot[7];
    const unsigned long long *part = scratch + 2;
    if (threadIdx.x < 7) {
        unsigned long long s = 0;
        for (int k = 0; k < n_items; ++k) s += part[(size_t)k * kSlot + threadIdx.x];
        tot[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        csg_result r;
        r.d = d;
        const bool failed = scratch[1] != 0;
        r.status = failed ? CSG_E_TIMEOUT : CSG_OK;
        r.N = N;
        // after a timed-out wait some slots hold an earlier call's counts: report zeros
        if (failed)
            for (int k = 0; k < 7; ++k) tot[k] = 0;
        for (int k = 0; k < 4; ++k) r.Nk[k] = tot[k];
        r.R = tot[4];
        r.sum_m = tot[5];
        r.W = tot[6];
        const long long n0 = (long long)tot[0], n1 = (long long)tot[1], n2 = (long long)tot[2],
                        n3 = (long long)tot[3];
        if (d == 2) {
            r.combo = N - 2 * n0 + 4 * n1 - 2 * n2;
            r.S = __dmul_rn(2.0, __ll2double_rn(r.combo));
        } else {
            r.combo = N - n0 + 9 * n1 - 16 * n2 + 8 * n3;
            r.S = __dmul_rn(__ddiv_rn(4.0, __dsqrt_rn(6.0)), __ll2double_rn(r.combo));
        }
        *out = r;
    }
}

// Device address of g_scratch for each device, found once per device.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned long long *g_scratch_addr[kMaxDevices] = {nullptr};

}  // namespace

unsigned long long check_word_noalloc() { return take_check_word(); }
}  // namespace csg

using namespace csg;

extern "C" int csg_action_noalloc(int d, int64_t N, const uint64_t *dev_rows, int64_t stride_words,
                                  csg_result *dev_out, void *stream) {
    if ((d != 2 && d != 4) || !dev_rows || !dev_out) {
        set_error("csg_action_noalloc: d must be 2 or 4 and the pointers non-null");
        return CSG_E_INVAL;
    }
    if (N < 1 || N > kMaxN) {
        set_error("csg_action_noalloc: N=%lld is outside [1, %lld], the largest set its fixed "
                  "%zu-byte scratch array holds (use csg_action for larger sets)",
                  (long long)N, (long long)kMaxN, kScratchBytes);
        return CSG_E_INVAL;
    }
    if (stride_words < (N + 63) / 64 || (stride_words & 1) ||
        (reinterpret_cast<uintptr_t>(dev_rows) & 15)) {
        set_error("csg_action_noalloc: rows must be 16-byte aligned with an even stride of at "
                  "least ceil(N/64) words");
        return CSG_E_INVAL;
    }
    int dev = 0;
    CSG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("csg_action_noalloc: device index %d out of range", dev);
        return CSG_E_INVAL;
    }
    unsigned long long *scratch = nullptr;
    {
        // first call on this device: look up the array's device address (a host-side
        // reference to g_scratch is not a device address)
        std::lock_guard<std::mutex> g(g_setup_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess || !p) {
                set_error("csg_action_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
                return CSG_E_CUDA;
            }
            g_scratch_addr[dev] = static_cast<unsigned long long *>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int n_items = (int)((N + kG - 1) / kG);
    const int64_t words = (N + 63) / 64 + 2;
    const int pitch = (int)((words + 1) & ~int64_t(1));
    const size_t smem = 256 + (size_t)kG * pitch * sizeof(uint64_t);
    CSG_CUDA_TRY(cudaFuncSetAttribute(noalloc_popc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    int sms = 0, per_sm = 0;
    CSG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CSG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, noalloc_popc_kernel, kThreads, smem));
    if (per_sm < 1) {
        set_error("csg_action_noalloc: %zu bytes of shared memory per CTA do not fit", smem);
        return CSG_E_INVAL;
    }
    int grid = sms * per_sm;
    if (grid > n_items) grid = n_items;
    // the queue counter and the error word must start at zero; item slots are
    // overwritten by their items
    CSG_CUDA_TRY(cudaMemsetAsync(scratch, 0, 2 * sizeof(unsigned long long), st));
    NaSet S{dev_rows, N, stride_words, d};
    noalloc_popc_kernel<<<grid, kThreads, smem, st>>>(S, n_items, pitch, scratch);
    CSG_CUDA_TRY(cudaGetLastError());
    noalloc_finalize_kernel<<<1, 32, 0, st>>>(d, N, n_items, scratch, dev_out);
    CSG_CUDA_TRY(cudaGetLastError());
    return CSG_OK;
}
