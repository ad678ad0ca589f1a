// Throughput probes for the rooflines of the interval counts.
//
// Population-count pipe, the bound of the popcount form (CSG_POPC: one 32-bit popcount per
// 32 candidate bits of every related pair's range):
// Every thread runs `iters` iterations of eight independent 32-bit popcounts (popc.b32) of
// values that change every iteration, summed with three-input adds, so the popcount pipe
// is the busiest one.  Two CTAs of 1024 threads per SM.  The result is popcounts per second
// over the whole GPU; divided by the SM count and the clock it gives the pipe's results per
// SM per clock (16 in the CUDA programming guide's throughput table).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "csg_internal.cuh"
#include "ptx.cuh"

namespace csg {
namespace {

__global__ void __launch_bounds__(1024) popc_probe_kernel(uint32_t seed, int iters, uint32_t *out) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t b[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) b[k] = (t ^ seed) * (2u * k + 3u) + k;
    uint32_t acc0 = 0, acc1 = 0;
    for (int i = 0; i < iters; ++i) {
        uint32_t p[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t x = b[k] ^ (uint32_t)i;
            asm volatile("popc.b32 %0, %1;" : "=r"(p[k]) : "r"(x));
        }
        acc0 += p[0] + p[1];
        acc1 += p[2] + p[3];
        acc0 += p[4] + p[5];
        acc1 += p[6] + p[7];
    }
    out[t] = acc0 + acc1;  // keeps the sums live
}

// Operand feed from L2 into shared memory, the second bound of the tensor form (each SM of a
// pair stages 32 KB of operands per 256-deep K step).  The probe issues the tensor kernel's
// kind of copy: 2D tensor-map loads of 128-row x 128-byte boxes with 128-byte swizzle, two per
// 32 KB stage, kFeedStages stages in flight, one CTA per SM (the stages fill most of its
// shared memory), from an 8192 x 4096-byte matrix (32 MB) that stays in L2; one thread
// re-issues each stage as soon as it lands.  Every wait is bounded: on expiry the thread
// counts it in *err, waits (bounded) for the copies still in flight and returns.
constexpr int kFeedStage = 32768, kFeedStages = 6, kFeedRows = 8192, kFeedRowBytes = 4096;

__global__ void __launch_bounds__(32, 1) feed_probe_kernel(const __grid_constant__ CUtensorMap map, int iters,
                                                           uint64_t limit, unsigned long long *err) {
    extern __shared__ __align__(1024) uint8_t stage[];
    __shared__ __align__(8) uint64_t bar[kFeedStages];
    if (threadIdx.x != 0) return;
    for (int s = 0; s < kFeedStages; ++s) ptx::mbar_init(&bar[s], 1);
    ptx::fence_mbar_init();
    int x = 0, y = (int)((blockIdx.x * 128u) % kFeedRows);
    uint32_t parity[kFeedStages] = {};
    auto issue = [&](int s) {
        ptx::mbar_arrive_expect_tx(&bar[s], kFeedStage);
        const int y2 = (y + kFeedRows / 2) % kFeedRows;
        const uint32_t b = ptx::smem_addr(&bar[s]);
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
                "r"(ptx::smem_addr(stage + (size_t)s * kFeedStage)),
            "l"(&map), "r"(x), "r"(y), "r"(b)
            : "memory");
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
                "r"(ptx::smem_addr(stage + (size_t)s * kFeedStage + kFeedStage / 2)),
            "l"(&map), "r"(x), "r"(y2), "r"(b)
            : "memory");
        x += 128;  // the next 128 bytes of the same rows, then the next 128 rows
        if (x == kFeedRowBytes) {
            x = 0;
            y = (y + 128) % kFeedRows;
        }
    };
    for (int s = 0; s < kFeedStages; ++s) issue(s);
    for (int it = 0; it < iters; ++it)
        for (int s = 0; s < kFeedStages; ++s) {
            if (!ptx::mbar_wait_bounded(&bar[s], parity[s], limit)) {
                atomicAdd(err, 1ull);
                for (int q = 0; q < kFeedStages; ++q) ptx::mbar_wait_bounded(&bar[q], parity[q], limit);
                return;
            }
            parity[s] ^= 1u;
            if (it + 1 < iters) issue(s);
        }
}

}  // namespace
}  // namespace csg

using namespace csg;

extern "C" int csg_measure_popc_rate(int device, double *popc_per_second) {
    if (device < 0 || !popc_per_second) {
        set_error("csg_measure_popc_rate: bad arguments");
        return CSG_E_INVAL;
    }
    CSG_CUDA_TRY(cudaSetDevice(device));
    int sms = 0;
    CSG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const int blocks = 2 * sms, threads = 1024;
    const int iters = 100000;
    uint32_t *out = nullptr;
    if (dev_malloc((void **)&out, (size_t)blocks * threads * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        set_error("csg_measure_popc_rate: allocation failed");
        return CSG_E_NOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = CSG_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = CSG_E_CUDA;
    float ms = 0.f;
    if (rc == CSG_OK) {
        popc_probe_kernel<<<blocks, threads>>>(1u, 1000, out);  // warm-up
        cudaEventRecord(e0);
        popc_probe_kernel<<<blocks, threads>>>(2u, iters, out);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
            rc = CSG_E_CUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (rc != CSG_OK) {
        set_error("csg_measure_popc_rate: the probe failed");
        return rc;
    }
    *popc_per_second = (double)blocks * threads * (double)iters * 8.0 / (ms * 1e-3);
    return CSG_OK;
}

extern "C" int csg_measure_l2_feed(int device, double *bytes_per_sm_per_second) {
    if (device < 0 || !bytes_per_sm_per_second) {
        set_error("csg_measure_l2_feed: bad arguments");
        return CSG_E_INVAL;
    }
    CSG_CUDA_TRY(cudaSetDevice(device));
    int sms = 0;
    CSG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        set_error("csg_measure_l2_feed: cuTensorMapEncodeTiled is unavailable");
        return CSG_E_CUDA;
    }
    const size_t buf_bytes = (size_t)kFeedRows * kFeedRowBytes;  // 32 MB: stays in L2
    const int smem = kFeedStage * kFeedStages, iters = 400;
    uint8_t *buf = nullptr;
    unsigned long long *err = nullptr;
    if (dev_malloc((void **)&buf, buf_bytes) != cudaSuccess || dev_malloc((void **)&err, 8) != cudaSuccess) {
        cudaGetLastError();
        if (buf) cudaFree(buf);
        set_error("csg_measure_l2_feed: allocation failed");
        return CSG_E_NOMEM;
    }
    CUtensorMap map;
    cuuint64_t dims[2] = {(cuuint64_t)kFeedRowBytes, (cuuint64_t)kFeedRows};
    cuuint64_t strides[1] = {(cuuint64_t)kFeedRowBytes};
    cuuint32_t box[2] = {128, 128};
    cuuint32_t estr[2] = {1, 1};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = CSG_OK;
    float ms = 0.f;
    unsigned long long h_err = 0;
    if (reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn)(
            &map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS ||
        cudaMemset(buf, 1, buf_bytes) != cudaSuccess || cudaMemset(err, 0, 8) != cudaSuccess ||
        cudaFuncSetAttribute(feed_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = CSG_E_CUDA;
    if (rc == CSG_OK) {
        const uint64_t limit = wait_limit_ns(2000000000ull);
        feed_probe_kernel<<<sms, 32, smem>>>(map, 20, limit, err);  // warm-up: the matrix into L2
        cudaEventRecord(e0);
        feed_probe_kernel<<<sms, 32, smem>>>(map, iters, limit, err);
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
    cudaFree(buf);
    cudaFree(err);
    if (rc != CSG_OK) {
        set_error(rc == CSG_E_TIMEOUT ? "csg_measure_l2_feed: a bounded wait expired"
                                      : "csg_measure_l2_feed: the probe failed");
        return rc;
    }
    *bytes_per_sm_per_second = (double)iters * kFeedStages * kFeedStage / (ms * 1e-3);
    return CSG_OK;
}
