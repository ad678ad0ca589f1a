// Throughput probe of the population-count pipe, the bound of the popcount interval counts
// (CSG_POPC: one 32-bit popcount per 32 candidate bits of every related pair's range).
//
// Every thread runs `iters` iterations of eight independent 32-bit popcounts (popc.b32) of
// values that change every iteration, summed with three-input adds, so the popcount pipe
// is the busiest one.  Two CTAs of 1024 threads per SM.  The result is popcounts per second
// over the whole GPU; divided by the SM count and the clock it gives the pipe's results per
// SM per clock (16 in the CUDA programming guide's throughput table).
#include <cuda_runtime.h>
#include <stdint.h>

#include "csg_internal.cuh"

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
