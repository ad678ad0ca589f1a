// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/csg.h"

namespace csg {

// ---------------------------------------------------------------- layout

// Row stride of a bitmap: ceil(N/64) words rounded up to 16 words (128 bytes), so
// every row starts on a 128-byte boundary for coalesced and bulk-copy access.
inline int64_t stride_for(int64_t N) {
    int64_t w = (N + 63) / 64;
    int64_t s = (w + 15) / 16 * 16;
    return s < 16 ? 16 : s;
}

// Counters written by the action kernels, one block per set (uint64 each).
enum : int {
    CNT_N0 = 0,
    CNT_N1,
    CNT_N2,
    CNT_N3,
    CNT_R,
    CNT_SUM_M,
    CNT_W,
    CNT_ERR,  // nonzero: a bounded device wait expired or an invariant failed
    CNT_WORDS = 8
};

// One set as the kernels see it.
struct SetDesc {
    const uint64_t *rows;  // N x stride words
    int64_t N;
    int64_t stride;        // words per row
    unsigned long long *counters;  // CNT_WORDS counters
    int64_t row_lo, row_hi;        // first elements i counted: [row_lo, row_hi)
};

// A unit of action work: rows [i0, i0 + G) of set `set`.
struct WorkItem {
    int32_t set;
    int32_t pad;
    int64_t i0;
};

// ---------------------------------------------------------------- kernels

// Sprinkle + sort for a batch of sets sharing one launch sequence.  coords[s] is
// [4][N_s] doubles (sorted output); seeds per set.  Returns CSG_OK or an error.
struct SprinkleSpec {
    int32_t d;
    int32_t pad;
    int64_t N;
    uint64_t seed, seq;
    double *coords;     // [4][N] sorted output
    int64_t key_off;    // offset of this set in the batch's sort arrays
};
int sprinkle_sort_batch(const SprinkleSpec *specs_host, int n, cudaStream_t st,
                        const double *const *host_coords /*null: sprinkle*/);

// Link a batch of sets (coords -> rows).
struct LinkSpec {
    int32_t d;
    int32_t pad;
    int64_t N;
    int64_t stride;
    const double *coords;
    uint64_t *rows;
    int64_t tile_off;  // first tile index of this set in the batch's tile space
    double coord_scale;  // max(1, max |coordinate|): scales the d=4 float-screen margin
};
int link_batch(const LinkSpec *specs_host, int n, cudaStream_t st);

// Popcount action over a list of sets.  counters must be zeroed by the caller.
// items == nullptr: one set, items implicit over its row range.
int action_popc(const SetDesc *sets_host, int n_sets, cudaStream_t st,
                unsigned long long *dev_hist, int64_t nbins);

// Tensor-core action (masked 0/1 product on tcgen05).  counters must be zeroed by
// the caller; dev_hist (optional) receives the full interval-size histogram.
int action_tc(const SetDesc *sets_host, int n_sets, cudaStream_t st, unsigned long long *dev_hist,
              int64_t nbins);

// ---------------------------------------------------------------- errors

void set_error(const char *fmt, ...);

// Stage timing hooks (no-ops unless a TimerScope with timing on is active).
void stage_begin(int stage, cudaStream_t st);
void stage_end(int stage, cudaStream_t st);
#define CSG_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t _e = (expr);                                                        \
        if (_e != cudaSuccess) {                                                        \
            ::csg::set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr,                 \
                             cudaGetErrorString(_e));                                   \
            return CSG_E_CUDA;                                                          \
        }                                                                               \
    } while (0)

// Device scratch owned by the caller of a launch sequence: allocated per call
// with the stream-ordered allocator.
template <typename T>
inline cudaError_t stream_alloc(T **p, size_t count, cudaStream_t st) {
    return cudaMallocAsync((void **)p, count * sizeof(T), st);
}

}  // namespace csg
