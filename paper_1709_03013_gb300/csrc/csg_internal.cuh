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
#include "arena.h"

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
    CNT_ERR,  // nonzero: CNT_ERR_TIMEOUT (a bounded device wait expired) or CNT_ERR_REJECT
    CNT_WORDS = 8
};
constexpr unsigned long long CNT_ERR_TIMEOUT = 1, CNT_ERR_REJECT = 2;

// One set as the kernels see it.
struct SetDesc {
    const uint64_t *rows;  // N x stride words
    int64_t N;
    int64_t stride;        // words per row
    unsigned long long *counters;  // CNT_WORDS counters
    int64_t row_lo, row_hi;        // first elements i counted: [row_lo, row_hi)
    // Optional d'Alembertian sums (Eq. b_local): for every related pair i < j with
    // m(i,j) <= 2, acc[j] += c_m phi[i] with c = (1, -2, 1); null when not wanted.
    const double *phi;
    double *acc;
};

// A unit of action work: rows [i0, i0 + G) of set `set`.
struct WorkItem {
    int32_t set;
    int32_t pad;
    int64_t i0;
};

// ---------------------------------------------------------------- kernels

// Sprinkle + sort for a batch of sets sharing one launch sequence.
// Geometry of a set: the flat diamonds (d = 2 or 4) or the 1+1 de Sitter slab of Sec. 5.1.
constexpr int GEOM_DS2 = 3;

struct SprinkleSpec {
    int32_t d;
    int32_t geom;              // 2, 4 or GEOM_DS2 (0: same as d)
    int64_t N;
    uint64_t seed, seq;
    double *coords;            // [4][N] sorted output
    unsigned long long *err;   // per-set error word (the set's CNT_ERR), or null
    double param;              // GEOM_DS2: tan(eta0)
};
struct SprinklePlan {
    int n = 0;
    int64_t E = 0, C = 0, maxN = 0;
    bool from_coords = false;
    size_t t_rows = 0, t_starts = 0, t_cstarts = 0;
    size_t s_tmp = 0, s_keys = 0, s_idx = 0, s_err = (size_t)-1;
    size_t s_counters = (size_t)-1;  // when set: set s reports into its counters' CNT_ERR
};
SprinklePlan sprinkle_plan(const SprinkleSpec *specs, int n, Arena &a, bool from_coords,
                           size_t s_counters = (size_t)-1);
void sprinkle_patch(const SprinklePlan &p, Arena &a);  // after allocation, before upload
void sprinkle_launch(const SprinklePlan &p, const Arena &a, cudaStream_t st);
// standalone: allocate, run and (sync) synchronise; host_coords (optional) replaces the
// sprinkle.  Without sync every spec must carry its own error word.
int sprinkle_sort_batch(const SprinkleSpec *specs_host, int n, cudaStream_t st,
                        const double *const *host_coords /*null: sprinkle*/, bool sync = true);

// Link a batch of sets (coords -> rows).
struct LinkSpec {
    int32_t d;  // geometry: 2, 4 or GEOM_DS2
    int32_t pad;
    int64_t N;
    int64_t stride;
    const double *coords;
    uint64_t *rows;
    int64_t tile_off;    // unused by callers (filled by the plan)
    double coord_scale;  // max(1, max |coordinate|): scales the d=4 float-screen margin
};
struct LinkPlan {
    struct Part {  // the sets of one geometry (part 0: d=2, 1: d=4, 2: 1+1 de Sitter)
        int n = 0;
        int64_t T = 0, E = 0;  // CTAs of the link kernel, elements
        int64_t RB = 0;        // d=2: row blocks, each sorted once by the pre-pass
        size_t t_rows = 0, t_starts = 0, t_estarts = 0, t_rbstarts = 0;
    } part[3];
    int64_t T = 0;
    size_t s_screen = 0;  // scratch: per-element float screen values of every set
    size_t s_sorted = 0;  // scratch: d=2 row blocks in u and v order
};
LinkPlan link_plan(const LinkSpec *specs, int n, Arena &a, int *rc);
void link_launch(const LinkPlan &p, const Arena &a, cudaStream_t st);
int link_batch(const LinkSpec *specs_host, int n, cudaStream_t st);

// Arena helpers (stream-ordered allocation; upload of the table image)
int arena_alloc(Arena &a, cudaStream_t st);
void arena_upload(Arena &a, cudaStream_t st);
void arena_free(Arena &a, cudaStream_t st);

// Popcount action over a list of sets.  Per-set counters live in the arena's scratch
// at s_counters (CNT_WORDS per set) and must be zeroed before the launch.
struct PopcPlan {
    std::vector<int> slot;  // counter slot of each set (empty: identity)
    int n_sets = 0, n_items = 0, G = 16, pitch = 0;
    bool phi = false;  // some set wants d'Alembertian sums (selects the kernel variant)
    size_t t_sets = 0, t_items = 0, s_queue = 0, s_counters = 0;
    unsigned long long *hist = nullptr;
    int64_t nbins = 0;
};
PopcPlan popc_plan(const SetDesc *sets, int n, Arena &a, size_t s_counters, unsigned long long *hist,
                   int64_t nbins, int *rc, const int *slots = nullptr);
void popc_patch(const PopcPlan &p, Arena &a);
int popc_launch(const PopcPlan &p, const Arena &a, cudaStream_t st);

// Tensor-core action (masked 0/1 product on tcgen05), many sets per launch.
struct TcSetDesc {
    const uint64_t *rows;
    int64_t N, stride, row_lo, row_hi;
    unsigned long long *counters;
    uint8_t *U, *P;  // 0/1 operands (strict future rows, strict past rows), N x kp bytes
    int64_t kp;      // operand row bytes: N rounded up to 128 (fp8) or to 256 elements / 2 (fp4)
    const double *phi;  // optional d'Alembertian sums, as in SetDesc
    double *acc;
};
struct TcPlan {
    struct Chunk {
        int set_lo = 0, set_hi = 0, n_tiles = 0;
        int64_t rows = 0;  // operand rows the expand pass writes (sum of N)
        size_t t_rstarts = 0, t_tiles = 0;
    };
    std::vector<int> slot;  // counter slot of each set (empty: identity)
    int n_sets = 0;
    int fmt = 0;            // operand format: 0 fp8 e4m3 (two TMEM accumulators), 1 fp4 e2m1 (block-scaled, one)
    size_t t_sets = 0, t_maps = 0, s_ops = 0, s_counters = 0, s_queues = 0;
    unsigned long long *hist = nullptr;
    int64_t nbins = 0;
    std::vector<Chunk> chunks;
};
// super: side of the square blocks (in elements) in which output tiles are rasterised
TcPlan tc_plan(const SetDesc *sets, int n, Arena &a, size_t s_counters, unsigned long long *hist,
               int64_t nbins, int *rc, const int *slots = nullptr, int super = 4096, int fmt = 0);
int tc_patch(const TcPlan &p, Arena &a);
int tc_launch(const TcPlan &p, const Arena &a, cudaStream_t st);

// ---------------------------------------------------------------- checked build
//
// The bounds-checked build (compiled with -DCSG_CHECKED; compute-sanitizer is not available
// to this project): CSG_IN_BOUNDS(cond, site, value) guards a memory access whose index the
// kernel computed.  In the checked build a false condition records the first failure of this
// translation unit -- the site number in the top 16 bits, the low 48 bits of the offending
// value below -- in a device word, and the access it guards is skipped; the host reads and
// clears the words with csg_check_words.  In the normal build the macro is `true` and
// compiles away.
#ifdef CSG_CHECKED
static __device__ unsigned long long g_csg_check;
__device__ __forceinline__ bool csg_in_bounds(bool ok, unsigned site, long long v) {
    if (!ok)
        atomicCAS(&g_csg_check, 0ull,
                  ((unsigned long long)site << 48) | ((unsigned long long)v & 0xFFFFFFFFFFFFull));
    return ok;
}
#define CSG_IN_BOUNDS(cond, site, v) ::csg::csg_in_bounds((cond), (site), (long long)(v))
// this translation unit's check word, read and cleared (host side)
static inline unsigned long long take_check_word() {
    unsigned long long v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_csg_check, sizeof v) != cudaSuccess) v = ~0ull;
    cudaMemcpyToSymbol(g_csg_check, &z, sizeof z);
    return v;
}
#else
#define CSG_IN_BOUNDS(cond, site, v) true
static inline unsigned long long take_check_word() { return 0; }
#endif
// Check words of the kernel groups, one per translation unit (0: no failure).
unsigned long long check_word_sprinkle();
unsigned long long check_word_link();
unsigned long long check_word_popc();
unsigned long long check_word_tc();
unsigned long long check_word_pipeline();
unsigned long long check_word_noalloc();

// ---------------------------------------------------------------- errors

void set_error(const char *fmt, ...);

// Failure injection for the library's own tests (csg_test_wait_expiry, csg_test_fail_alloc);
// process-wide and off by default.
struct TestHooks {
    std::atomic<unsigned long long> wait_ns{0};  // nonzero: limit of every bounded device wait
    std::atomic<int> starve{0};                  // producers skip the copies of their first stage
    std::atomic<int> fail_alloc{0};              // the next n device allocations fail
};
TestHooks &test_hooks();
// The wait limit a kernel launch gets: the test setting, else the kernel's own default.
inline unsigned long long wait_limit_ns(unsigned long long dflt) {
    const unsigned long long t = test_hooks().wait_ns.load(std::memory_order_relaxed);
    return t ? t : dflt;
}
inline int starve_first_stage() { return test_hooks().starve.load(std::memory_order_relaxed); }
// cudaMallocAsync / cudaMalloc, or cudaErrorMemoryAllocation while an injected failure count lasts.
cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t st);
cudaError_t dev_malloc(void **p, size_t bytes);

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
    return dev_malloc_async((void **)p, count * sizeof(T), st);
}

}  // namespace csg
