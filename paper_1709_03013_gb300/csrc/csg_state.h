// Host-side state behind the opaque handles of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <set>

#include "../../include/csg.h"

struct csg_set {
    csg_ctx *ctx = nullptr;
    int d = 0;
    int64_t N = 0;
    int64_t stride = 0;          // words per bitmap row
    double *coords = nullptr;    // [4][N] sorted coordinates (device)
    uint64_t *rows = nullptr;    // N x stride bitmap words (device)
    size_t bytes = 0;            // charged against the context budget
    bool linked = false;
    bool from_bitmap = false;
    double coord_scale = 1.0;    // max(1, max |coordinate|)
    int geom = 0;                // 0: flat diamond of dimension d; 3: 1+1 de Sitter slab
    cudaStream_t stream = nullptr;      // the stream the set was created on; its memory is freed there
    unsigned long long *err = nullptr;  // device word after the coordinates: nonzero if the sprinkle failed
};

namespace csg {
struct ServeState;
struct StageTimer;
struct BatchGraph;
}

struct csg_ctx {
    int device = 0;
    size_t budget = 0;  // 0 = unlimited
    size_t used = 0;
    std::mutex mu;      // guards used and sets
    std::set<csg_set *> sets;
    std::mutex serve_mu;
    csg::ServeState *serve = nullptr;
    csg::StageTimer *timer = nullptr;  // per-stage CUDA events when timing is on
    csg::BatchGraph *batch = nullptr;  // the last batch's captured graph and memory
};

namespace csg {

int alloc_set(csg_ctx *ctx, int d, int64_t N, csg_set **out, cudaStream_t st);
void free_set(csg_set *s, bool device_synced = false);

// Action for n linked sets; writes n host results and synchronises st.
// Interval-count methods of the ABI and the tensor operand format each one selects.
inline bool method_ok(int m) { return m == CSG_POPC || m == CSG_TC || m == CSG_TC_FP8 || m == CSG_TC_FP4; }
constexpr int kTcDefaultFmt = 1;  // format of CSG_TC: 0 fp8, 1 fp4 (measured faster on GB300)
inline int tc_format(int m) { return m == CSG_TC_FP4 ? 1 : (m == CSG_TC_FP8 ? 0 : kTcDefaultFmt); }
int run_dalembertian(csg_set *set, int method, const double *phi, double l, double *Bphi, csg_result *out,
                     cudaStream_t st);
int run_actions(csg_set *const *sets, int n, int method, int64_t row_lo, int64_t row_hi,
                unsigned long long *dev_hist, int64_t nbins, csg_result *out, cudaStream_t st);

// Sprinkle + sort + link + action for n allocated sets with the given seeds, all
// steps batched across the sets; synchronises st.
int run_pipeline(csg_set *const *sets, int n, const uint64_t *seed, const uint64_t *seq, int method,
                 csg_result *out, cudaStream_t st);

void serve_shutdown(csg_ctx *ctx);
int run_smeared(csg_set *set, int method, double eps, double *S_eps, csg_result *out, cudaStream_t st);
void free_batch_graph(csg_ctx *ctx);
int run_batch_graph(csg_ctx *ctx, int n, const int32_t *d, const int64_t *N, const uint64_t *seed,
                    const uint64_t *seq, int method, csg_result *out, cudaStream_t st);
void destroy_timer(csg_ctx *ctx);

// Makes the context's stage timer (if any) current for the calling thread.
struct TimerScope {
    explicit TimerScope(csg_ctx *ctx);
    ~TimerScope();
    StageTimer *prev;
};

}  // namespace csg
