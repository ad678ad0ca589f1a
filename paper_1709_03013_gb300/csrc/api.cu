// C ABI: contexts, sets, and the single-set and batch entry points.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <set>

#include "csg_internal.cuh"
#include "csg_state.h"

namespace csg {

static thread_local char g_last_error[512];

TestHooks &test_hooks() {
    static TestHooks h;
    return h;
}

static bool injected_alloc_failure() {
    std::atomic<int> &n = test_hooks().fail_alloc;
    int v = n.load();
    while (v > 0)
        if (n.compare_exchange_weak(v, v - 1)) return true;
    return false;
}

cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t st) {
    if (injected_alloc_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocAsync(p, bytes, st);
}

cudaError_t dev_malloc(void **p, size_t bytes) {
    if (injected_alloc_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
}

// ------------------------------------------------------------------ sets

// Set memory comes from the stream-ordered pool on the creating stream (no device-wide
// synchronisation on free); a word after the coordinates carries the sprinkle's error flag.
int alloc_set(csg_ctx *ctx, int d, int64_t N, csg_set **out, cudaStream_t st) {
    if (!ctx || !out || (d != 2 && d != 4) || N < 1 || N > CSG_MAX_N) {
        set_error("bad set arguments (d=%d, N=%lld)", d, (long long)N);
        return CSG_E_INVAL;
    }
    csg_set *s = new csg_set();
    s->ctx = ctx;
    s->d = d;
    s->N = N;
    s->stride = stride_for(N);
    s->bytes = (size_t)N * 4 * sizeof(double) + (size_t)N * s->stride * sizeof(uint64_t);
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        if (ctx->budget && ctx->used + s->bytes > ctx->budget) {
            set_error("set of %zu bytes exceeds the context budget", s->bytes);
            delete s;
            return CSG_E_NOMEM;
        }
        ctx->used += s->bytes;
    }
    s->stream = st;
    cudaError_t e1 = dev_malloc_async((void **)&s->coords, (size_t)N * 4 * sizeof(double) + 256, st);
    cudaError_t e2 = dev_malloc_async((void **)&s->rows, (size_t)N * s->stride * sizeof(uint64_t), st);
    if (e1 == cudaSuccess && e2 == cudaSuccess) {
        s->err = reinterpret_cast<unsigned long long *>(s->coords + (size_t)N * 4);
        e1 = cudaMemsetAsync(s->err, 0, sizeof(unsigned long long), st);
    }
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        if (s->coords) cudaFreeAsync(s->coords, st);
        if (s->rows) cudaFreeAsync(s->rows, st);
        {
            std::lock_guard<std::mutex> g(ctx->mu);
            ctx->used -= s->bytes;
        }
        delete s;
        cudaGetLastError();
        set_error("device allocation of a set with N=%lld failed", (long long)N);
        return CSG_E_NOMEM;
    }
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->sets.insert(s);
    }
    *out = s;
    return CSG_OK;
}

void free_set(csg_set *s, bool device_synced) {
    if (!s) return;
    csg_ctx *ctx = s->ctx;
    cudaSetDevice(ctx->device);
    // stream-ordered on the creating stream; after a device-wide synchronisation (context
    // teardown, where that stream may no longer exist) on the legacy stream instead
    cudaStream_t st = device_synced ? nullptr : s->stream;
    if (s->coords) cudaFreeAsync(s->coords, st);
    if (s->rows) cudaFreeAsync(s->rows, st);
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->used -= s->bytes;
        ctx->sets.erase(s);
    }
    delete s;
}

}  // namespace csg

using namespace csg;

extern "C" {

const char *csg_strerror(int code) {
    switch (code) {
        case CSG_OK: return "ok";
        case CSG_PENDING: return "pending";
        case CSG_E_INVAL: return "invalid argument";
        case CSG_E_NOMEM: return "out of device memory or over budget";
        case CSG_E_CUDA: return "CUDA error";
        case CSG_E_TIMEOUT: return "bounded wait expired";
        case CSG_E_BUSY: return "service queue full";
        case CSG_E_REJECT: return "rejection sampling cap reached";
        case CSG_E_NOTFOUND: return "unknown ticket";
        case CSG_E_CANCELLED: return "request cancelled";
        default: return "unknown error";
    }
}

const char *csg_last_error(void) { return g_last_error; }

int csg_init(int device, size_t hbm_budget_bytes, csg_ctx **out) {
    if (!out || device < 0) {
        set_error("csg_init: bad arguments");
        return CSG_E_INVAL;
    }
    int count = 0;
    CSG_CUDA_TRY(cudaGetDeviceCount(&count));
    if (device >= count) {
        set_error("csg_init: device %d of %d", device, count);
        return CSG_E_INVAL;
    }
    CSG_CUDA_TRY(cudaSetDevice(device));
    // keep stream-ordered scratch (the tensor form's operands) cached between calls
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    csg_ctx *c = new csg_ctx();
    c->device = device;
    c->budget = hbm_budget_bytes;
    c->used = 0;
    *out = c;
    return CSG_OK;
}

void csg_finalize(csg_ctx *ctx) {
    if (!ctx) return;
    serve_shutdown(ctx);
    cudaSetDevice(ctx->device);
    destroy_timer(ctx);
    free_batch_graph(ctx);
    std::vector<csg_set *> all;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        all.assign(ctx->sets.begin(), ctx->sets.end());
    }
    cudaDeviceSynchronize();
    for (csg_set *s : all) free_set(s, true);
    cudaDeviceSynchronize();
    delete ctx;
}

int csg_sprinkle(csg_ctx *ctx, int d, int64_t N, uint64_t seed, uint64_t seq, void *stream,
                 csg_set **out) {
    if (!ctx) return CSG_E_INVAL;
    TimerScope ts(ctx);
    CSG_CUDA_TRY(cudaSetDevice(ctx->device));
    csg_set *s = nullptr;
    int rc = alloc_set(ctx, d, N, &s, (cudaStream_t)stream);
    if (rc != CSG_OK) return rc;
    SprinkleSpec sp{d, 0, N, seed, seq, s->coords, s->err};
    rc = sprinkle_sort_batch(&sp, 1, (cudaStream_t)stream, nullptr, /*sync=*/false);
    if (rc != CSG_OK) {
        free_set(s);
        return rc;
    }
    s->coord_scale = 1.0;
    *out = s;
    return CSG_OK;
}

int csg_sprinkle_desitter(csg_ctx *ctx, int64_t N, double eta0, uint64_t seed, uint64_t seq,
                          void *stream, csg_set **out) {
    if (!ctx || !out || !(eta0 > 0.0 && eta0 < 1.5707963267948966)) {
        set_error("csg_sprinkle_desitter: bad arguments (0 < eta0 < pi/2)");
        return CSG_E_INVAL;
    }
    TimerScope ts(ctx);
    CSG_CUDA_TRY(cudaSetDevice(ctx->device));
    csg_set *s = nullptr;
    int rc = alloc_set(ctx, 2, N, &s, (cudaStream_t)stream);
    if (rc != CSG_OK) return rc;
    s->geom = GEOM_DS2;
    SprinkleSpec sp{2, GEOM_DS2, N, seed, seq, s->coords, s->err, tan(eta0)};
    rc = sprinkle_sort_batch(&sp, 1, (cudaStream_t)stream, nullptr, /*sync=*/false);
    if (rc != CSG_OK) {
        free_set(s);
        return rc;
    }
    *out = s;
    return CSG_OK;
}

int csg_set_from_coords(csg_ctx *ctx, int d, int64_t N, const double *host_coords, void *stream,
                        csg_set **out) {
    if (!ctx || !host_coords) {
        set_error("csg_set_from_coords: null argument");
        return CSG_E_INVAL;
    }
    TimerScope ts(ctx);
    double scale = 1.0;
    for (int64_t q = 0; q < 4 * N; ++q) {
        double a = fabs(host_coords[q]);
        if (!(a <= 1e15)) {
            set_error("csg_set_from_coords: coordinate %lld is not finite or exceeds 1e15",
                      (long long)q);
            return CSG_E_INVAL;
        }
        if (a > scale) scale = a;
    }
    CSG_CUDA_TRY(cudaSetDevice(ctx->device));
    csg_set *s = nullptr;
    int rc = alloc_set(ctx, d, N, &s, (cudaStream_t)stream);
    if (rc != CSG_OK) return rc;
    SprinkleSpec sp{d, 0, N, 0, 0, s->coords, nullptr};
    const double *hc[1] = {host_coords};
    rc = sprinkle_sort_batch(&sp, 1, (cudaStream_t)stream, hc);
    if (rc != CSG_OK) {
        free_set(s);
        return rc;
    }
    s->coord_scale = scale;
    *out = s;
    return CSG_OK;
}

int csg_link(csg_ctx *ctx, csg_set *set, void *stream) {
    if (!ctx || !set || set->ctx != ctx) {
        set_error("csg_link: bad handle");
        return CSG_E_INVAL;
    }
    if (set->from_bitmap) {
        set_error("csg_link: set was made from a bitmap and has no coordinates");
        return CSG_E_INVAL;
    }
    CSG_CUDA_TRY(cudaSetDevice(ctx->device));
    TimerScope ts(ctx);
    LinkSpec L{set->geom ? set->geom : set->d, 0, set->N, set->stride, set->coords, set->rows, 0,
               set->coord_scale};
    int rc = link_batch(&L, 1, (cudaStream_t)stream);
    if (rc == CSG_OK) set->linked = true;
    return rc;
}

int csg_set_from_bitmap(csg_ctx *ctx, int d, int64_t N, const uint64_t *dev_rows,
                        int64_t stride_words, void *stream, csg_set **out) {
    if (!ctx || !dev_rows || !out || stride_words < (N + 63) / 64) {
        set_error("csg_set_from_bitmap: bad arguments");
        return CSG_E_INVAL;
    }
    CSG_CUDA_TRY(cudaSetDevice(ctx->device));
    csg_set *s = nullptr;
    int rc = alloc_set(ctx, d, N, &s, (cudaStream_t)stream);
    if (rc != CSG_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t wN = (N + 63) / 64;
    cudaError_t e = cudaMemsetAsync(s->rows, 0, (size_t)N * s->stride * sizeof(uint64_t), st);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(s->rows, s->stride * sizeof(uint64_t), dev_rows,
                              stride_words * sizeof(uint64_t), wN * sizeof(uint64_t), N,
                              cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->coords, 0, (size_t)N * 4 * sizeof(double), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_error("csg_set_from_bitmap: %s", cudaGetErrorString(e));
        free_set(s);
        return CSG_E_CUDA;
    }
    s->linked = true;
    s->from_bitmap = true;
    *out = s;
    return CSG_OK;
}

static int action_common(csg_ctx *ctx, csg_set *set, int method, int64_t lo, int64_t hi,
                         unsigned long long *hist, int64_t nbins, csg_result *out, void *stream) {
    if (!ctx || !set || !out || set->ctx != ctx || !method_ok(method)) {
        set_error("csg_action: bad arguments");
        return CSG_E_INVAL;
    }
    if (!set->linked) {
        set_error("csg_action: set has no bitmap (call csg_link)");
        return CSG_E_INVAL;
    }
    CSG_CUDA_TRY(cudaSetDevice(ctx->device));
    TimerScope ts(ctx);
    csg_set *one[1] = {set};
    return run_actions(one, 1, method, lo, hi, hist, nbins, out, (cudaStream_t)stream);
}

int csg_action(csg_ctx *ctx, csg_set *set, int method, csg_result *out, void *stream) {
    return action_common(ctx, set, method, -1, -1, nullptr, 0, out, stream);
}

int csg_action_rows(csg_ctx *ctx, csg_set *set, int method, int64_t row_lo, int64_t row_hi,
                    csg_result *out, void *stream) {
    if (row_lo < 0 || row_hi < row_lo) {
        set_error("csg_action_rows: bad row range");
        return CSG_E_INVAL;
    }
    return action_common(ctx, set, method, row_lo, row_hi, nullptr, 0, out, stream);
}

int csg_action_hist(csg_ctx *ctx, csg_set *set, int method, uint64_t *dev_hist, int64_t nbins,
                    csg_result *out, void *stream) {
    if (!dev_hist || nbins < 1) {
        set_error("csg_action_hist: bad histogram");
        return CSG_E_INVAL;
    }
    if (cudaMemsetAsync(dev_hist, 0, nbins * sizeof(uint64_t), (cudaStream_t)stream) != cudaSuccess) {
        set_error("csg_action_hist: histogram memset failed");
        return CSG_E_CUDA;
    }
    return action_common(ctx, set, method, -1, -1, (unsigned long long *)dev_hist, nbins, out,
                         stream);
}

int csg_action_smeared(csg_ctx *ctx, csg_set *set, int method, double eps, double *S_eps,
                       csg_result *out, void *stream) {
    if (!ctx || !set || !S_eps || set->ctx != ctx || !method_ok(method) ||
        !(eps > 0.0 && eps < 1.0)) {
        set_error("csg_action_smeared: bad arguments (0 < eps < 1, method POPC or TC)");
        return CSG_E_INVAL;
    }
    if (set->d != 2) {
        set_error("csg_action_smeared: the smeared action is defined here for d=2 only");
        return CSG_E_INVAL;
    }
    if (!set->linked) {
        set_error("csg_action_smeared: set has no bitmap (call csg_link)");
        return CSG_E_INVAL;
    }
    CSG_CUDA_TRY(cudaSetDevice(ctx->device));
    TimerScope ts(ctx);
    return run_smeared(set, method, eps, S_eps, out, (cudaStream_t)stream);
}

int csg_dalembertian(csg_ctx *ctx, csg_set *set, int method, const double *phi, double l, double *Bphi,
                     csg_result *out, void *stream) {
    if (!ctx || !set || set->ctx != ctx || !phi || !Bphi || !method_ok(method) ||
        !(l > 0.0 && l < INFINITY)) {
        set_error("csg_dalembertian: bad arguments (device phi and Bphi, 0 < l < inf, method POPC or TC)");
        return CSG_E_INVAL;
    }
    if (set->d != 2) {
        set_error("csg_dalembertian: the d'Alembertian of Eq. b_local is defined for 1+1 sets only");
        return CSG_E_INVAL;
    }
    if (!set->linked) {
        set_error("csg_dalembertian: set has no bitmap (call csg_link)");
        return CSG_E_INVAL;
    }
    const uintptr_t a0 = (uintptr_t)phi, b0 = (uintptr_t)Bphi, len = (uintptr_t)set->N * sizeof(double);
    if (a0 < b0 + len && b0 < a0 + len) {
        set_error("csg_dalembertian: phi and Bphi overlap");
        return CSG_E_INVAL;
    }
    CSG_CUDA_TRY(cudaSetDevice(ctx->device));
    TimerScope ts(ctx);
    return run_dalembertian(set, method, phi, l, Bphi, out, (cudaStream_t)stream);
}

int csg_action_batch(csg_ctx *ctx, csg_set *const *sets, int n, int method, csg_result *out,
                     void *stream) {
    if (!ctx || (n > 0 && (!sets || !out)) || n < 0 || !method_ok(method)) {
        set_error("csg_action_batch: bad arguments");
        return CSG_E_INVAL;
    }
    for (int s = 0; s < n; ++s)
        if (!sets[s] || sets[s]->ctx != ctx || !sets[s]->linked) {
            set_error("csg_action_batch: set %d is not a linked set of this context", s);
            return CSG_E_INVAL;
        }
    CSG_CUDA_TRY(cudaSetDevice(ctx->device));
    TimerScope ts(ctx);
    return run_actions(sets, n, method, -1, -1, nullptr, 0, out, (cudaStream_t)stream);
}

int csg_run_batch(csg_ctx *ctx, int n, const int32_t *d, const int64_t *N, const uint64_t *seed,
                  const uint64_t *seq, int method, csg_result *out, void *stream) {
    if (!ctx || n < 0 || (n > 0 && (!d || !N || !seed || !seq || !out))) {
        set_error("csg_run_batch: bad arguments");
        return CSG_E_INVAL;
    }
    for (int s = 0; s < n; ++s)
        if ((d[s] != 2 && d[s] != 4) || N[s] < 1 || N[s] > CSG_MAX_N) {
            set_error("csg_run_batch: bad spec %d (d=%d, N=%lld)", s, d[s], (long long)N[s]);
            return CSG_E_INVAL;
        }
    if (!method_ok(method)) {
        set_error("csg_run_batch: bad method");
        return CSG_E_INVAL;
    }
    CSG_CUDA_TRY(cudaSetDevice(ctx->device));
    if (n == 0) return CSG_OK;
    return run_batch_graph(ctx, n, d, N, seed, seq, method, out, (cudaStream_t)stream);
}

// The sprinkle of a set reports a rejection-cap failure in the set's error word; calls
// that read the set back check it after they synchronise.
static int check_set_err(const csg_set *set) {
    unsigned long long e = 0;
    CSG_CUDA_TRY(cudaMemcpy(&e, set->err, sizeof e, cudaMemcpyDeviceToHost));
    if (e != 0) {
        set_error("sprinkle: an element hit the 256-attempt rejection cap");
        return CSG_E_REJECT;
    }
    return CSG_OK;
}

int csg_export_coords(csg_set *set, double *host, size_t cap) {
    if (!set || !host || cap < (size_t)(4 * set->N)) {
        set_error("csg_export_coords: bad arguments");
        return CSG_E_INVAL;
    }
    CSG_CUDA_TRY(cudaSetDevice(set->ctx->device));
    CSG_CUDA_TRY(cudaDeviceSynchronize());
    CSG_CUDA_TRY(cudaMemcpy(host, set->coords, 4 * set->N * sizeof(double), cudaMemcpyDeviceToHost));
    return check_set_err(set);
}

int csg_export_bitmap(csg_set *set, uint64_t *host, size_t cap) {
    if (!set || !host || cap < (size_t)(set->N * set->stride)) {
        set_error("csg_export_bitmap: bad arguments");
        return CSG_E_INVAL;
    }
    if (!set->linked) {
        set_error("csg_export_bitmap: set has no bitmap");
        return CSG_E_INVAL;
    }
    CSG_CUDA_TRY(cudaSetDevice(set->ctx->device));
    CSG_CUDA_TRY(cudaDeviceSynchronize());
    CSG_CUDA_TRY(cudaMemcpy(host, set->rows, set->N * set->stride * sizeof(uint64_t),
                            cudaMemcpyDeviceToHost));
    return check_set_err(set);
}

int csg_set_info(const csg_set *set, int *d, int64_t *N, int64_t *stride_words,
                 const uint64_t **dev_rows, const double **dev_coords) {
    if (!set) return CSG_E_INVAL;
    if (d) *d = set->d;
    if (N) *N = set->N;
    if (stride_words) *stride_words = set->stride;
    if (dev_rows) *dev_rows = set->rows;
    if (dev_coords) *dev_coords = set->coords;
    return CSG_OK;
}

void csg_set_free(csg_set *set) { free_set(set); }

int csg_check_words(uint64_t *words, int n) {
    if (!words || n < 0) {
        set_error("csg_check_words: bad arguments");
        return CSG_E_INVAL;
    }
#ifdef CSG_CHECKED
    cudaDeviceSynchronize();
    const unsigned long long w[6] = {check_word_sprinkle(), check_word_link(), check_word_popc(),
                                     check_word_tc(), check_word_pipeline(), check_word_noalloc()};
    const int k = n < 6 ? n : 6;
    for (int q = 0; q < k; ++q) words[q] = w[q];
    return k;
#else
    (void)words;
    return 0;  // the normal build compiles no checks
#endif
}

int csg_test_wait_expiry(uint64_t limit_ns, int starve) {
    if (starve && limit_ns == 0) {
        set_error("csg_test_wait_expiry: starving a stage needs a wait limit");
        return CSG_E_INVAL;
    }
    test_hooks().wait_ns.store(limit_ns);
    test_hooks().starve.store(starve ? 1 : 0);
    return CSG_OK;
}

int csg_test_fail_alloc(int n) {
    if (n < 0) {
        set_error("csg_test_fail_alloc: n < 0");
        return CSG_E_INVAL;
    }
    test_hooks().fail_alloc.store(n);
    return CSG_OK;
}

}  // extern "C"
