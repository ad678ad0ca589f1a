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

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
}

namespace {

// Forms the action from the counters (a6 of the path): the integer combination in
// int64, then one double multiply (Eq. s_local for d=2; (4/sqrt6) for d=4).
struct FinRow {
    int32_t d;
    int32_t pad;
    int64_t N;
    const unsigned long long *counters;
};

__global__ void finalize_kernel(const FinRow *__restrict__ rows, int n, csg_result *__restrict__ out) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const FinRow F = rows[s];
        const unsigned long long *c = F.counters;
        csg_result r;
        r.d = F.d;
        r.status = c[CNT_ERR] ? CSG_E_TIMEOUT : CSG_OK;
        r.N = F.N;
        r.R = c[CNT_R];
        for (int k = 0; k < 4; ++k) r.Nk[k] = c[CNT_N0 + k];
        r.sum_m = c[CNT_SUM_M];
        r.W = c[CNT_W];
        const long long n0 = (long long)c[CNT_N0], n1 = (long long)c[CNT_N1],
                        n2 = (long long)c[CNT_N2], n3 = (long long)c[CNT_N3];
        if (F.d == 2) {
            r.combo = F.N - 2 * n0 + 4 * n1 - 2 * n2;
            r.S = __dmul_rn(2.0, __ll2double_rn(r.combo));
        } else {
            r.combo = F.N - n0 + 9 * n1 - 16 * n2 + 8 * n3;
            r.S = __dmul_rn(__ddiv_rn(4.0, __dsqrt_rn(6.0)), __ll2double_rn(r.combo));
        }
        out[s] = r;
    }
}

}  // namespace

// Runs the action for n sets (already linked) and writes n results to host `out`.
int run_actions(csg_set *const *sets, int n, int method, int64_t row_lo, int64_t row_hi,
                unsigned long long *dev_hist, int64_t nbins, csg_result *out, cudaStream_t st) {
    if (n <= 0) return CSG_OK;
    std::vector<SetDesc> desc(n);
    std::vector<FinRow> fin(n);
    char *scratch = nullptr;
    const size_t cnt_bytes = (size_t)n * CNT_WORDS * sizeof(unsigned long long);
    const size_t bytes = cnt_bytes + n * sizeof(FinRow) + n * sizeof(csg_result) + 64;
    CSG_CUDA_TRY(cudaMallocAsync((void **)&scratch, bytes, st));
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(scratch);
    FinRow *d_fin = reinterpret_cast<FinRow *>(scratch + cnt_bytes);
    csg_result *d_out = reinterpret_cast<csg_result *>(scratch + cnt_bytes + n * sizeof(FinRow));
    for (int s = 0; s < n; ++s) {
        desc[s].rows = sets[s]->rows;
        desc[s].N = sets[s]->N;
        desc[s].stride = sets[s]->stride;
        desc[s].counters = cnt + (size_t)s * CNT_WORDS;
        desc[s].row_lo = row_lo < 0 ? 0 : row_lo;
        desc[s].row_hi = row_hi < 0 ? sets[s]->N : std::min<int64_t>(row_hi, sets[s]->N);
        fin[s].d = sets[s]->d;
        fin[s].pad = 0;
        fin[s].N = sets[s]->N;
        fin[s].counters = desc[s].counters;
    }
    cudaMemsetAsync(cnt, 0, cnt_bytes, st);
    cudaMemcpyAsync(d_fin, fin.data(), n * sizeof(FinRow), cudaMemcpyHostToDevice, st);
    int rc;
    if (method == CSG_POPC)
        rc = action_popc(desc.data(), n, st, dev_hist, nbins);
    else
        rc = action_tc(desc.data(), n, st, dev_hist, nbins);
    if (rc == CSG_OK) {
        stage_begin(CSG_STAGE_FINALIZE, st);
        finalize_kernel<<<(n + 127) / 128, 128, 0, st>>>(d_fin, n, d_out);
        stage_end(CSG_STAGE_FINALIZE, st);
        cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) {
            set_error("finalize launch: %s", cudaGetErrorString(le));
            rc = CSG_E_CUDA;
        } else {
            cudaMemcpyAsync(out, d_out, n * sizeof(csg_result), cudaMemcpyDeviceToHost, st);
        }
    }
    cudaFreeAsync(scratch, st);
    cudaError_t se = cudaStreamSynchronize(st);
    if (rc == CSG_OK && se != cudaSuccess) {
        set_error("action: %s", cudaGetErrorString(se));
        rc = CSG_E_CUDA;
    }
    if (rc == CSG_OK) {
        for (int s = 0; s < n; ++s)
            if (out[s].status != CSG_OK) {
                set_error("action: a bounded device wait expired (set %d)", s);
                rc = out[s].status;
            }
    }
    return rc;
}

// ------------------------------------------------------------------ sets

int alloc_set(csg_ctx *ctx, int d, int64_t N, csg_set **out) {
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
    cudaError_t e1 = cudaMalloc((void **)&s->coords, (size_t)N * 4 * sizeof(double));
    cudaError_t e2 = cudaMalloc((void **)&s->rows, (size_t)N * s->stride * sizeof(uint64_t));
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        if (s->coords) cudaFree(s->coords);
        if (s->rows) cudaFree(s->rows);
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

void free_set(csg_set *s) {
    if (!s) return;
    csg_ctx *ctx = s->ctx;
    cudaSetDevice(ctx->device);
    if (s->coords) cudaFree(s->coords);
    if (s->rows) cudaFree(s->rows);
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
    std::vector<csg_set *> all;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        all.assign(ctx->sets.begin(), ctx->sets.end());
    }
    for (csg_set *s : all) free_set(s);
    delete ctx;
}

int csg_sprinkle(csg_ctx *ctx, int d, int64_t N, uint64_t seed, uint64_t seq, void *stream,
                 csg_set **out) {
    if (!ctx) return CSG_E_INVAL;
    TimerScope ts(ctx);
    CSG_CUDA_TRY(cudaSetDevice(ctx->device));
    csg_set *s = nullptr;
    int rc = alloc_set(ctx, d, N, &s);
    if (rc != CSG_OK) return rc;
    SprinkleSpec sp{d, 0, N, seed, seq, s->coords, 0};
    rc = sprinkle_sort_batch(&sp, 1, (cudaStream_t)stream, nullptr);
    if (rc != CSG_OK) {
        free_set(s);
        return rc;
    }
    s->coord_scale = 1.0;
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
    int rc = alloc_set(ctx, d, N, &s);
    if (rc != CSG_OK) return rc;
    SprinkleSpec sp{d, 0, N, 0, 0, s->coords, 0};
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
    LinkSpec L{set->d, 0, set->N, set->stride, set->coords, set->rows, 0, set->coord_scale};
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
    int rc = alloc_set(ctx, d, N, &s);
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
    if (!ctx || !set || !out || set->ctx != ctx || (method != CSG_POPC && method != CSG_TC)) {
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

int csg_action_batch(csg_ctx *ctx, csg_set *const *sets, int n, int method, csg_result *out,
                     void *stream) {
    if (!ctx || (n > 0 && (!sets || !out)) || n < 0 || (method != CSG_POPC && method != CSG_TC)) {
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
    CSG_CUDA_TRY(cudaSetDevice(ctx->device));
    TimerScope ts(ctx);
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<csg_set *> sets;
    int rc = CSG_OK;
    for (int s = 0; s < n && rc == CSG_OK; ++s) {
        csg_set *x = nullptr;
        rc = alloc_set(ctx, d[s], N[s], &x);
        if (rc == CSG_OK) {
            x->coord_scale = 1.0;
            sets.push_back(x);
        }
    }
    if (rc == CSG_OK) rc = run_pipeline(sets.data(), n, seed, seq, method, out, st);
    for (csg_set *x : sets) free_set(x);
    return rc;
}

int csg_export_coords(csg_set *set, double *host, size_t cap) {
    if (!set || !host || cap < (size_t)(4 * set->N)) {
        set_error("csg_export_coords: bad arguments");
        return CSG_E_INVAL;
    }
    CSG_CUDA_TRY(cudaSetDevice(set->ctx->device));
    CSG_CUDA_TRY(cudaDeviceSynchronize());
    CSG_CUDA_TRY(cudaMemcpy(host, set->coords, 4 * set->N * sizeof(double), cudaMemcpyDeviceToHost));
    return CSG_OK;
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
    return CSG_OK;
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

}  // extern "C"
