// Per-stage device timing: CUDA events recorded on the call's own stream around the
// kernels of each stage (sprinkle+sort, link, operand expansion, the action kernel,
// finalize) when timing is switched on for a context.
#include <cuda_runtime.h>

#include "csg_internal.cuh"
#include "csg_state.h"

namespace csg {

struct StageTimer {
    cudaEvent_t start[CSG_STAGE_COUNT], stop[CSG_STAGE_COUNT];
    bool recorded[CSG_STAGE_COUNT];
    bool begun[CSG_STAGE_COUNT];
};

static thread_local StageTimer *t_timer = nullptr;

TimerScope::TimerScope(csg_ctx *ctx) : prev(t_timer) {
    t_timer = ctx ? ctx->timer : nullptr;
    if (t_timer)
        for (int s = 0; s < CSG_STAGE_COUNT; ++s) t_timer->begun[s] = false;
}

TimerScope::~TimerScope() { t_timer = prev; }

void stage_begin(int stage, cudaStream_t st) {
    if (!t_timer || t_timer->begun[stage]) return;
    cudaEventRecord(t_timer->start[stage], st);
    t_timer->begun[stage] = true;
}

void stage_end(int stage, cudaStream_t st) {
    if (!t_timer || !t_timer->begun[stage]) return;
    cudaEventRecord(t_timer->stop[stage], st);
    t_timer->recorded[stage] = true;
}

void destroy_timer(csg_ctx *ctx) {
    if (!ctx->timer) return;
    for (int s = 0; s < CSG_STAGE_COUNT; ++s) {
        cudaEventDestroy(ctx->timer->start[s]);
        cudaEventDestroy(ctx->timer->stop[s]);
    }
    delete ctx->timer;
    ctx->timer = nullptr;
}

}  // namespace csg

using namespace csg;

extern "C" int csg_set_timing(csg_ctx *ctx, int enable) {
    if (!ctx) {
        set_error("csg_set_timing: null context");
        return CSG_E_INVAL;
    }
    CSG_CUDA_TRY(cudaSetDevice(ctx->device));
    if (!enable) {
        destroy_timer(ctx);
        return CSG_OK;
    }
    if (ctx->timer) return CSG_OK;
    StageTimer *t = new StageTimer();
    for (int s = 0; s < CSG_STAGE_COUNT; ++s) {
        if (cudaEventCreate(&t->start[s]) != cudaSuccess || cudaEventCreate(&t->stop[s]) != cudaSuccess) {
            delete t;
            set_error("csg_set_timing: cudaEventCreate failed");
            return CSG_E_CUDA;
        }
        t->recorded[s] = false;
        t->begun[s] = false;
    }
    ctx->timer = t;
    return CSG_OK;
}

extern "C" int csg_stage_times(csg_ctx *ctx, double *ms, int n) {
    if (!ctx || !ms || n < 0) {
        set_error("csg_stage_times: bad arguments");
        return CSG_E_INVAL;
    }
    if (!ctx->timer) {
        set_error("csg_stage_times: timing is off (csg_set_timing)");
        return CSG_E_INVAL;
    }
    CSG_CUDA_TRY(cudaSetDevice(ctx->device));
    for (int s = 0; s < n && s < CSG_STAGE_COUNT; ++s) {
        ms[s] = -1.0;
        if (!ctx->timer->recorded[s]) continue;
        float f = 0.f;
        CSG_CUDA_TRY(cudaEventSynchronize(ctx->timer->stop[s]));
        CSG_CUDA_TRY(cudaEventElapsedTime(&f, ctx->timer->start[s], ctx->timer->stop[s]));
        ms[s] = (double)f;
    }
    return CSG_OK;
}
