// Batched pipeline (sprinkle + sort + link + action for many sets) and the request
// service built on it.
//
// The service does continuous batching: csg_serve_submit only queues a request.
// A small pool of worker threads repeatedly takes queued requests that fit the
// context's memory budget (admission by the set's footprint, N*N/8 bytes of bitmap plus
// coordinates), up to a work cap per batch, and runs the whole path for them in shared
// launches.  The smallest queued request opens each batch (shortest job first, which keeps
// the many small requests from queueing behind a few large ones), unless a request has
// waited longer than the age limit, in which case the oldest such request opens it (no
// request starves, even above capacity); only requests within a factor of two of the
// opener's size join it, so small requests are not held back by a large one's results;
// batches of small sets run on a high-priority stream.  Requests that arrive
// while other batches are on the GPU are admitted by the next free worker as soon as
// memory frees up, so their kernels overlap on the device.  Results are kept per ticket
// until csg_serve_poll collects them.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>
#include <vector>

#include "csg_internal.cuh"
#include "csg_state.h"

namespace csg {

// ------------------------------------------------------------------ service

namespace {

enum ReqState { Q_QUEUED, Q_RUNNING, Q_DONE, Q_CANCELLED };

struct Req {
    int d;
    int64_t N;
    uint64_t seed, seq;
    ReqState state;
    int rc;
    csg_result res;
    std::chrono::steady_clock::time_point submitted;
};

size_t footprint(int64_t N) {
    return (size_t)N * 4 * sizeof(double) + (size_t)N * stride_for(N) * sizeof(uint64_t);
}

// work of a request for the tensor form: the triangle-restricted contraction, N^3/3 flops
double work_of(int d, int64_t N) {
    (void)d;
    const double n = (double)N;
    return n * n * n / 3.0;
}

}  // namespace

struct ServeState {
    csg_ctx *ctx = nullptr;
    std::mutex mu;
    std::condition_variable cv_work;   // workers wait for queued requests / memory
    std::condition_variable cv_done;   // pollers wait for results
    std::deque<uint64_t> queue;        // queued tickets, arrival order
    std::map<uint64_t, Req> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    size_t reserved = 0;               // bytes admitted by running batches
    std::vector<std::thread> workers;
    size_t max_queue = 1 << 20;
    double batch_work_cap = 1e14;      // flops per batch (12 ms at the tensor form's large-set rate)
    int batch_max_sets = 4096;
    int64_t small_n = 16384;           // batches of sets up to this size run at high priority
    std::chrono::milliseconds max_age{250};  // a request waiting longer opens the next batch
};

namespace {

void worker_main(ServeState *S) {
    csg_ctx *ctx = S->ctx;
    cudaSetDevice(ctx->device);
    // two streams: batches of small sets go on the high-priority one, so their kernels'
    // blocks are scheduled first whenever a large batch's short kernels leave SMs free
    // (if only one stream can be made, both classes share it; with none, every batch this
    // worker takes fails with CSG_E_CUDA, so its requests still complete)
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    cudaStream_t st_lo = nullptr, st_hi = nullptr;
    const bool own_lo = cudaStreamCreateWithPriority(&st_lo, cudaStreamNonBlocking, prio_lo) == cudaSuccess;
    const bool own_hi = cudaStreamCreateWithPriority(&st_hi, cudaStreamNonBlocking, prio_hi) == cudaSuccess;
    if (!own_lo) st_lo = own_hi ? st_hi : nullptr;
    if (!own_hi) st_hi = own_lo ? st_lo : nullptr;
    const int stream_rc = own_lo || own_hi ? CSG_OK : CSG_E_CUDA;
    cudaGetLastError();  // a failed creation leaves no sticky error behind
    std::vector<uint64_t> batch;
    for (;;) {
        batch.clear();
        size_t bytes = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (;;) {
                if (S->stop) break;
                // The opener: the oldest request past the age limit, else the smallest (the
                // oldest of equal size).  Others join it while memory and the work cap allow, in
                // arrival order, if their size is within a factor of two of the opener's, so a
                // small request never waits for a large one's results (a batch's results are
                // ready together).  Requests passed over keep their place in the queue.
                // tickets that were cancelled (or cancelled and already collected) leave the queue
                // first, in a pass of their own: erasing from the deque invalidates its iterators
                S->queue.erase(std::remove_if(S->queue.begin(), S->queue.end(),
                                              [&](uint64_t t) {
                                                  auto f = S->reqs.find(t);
                                                  return f == S->reqs.end() || f->second.state == Q_CANCELLED;
                                              }),
                               S->queue.end());
                const auto now = std::chrono::steady_clock::now();
                uint64_t opener = 0;
                int64_t opener_n = 0;
                for (uint64_t t : S->queue) {
                    const Req &r = S->reqs.find(t)->second;
                    if (now - r.submitted > S->max_age) {  // the queue is in arrival order
                        opener = t;
                        break;
                    }
                    if (opener == 0 || r.N < opener_n) {
                        opener = t;
                        opener_n = r.N;
                    }
                }
                double work = 0.0;
                int64_t n_lo = 0, n_hi = 0;
                auto fits = [&](const Req &r) {
                    size_t used;
                    {
                        std::lock_guard<std::mutex> g(ctx->mu);
                        used = ctx->used;
                    }
                    return ctx->budget == 0 || used + S->reserved + bytes + footprint(r.N) <= ctx->budget;
                };
                auto take = [&](std::deque<uint64_t>::iterator it) {
                    Req &r = S->reqs.find(*it)->second;
                    r.state = Q_RUNNING;
                    batch.push_back(*it);
                    bytes += footprint(r.N);
                    work += work_of(r.d, r.N);
                    return S->queue.erase(it);
                };
                if (opener != 0 && fits(S->reqs.find(opener)->second)) {
                    n_lo = S->reqs.find(opener)->second.N / 2;
                    n_hi = S->reqs.find(opener)->second.N * 2;
                    take(std::find(S->queue.begin(), S->queue.end(), opener));
                    for (auto it = S->queue.begin(); it != S->queue.end() && (int)batch.size() < S->batch_max_sets;) {
                        const Req &r = S->reqs.find(*it)->second;
                        if (r.N < n_lo || r.N > n_hi) {
                            ++it;
                            continue;
                        }
                        if (!fits(r) || work + work_of(r.d, r.N) > S->batch_work_cap) break;
                        it = take(it);
                    }
                }
                if (!batch.empty()) break;
                S->cv_work.wait(lk);
            }
            if (batch.empty() && S->stop) break;
            S->reserved += bytes;
        }
        // run the batch
        const int n = (int)batch.size();
        int64_t n_max = 0;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (uint64_t t : batch) n_max = std::max<int64_t>(n_max, S->reqs[t].N);
        }
        cudaStream_t st = n_max <= S->small_n ? st_hi : st_lo;
        std::vector<csg_set *> sets;
        std::vector<uint64_t> seeds(n), seqs(n);
        std::vector<csg_result> res(n);
        int rc = stream_rc;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (int q = 0; q < n; ++q) {
                const Req &r = S->reqs[batch[q]];
                seeds[q] = r.seed;
                seqs[q] = r.seq;
            }
        }
        for (int q = 0; q < n && rc == CSG_OK; ++q) {
            int d;
            int64_t N;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                d = S->reqs[batch[q]].d;
                N = S->reqs[batch[q]].N;
            }
            csg_set *x = nullptr;
            rc = alloc_set(ctx, d, N, &x, st);
            if (rc == CSG_OK) sets.push_back(x);
        }
        {
            // the sets now hold the memory that admission reserved
            std::lock_guard<std::mutex> lk(S->mu);
            S->reserved -= bytes;
        }
        // the tensor form is the faster one; above N = 2^17 its operand scratch (N^2 bytes, 16 to
        // 64 GiB a set) is not part of the admission budget, so such batches take the popcount form
        int method = CSG_TC;
        for (csg_set *x : sets)
            if (x->N > (1 << 17)) method = CSG_POPC;
        if (rc == CSG_OK) rc = run_pipeline(sets.data(), n, seeds.data(), seqs.data(), method,
                                            res.data(), st);
        for (csg_set *x : sets) free_set(x);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (int q = 0; q < n; ++q) {
                Req &r = S->reqs[batch[q]];
                r.state = Q_DONE;
                r.rc = rc;
                if (rc == CSG_OK) r.res = res[q];
            }
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
    if (own_lo) cudaStreamDestroy(st_lo);
    if (own_hi) cudaStreamDestroy(st_hi);
}

// the running service, or null before the first request (polls and cancels do not start it)
ServeState *find_serve(csg_ctx *ctx) {
    std::lock_guard<std::mutex> g(ctx->serve_mu);
    return ctx->serve;
}

ServeState *ensure_serve(csg_ctx *ctx) {
    std::lock_guard<std::mutex> g(ctx->serve_mu);
    if (!ctx->serve) {
        ServeState *S = new ServeState();
        S->ctx = ctx;
        const int workers = 3;
        for (int w = 0; w < workers; ++w) S->workers.emplace_back(worker_main, S);
        ctx->serve = S;
    }
    return ctx->serve;
}

}  // namespace

void serve_shutdown(csg_ctx *ctx) {
    ServeState *S = nullptr;
    {
        std::lock_guard<std::mutex> g(ctx->serve_mu);
        S = ctx->serve;
        ctx->serve = nullptr;
    }
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto &t : S->workers) t.join();
    delete S;
}

}  // namespace csg

using namespace csg;

extern "C" {

int csg_serve_submit(csg_ctx *ctx, int d, int64_t N, uint64_t seed, uint64_t seq, uint64_t *ticket) {
    if (!ctx || !ticket || (d != 2 && d != 4) || N < 1 || N > CSG_MAX_N) {
        set_error("csg_serve_submit: bad arguments");
        return CSG_E_INVAL;
    }
    if (ctx->budget && footprint(N) > ctx->budget) {
        set_error("csg_serve_submit: request of %zu bytes can never fit the budget", footprint(N));
        return CSG_E_NOMEM;
    }
    ServeState *S = ensure_serve(ctx);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->queue.size() >= S->max_queue) {
            set_error("csg_serve_submit: queue full");
            return CSG_E_BUSY;
        }
        const uint64_t t = S->next_ticket++;
        Req r{};
        r.d = d;
        r.N = N;
        r.seed = seed;
        r.seq = seq;
        r.state = Q_QUEUED;
        r.rc = CSG_PENDING;
        r.submitted = std::chrono::steady_clock::now();
        S->reqs[t] = r;
        S->queue.push_back(t);
        *ticket = t;
    }
    S->cv_work.notify_one();
    return CSG_OK;
}

int csg_serve_poll(csg_ctx *ctx, uint64_t ticket, csg_result *out, int timeout_ms) {
    if (!ctx || !out) return CSG_E_INVAL;
    ServeState *S = find_serve(ctx);
    if (!S) return CSG_E_NOTFOUND;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return CSG_E_NOTFOUND;
    auto ready = [&] {
        auto f = S->reqs.find(ticket);
        return f == S->reqs.end() || f->second.state == Q_DONE || f->second.state == Q_CANCELLED;
    };
    if (!ready()) {
        if (timeout_ms == 0) return CSG_PENDING;
        if (timeout_ms < 0)
            S->cv_done.wait(lk, ready);
        else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
            return CSG_PENDING;
    }
    it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return CSG_E_NOTFOUND;
    if (it->second.state == Q_CANCELLED) {
        S->reqs.erase(it);
        return CSG_E_CANCELLED;
    }
    const int rc = it->second.rc;
    if (rc == CSG_OK) *out = it->second.res;
    S->reqs.erase(it);
    return rc;
}

int csg_serve_cancel(csg_ctx *ctx, uint64_t ticket) {
    if (!ctx) return CSG_E_INVAL;
    ServeState *S = find_serve(ctx);
    if (!S) return CSG_E_NOTFOUND;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return CSG_E_NOTFOUND;
        if (it->second.state != Q_QUEUED) return CSG_E_BUSY;  // already admitted
        it->second.state = Q_CANCELLED;
    }
    S->cv_done.notify_all();
    return CSG_OK;
}

}  // extern "C"
