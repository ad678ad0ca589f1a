/*
 * csg.h -- C ABI of the GB300 causal-set library.
 *
 * The library runs the data-parallel path of Cunningham & Krioukov, "Causal Set
 * Generator and Action Computer" (arXiv:1709.03013) on one GPU:
 *
 *   csg_sprinkle  sprinkle N elements into a flat causal diamond and sort them by
 *                 time (Sec. 2.1; Sec. 2.2 for the time order)
 *   csg_link      build the symmetric bit-packed causal matrix (Sec. 2.2,
 *                 "Optimized GPU Linking Algorithm")
 *   csg_action    count, for every related pair i < j, the elements strictly
 *                 between them, histogram the counts into N_0..N_3 and form the
 *                 Benincasa-Dowker action (Sec. 4, Alg. 5; Eq. s_local)
 *   csg_action_batch, csg_serve_submit / csg_serve_poll
 *                 the same for many sets at once, and as a request service
 *
 * Conventions shared by every call
 *   - Return value: CSG_OK (0) on success, CSG_PENDING (1) from csg_serve_poll while a
 *     request is unfinished, a negative CSG_E_* code otherwise.  No C++ exception
 *     crosses the ABI.  csg_strerror() names a code; csg_last_error() gives the
 *     message of the last failure on the calling thread.
 *   - Ownership: a context owns every device allocation it makes; a set handle stays
 *     valid until csg_set_free (or csg_finalize of its context).  Result structs and
 *     host buffers are caller-owned.
 *   - Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     enqueue their kernels on it; calls that return results (csg_action,
 *     csg_action_batch, exports) synchronise that stream before returning.
 *   - Bitmap layout: row i of the N x N symmetric matrix is `stride_words` uint64
 *     words at dev_rows + i*stride_words; entry (i,k) is bit k%64 of word k/64
 *     (LSB first).  The diagonal is 0, bits k >= N are 0.  Elements are labelled in
 *     time order, so i < k related means i precedes k (Sec. 2.2).  The library's own
 *     sets use stride_words = ceil(N/64) rounded up to a multiple of 16 (128 bytes).
 *   - Coordinates: [4][N] doubles on the device, rows (t, x, u, v) for d=2 and
 *     (t, x, y, z) for d=4, sorted by time.
 */
#ifndef CSG_H
#define CSG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CSG_OK 0
#define CSG_PENDING 1
#define CSG_E_INVAL (-1)   /* bad argument: d not 2/4, N out of range, NULL pointer ... */
#define CSG_E_NOMEM (-2)   /* device allocation failed or over the context's HBM budget */
#define CSG_E_CUDA (-3)    /* a CUDA runtime call or kernel launch failed */
#define CSG_E_TIMEOUT (-4) /* a bounded wait expired (device-side or in csg_serve_poll) */
#define CSG_E_BUSY (-5)    /* the service queue is full */
#define CSG_E_REJECT (-6)  /* the d=4 sprinkle hit its 256-attempt rejection cap */
#define CSG_E_NOTFOUND (-7) /* unknown or already collected ticket */
#define CSG_E_CANCELLED (-8) /* request cancelled before it ran */

/* Methods for the interval counts (csg_action, csg_action_batch). */
#define CSG_POPC 0 /* AND + popcount of packed row words (Alg. 5 restated for the GPU) */
#define CSG_TC 1   /* the same counts as a masked 0/1 matrix product on tensor cores (currently CSG_TC_FP4) */
#define CSG_TC_FP8 2 /* tensor cores, 0/1 operands in fp8 e4m3 (kind::f8f6f4), two TMEM accumulators */
#define CSG_TC_FP4 3 /* tensor cores, 0/1 operands in packed fp4 e2m1 with unit block scales (kind::mxf4) */

/* Largest N a set may have. */
#define CSG_MAX_N (1 << 18)

typedef struct csg_ctx csg_ctx; /* opaque, library-owned */
typedef struct csg_set csg_set; /* opaque, library-owned */

/* Result of one action computation.
 *   R      number of related pairs i < j
 *   Nk[k]  number of related pairs with exactly k elements strictly between them
 *          (the paper's 1-based n_{k+1}; Sec. 1.2, Alg. 5)
 *   sum_m  sum over related pairs of the interval size m
 *   W      sum over related pairs of (j - i - 1): candidate bits inspected, the
 *          algorithmic work of Alg. 5 in bit operations
 *   combo  d=2: N - 2N0 + 4N1 - 2N2 (S = 2*combo, Eq. s_local)
 *          d=4: N - N0 + 9N1 - 16N2 + 8N3 (S = 4/sqrt(6)*combo, the 3+1 BD action)
 *   S      the action, formed once in double from the exact integer combo
 *   status CSG_OK or the error of this set (batch and serve paths) */
typedef struct {
    int32_t d;
    int32_t status;
    int64_t N;
    uint64_t R;
    uint64_t Nk[4];
    uint64_t sum_m;
    uint64_t W;
    int64_t combo;
    double S;
} csg_result;

/* Create a context on `device` that may hold at most hbm_budget_bytes of set
 * memory (0 = no limit).  *out receives the handle. */
int csg_init(int device, size_t hbm_budget_bytes, csg_ctx **out);

/* Stop the service thread (if any), free every set and all device memory. */
void csg_finalize(csg_ctx *ctx);

const char *csg_strerror(int code);
const char *csg_last_error(void);

/* Sprinkle N elements into the flat causal diamond of dimension d (2 or 4) and
 * sort them by time (Secs. 2.1-2.2).  Element e draws Philox4x64-10 blocks with
 * counter (e, attempt, 0, 0) and key (seed, seq):
 *   d=2: u, v = top 53 bits of words 0, 1 of attempt 0 scaled by 2^-53;
 *        t = (u+v)/2, x = (v-u)/2.
 *   d=4: (t,x,y,z) = 2U-1 from the four words; the first attempt with
 *        |t| + sqrt((x*x + y*y) + z*z) <= 1 is kept (at most 256, else CSG_E_REJECT).
 * Sorting key: (t, u, e) for d=2, (t, e) for d=4.  1 <= N <= CSG_MAX_N.
 * The new set has coordinates but no bitmap until csg_link.  The call enqueues the work
 * on `stream` and returns without waiting; the set's memory comes from the stream-ordered
 * pool on that stream.  An element that exhausts the rejection cap (probability below
 * 1e-15 per element) is reported as CSG_E_REJECT by the next call that reads the set's
 * results (csg_action and its variants, csg_export_*). */
int csg_sprinkle(csg_ctx *ctx, int d, int64_t N, uint64_t seed, uint64_t seq, void *stream,
                 csg_set **out);

/* Sprinkle N elements into the 1+1 de Sitter slab of Sec. 5.1 (Eq. ds_metric,
 * ds^2 = sec^2(eta) (-d eta^2 + d theta^2)), the paper's benchmark manifold: eta in
 * [-eta0, eta0] with density sec^2(eta) / (2 tan eta0), drawn as
 * eta = atan(tan(eta0) (2U - 1)) from word 0 of the Philox block (e, 0, 0, 0) with key
 * (seed, seq), and theta = 2 pi U' from word 1.  Coordinates are stored as rows
 * (eta, theta, 0, 0), sorted by (eta, e).  Two elements are related when
 * pi - |pi - |d theta|| < |d eta|.  The set uses the 1+1 action (d = 2).
 * 0 < eta0 < pi/2, 1 <= N <= CSG_MAX_N.  Enqueues and returns like csg_sprinkle. */
int csg_sprinkle_desitter(csg_ctx *ctx, int64_t N, double eta0, uint64_t seed, uint64_t seq,
                          void *stream, csg_set **out);

/* Make a set from host coordinates [4][N] (layout above, any order): copies them
 * to the device and sorts them by time like csg_sprinkle. */
int csg_set_from_coords(csg_ctx *ctx, int d, int64_t N, const double *host_coords,
                        void *stream, csg_set **out);

/* Build the symmetric bit-packed causal matrix of a sprinkled set (Sec. 2.2):
 *   d=2: i < k related iff u_i < u_k and v_i < v_k
 *   d=4: i < k related iff t_k > t_i and dt*dt > (dx*dx + dy*dy) + dz*dz in IEEE
 *        double without fused multiply-add (decided exactly; an fp32 screen with a
 *        proven error margin settles most pairs first).
 * Every row word up to the stride, padding included, is written. */
int csg_link(csg_ctx *ctx, csg_set *set, void *stream);

/* Wrap a caller-built bitmap (any time-ordered causal matrix, Sec. 1.3: the action
 * uses the adjacency matrix only).  dev_rows is copied into library memory with
 * the library's stride; stride_words >= ceil(N/64). d (2 or 4) picks the action's
 * formula.  The caller keeps ownership of dev_rows. */
int csg_set_from_bitmap(csg_ctx *ctx, int d, int64_t N, const uint64_t *dev_rows,
                        int64_t stride_words, void *stream, csg_set **out);

/* Interval abundances and action of one set (Alg. 5; Eq. s_local).  method is
 * CSG_POPC, CSG_TC, CSG_TC_FP8 or CSG_TC_FP4.  The tensor methods take N^2 bytes of
 * device scratch for their operands (fp4; 2 N^2 for fp8), allocated on `stream` and
 * freed before return; CSG_E_NOMEM if it cannot be allocated.  Synchronises `stream`,
 * then fills *out. */
int csg_action(csg_ctx *ctx, csg_set *set, int method, csg_result *out, void *stream);

/* The same restricted to first elements i in [row_lo, row_hi): counts only pairs
 * whose earlier element lies in the range (used to check sampled rows). */
int csg_action_rows(csg_ctx *ctx, csg_set *set, int method, int64_t row_lo, int64_t row_hi,
                    csg_result *out, void *stream);

/* Full interval-size histogram (the abundances the smeared action of Eq. s_smeared
 * needs, Sec. 4.1): dev_hist[m] (m < nbins, device uint64 array owned by the caller,
 * zeroed by the call) receives the number of related pairs with m interior elements;
 * bins m >= nbins are not recorded.  Fills *out like csg_action. */
int csg_action_hist(csg_ctx *ctx, csg_set *set, int method, uint64_t *dev_hist, int64_t nbins,
                    csg_result *out, void *stream);

/* Smeared (non-local) 1+1 action of Eq. s_smeared:
 *   S_eps = 2 eps [N - 2 eps sum_{i=1}^{N-1} n_i f2(i-1, eps)],
 *   f2(i, eps) = (1-eps)^i [1 - 2 eps i/(1-eps) + eps^2 i (i-1) / (2 (1-eps)^2)],
 * where n_i is the number of related pairs with i-1 elements between them (the full
 * histogram, Sec. 4.1).  0 < eps < 1; the set must have d = 2 (the paper gives the
 * smeared form in 1+1 dimensions only).  *S_eps receives the action; *out (optional)
 * the local counts as from csg_action.  The histogram uses N 64-bit words of
 * stream-ordered scratch. */
int csg_action_smeared(csg_ctx *ctx, csg_set *set, int method, double eps, double *S_eps,
                       csg_result *out, void *stream);

/* Discrete d'Alembertian of Eq. b_local (Sec. 1.2) at every element of a 1+1 set:
 *   Bphi[x] = (2 / l^2) ( -phi[x] + 2 [ sum_{y in L_1} - 2 sum_{y in L_2} + sum_{y in L_3} ] phi[y] ),
 * where L_i holds the elements y preceding x with exactly i-1 elements strictly between
 * them.  phi and Bphi are caller-owned DEVICE arrays of N doubles in the set's element
 * order (time order for sprinkled sets, the caller's order for bitmaps); they must not
 * overlap.  l > 0 is the discreteness scale.  The layer sums come from the same pass
 * that counts the intervals (method CSG_POPC or CSG_TC); they are accumulated with
 * atomic adds, so their rounding order is unspecified (each result is within the
 * recursive-summation bound of the exact value; with integer phi, |phi| < 2^32, and l a
 * power of two every step is exact).
 * The set must have d = 2 (the paper gives the 1+1 form only) and a bitmap.  *out
 * (optional) receives the action counts as from csg_action.  Synchronises the stream. */
int csg_dalembertian(csg_ctx *ctx, csg_set *set, int method, const double *phi, double l, double *Bphi,
                     csg_result *out, void *stream);

/* Actions of n sets in one pass: all sets' work in one persistent launch over a
 * queue of (set, row group) items, longest first.  out[n] is filled in order. */
int csg_action_batch(csg_ctx *ctx, csg_set *const *sets, int n, int method, csg_result *out,
                     void *stream);

/* Sprinkle + link + action for n (d, N, seed, seq) specs at once, with every step
 * batched across the sets; the sets are freed before returning. */
int csg_run_batch(csg_ctx *ctx, int n, const int32_t *d, const int64_t *N, const uint64_t *seed,
                  const uint64_t *seq, int method, csg_result *out, void *stream);

/* Request service (continuous batching).  submit queues a (d, N, seed, seq) request
 * without blocking and returns a ticket; a worker thread admits queued requests
 * while their bitmaps (N*N/8 bytes each) fit the context's budget, runs sprinkle,
 * link and action for every admitted request in shared launches, and retires them.
 * poll waits up to timeout_ms (0 = no wait, <0 = forever) and returns CSG_OK with
 * *out filled, CSG_PENDING, or an error; a collected ticket is forgotten.  cancel
 * drops a request that is still queued (CSG_E_BUSY once it is admitted; its poll
 * then returns CSG_E_CANCELLED).  Both return CSG_E_NOTFOUND for a ticket the
 * context never issued or already forgot; neither starts the service. */
int csg_serve_submit(csg_ctx *ctx, int d, int64_t N, uint64_t seed, uint64_t seq,
                     uint64_t *ticket);
int csg_serve_poll(csg_ctx *ctx, uint64_t ticket, csg_result *out, int timeout_ms);
int csg_serve_cancel(csg_ctx *ctx, uint64_t ticket);

/* Copy a set's sorted coordinates ([4][N] doubles) or bitmap (N*stride words) to
 * host memory; cap is the host buffer's capacity in elements.  Waits for the device;
 * returns CSG_E_REJECT if the set's sprinkle hit the rejection cap. */
int csg_export_coords(csg_set *set, double *host, size_t cap_doubles);
int csg_export_bitmap(csg_set *set, uint64_t *host, size_t cap_words);

/* Shape and device pointers of a set (pointers stay owned by the library). */
int csg_set_info(const csg_set *set, int *d, int64_t *N, int64_t *stride_words,
                 const uint64_t **dev_rows, const double **dev_coords);

/* Release a set.  Its device memory returns to the pool in stream order on the stream
 * the set was created with; work that uses the set on other streams must be complete
 * (or ordered before that stream) when this is called. */
void csg_set_free(csg_set *set);

/* Per-stage device timing (a tracing aid; Sec. 5 of the paper reports stage times).
 * With timing on, every call on the context records CUDA events on its own stream
 * around the kernels of each stage it runs; csg_stage_times(ctx, ms, n) waits for the
 * last recorded events and writes the elapsed milliseconds of stages 0..n-1 (-1 for a
 * stage not run since timing was switched on). */
#define CSG_STAGE_SPRINKLE 0 /* sprinkle + time order */
#define CSG_STAGE_LINK 1     /* causal matrix */
#define CSG_STAGE_EXPAND 2   /* 0/1 operand expansion of the tensor form (fp4, or fp8) */
#define CSG_STAGE_ACTION 3   /* the interval-count kernel itself */
#define CSG_STAGE_FINALIZE 4 /* counters -> action */
#define CSG_STAGE_COUNT 5
int csg_set_timing(csg_ctx *ctx, int enable);
int csg_stage_times(csg_ctx *ctx, double *ms, int n);

/* The popcount action for callers that cannot let the library allocate device
 * memory.  The paper has no counterpart to this call; it exists for callers such as
 * code recording a CUDA graph (a cudaMalloc there breaks the capture), applications
 * that give all of HBM to their own arena, and multi-stream servers that cannot
 * afford the device-wide synchronisation of a cudaFree.
 *
 * Inputs: dev_rows, an N x stride_words bitmap in the layout above (16-byte aligned,
 * even stride_words >= ceil(N/64)), and d (2 or 4) for the action's formula.
 * Output: *dev_out, a csg_result in device memory owned by the caller, written when
 * the stream reaches the call's kernels; the call returns without synchronising.
 * The result equals csg_action(..., CSG_POPC, ...) on the same bitmap.
 *
 * The call allocates nothing: its scratch (a work-queue counter and partial counters
 * for each group of 16 rows) lives in one fixed device array of 256 KiB + 16 bytes,
 * which every GPU that loads the library holds until the process exits.  Hence N is
 * limited to 1 <= N <= 65536; larger N returns CSG_E_INVAL with a message.  The
 * first call on a device looks up that array's device address (cudaGetSymbolAddress)
 * and caches it, so make that first call before any stream capture.  All calls on a
 * device share the array and each call clears the parts that must start at zero;
 * calls whose kernels overlap on the GPU (different streams, no ordering between
 * them) race on it and must not be issued.  If a bounded wait of the call's kernel runs
 * out, *dev_out gets status CSG_E_TIMEOUT with every count (and combo and S) zero. */
int csg_action_noalloc(int d, int64_t N, const uint64_t *dev_rows, int64_t stride_words,
                       csg_result *dev_out, void *stream);

/* Bounds checks (the library built with CSG_CHECKED defined, e.g. by
 * paper_1709_03013_gb300/_build.py's build(checked=True) into libcsg_checked.so): the kernels
 * test the indices they compute before each guarded access, skip an access that would leave
 * its buffer, and record the first such failure of each kernel group -- the check site in the
 * top 16 bits, the low 48 bits of the offending index below -- in a device word.
 * csg_check_words synchronises the device, copies up to n of the words (sprinkle/sort, link,
 * popcount, tensor, pipeline, allocation-free, in that order) to words[], clears them and
 * returns how many it wrote; 0 means no failure.  The normal build compiles no checks and
 * returns 0. */
int csg_check_words(uint64_t *words, int n);

/* Measurement aid for the roofline of CSG_POPC: the sustained throughput of this GPU's
 * 32-bit population-count pipe, in popcounts per second over the whole device, from a
 * dedicated loop of independent popcounts (two 1024-thread CTAs per SM, about 50 ms).
 * Divided by the SM count and the SM clock it gives results per SM per clock; the CUDA
 * programming guide lists 16.  Allocates and frees a small output buffer; synchronises the
 * device. */
int csg_measure_popc_rate(int device, double *popc_per_second);

/* Throughput probe of the operand feed from L2 into shared memory, the second bound of the
 * tensor-core interval counts (each SM of a CTA pair stages 32 KB of operands per 256-deep K
 * step).  One CTA per SM keeps six 32 KB stages in flight, each two 2D tensor-map loads of
 * 128 rows x 128 bytes with 128-byte swizzle (the tensor kernel's kind of copy), from a 32 MB
 * matrix that stays in L2; *bytes_per_sm_per_second receives the bytes one SM receives per
 * second with every SM pulling at once.  Allocates and frees the matrix; synchronises the
 * device; every device wait is bounded (CSG_E_TIMEOUT if one runs out). */
int csg_measure_l2_feed(int device, double *bytes_per_sm_per_second);

/* Throughput probe of the tensor cores as the interval counts use them: the same 2-SM MMA
 * (tcgen05.mma.cta_group::2, M = 256, N = 256; method CSG_TC or CSG_TC_FP4: kind::mxf4 with
 * unit block scales, CSG_TC_FP8: kind::f8f6f4), instruction descriptor and TMEM layout as the
 * product kernel, issued back to back on operands resident in shared memory by one CTA pair
 * per two SMs.  *flops_per_second receives the whole GPU's rate (2 flops per product).
 * Synchronises the device; every device wait is bounded (CSG_E_TIMEOUT if one runs out);
 * CSG_E_INVAL for another method. */
int csg_measure_mma_rate(int device, int method, double *flops_per_second);

/* Failure injection for tests of the error paths (not for production use; process-wide,
 * off by default).  No GPU faults, traps or hangs in either: the failures are made on the
 * host or by a wait that nothing completes, and every device wait is bounded.
 *
 * csg_test_wait_expiry(limit_ns, starve): every bounded wait of the interval-count kernels
 * (csg_action and its variants with CSG_POPC or a tensor method) gives up after limit_ns
 * nanoseconds (0 restores the built-in limits of 2-4 s).  With starve nonzero (limit_ns must
 * then be nonzero), the producer of every CTA skips the bulk copies of its first stage: the
 * stage's barrier never completes, the first wait on it runs out with no copy in flight, the
 * kernel records the expiry in the set's error word and returns, and the call returns
 * CSG_E_TIMEOUT.  The context stays usable; csg_test_wait_expiry(0, 0) switches it off.
 *
 * csg_test_fail_alloc(n): the next n device allocations the library makes (set memory,
 * stream-ordered scratch, batch arenas) fail as if the allocator were out of memory, so the
 * calls that needed them return CSG_E_NOMEM.  n = 0 clears the count. */
int csg_test_wait_expiry(uint64_t limit_ns, int starve);
int csg_test_fail_alloc(int n);

#ifdef __cplusplus
}
#endif
#endif /* CSG_H */
