/*
 * stag_kde.h — exact Gaussian kernel density estimation on one GB300 GPU (sm_103a).
 *
 * Computes, for every query q_j of a batch Q against a resident point set X,
 *
 *     K(q_j) = sum_{i=1..n} exp(-a * ||q_j - x_i||^2)
 *
 * which is the paper's kernel density (Sec. 3) with the Gaussian kernel
 * k(x) = exp(-a x^2) (Sec. 3), computed exactly ("naive", O(dmn), Sec. 3 and Sec. 6.1)
 * rather than estimated. The 1/n factor of the paper's definition is applied only when
 * the `normalise` option is set; by default the unnormalised sum is returned (the form
 * the similarity-graph degrees of Sec. 4 and the subset estimators of Sec. 3.1 use).
 * The create/query/destroy life cycle mirrors the paper's ExactGaussianKDE class
 * (Sec. 5.3: constructor taking the data and a; query of one point or of a matrix).
 *
 * Conventions shared by every entry point:
 *   - Matrices are dense row-major, rows = points, `d` contiguous coordinates per row.
 *   - Host pointers are plain CPU memory (pageable or pinned); device pointers are CUDA
 *     global memory on the handle's device. Nothing is retained: the library copies X
 *     at create time; Q and out are used only during the call (host API) or until the
 *     work queued on the given stream completes (device API).
 *   - Return codes: 0 on success, a negative STAG_KDE_E* code on failure. Functions
 *     returning a pointer return NULL on failure. stag_kde_last_error() gives a
 *     human-readable reason for the calling thread's most recent failure.
 *   - On failure the output buffer is left untouched (host API).
 *   - Inputs must be finite with |coordinate| <= 1e15 (so that squared distances are
 *     finite in FP32); a must be finite and >= 0 (a < 0 would break k(x) in [0, 1],
 *     Sec. 3). Violations return STAG_KDE_EINVAL.
 *   - m = 0 is a valid no-op. n >= 1 and d >= 1 are required.
 *   - A handle may be used by one thread at a time. Results are deterministic: the same
 *     handle, inputs and options give bitwise-identical outputs on every call.
 */
#ifndef STAG_KDE_H
#define STAG_KDE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STAG_KDE_OK 0
#define STAG_KDE_EINVAL (-1)     /* bad argument (sizes, NULL pointer, non-finite value)  */
#define STAG_KDE_ENOMEM (-2)     /* device or host allocation failed (also: admission)     */
#define STAG_KDE_ECUDA (-3)      /* a CUDA call failed (message has the CUDA error string) */
#define STAG_KDE_ETIMEDOUT (-4)  /* a bounded wait expired                                 */
#define STAG_KDE_ECANCELED (-5)  /* request cancelled or server stopped                    */
#define STAG_KDE_EUNSUPPORTED (-6) /* form not available for this shape / dtype           */

/* Element type of X and Q. */
#define STAG_KDE_F32 0
#define STAG_KDE_F64 1

/*
 * Kernel function k of the distance r = ||q - x|| (Sec. 3 lists three):
 *   GAUSSIAN     k = exp(-a r^2)                       (the default; every form)
 *   EXPONENTIAL  k = exp(-a r)                         (plain FP32 and FP64 forms)
 *   LOGISTIC     k = 4 / (2 + exp(a r) + exp(-a r))    (plain FP32 and FP64 forms)
 * The paper writes the logistic kernel without a bandwidth; here its argument is a*r, so
 * a = 1 gives the paper's k(r). The tensor-core form serves only the Gaussian kernel: the
 * other two take sqrt of the squared distance, which turns the split products' absolute
 * error in r^2 into a large relative error near r = 0. AUTO picks the plain FP32 form
 * for them; an explicit STAG_KDE_FORM_TC returns STAG_KDE_EUNSUPPORTED.
 */
#define STAG_KDE_KERNEL_GAUSSIAN 0
#define STAG_KDE_KERNEL_EXPONENTIAL 1
#define STAG_KDE_KERNEL_LOGISTIC 2

/* Evaluation form ("precision form"). */
#define STAG_KDE_FORM_AUTO 0     /* library picks (tensor-core form where its error model allows) */
#define STAG_KDE_FORM_SIMT_F32 1 /* plain FP32 CUDA-core kernel, direct differences              */
#define STAG_KDE_FORM_TC 2       /* tcgen05/TMEM tensor-core kernel, split-FP16 products         */
#define STAG_KDE_FORM_SIMT_F64 3 /* FP64 direct differences (for FP64 inputs)                     */

typedef struct stag_kde stag_kde_t; /* opaque handle */

typedef struct stag_kde_opts {
    int form;       /* STAG_KDE_FORM_*; 0 = AUTO                                    */
    int normalise;  /* 1: return (1/n) * sum (the paper's K(q)); 0: the plain sum     */
    int device;     /* CUDA device ordinal; -1 = the calling thread's current device  */
    int tc_no_check;/* tensor-core form only. 0 (default): every query gets an error   *
                     * estimate; those above 7.5e-5 relative are recomputed with the    *
                     * plain FP32 form. 1: skip the estimate and keep every result.     */
    int kernel;     /* STAG_KDE_KERNEL_*; 0 = Gaussian                                */
    int reserved[3];/* must be zero                                                   */
} stag_kde_opts;

/* Fills *o with the defaults (AUTO form, unnormalised, current device, Gaussian kernel). */
void stag_kde_opts_init(stag_kde_opts *o);

/*
 * Creates a handle holding a device copy of X (n x d, FP32, host memory) with
 * bandwidth a. The caller may free X on return. Default options.
 * Device memory held for the point set: the plain form's tiled copy (about n * d_pad * 4
 * bytes, d_pad = d rounded up to 4); the tensor-core form adds the FP16 splits of the
 * points (about n * (2 * Kp + 16) * 2 bytes, Kp = d rounded up to 16, 32, 64 or 128),
 * per-tile centres and radii, and for d <= 16 a k-d ordered FP32 copy (n * d * 4 bytes)
 * from which flagged queries are recomputed. Per-query scratch comes on top
 * (stag_kde_reserve).
 * Returns NULL on error (see stag_kde_last_error()).
 */
stag_kde_t *stag_kde_create(const float *X, int64_t n, int64_t d, double a);

/*
 * As stag_kde_create with an explicit element type (STAG_KDE_F32 or STAG_KDE_F64) and
 * options (NULL = defaults). FP64 data selects STAG_KDE_FORM_SIMT_F64 under AUTO.
 */
stag_kde_t *stag_kde_create_ex(const void *X, int dtype, int64_t n, int64_t d, double a,
                               const stag_kde_opts *opts);

/*
 * Synchronous query with host buffers: Q is m x d in the handle's element type (FP32
 * for stag_kde_create), out receives m doubles. Copies Q to the device, runs the
 * kernels on the handle's own stream, copies the result back and waits.
 * Returns 0, or a negative code with out untouched.
 */
int stag_kde_query(stag_kde_t *h, const void *Q, int64_t m, double *out);

/*
 * Asynchronous query on device buffers: dQ (m x d, handle's element type) and dOut
 * (m doubles) are device pointers on the handle's device; `stream` is a cudaStream_t
 * (NULL = the legacy default stream). Work is queued and the call returns; dOut is
 * valid once the stream reaches that point. Only sizes and pointers are validated;
 * non-finite values in dQ propagate to the outputs instead of being rejected.
 * Scratch memory is owned by the handle and grown on demand (a growth synchronises the
 * handle's device); stag_kde_reserve() pre-sizes it, after which the call allocates
 * nothing for m <= the reserved size.
 */
int stag_kde_query_dev(stag_kde_t *h, const void *dQ, int64_t m, double *dOut, void *stream);

/*
 * Weighted subset sums, the estimator that random sampling (every sampled point
 * weighted n/s) and the CKNS scheme (weights 2^i on hashed candidates) evaluate
 * (Sec. 3.1): for every query j, over its own list of (point index, weight) pairs,
 *     out[j] = sum_{p = off[j] .. off[j+1]-1} W[p] k(||q_j - x_{idx[p]}||)
 * (times 1/n when the handle normalises), in the handle's kernel function k. Q is
 * m x d FP32; off has m + 1 entries (off[0] = 0, non-decreasing; query j owns entries
 * off[j] .. off[j+1]-1, an empty list gives 0); idx has off[m] entries, each a row of X
 * as given at create (repeats allowed); W has off[m] weights, or NULL for all 1. Each
 * term is evaluated in FP32 by direct differences (the plain form's arithmetic, so the
 * same error bound) with a per-query power-of-two shift and FP64 accumulation. FP32
 * handles of any form (the point set is gathered from a row-major copy built on the
 * first call); FP64 handles return STAG_KDE_EUNSUPPORTED.
 *
 * Host variant: all buffers in host memory (pinned memory copies fastest), synchronous;
 * validates everything (the offsets on the host before any work; Q finite, indices in
 * [0, n) and finite W >= 0 on the device before the results are copied out) and returns
 * STAG_KDE_EINVAL on a violation with out untouched.
 */
int stag_kde_query_subset(stag_kde_t *h, const float *Q, int64_t m, const int64_t *off, const int64_t *idx,
                          const float *W, double *out);

/*
 * Device variant: dQ, dOff, dIdx, dW (or NULL) and dOut are device pointers on the
 * handle's device; work is queued on `stream` (a cudaStream_t) and the call returns.
 * Only pointers and m are validated; an entry whose index lies outside [0, n)
 * contributes nothing, and offsets must satisfy the host variant's rules (not checked).
 */
int stag_kde_query_subset_dev(stag_kde_t *h, const float *dQ, int64_t m, const int64_t *dOff, const int64_t *dIdx,
                              const float *dW, double *dOut, void *stream);

/*
 * ------------------------------------------------------------------ Euclidean LSH
 * E2LSH tables (Sec. 2), the candidate generator of the LSH-based estimators (Sec. 3.1):
 * L tables, each keyed by K hash functions h_{a,b}(x) = floor((<x, a> + b) / 4). The
 * caller supplies the L*K functions: A (L*K x d, row-major; row l*K + k is function k of
 * table l; drawn from N(0, I)) and B (L*K offsets, drawn from U(0, 4)); the library
 * draws no random numbers. Each hash value is decided in FP32 with a fixed order
 * (s = 0; s = fma(x_k, a_k, s) for k = 0..d-1; floor((s + b) * 0.25), saturated to int32),
 * so values are reproducible bit for bit. A point and a query share table l's bucket when
 * their K values of that table agree (buckets are keyed by a 58-bit mix of the K values;
 * two different K-tuples collide with probability ~2^-58 per pair).
 */
typedef struct stag_lsh stag_lsh_t; /* opaque handle */

/* Builds the L tables over X (n x d FP32, host; copied, not retained) on `device`
 * (-1 = current). Requires n < 2^32, d <= 384, K >= 1, 1 <= L <= 63, K*L <= 4096, finite
 * inputs. Returns NULL on error (stag_kde_last_error / stag_kde_last_error_code). */
stag_lsh_t *stag_lsh_create(const float *X, int64_t n, int64_t d, int K, int L, const float *A, const float *B,
                            int device);

/* Hash values of the rows of dQ (m x d FP32, device) under all L*K functions into dH
 * (m x L*K int32, device, row-major), queued on `stream`. */
int stag_lsh_hash_dev(stag_lsh_t *h, const float *dQ, int64_t m, int32_t *dH, void *stream);

/*
 * Near-neighbour candidates: for every query, the distinct points that share its bucket
 * in at least one table, in increasing index order, as CSR lists (off has m + 1 entries).
 * Host variant: Q (m x d FP32, host) is validated (finite); off always receives the
 * offsets and *total the number of candidates; idx receives the indices only when it is
 * not NULL and cap >= *total (otherwise call again with a large enough buffer).
 * Device variant: dQ, dOff (m + 1 int64) and dIdx (cap int64, or NULL) are device
 * buffers; dOff and *total are always written, the indices only when cap >= *total. The
 * handle keeps the last query's lists (either variant): stag_lsh_fetch (host memory,
 * synchronous) and stag_lsh_fetch_dev (device memory, on `stream`) copy them into a
 * large enough buffer without recomputing. Both variants synchronise the stream (the
 * list sizes decide allocations). The lists feed stag_kde_query_subset[_dev] directly.
 */
int stag_lsh_query(stag_lsh_t *h, const float *Q, int64_t m, int64_t *off, int64_t *idx, int64_t cap,
                   int64_t *total);
int stag_lsh_query_dev(stag_lsh_t *h, const float *dQ, int64_t m, int64_t *dOff, int64_t *dIdx, int64_t cap,
                       int64_t *total, void *stream);
int stag_lsh_fetch(stag_lsh_t *h, int64_t *idx, int64_t cap);
int stag_lsh_fetch_dev(stag_lsh_t *h, int64_t *dIdx, int64_t cap, void *stream);

/* Sizes of the handle (any pointer may be NULL). */
int stag_lsh_info(const stag_lsh_t *h, int64_t *n, int64_t *d, int *K, int *L);

/* Releases the tables. NULL-safe. */
void stag_lsh_destroy(stag_lsh_t *h);

/*
 * Batched evaluation: instance i evaluates the device query matrix dQs[i] (ms[i] rows,
 * the handle's element type and d) against handle hs[i] into dOuts[i] (ms[i] doubles).
 * The handles must be distinct and live on one device; ms[i] may differ, and so may the
 * handles' n, d and a. All tensor-core instances share ONE persistent kernel launch:
 * its CTAs are split into one range per operand width (sized by the width's share of the
 * work), and each range walks the (query tile, point range) units of every instance of
 * its width; every instance keeps its own partial sums and FP64 combine, so its results
 * equal a solo call on the same handle within the form's tolerance.
 * The first call with a given (handles, pointers, sizes) tunes the tensor-core launch
 * settings on the batch, reserves all scratch and captures the whole batch into a CUDA
 * graph (it synchronises the device and must not be made while a stream capture is in
 * progress); later calls with the same arguments replay the graph on `stream` without
 * allocating. A handle's later query of larger m (scratch growth) or destruction
 * invalidates the cached graph (it is rebuilt on the next call). Work is asynchronous:
 * results are valid once `stream` reaches this point. STAG_KDE_ETIMEDOUT reports a
 * bounded wait that expired during the previous replay of the same batch.
 */
int stag_kde_query_batch(stag_kde_t *const *hs, const void *const *dQs, const int64_t *ms,
                         double *const *dOuts, int64_t count, void *stream);

/*
 * Times the tensor-core form's launch settings (epilogue warp groups, point tiles per
 * work unit) on the given device query batch and keeps the fastest for this handle's
 * later queries. No-op for other forms. Synchronises; allocates a temporary output.
 */
int stag_kde_autotune(stag_kde_t *h, const void *dQ, int64_t m);

/*
 * Degrees of the fully connected similarity graph on the handle's own points (Sec. 4.1):
 * dOut[i] = sum_{j=1..n} exp(-a ||x_i - x_j||^2) for every point i in its original order
 * (the density at every data point; the j = i term is exp(0) = 1). exclude_self = 1
 * subtracts that term (1, or 1/n when normalised) afterwards, so its absolute error is that
 * of the full sum. dOut: n doubles in device memory; asynchronous on `stream`. FP32
 * handles only; uses the handle's query scratch.
 */
int stag_kde_degrees(stag_kde_t *h, int exclude_self, double *dOut, void *stream);

/* Pre-sizes the handle's scratch for queries of up to m rows. */
int stag_kde_reserve(stag_kde_t *h, int64_t m);

/* Reads back the handle's parameters; any pointer may be NULL. `form` is the form the
 * handle evaluates with (AUTO resolved). */
int stag_kde_info(const stag_kde_t *h, int64_t *n, int64_t *d, double *a, int *dtype, int *form);

/* Number of queries of the handle's most recent query call that the tensor-core
 * form's error estimate handed to the plain FP32 form (0 for other forms).
 * Synchronises with the device. */
int stag_kde_last_recomputed(stag_kde_t *h, int64_t *count);

/*
 * Limit, in nanoseconds, of each bounded wait inside the tensor-core kernel (its warps
 * hand shared-memory stages and TMEM accumulators to one another through mbarriers;
 * every wait on one gives up after this long). On expiry the kernel records an error,
 * makes its other warps stop, waits (again bounded) for its own copies and MMAs in
 * flight, frees its TMEM and returns; the call that synchronises on the result reports
 * STAG_KDE_ETIMEDOUT and the handle stays usable. 0 restores the default of 2 s; the
 * limit must not exceed 60 s. A watchdog for deployments, and the way tests make a wait
 * expire without faulting the GPU. No effect on the other forms.
 */
int stag_kde_set_wait_limit(stag_kde_t *h, int64_t limit_ns);

/* Releases the handle and its device memory. NULL-safe. */
void stag_kde_destroy(stag_kde_t *h);

/* Thread-local description of the calling thread's last failure ("" if none). */
const char *stag_kde_last_error(void);

/* Thread-local STAG_KDE_E* code of the calling thread's last failure (0 if none): the
 * code behind a NULL from stag_kde_create / stag_kde_create_ex / stag_srv_start.
 * Failures that only set a message (argument checks) report STAG_KDE_EINVAL. */
int stag_kde_last_error_code(void);

/* Library version string. */
const char *stag_kde_version(void);

/*
 * Per-handle timing of the main (pairwise) kernel with CUDA events recorded on the
 * stream it is launched on. stag_kde_profile_begin() enables recording and clears the
 * record; stag_kde_profile_end() waits for the recorded events, returns the summed
 * kernel time in milliseconds, the number of main-kernel launches and the number of
 * query-point pairs they evaluated, and disables recording. Either pointer may be NULL.
 */
int stag_kde_profile_begin(stag_kde_t *h);
int stag_kde_profile_end(stag_kde_t *h, double *ms, int64_t *launches, double *pairs);

/*
 * Measures the ex2.approx throughput of the current device (the MUFU unit that bounds
 * the Gaussian kernel's epilogue: one ex2 per query-point pair): 8 independent chains
 * of `iters` steps per thread, 8 blocks of 256 threads per SM, timed with CUDA events
 * after a warm-up launch. Writes the kernel time (ms) and the ex2 results per second.
 * Synchronises the device; 1 <= iters <= 2^24. Not part of the paper's method: it is the
 * measured peak the benchmark reports the kernels' fraction of roofline against.
 */
int stag_kde_probe_ex2(int64_t iters, double *ms, double *ex2_per_s);

/* Number of CUDA kernels this library has launched in this process (all handles,
 * all threads). Lets a caller count the device work behind a sequence of calls. */
uint64_t stag_kde_launch_count(void);

/*
 * Allocation-free evaluation. The paper has no counterpart; this is a deployment aid.
 *
 * For callers that cannot allocate GPU memory at call time: code running inside its
 * own memory-pool or allocator callback (a nested cudaMalloc would recurse or
 * deadlock), latency-critical loops that cannot afford the device-wide
 * synchronisation cudaMalloc/cudaFree may cause, or processes whose device memory is
 * budgeted up front. The handle API above allocates (its copy of X and its scratch);
 * this call allocates nothing: no cudaMalloc, no cudaFree, no allocating library call.
 *
 * Computes out[j] = sum_i exp(-a ||q_j - x_i||^2) (unnormalised) with the plain FP32
 * form. dX (n x d), dQ (m x d) and dOut (m doubles) are device pointers on the current
 * device, row-major, owned by the caller; work is queued on `stream` (a cudaStream_t,
 * NULL = legacy default stream) and the call returns without waiting.
 *
 * Scratch: a fixed 8 MiB array in the library's device memory (every GPU that loads
 * the library holds it until the process exits) stores the per-split partial sums.
 * It limits m to at most 699050 queries per call; larger m returns STAG_KDE_EINVAL
 * with a message saying so. All calls in the process share that array, so calls whose
 * GPU work overlaps (different streams or host threads) race and give wrong results:
 * serialise them. The array needs no clearing between calls.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before any
 * CUDA stream capture. Returns 0 or a negative STAG_KDE_E* code (sizes, NULL pointers,
 * a < 0 or non-finite are rejected; values in dX/dQ are not inspected).
 */
int stag_kde_eval_noalloc(const float *dX, int64_t n, const float *dQ, int64_t m, int64_t d, double a,
                          double *dOut, void *stream);

/*
 * Serving with continuous batching. The caller creates a handle per dataset (they stay
 * resident) and starts a server over them; any thread may then submit query batches.
 * A dispatcher thread merges pending requests for the same dataset, in arrival order, into
 * launch groups of at most max_rows rows, admits a group when one of `slots` execution
 * slots is free and the device memory of the groups in flight stays within
 * mem_budget_bytes (a group larger than the budget runs alone), and runs groups of
 * different slots concurrently (one CUDA stream per slot; each slot has its own scratch
 * for every dataset). Requests arriving while others are on the GPU join the next
 * groups. Results equal a solo stag_kde_query on the same handle within the form's
 * tolerance.
 */
typedef struct stag_srv stag_srv_t;

typedef struct stag_srv_opts {
    stag_kde_t *const *datasets; /* handles (created by the caller, kept alive until stop) */
    int n_datasets;
    int slots;                   /* concurrent launch groups (default 4, at most 64)      */
    int64_t max_rows;            /* rows per launch group and per request (default 8192) */
    int64_t mem_budget_bytes;    /* device memory of the groups in flight (default 1 GiB)*/
    int reserved[4];             /* must be zero                                         */
} stag_srv_opts;

void stag_srv_opts_init(stag_srv_opts *o);

/* Starts the server: allocates the slots (streams, device and pinned staging buffers)
 * and the dispatcher thread. Returns NULL on error (stag_kde_last_error()). */
stag_srv_t *stag_srv_start(const stag_srv_opts *o);

/* Queues Q (m x d host rows in the dataset's element type, 1 <= m <= max_rows) for
 * dataset index `dataset`; out (m doubles, host) receives the densities. Q and out must
 * stay valid until stag_srv_wait returns for *ticket. */
int stag_srv_submit(stag_srv_t *s, int dataset, const void *Q, int64_t m, double *out, uint64_t *ticket);

/* Waits for a request (timeout_us < 0: no limit). Returns 0 when out is filled,
 * STAG_KDE_ETIMEDOUT if it did not finish in time (the ticket stays valid), or the
 * request's error (STAG_KDE_ECANCELED for a cancelled request). A ticket is released
 * by the wait that returns its final status. */
int stag_srv_wait(stag_srv_t *s, uint64_t ticket, int64_t timeout_us);

/* Cancels a request that has not been dispatched yet; its wait returns ECANCELED. */
int stag_srv_cancel(stag_srv_t *s, uint64_t ticket);

/* Completed requests, rows, and the median / 99th-percentile latency (submit to results
 * copied out) in microseconds, since start or the last reset. */
int stag_srv_stats(stag_srv_t *s, int64_t *completed, int64_t *rows, double *p50_us, double *p99_us);
int stag_srv_reset_stats(stag_srv_t *s);

/* Stops accepting requests, cancels those not yet dispatched, waits for the groups in
 * flight and releases the server. No wait or submit may follow. NULL-safe. */
int stag_srv_stop(stag_srv_t *s);

#ifdef __cplusplus
}
#endif
#endif /* STAG_KDE_H */
