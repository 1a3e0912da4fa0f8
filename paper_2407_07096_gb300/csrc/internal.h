// Internal declarations shared by the library's translation units (not installed).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "stag_kde.h"

namespace stagkde {

// ---------------------------------------------------------------------------------
// Error reporting (thread-local last error).
// ---------------------------------------------------------------------------------
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define STAG_CUDA_TRY(expr)                                               \
    do {                                                                  \
        cudaError_t _e = (expr);                                          \
        if (_e != cudaSuccess) return ::stagkde::cuda_fail(_e, #expr);    \
    } while (0)

// ---------------------------------------------------------------------------------
// Layout constants of the plain CUDA-core kernel.
// Points and queries are stored "tile-transposed": tile t of 64 rows is a d_pad x 64
// block, coordinate k of row r at [t][k][r]. d_pad = d rounded up to 4; the padding
// coordinates are zero in both X and Q, so they add (0 - 0)^2 = 0 to every distance.
// ---------------------------------------------------------------------------------
constexpr int kSimtTile = 64;  // rows per tile (queries per block, points per tile)
constexpr int kSimtKC = 32;    // coordinates per shared-memory chunk
// Up to this d_pad the plain form keeps a block's whole query tile in shared memory
// (d_pad x 64 floats, 32 KB at 128) and streams only the point chunks; beyond it the
// query tile is streamed chunk by chunk beside the points.
constexpr int kSimtResidentMaxD = 128;
inline size_t simt_resident_bytes(int d_pad) { return (size_t)d_pad * kSimtTile * sizeof(float); }

// Every device allocation of the library goes through dev_malloc. It is also the
// library's host-side fault-injection point: while the environment variable
// STAG_KDE_INJECT_ALLOC_FAIL holds a positive integer k, the k-th device allocation
// counted from the moment the variable took that value fails as cudaErrorMemoryAllocation
// (reported as STAG_KDE_ENOMEM), so tests can fail each allocation of a call in turn
// without exhausting the GPU.
cudaError_t dev_malloc_bytes(void **p, size_t bytes);
template <typename T>
inline cudaError_t dev_malloc(T **p, size_t bytes) {
    return dev_malloc_bytes(reinterpret_cast<void **>(p), bytes);
}

// Process-wide count of kernel launches (reported by stag_kde_launch_count).
void count_launch(int k = 1);
void uncount_launches(uint64_t k);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// Per-split partial results: sum (FP64) and an integer power-of-two shift (stored as
// float). The true partial is sum * 2^shift.
struct Partials {
    double *sum = nullptr;
    float *shift = nullptr;
    int64_t cap = 0;  // capacity in (split, query) entries
};

struct TcData;  // tensor-core form data (kde_tc.cu)

}  // namespace stagkde

struct stag_kde {
    int device = 0;
    int64_t n = 0, d = 0;
    double a = 0.0;
    int dtype = STAG_KDE_F32;
    int form = STAG_KDE_FORM_SIMT_F32;
    int normalise = 0;
    int kernel = STAG_KDE_KERNEL_GAUSSIAN;  // k(r): Gaussian, exponential or logistic
    bool tc_check = true;  // recompute queries the tensor-core error estimate flags
    uint64_t scratch_epoch = 0;    // bumped whenever scratch is reallocated (graphs hold pointers)
    bool is_view = false;          // shares another handle's point-set data (serving slots)
    int tune_eg = 0;               // tensor-core epilogue warp groups (0 = default)
    int tune_tiles_per_unit = 0;   // point tiles per work unit (0 = heuristic)
    uint64_t wait_ns = 2000000000ull;  // limit of each bounded device wait (stag_kde_set_wait_limit)
    cudaStream_t stream = nullptr;  // the handle's own stream (host API)

    // plain FP32 form: tile-transposed points
    float *xt = nullptr;
    int64_t n_tiles = 0;
    int d_pad = 0;

    // FP64 form: row-major points
    double *x64 = nullptr;

    // tensor-core form
    stagkde::TcData *tc = nullptr;

    // scratch (grown on demand, owned by the handle)
    void *q_dev = nullptr;  // device copy of host queries
    int64_t q_dev_cap = 0;  // bytes
    float *qt = nullptr;    // tile-transposed queries
    int64_t qt_cap = 0;     // floats
    double *out_dev = nullptr;
    int64_t out_cap = 0;  // bytes
    stagkde::Partials part;
    float *xrow = nullptr;    // row-major FP32 point set for gathers (subset sums), built on first use
    void *sub_dev = nullptr;  // host subset call: device copies of offsets, indices, weights
    int64_t sub_dev_cap = 0;  // bytes
    int *flag_dev = nullptr;  // input-validation flag
    cudaStream_t copy_stream[2] = {nullptr, nullptr};  // host subset call: extra streams for the list copies
    cudaEvent_t copy_done[2] = {nullptr, nullptr};
    int *flag_host = nullptr; // pinned mirror
    int sm_count = 0;

    // main-kernel timing (stag_kde_profile_begin/end)
    bool profiling = false;
    std::vector<cudaEvent_t> prof_events;  // start/stop pairs
    std::vector<cudaEvent_t> prof_pool;    // reusable events
    int64_t prof_launches = 0;
    double prof_pairs = 0.0;
};

namespace stagkde {

// Brackets a main-kernel launch with events when the handle is profiling.
void prof_start(stag_kde *h, cudaStream_t s);
void prof_stop(stag_kde *h, cudaStream_t s, double pairs);

// kde_simt.cu
int simt_prepare_points(stag_kde *h, const float *dX);  // dX: device row-major n x d
int simt_query_f32(stag_kde *h, const float *dQ, int64_t m, double *dOut, cudaStream_t s,
                   int *dflag);
int simt_query_f64(stag_kde *h, const double *dQ, int64_t m, double *dOut, cudaStream_t s,
                   int *dflag);
int ensure_partials(stag_kde *h, int64_t entries);
// The point set in its original order, row-major (from the plain form's tiled copy).
int simt_points_rows(stag_kde *h, float *out, cudaStream_t s);
int launch_subtract(double *v, int64_t count, double one, cudaStream_t s);
// Sizes the plain form's scratch (tiled queries, partials) for queries of up to m rows.
int simt_reserve(stag_kde *h, int64_t m);
int ensure_qt(stag_kde *h, int64_t floats);
// Grouped pruned recompute (tensor-core form, d > 16): the plain form's register-tiled
// kernel over lists of kept point tiles per query group (see kde_simt.cu), the gather of
// rows idx[0 .. *count) into tile-transposed query tiles, and a tile-transposed copy of
// row-major points (the k-d ordered set).
int simt_list_launch(const stag_kde *h, const float *xt, const float *qt, const int *kept, int64_t kstride,
                     const int *kcount, const int *item_off, const int *n_groups, int seg, int per, double *part_sum,
                     float *part_shift, cudaStream_t s);
int simt_gather_rows(const stag_kde *h, const float *dQ, const int *idx, const int *count, int64_t m_cap, float *qt,
                     cudaStream_t s);
int simt_tiles_from_rows(const stag_kde *h, const float *rows, float *out, cudaStream_t s);
int launch_check_finite_f32(const float *p, int64_t count, int *dflag, cudaStream_t s, int bit = 1);
int launch_check_finite_f64(const double *p, int64_t count, int *dflag, cudaStream_t s);

// kde_subset.cu: weighted subset sums over per-query (index, weight) lists. `entries`
// (the list entries, if known on the host) only feeds the profiling counters.
int subset_prepare(stag_kde *h, cudaStream_t s);
// Sets bit 0 of *dflag if an index lies outside [0, n), bit 1 if a weight is negative
// or not finite.
int subset_check_entries(const int64_t *dIdx, const float *dW, int64_t nnz, int64_t n, int *dflag, cudaStream_t s);
int subset_query(stag_kde *h, const float *dQ, int64_t m, const int64_t *dOff, const int64_t *dIdx, const float *dW,
                 double *dOut, cudaStream_t s, double entries);

// kde_combine.cu
int launch_combine(const double *part_sum, const float *part_shift, int64_t m, int splits,
                   double scale, double *out, cudaStream_t s);

// kd_order.cu
// Stable LSD radix sort of (64-bit key, 32-bit value) pairs by key bits [0, bits); the
// result ends in (keys, vals); hist holds radix_sort_hist_entries(n) entries (the digit
// histogram, 256 per block of 4096 keys, and the totals of its scan chunks).
// With dcount (device memory) only the first min(n, *dcount) entries are sorted (the
// buffers are still sized for n; the rest is left as it is).
int radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *ktmp, uint32_t *vtmp, uint32_t *hist, int64_t n,
                     int bits, cudaStream_t s, const int *dcount = nullptr);
inline int64_t radix_sort_blocks(int64_t n) { return ceil_div(n, 4096); }
inline int64_t radix_sort_hist_entries(int64_t n) {
    const int64_t e = 256 * radix_sort_blocks(n);
    return e + ceil_div(e, 4096) + 1;
}
int kd_reorder(const float *dX, int64_t n, int64_t d, int BN, float *dXs, cudaStream_t s);

// kde_tc.cu
int tc_tile_points(int64_t d);
int tc_prepare_points(stag_kde *h, const float *dX);
int tc_query(stag_kde *h, const float *dQ, int64_t m, double *dOut, cudaStream_t s, int *dflag);
void tc_free(stag_kde *h);
// The kernel's error code (a bounded wait that expired): tc_error_enqueue queues its copy
// to the host on s; after s has been synchronised, tc_error_take reports and clears it.
int tc_error_enqueue(stag_kde *h, cudaStream_t s);
int tc_error_take(stag_kde *h, cudaStream_t s);
int tc_reserve(stag_kde *h, int64_t m, int tiles_per_unit);
int tc_make_view(const stag_kde *base, stag_kde *view);
// Pieces of a tensor-core query for the batched path (kde_tc.cu).
int tc_operand_width(const stag_kde *h);
int tc_epilogue_groups();
size_t tc_inst_size();
int tc_prep_public(stag_kde *h, const float *dQ, int64_t m, cudaStream_t s);
int64_t tc_fill_inst(const stag_kde *h, int64_t m, int tiles_per_unit, int64_t unit_begin, void *inst,
                     int64_t *splits);
// One persistent launch for every operand width (16, 32, 64, 128 at index 0..3): table c
// holds n_inst[c] instances with units[c] units in all; work[c] (any unit, 0 for an empty
// width) sizes the width's share of the CTAs.
int tc_launch_multi(int eg, const void *const tables[4], const int n_inst[4], const int64_t units[4],
                    const double work[4], int *err, int sm_count, uint64_t wait_ns, cudaStream_t s);
int tc_finish_public(stag_kde *h, const float *dQ, int64_t m, int64_t splits, double *dOut, cudaStream_t s);
// kde_batch.cu
void batch_forget_handle(stag_kde *h);

// stag_kde_api.cu: views (same point set, separate scratch) and their release
stag_kde *make_view(stag_kde *base);
void free_view(stag_kde *view);
int tc_fixed_rows(stag_kde *h, int64_t *count);
bool tc_supported(int64_t d);

}  // namespace stagkde
