// Weighted subset sums: the estimator that random sampling (every point weighted n/s)
// and the CKNS scheme (weights 2^i on hashed candidates) evaluate (Sec. 3.1),
//     out[j] = sum_{p = off[j] .. off[j+1]-1} w[p] k(||q_j - x_{idx[p]}||),
// with each query's own list of (point index, weight) pairs, gather-fed.
//
// Layout and work split: the point set is kept row-major (FP32, built once per handle
// from the plain form's tiled copy), so a list entry is one contiguous d-float row. One
// warp owns one query at a time (grid-stride over queries); the query sits in shared
// memory and each lane takes every 32nd entry of the list: it gathers the row with
// 16-byte loads when d is a multiple of 4, forms d2 by direct differences in FP32 and
// adds w k(r) 2^-s with its own integer shift s (kernel_fn.cuh; rescaled exactly by a
// power of two when a term would exceed 2^64), flushing to FP64 every 16 terms. The 32
// lanes are merged in FP64 with a fixed shuffle order, so results are deterministic.
// The gathers dominate: per entry d*4 bytes of row (from L2 when X fits there) plus 8 + 4
// bytes of index and weight streamed from HBM. (Four entries per lane in flight, with all
// their loads issued first, measured slower: the extra registers cost more occupancy
// than the added loads in flight gained.)
#include <math.h>

#include <algorithm>

#include "internal.h"
#include "kernel_fn.cuh"

namespace stagkde {

namespace {

constexpr int kSubsetWarps = 8;  // warps per block
constexpr float kShiftInit = -0x1p100f;
constexpr float kGuard = 0x1p64f;
constexpr int kFlush = 16;

__device__ __forceinline__ int clampe(float e) { return (int)fminf(fmaxf(e, -4000.f), 4000.f); }

template <int KERN, bool kVec4>
__global__ void __launch_bounds__(32 * kSubsetWarps)
kde_subset_kernel(const float *__restrict__ X, int64_t n, int d, const float *__restrict__ Q, int64_t m,
                  const int64_t *__restrict__ off, const int64_t *__restrict__ idx, const float *__restrict__ W,
                  float negc, double scale, double *__restrict__ out) {
    extern __shared__ __align__(16) float sq_all[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *sq = sq_all + warp * d;
    const int64_t warps = (int64_t)gridDim.x * kSubsetWarps;
    for (int64_t j = (int64_t)blockIdx.x * kSubsetWarps + warp; j < m; j += warps) {
        __syncwarp();
        for (int k = lane; k < d; k += 32) sq[k] = Q[j * d + k];
        __syncwarp();
        const int64_t p0 = off[j], p1 = off[j + 1];
        float shift = kShiftInit, acc32 = 0.f;
        double acc64 = 0.0;
        int cnt = 0;
        for (int64_t p = p0 + lane; p < p1; p += 32) {
            const int64_t i = idx[p];
            if (i < 0 || i >= n) continue;  // out-of-range entries contribute nothing
            const float w = W ? W[p] : 1.f;
            const float *x = X + i * d;
            // FP32 chains over blocks of 16 coordinates, block sums added (the plain
            // form's order and error bound)
            float d2 = 0.f, b2 = 0.f;
            if constexpr (kVec4) {
                for (int k = 0; k < d; k += 4) {
                    const float4 xv = *reinterpret_cast<const float4 *>(x + k);
                    const float4 qv = *reinterpret_cast<const float4 *>(sq + k);
                    float t = qv.x - xv.x;
                    b2 = fmaf(t, t, b2);
                    t = qv.y - xv.y;
                    b2 = fmaf(t, t, b2);
                    t = qv.z - xv.z;
                    b2 = fmaf(t, t, b2);
                    t = qv.w - xv.w;
                    b2 = fmaf(t, t, b2);
                    if (((k + 4) & 15) == 0) {
                        d2 += b2;
                        b2 = 0.f;
                    }
                }
            } else {
                for (int k = 0; k < d; ++k) {
                    const float t = sq[k] - x[k];
                    b2 = fmaf(t, t, b2);
                    if (((k + 1) & 15) == 0) {
                        d2 += b2;
                        b2 = 0.f;
                    }
                }
            }
            d2 += b2;
            float e = w * kfn::term<KERN>(negc, d2, shift);
            if (!(fabsf(e) <= kGuard)) {
                // first term, or one far above the current shift: move the shift up
                const float s_new = fmaxf(ceilf(kfn::term_log2<KERN>(negc, d2)), kShiftInit);
                if (s_new > shift) {
                    const int de = clampe(shift - s_new);
                    acc32 = ldexpf(acc32, de);
                    acc64 = ldexp(acc64, de);
                    shift = s_new;
                }
                e = w * kfn::term<KERN>(negc, d2, shift);
            }
            acc32 += e;
            if (++cnt == kFlush) {
                acc64 += (double)acc32;
                acc32 = 0.f;
                cnt = 0;
            }
        }
        acc64 += (double)acc32;
        // merge the lanes: common shift = the largest, fixed butterfly order
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const double oa = __shfl_xor_sync(0xffffffffu, acc64, o);
            const float os = __shfl_xor_sync(0xffffffffu, shift, o);
            const float sm = fmaxf(shift, os);
            acc64 = ldexp(acc64, clampe(shift - sm)) + ldexp(oa, clampe(os - sm));
            shift = sm;
        }
        if (lane == 0) out[j] = ldexp(acc64, clampe(shift)) * scale;
    }
}

template <int KERN>
void launch_kern(const stag_kde *h, const float *dQ, int64_t m, const int64_t *dOff, const int64_t *dIdx,
                 const float *dW, double *dOut, cudaStream_t s) {
    const float negc = (float)(-h->a * 1.4426950408889634);  // -a log2(e)
    const double scale = h->normalise ? 1.0 / (double)h->n : 1.0;
    const unsigned grid =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(m, kSubsetWarps), (int64_t)h->sm_count * 16));
    const size_t smem = (size_t)kSubsetWarps * h->d * sizeof(float);
    if (h->d % 4 == 0)
        kde_subset_kernel<KERN, true><<<grid, 32 * kSubsetWarps, smem, s>>>(h->xrow, h->n, (int)h->d, dQ, m, dOff,
                                                                             dIdx, dW, negc, scale, dOut);
    else
        kde_subset_kernel<KERN, false><<<grid, 32 * kSubsetWarps, smem, s>>>(h->xrow, h->n, (int)h->d, dQ, m, dOff,
                                                                              dIdx, dW, negc, scale, dOut);
}

// Flags (bit 0) an index outside [0, n) and (bit 1) a weight that is negative or not
// finite, over the nnz list entries.
__global__ void subset_check_kernel(const int64_t *__restrict__ idx, const float *__restrict__ W, int64_t nnz,
                                    int64_t n, int *flag) {
    int bad = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx[p];
        if (i < 0 || i >= n) bad |= 1;
        if (W) {
            const float w = W[p];
            if (!(w >= 0.f) || !isfinite(w)) bad |= 2;
        }
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (bad && (threadIdx.x & 31) == 0) atomicOr(flag, bad);
}

}  // namespace

int subset_check_entries(const int64_t *dIdx, const float *dW, int64_t nnz, int64_t n, int *dflag, cudaStream_t s) {
    if (nnz <= 0) return 0;
    count_launch();
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nnz, 256), 152 * 16));
    subset_check_kernel<<<grid, 256, 0, s>>>(dIdx, dW, nnz, n, dflag);
    STAG_CUDA_TRY(cudaGetLastError());
    return 0;
}

int subset_prepare(stag_kde *h, cudaStream_t s) {
    if (h->xrow) return 0;
    if (h->dtype != STAG_KDE_F32 || !h->xt) return fail(STAG_KDE_EUNSUPPORTED, "subset sums: FP32 handles only");
    if ((size_t)kSubsetWarps * h->d * sizeof(float) > 48 * 1024)
        return fail(STAG_KDE_EUNSUPPORTED, "subset sums: d too large");
    STAG_CUDA_TRY(dev_malloc(&h->xrow, (size_t)(h->n * h->d) * sizeof(float)));
    int rc = simt_points_rows(h, h->xrow, s);
    if (rc) return rc;
    // later calls may come on other streams: the copy must be complete before them
    STAG_CUDA_TRY(cudaStreamSynchronize(s));
    return 0;
}

int subset_query(stag_kde *h, const float *dQ, int64_t m, const int64_t *dOff, const int64_t *dIdx, const float *dW,
                 double *dOut, cudaStream_t s, double entries) {
    int rc = subset_prepare(h, s);
    if (rc) return rc;
    count_launch();
    prof_start(h, s);
    switch (h->kernel) {
        case STAG_KDE_KERNEL_EXPONENTIAL:
            launch_kern<STAG_KDE_KERNEL_EXPONENTIAL>(h, dQ, m, dOff, dIdx, dW, dOut, s);
            break;
        case STAG_KDE_KERNEL_LOGISTIC:
            launch_kern<STAG_KDE_KERNEL_LOGISTIC>(h, dQ, m, dOff, dIdx, dW, dOut, s);
            break;
        default:
            launch_kern<STAG_KDE_KERNEL_GAUSSIAN>(h, dQ, m, dOff, dIdx, dW, dOut, s);
    }
    prof_stop(h, s, entries);
    STAG_CUDA_TRY(cudaGetLastError());
    return 0;
}

}  // namespace stagkde
