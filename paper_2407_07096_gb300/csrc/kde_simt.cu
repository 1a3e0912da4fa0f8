// Plain CUDA-core forms of exact KDE (Sec. 3: K(q) = sum_i k(||q - x_i||), by default the
// Gaussian kernel k(r) = exp(-a r^2); also the exponential and logistic kernels of Sec. 3),
// evaluated over every data point, the "naive" exact method of Sec. 3 / Sec. 6.1.
//
//  * kde_simt_f32_kernel: FP32 direct differences sum_k (q_k - x_k)^2, register-tiled
//    4 queries x 4 points per thread, 64 x 64 pairs per 256-thread block, shared-memory
//    chunks of 32 coordinates fed by cp.async; the exp and the row sum are fused, so no
//    m x n matrix is ever written.
//  * kde_simt_f64_kernel: FP64 direct differences and FP64 exp, for FP64 inputs.
//
// Exponent arithmetic (FP32 form). With c = a log2(e), every term is evaluated as
//     e = 2^(-c d2 - s)      (one fused multiply-add, then ex2.approx)
// where s is a per-row integer shift, so that terms near the row maximum are computed
// with a small argument (accurate) and rows whose every term is below FP32's range
// (a d2 > 87, e.g. d = 128, a = 1) are still represented. s starts at -2^100, which
// forces the first tile through the rescale path; a tile whose FP32 sum exceeds 2^64
// (or is not finite) recomputes with s = ceil(max of its exponents) after rescaling
// the row's accumulators by the exact power of two 2^(s_old - s_new). Terms more than
// 2^-126 below the shift flush to zero (relative contribution < n 2^-126).
//
// Other kernel functions (Sec. 3): the exponential and logistic kernels of r = sqrt(d2),
// in the same shifted form (kernel_fn.cuh).
//
// Squared distances: FP32 FMA chains over blocks of 16 coordinates, block sums added
// (about half the rounding error of a single chain at d >= 32).
// Summation: per thread, FP32 over 16 tiles (64 terms), then FP64; the 16 threads that
// share a row are combined in FP64 with a fixed shuffle pattern; splits of the point set
// are combined in FP64 by kde_combine.cu. Every order is fixed, so results are
// bitwise reproducible.
#include <math.h>

#include "f32x2.cuh"
#include "internal.h"
#include "kernel_fn.cuh"

namespace stagkde {

namespace {

constexpr float kShiftFloor = -0x1p100f;  // initial shift (an exact integer)
constexpr float kOverflowGuard = 0x1p64f;
constexpr int kFlushTiles = 16;
constexpr int kSumBlock = 16;  // coordinates per partial chain of a squared distance

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ int clamp_exp(float e) {
    return (int)fminf(fmaxf(e, -4000.f), 4000.f);
}

// Row state: value = (acc64 + acc32) * 2^shift.
struct RowAcc {
    float shift;
    float acc32;
    double acc64;
};

__device__ __forceinline__ void rescale(RowAcc &r, float s_new) {
    int de = clamp_exp(r.shift - s_new);  // <= 0
    r.acc32 = ldexpf(r.acc32, de);
    r.acc64 = ldexp(r.acc64, de);
    r.shift = s_new;
}

using kfn::term;
using kfn::term_log2;

// Adds the four terms k(r_j) 2^-shift (j < valid) to row r.
template <int KERN>
__device__ __forceinline__ void add_terms(RowAcc &r, const float d2[4], float negc, int valid) {
    float ts = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float e = term<KERN>(negc, d2[j], r.shift);
        ts += (j < valid) ? e : 0.f;
    }
    if (!(ts <= kOverflowGuard)) {
        float mx = -INFINITY;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j < valid) mx = fmaxf(mx, term_log2<KERN>(negc, d2[j]));
        float s_new = fmaxf(ceilf(mx), kShiftFloor);
        if (s_new > r.shift) rescale(r, s_new);
        ts = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float e = term<KERN>(negc, d2[j], r.shift);
            ts += (j < valid) ? e : 0.f;
        }
    }
    r.acc32 += ts;
}

__device__ __forceinline__ void merge(RowAcc &r, double oacc, float oshift) {
    float sm = fmaxf(r.shift, oshift);
    r.acc64 = ldexp(r.acc64, clamp_exp(r.shift - sm)) + ldexp(oacc, clamp_exp(oshift - sm));
    r.shift = sm;
}

// One work item: a query tile of 64 rows (qbase, tile-transposed) against `ntiles` point
// tiles, tile_at(i) giving the index of the i-th. Rows at or past rows_valid are
// computed on zero padding and not stored; the partials of row r go to out_sum[r] and
// out_shift[r].
template <bool kQResident, int KERN, class TileAt>
__device__ __forceinline__ void simt_item(float (*sX)[kSimtKC * kSimtTile], float (*sQ)[kSimtKC * kSimtTile],
                                          const float *__restrict__ xt, int64_t n, const float *__restrict__ qbase,
                                          int d_pad, float negc, int64_t ntiles, TileAt tile_at, int64_t rows_valid,
                                          double *__restrict__ out_sum, float *__restrict__ out_shift) {
    const int tid = threadIdx.x;
    const int tx = tid & 15;  // point group: points 4*tx .. 4*tx+3 of the tile
    const int ty = tid >> 4;  // query group: rows 4*ty .. 4*ty+3 of the block
    const int nch = (d_pad + kSimtKC - 1) / kSimtKC;

    RowAcc row[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) row[i] = RowAcc{kShiftFloor, 0.f, 0.0};

    auto load = [&](int stage, int64_t t, int ch) {
        const int k0 = ch * kSimtKC;
        const int klen = min(kSimtKC, d_pad - k0);
        const int nvec = klen * (kSimtTile / 4);
        const float *src = xt + (t * d_pad + k0) * kSimtTile;
        for (int v = tid; v < nvec; v += 256) cp_async16(&sX[stage][v * 4], src + v * 4);
        if (!kQResident) {
            const float *qs = qbase + (int64_t)k0 * kSimtTile;
            for (int v = tid; v < nvec; v += 256) cp_async16(&sQ[kQResident ? 0 : stage][v * 4], qs + v * 4);
        }
    };

    if (kQResident) {
        const int nvec = d_pad * (kSimtTile / 4);
        for (int v = tid; v < nvec; v += 256) cp_async16(&sQ[0][v * 4], qbase + v * 4);
    }
    const int64_t iters = ntiles * nch;
    if (iters > 0) load(0, tile_at(0), 0);
    cp_async_commit();

    // squared distances of the 4 x 4 pairs, as packed column pairs (4*tx+0,1) and (+2,3)
    uint64_t d2p[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i) d2p[i][0] = d2p[i][1] = 0ull;

    int group = 0;
    for (int64_t it = 0; it < iters; ++it) {
        const int stage = (int)(it & 1);
        if (it + 1 < iters) {
            load(stage ^ 1, tile_at((it + 1) / nch), (int)((it + 1) % nch));
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();

        const int ch = (int)(it % nch);
        const int klen = min(kSimtKC, d_pad - ch * kSimtKC);
        const float *xs = sX[stage];
        const float *qs = kQResident ? sQ[0] + ch * kSimtKC * kSimtTile : sQ[kQResident ? 0 : stage];
        // blocks of kSumBlock coordinates: each block's squares are summed in a chain of
        // its own and the block sum is added to the pair's total, which keeps the
        // accumulated rounding error of d2 about half that of one chain over all d
        for (int kb = 0; kb < klen; kb += kSumBlock) {
            const int ke = min(klen, kb + kSumBlock);
            uint64_t b2p[4][2];
#pragma unroll
            for (int i = 0; i < 4; ++i) b2p[i][0] = b2p[i][1] = 0ull;
#pragma unroll 4
            for (int k = kb; k < ke; ++k) {
                const float4 qv = *reinterpret_cast<const float4 *>(&qs[k * kSimtTile + ty * 4]);
                const float4 xv = *reinterpret_cast<const float4 *>(&xs[k * kSimtTile + tx * 4]);
                const float qa[4] = {qv.x, qv.y, qv.z, qv.w};
                const uint64_t x01 = f2::pack(xv.x, xv.y), x23 = f2::pack(xv.z, xv.w);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint64_t qq = f2::pack(qa[i], qa[i]);
                    const uint64_t df0 = f2::sub(qq, x01), df1 = f2::sub(qq, x23);
                    b2p[i][0] = f2::fma(df0, df0, b2p[i][0]);
                    b2p[i][1] = f2::fma(df1, df1, b2p[i][1]);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                d2p[i][0] = f2::add(d2p[i][0], b2p[i][0]);
                d2p[i][1] = f2::add(d2p[i][1], b2p[i][1]);
            }
        }
        __syncthreads();

        if (ch == nch - 1) {
            const int64_t t = tile_at(it / nch);
            const int64_t col0 = t * kSimtTile + tx * 4;
            const int valid = (int)max((int64_t)0, min((int64_t)4, n - col0));
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float d2[4];
                f2::unpack(d2p[i][0], d2[0], d2[1]);
                f2::unpack(d2p[i][1], d2[2], d2[3]);
                add_terms<KERN>(row[i], d2, negc, valid);
                d2p[i][0] = d2p[i][1] = 0ull;
            }
            if (++group == kFlushTiles) {
                group = 0;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    row[i].acc64 += (double)row[i].acc32;
                    row[i].acc32 = 0.f;
                }
            }
        }
    }

#pragma unroll
    for (int i = 0; i < 4; ++i) {
        row[i].acc64 += (double)row[i].acc32;
        row[i].acc32 = 0.f;
    }
    // Combine the 16 threads of the half-warp that share rows 4*ty..4*ty+3.
#pragma unroll
    for (int off = 8; off >= 1; off >>= 1) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const double oa = __shfl_xor_sync(0xffffffffu, row[i].acc64, off);
            const float os = __shfl_xor_sync(0xffffffffu, row[i].shift, off);
            merge(row[i], oa, os);
        }
    }
    if (tx == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = ty * 4 + i;
            if (r < rows_valid) {
                out_sum[r] = row[i].acc64;
                out_shift[r] = row[i].shift;
            }
        }
    }
}

// The contiguous point tiles of split `split` against query tile `qtile`; partials of
// query q at part_sum[split * m + q] (rows from m_real on are not stored).
template <bool kQResident, int KERN>
__device__ __forceinline__ void simt_split_item(float (*sX)[kSimtKC * kSimtTile], float (*sQ)[kSimtKC * kSimtTile],
                                                const float *__restrict__ xt, int64_t n, int64_t n_tiles,
                                                const float *__restrict__ qt, int64_t m, int64_t m_real, int d_pad,
                                                float negc, int64_t tiles_per_split, double *__restrict__ part_sum,
                                                float *__restrict__ part_shift, int64_t qtile, int64_t split) {
    const int64_t t0 = split * tiles_per_split;
    const int64_t t1 = min(n_tiles, t0 + tiles_per_split);
    const int64_t off = split * m + qtile * kSimtTile;
    simt_item<kQResident, KERN>(sX, sQ, xt, n, qt + qtile * (int64_t)d_pad * kSimtTile, d_pad, negc,
                                  max((int64_t)0, t1 - t0), [t0](int64_t i) { return t0 + i; },
                                  m_real - qtile * kSimtTile, part_sum + off, part_shift + off);
}

template <bool kQResident, int KERN>
__global__ void __launch_bounds__(256, 2)
kde_simt_f32_kernel(const float *__restrict__ xt, int64_t n, int64_t n_tiles, const float *__restrict__ qt, int64_t m,
                    int d_pad, float negc, int64_t tiles_per_split, double *__restrict__ part_sum,
                    float *__restrict__ part_shift) {
    __shared__ __align__(16) float sX[2][kSimtKC * kSimtTile];
    // resident query tile: all d_pad coordinates (dynamic, d_pad x 64 floats); otherwise
    // double-buffered chunks of the query tile
    extern __shared__ __align__(16) float sQres[];
    __shared__ __align__(16) float sQchunk[kQResident ? 1 : 2][kQResident ? 4 : kSimtKC * kSimtTile];
    auto sQ = kQResident ? reinterpret_cast<float (*)[kSimtKC * kSimtTile]>(sQres)
                         : reinterpret_cast<float (*)[kSimtKC * kSimtTile]>(&sQchunk[0][0]);
    // one block per (query tile, split)
    simt_split_item<kQResident, KERN>(sX, sQ, xt, n, n_tiles, qt, m, m, d_pad, negc, tiles_per_split, part_sum,
                                        part_shift, blockIdx.x, blockIdx.y);
}

// The grouped recompute of the tensor-core form's flagged queries (kde_tc.cu): work item
// w belongs to query group g (item_off[g] <= w < item_off[g + 1]; groups = *n_groups) and
// covers the group's kept point tiles [s * seg, min(kcount[g], (s + 1) * seg)) of the
// list kept[g * kstride ..], s = w - item_off[g]; each kept tile is `per` consecutive
// 64-point tiles of xt. Query group g is tile g of qt (64 gathered rows). The partials of
// row r go to part_sum[w * 64 + r]. A fixed grid walks the items (counts on the device).
template <bool kQResident, int KERN>
__global__ void __launch_bounds__(256, 2)
kde_simt_f32_list_kernel(const float *__restrict__ xt, int64_t n, int64_t n_tiles, const float *__restrict__ qt,
                         int d_pad, float negc, const int *__restrict__ kept, int64_t kstride,
                         const int *__restrict__ kcount, const int *__restrict__ item_off,
                         const int *__restrict__ n_groups, int seg, int per, double *__restrict__ part_sum,
                         float *__restrict__ part_shift) {
    __shared__ __align__(16) float sX[2][kSimtKC * kSimtTile];
    // resident query tile: all d_pad coordinates (dynamic, d_pad x 64 floats); otherwise
    // double-buffered chunks of the query tile
    extern __shared__ __align__(16) float sQres[];
    __shared__ __align__(16) float sQchunk[kQResident ? 1 : 2][kQResident ? 4 : kSimtKC * kSimtTile];
    auto sQ = kQResident ? reinterpret_cast<float (*)[kSimtKC * kSimtTile]>(sQres)
                         : reinterpret_cast<float (*)[kSimtKC * kSimtTile]>(&sQchunk[0][0]);
    const int G = *n_groups;
    const int total = G > 0 ? item_off[G] : 0;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        __syncthreads();  // the previous item's shared-memory reads are done
        int lo = 0, hi = G - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (item_off[mid] <= w)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int g = lo;
        const int k0 = (w - item_off[g]) * seg;
        const int k1 = min(kcount[g], k0 + seg);
        const int *list = kept + (int64_t)g * kstride + k0;
        // the point set's last tile may cover fewer than `per` 64-point tiles; it can only
        // be the list's last entry (the lists ascend), whose tail is enumerated last
        int64_t nt = (int64_t)(k1 - k0) * per;
        if (k1 > k0) nt -= max((int64_t)0, ((int64_t)list[k1 - k0 - 1] + 1) * per - n_tiles);
        simt_item<kQResident, KERN>(
            sX, sQ, xt, n, qt + (int64_t)g * d_pad * kSimtTile, d_pad, negc, nt,
            [list, per](int64_t i) { return (int64_t)list[i / per] * per + i % per; }, kSimtTile,
            part_sum + (int64_t)w * kSimtTile, part_shift + (int64_t)w * kSimtTile);
    }
}

// Row-major n x d -> tile-transposed [tile][d_pad][64], zero padded.
template <typename T>
__global__ void to_tiles_kernel(const T *__restrict__ src, int64_t rows, int64_t d, int d_pad,
                                int64_t n_tiles, float *__restrict__ dst) {
    const int64_t total = n_tiles * d_pad * kSimtTile;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx % kSimtTile);
        const int64_t rest = idx / kSimtTile;
        const int k = (int)(rest % d_pad);
        const int64_t t = rest / d_pad;
        const int64_t row = t * kSimtTile + r;
        float v = 0.f;
        if (row < rows && k < d) v = (float)src[row * d + k];
        dst[idx] = v;
    }
}

// ORs `bit` into *flag when a value is not finite or exceeds 1e15 in magnitude.
template <typename T>
__global__ void check_finite_kernel(const T *__restrict__ p, int64_t count, int *flag, int bit) {
    int bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)p[i];
        bad |= !(fabs(v) <= 1e15);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, bit);
}

// FP64 form: one thread per query, points staged through shared memory, summed in
// index order with FP64 exp (plain double arithmetic, for FP64 inputs).
__global__ void __launch_bounds__(128)
kde_simt_f64_kernel(const double *__restrict__ X, int64_t n, const double *__restrict__ Q,
                    int64_t m, int64_t d, double a, int kern, double *__restrict__ out) {
    extern __shared__ double sx[];
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t tp = max((int64_t)1, (int64_t)(4096 / d));  // points per staged tile
    double s = 0.0;
    for (int64_t i0 = 0; i0 < n; i0 += tp) {
        const int64_t cnt = min(tp, n - i0);
        __syncthreads();
        for (int64_t e = threadIdx.x; e < cnt * d; e += blockDim.x) sx[e] = X[i0 * d + e];
        __syncthreads();
        if (j < m) {
            const double *q = Q + j * d;
            for (int64_t i = 0; i < cnt; ++i) {
                double d2 = 0.0;
                for (int64_t k = 0; k < d; ++k) {
                    const double t = q[k] - sx[i * d + k];
                    d2 = fma(t, t, d2);
                }
                if (kern == STAG_KDE_KERNEL_GAUSSIAN) {
                    s += exp(-a * d2);
                } else {
                    const double x = a * sqrt(d2);
                    s += kern == STAG_KDE_KERNEL_EXPONENTIAL ? exp(-x) : 4.0 / (2.0 + exp(x) + exp(-x));
                }
            }
        }
    }
    if (j < m) out[j] = s;
}

// Rows idx[0 .. *count) of the row-major Q, in that order, into the tile-transposed
// layout (rows past *count are zero).
__global__ void gather_rows_tiles_kernel(const float *__restrict__ Q, int64_t d, int d_pad,
                                         const int *__restrict__ idx, const int *__restrict__ count, int64_t m_cap,
                                         float *__restrict__ qt) {
    const int64_t cnt = *count;
    const int64_t total = ((min(cnt, m_cap) + kSimtTile - 1) / kSimtTile) * d_pad * kSimtTile;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % kSimtTile);
        const int64_t rest = e / kSimtTile;
        const int k = (int)(rest % d_pad);
        const int64_t j = (rest / d_pad) * kSimtTile + r;
        qt[e] = (j < cnt && k < d) ? Q[(int64_t)idx[j] * d + k] : 0.f;
    }
}

int grid_for(int64_t total, int threads) {
    return (int)std::min<int64_t>(ceil_div(total, threads), 152 * 16);
}

}  // namespace

int ensure_partials(stag_kde *h, int64_t entries) {
    if (h->part.cap >= entries) return 0;
    ++h->scratch_epoch;
    if (h->part.sum) cudaFree(h->part.sum);
    if (h->part.shift) cudaFree(h->part.shift);
    h->part = Partials{};
    STAG_CUDA_TRY(dev_malloc(&h->part.sum, entries * sizeof(double)));
    STAG_CUDA_TRY(dev_malloc(&h->part.shift, entries * sizeof(float)));
    h->part.cap = entries;
    return 0;
}

int ensure_qt(stag_kde *h, int64_t floats) {
    if (h->qt_cap >= floats) return 0;
    ++h->scratch_epoch;
    if (h->qt) cudaFree(h->qt);
    h->qt = nullptr;
    h->qt_cap = 0;
    STAG_CUDA_TRY(dev_malloc(&h->qt, floats * sizeof(float)));
    h->qt_cap = floats;
    return 0;
}

int launch_check_finite_f32(const float *p, int64_t count, int *dflag, cudaStream_t s, int bit) {
    if (count <= 0) return 0;
    count_launch();
    check_finite_kernel<float><<<grid_for(count, 256), 256, 0, s>>>(p, count, dflag, bit);
    STAG_CUDA_TRY(cudaGetLastError());
    return 0;
}

int launch_check_finite_f64(const double *p, int64_t count, int *dflag, cudaStream_t s) {
    if (count <= 0) return 0;
    count_launch();
    check_finite_kernel<double><<<grid_for(count, 256), 256, 0, s>>>(p, count, dflag, 1);
    STAG_CUDA_TRY(cudaGetLastError());
    return 0;
}

int simt_prepare_points(stag_kde *h, const float *dX) {
    h->d_pad = (int)round_up(h->d, 4);
    h->n_tiles = ceil_div(h->n, kSimtTile);
    const int64_t total = h->n_tiles * h->d_pad * kSimtTile;
    STAG_CUDA_TRY(dev_malloc(&h->xt, total * sizeof(float)));
    count_launch();
    to_tiles_kernel<float><<<grid_for(total, 256), 256, 0, h->stream>>>(dX, h->n, h->d, h->d_pad,
                                                                        h->n_tiles, h->xt);
    STAG_CUDA_TRY(cudaGetLastError());
    return 0;
}

// Launches the FP32 kernel instance for the handle's operand width and kernel function.
template <int KERN>
void launch_simt_kern(const stag_kde *h, dim3 grid, cudaStream_t s, int64_t m, float negc, int64_t tps) {
    if (h->d_pad <= kSimtResidentMaxD)
        kde_simt_f32_kernel<true, KERN><<<grid, 256, simt_resident_bytes(h->d_pad), s>>>(h->xt, h->n, h->n_tiles, h->qt, m, h->d_pad, negc, tps,
                                                             h->part.sum, h->part.shift);
    else
        kde_simt_f32_kernel<false, KERN><<<grid, 256, 0, s>>>(h->xt, h->n, h->n_tiles, h->qt, m, h->d_pad, negc, tps,
                                                              h->part.sum, h->part.shift);
}
void launch_simt(const stag_kde *h, dim3 grid, cudaStream_t s, int64_t m, int64_t tps) {
    const float negc = (float)(-h->a * 1.4426950408889634);  // -a log2(e)
    switch (h->kernel) {
        case STAG_KDE_KERNEL_EXPONENTIAL:
            return launch_simt_kern<STAG_KDE_KERNEL_EXPONENTIAL>(h, grid, s, m, negc, tps);
        case STAG_KDE_KERNEL_LOGISTIC:
            return launch_simt_kern<STAG_KDE_KERNEL_LOGISTIC>(h, grid, s, m, negc, tps);
        default:
            return launch_simt_kern<STAG_KDE_KERNEL_GAUSSIAN>(h, grid, s, m, negc, tps);
    }
}

// Number of point-set splits: enough blocks for several waves of 2 blocks per SM.
static int64_t choose_tiles_per_split(const stag_kde *h, int64_t q_tiles) {
    const int64_t target_blocks = (int64_t)h->sm_count * 2 * 6;
    int64_t splits = std::max<int64_t>(1, ceil_div(target_blocks, q_tiles));
    splits = std::min<int64_t>(splits, h->n_tiles);
    // keep at least 8 tiles (512 points) per split so per-block set-up stays amortised
    splits = std::min<int64_t>(splits, std::max<int64_t>(1, h->n_tiles / 8));
    return ceil_div(h->n_tiles, splits);
}

int simt_query_f32(stag_kde *h, const float *dQ, int64_t m, double *dOut, cudaStream_t s,
                   int *dflag) {
    const int64_t q_tiles = ceil_div(m, kSimtTile);
    int rc = ensure_qt(h, q_tiles * h->d_pad * kSimtTile);
    if (rc) return rc;
    const int64_t total = q_tiles * h->d_pad * kSimtTile;
    count_launch();
    to_tiles_kernel<float><<<grid_for(total, 256), 256, 0, s>>>(dQ, m, h->d, h->d_pad, q_tiles, h->qt);
    STAG_CUDA_TRY(cudaGetLastError());
    if (dflag) {
        rc = launch_check_finite_f32(dQ, m * h->d, dflag, s);
        if (rc) return rc;
    }
    const int64_t tps = choose_tiles_per_split(h, q_tiles);
    const int64_t splits = ceil_div(h->n_tiles, tps);
    rc = ensure_partials(h, splits * m);
    if (rc) return rc;
    if (q_tiles > 0x7fffffff || splits > 65535) return fail(STAG_KDE_EINVAL, "query batch too large");
    dim3 grid((unsigned)q_tiles, (unsigned)splits);
    count_launch();
    prof_start(h, s);
    launch_simt(h, grid, s, m, tps);
    prof_stop(h, s, (double)m * (double)h->n);
    STAG_CUDA_TRY(cudaGetLastError());
    return launch_combine(h->part.sum, h->part.shift, m, (int)splits, h->normalise ? 1.0 / (double)h->n : 1.0,
                          dOut, s);
}

int simt_reserve(stag_kde *h, int64_t m) {
    const int64_t q_tiles = ceil_div(m, kSimtTile);
    int rc = ensure_qt(h, q_tiles * h->d_pad * kSimtTile);
    if (rc) return rc;
    const int64_t tps = choose_tiles_per_split(h, q_tiles);
    return ensure_partials(h, ceil_div(h->n_tiles, tps) * m);
}

// Tile-transposed [tile][d_pad][64] back to row-major n x d.
__global__ void tiles_to_rows_kernel(const float *__restrict__ xt, int64_t n, int64_t d, int d_pad,
                                     float *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * d; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / d, k = i % d;
        out[i] = xt[((row / kSimtTile) * d_pad + k) * kSimtTile + row % kSimtTile];
    }
}

__global__ void subtract_one_kernel(double *__restrict__ v, int64_t count, double one) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        v[i] -= one;
}

int simt_points_rows(stag_kde *h, float *out, cudaStream_t s) {
    count_launch();
    tiles_to_rows_kernel<<<grid_for(h->n * h->d, 256), 256, 0, s>>>(h->xt, h->n, h->d, h->d_pad, out);
    STAG_CUDA_TRY(cudaGetLastError());
    return 0;
}

int launch_subtract(double *v, int64_t count, double one, cudaStream_t s) {
    count_launch();
    subtract_one_kernel<<<grid_for(count, 256), 256, 0, s>>>(v, count, one);
    STAG_CUDA_TRY(cudaGetLastError());
    return 0;
}

int simt_list_launch(const stag_kde *h, const float *xt, const float *qt, const int *kept, int64_t kstride,
                     const int *kcount, const int *item_off, const int *n_groups, int seg, int per, double *part_sum,
                     float *part_shift, cudaStream_t s) {
    const float negc = (float)(-h->a * 1.4426950408889634);  // -a log2(e)
    const dim3 grid((unsigned)(h->sm_count * 2));
    count_launch();
    if (h->d_pad <= kSimtResidentMaxD)
        kde_simt_f32_list_kernel<true, STAG_KDE_KERNEL_GAUSSIAN><<<grid, 256, simt_resident_bytes(h->d_pad), s>>>(
            xt, h->n, h->n_tiles, qt, h->d_pad, negc, kept, kstride, kcount, item_off, n_groups, seg, per, part_sum,
            part_shift);
    else
        kde_simt_f32_list_kernel<false, STAG_KDE_KERNEL_GAUSSIAN><<<grid, 256, 0, s>>>(
            xt, h->n, h->n_tiles, qt, h->d_pad, negc, kept, kstride, kcount, item_off, n_groups, seg, per, part_sum,
            part_shift);
    STAG_CUDA_TRY(cudaGetLastError());
    return 0;
}

int simt_gather_rows(const stag_kde *h, const float *dQ, const int *idx, const int *count, int64_t m_cap, float *qt,
                     cudaStream_t s) {
    count_launch();
    gather_rows_tiles_kernel<<<grid_for(ceil_div(m_cap, kSimtTile) * h->d_pad * kSimtTile, 256), 256, 0, s>>>(
        dQ, h->d, h->d_pad, idx, count, m_cap, qt);
    STAG_CUDA_TRY(cudaGetLastError());
    return 0;
}

int simt_tiles_from_rows(const stag_kde *h, const float *rows, float *out, cudaStream_t s) {
    const int64_t total = h->n_tiles * h->d_pad * kSimtTile;
    count_launch();
    to_tiles_kernel<float><<<grid_for(total, 256), 256, 0, s>>>(rows, h->n, h->d, h->d_pad, h->n_tiles, out);
    STAG_CUDA_TRY(cudaGetLastError());
    return 0;
}

int simt_query_f64(stag_kde *h, const double *dQ, int64_t m, double *dOut, cudaStream_t s, int *dflag) {
    if (dflag) {
        int rc = launch_check_finite_f64(dQ, m * h->d, dflag, s);
        if (rc) return rc;
    }
    const int64_t tp = std::max<int64_t>(1, 4096 / h->d);
    const size_t smem = (size_t)(tp * h->d) * sizeof(double);
    if (smem > 48 * 1024) return fail(STAG_KDE_EUNSUPPORTED, "FP64 form: d too large");
    count_launch();
    prof_start(h, s);
    kde_simt_f64_kernel<<<(unsigned)ceil_div(m, 128), 128, smem, s>>>(h->x64, h->n, dQ, m, h->d, h->a, h->kernel,
                                                                       dOut);
    prof_stop(h, s, (double)m * (double)h->n);
    STAG_CUDA_TRY(cudaGetLastError());
    if (h->normalise) {
        // (1/n) applied by the combine kernel with a single split of FP64 partials
        int rc = ensure_partials(h, m);
        if (rc) return rc;
        STAG_CUDA_TRY(cudaMemcpyAsync(h->part.sum, dOut, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
        STAG_CUDA_TRY(cudaMemsetAsync(h->part.shift, 0, m * sizeof(float), s));
        return launch_combine(h->part.sum, h->part.shift, m, 1, 1.0 / (double)h->n, dOut, s);
    }
    return 0;
}

}  // namespace stagkde
