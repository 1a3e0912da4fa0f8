// Allocation-free exact-KDE entry point (stag_kde_eval_noalloc, include/stag_kde.h).
//
// Who needs this: code that must not allocate GPU memory at call time, for example a
// caller running inside a memory pool or allocator hook of its own (where a nested
// cudaMalloc would recurse or deadlock), a real-time loop that forbids the implicit
// device synchronisation cudaMalloc/cudaFree can cause, or a host process whose
// allocator budget is fixed up front. The handle-based API allocates its data copy and
// scratch on the device; this entry point allocates nothing.
//
// How: the caller passes X, Q and out in device memory (row-major, no data copy). The
// only scratch the computation needs is the per-split partial sums; they live in the
// file-scope __device__ array below, a fixed 8 MiB that every GPU which loads this
// library holds until the process exits. Its device address is looked up once per
// device with cudaGetSymbolAddress (the array's name is only a host-side stand-in in
// host code). Every call shares the array, so calls whose work overlaps on the GPU (two
// streams, or two host threads) race and corrupt each other's results: serialise them.
// No part of the scratch needs to start at zero: every (split, query) entry the kernel
// reads is written by the same call first.
//
// The arithmetic is the plain FP32 form's (direct differences, per-row integer shift,
// FP32 within a tile group and FP64 across, FP64 combine); the kernel is a variant that
// reads X and Q in their row-major layout instead of the handle's tiled copies.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "internal.h"

namespace stagkde {
namespace {

constexpr int64_t kNoallocScratchBytes = 8ll << 20;  // 8 MiB
constexpr int64_t kEntryBytes = sizeof(double) + sizeof(float);
constexpr int64_t kNoallocMaxEntries = kNoallocScratchBytes / kEntryBytes;

// Partials: splits*m doubles, then splits*m floats packed right behind them (8-byte
// aligned), so splits*m <= 8 MiB / 12 bytes = 699050 entries always fit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_ptr[kMaxDevices] = {};

constexpr int T = 64;        // rows per tile
constexpr int KC = 32;       // coordinates per shared-memory chunk
constexpr float kFloor = -0x1p100f;
constexpr float kGuard = 0x1p64f;

__device__ __forceinline__ float ex2a(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ int cexp(float e) { return (int)fminf(fmaxf(e, -4000.f), 4000.f); }

struct Acc {
    float shift, acc32;
    double acc64;
};

__device__ __forceinline__ void add4(Acc &r, const float d2[4], float negc, int valid) {
    float ts = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float e = ex2a(fmaf(negc, d2[j], -r.shift));
        ts += (j < valid) ? e : 0.f;
    }
    if (!(ts <= kGuard)) {
        float mx = -INFINITY;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j < valid) mx = fmaxf(mx, negc * d2[j]);
        const float s_new = fmaxf(ceilf(mx), kFloor);
        if (s_new > r.shift) {
            const int de = cexp(r.shift - s_new);
            r.acc32 = ldexpf(r.acc32, de);
            r.acc64 = ldexp(r.acc64, de);
            r.shift = s_new;
        }
        ts = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float e = ex2a(fmaf(negc, d2[j], -r.shift));
            ts += (j < valid) ? e : 0.f;
        }
    }
    r.acc32 += ts;
}

// One block: 64 queries x one contiguous range of point tiles; 4 x 4 pairs per thread.
__global__ void __launch_bounds__(256, 2)
kde_noalloc_kernel(const float *__restrict__ X, int64_t n, const float *__restrict__ Q, int64_t m, int64_t d,
                   float negc, int64_t tiles_per_split, double *__restrict__ part_sum,
                   float *__restrict__ part_shift) {
    __shared__ __align__(16) float sX[KC * T];
    __shared__ __align__(16) float sQ[KC * T];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t q0 = (int64_t)blockIdx.x * T;
    const int split = blockIdx.y;
    const int64_t n_tiles = (n + T - 1) / T;
    const int64_t t0 = (int64_t)split * tiles_per_split;
    const int64_t t1 = min(n_tiles, t0 + tiles_per_split);
    Acc row[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) row[i] = Acc{kFloor, 0.f, 0.0};
    int group = 0;
    for (int64_t t = t0; t < t1; ++t) {
        float d2[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) d2[i][j] = 0.f;
        for (int64_t k0 = 0; k0 < d; k0 += KC) {
            __syncthreads();
            for (int e = tid; e < KC * T; e += 256) {
                const int r = e / KC, k = e % KC;  // consecutive threads: consecutive coordinates
                const int64_t px = t * T + r, qy = q0 + r, kk = k0 + k;
                sX[k * T + r] = (px < n && kk < d) ? X[px * d + kk] : 0.f;
                sQ[k * T + r] = (qy < m && kk < d) ? Q[qy * d + kk] : 0.f;
            }
            __syncthreads();
            const int klen = (int)min((int64_t)KC, d - k0);
            // chains of 16 coordinates, block sums added (the plain form's order)
            for (int kb = 0; kb < klen; kb += 16) {
                const int ke = min(klen, kb + 16);
                float b2[4][4];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) b2[i][j] = 0.f;
                for (int k = kb; k < ke; ++k) {
                    const float4 qv = *reinterpret_cast<const float4 *>(&sQ[k * T + ty * 4]);
                    const float4 xv = *reinterpret_cast<const float4 *>(&sX[k * T + tx * 4]);
                    const float qa[4] = {qv.x, qv.y, qv.z, qv.w};
                    const float xa[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float df = qa[i] - xa[j];
                            b2[i][j] = fmaf(df, df, b2[i][j]);
                        }
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) d2[i][j] += b2[i][j];
            }
        }
        const int64_t col0 = t * T + tx * 4;
        const int valid = (int)max((int64_t)0, min((int64_t)4, n - col0));
#pragma unroll
        for (int i = 0; i < 4; ++i) add4(row[i], d2[i], negc, valid);
        if (++group == 16) {
            group = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                row[i].acc64 += (double)row[i].acc32;
                row[i].acc32 = 0.f;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        row[i].acc64 += (double)row[i].acc32;
        row[i].acc32 = 0.f;
    }
#pragma unroll
    for (int off = 8; off >= 1; off >>= 1) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const double oa = __shfl_xor_sync(0xffffffffu, row[i].acc64, off);
            const float os = __shfl_xor_sync(0xffffffffu, row[i].shift, off);
            const float sm = fmaxf(row[i].shift, os);
            row[i].acc64 = ldexp(row[i].acc64, cexp(row[i].shift - sm)) + ldexp(oa, cexp(os - sm));
            row[i].shift = sm;
        }
    }
    if (tx == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t q = q0 + ty * 4 + i;
            if (q < m) {
                part_sum[(int64_t)split * m + q] = row[i].acc64;
                part_shift[(int64_t)split * m + q] = row[i].shift;
            }
        }
    }
}

// Device address of the scratch array for `dev` (which must be current), looked up once.
int scratch_for_device(int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(STAG_KDE_EUNSUPPORTED, "device ordinal beyond 63");
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return 0;
}

}  // namespace
}  // namespace stagkde

using namespace stagkde;

extern "C" int stag_kde_eval_noalloc(const float *dX, int64_t n, const float *dQ, int64_t m, int64_t d, double a,
                                     double *dOut, void *stream) {
    if (n < 1 || d < 1) return fail(STAG_KDE_EINVAL, "need n >= 1 and d >= 1");
    if (m < 0) return fail(STAG_KDE_EINVAL, "m < 0");
    if (!(a >= 0.0) || !isfinite(a)) return fail(STAG_KDE_EINVAL, "bandwidth a must be finite and >= 0");
    if (m == 0) return 0;
    if (!dX || !dQ || !dOut) return fail(STAG_KDE_EINVAL, "dX, dQ or dOut is NULL");
    if (m > kNoallocMaxEntries)
        return fail(STAG_KDE_EINVAL, "m exceeds the no-alloc scratch capacity (" +
                                         std::to_string(kNoallocMaxEntries) + " queries per call)");
    int dev = 0;
    STAG_CUDA_TRY(cudaGetDevice(&dev));
    void *base = nullptr;
    int rc = scratch_for_device(dev, &base);
    if (rc) return rc;
    int sms = 0;
    STAG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

    // splits: enough blocks for several waves, bounded by the scratch capacity
    const int64_t q_tiles = ceil_div(m, T);
    const int64_t n_tiles = ceil_div(n, T);
    int64_t splits = std::max<int64_t>(1, ceil_div((int64_t)sms * 12, q_tiles));
    splits = std::min<int64_t>(splits, n_tiles);
    splits = std::min<int64_t>(splits, std::max<int64_t>(1, n_tiles / 8));
    splits = std::min<int64_t>(splits, kNoallocMaxEntries / m);
    splits = std::min<int64_t>(splits, 65535);
    const int64_t tps = ceil_div(n_tiles, splits);
    splits = ceil_div(n_tiles, tps);
    if (q_tiles > 0x7fffffff) return fail(STAG_KDE_EINVAL, "m too large");

    // splits * m <= kNoallocMaxEntries by construction: the packed layout fits exactly
    double *psum = reinterpret_cast<double *>(base);
    float *pshift = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(base) +
                                              splits * m * (int64_t)sizeof(double));

    cudaStream_t s = (cudaStream_t)stream;
    const float negc = (float)(-a * 1.4426950408889634);
    count_launch();
    kde_noalloc_kernel<<<dim3((unsigned)q_tiles, (unsigned)splits), 256, 0, s>>>(dX, n, dQ, m, d, negc, tps, psum,
                                                                                  pshift);
    STAG_CUDA_TRY(cudaGetLastError());
    return launch_combine(psum, pshift, m, (int)splits, 1.0, dOut, s);
}
