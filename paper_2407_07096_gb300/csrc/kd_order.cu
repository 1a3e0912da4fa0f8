// Spatially coherent ordering of the point set for the tensor-core form.
//
// The tensor-core form centres every tile of BN consecutive points on the tile's mean
// and its rounding error grows with the tile's radius (kde_tc.cu), so points that are
// close in space should share tiles. This file computes a permutation by the classic
// k-d tree construction: the tile range [0, T) is halved recursively (left half
// [a, a + (b-a)/2), right half the rest); at every level each segment's points are
// sorted by their coordinate of largest spread (max - min within the segment) and cut
// at the segment's middle tile boundary. After ceil(log2 T) levels every tile is a leaf.
//
// All levels run on the GPU: per-tile min/max reductions with one atomic per tile and
// coordinate, a per-segment choice of the split coordinate, and a stable LSD radix sort
// of 64-bit keys (segment id in the high bits, the order-preserving bits of the
// coordinate in the low 32) carrying the point indices. Segment ids are the left/right
// path bits of the recursion, so sorting by them keeps segments in place.
#include <stdint.h>

#include <algorithm>
#include <utility>

#include "internal.h"

namespace stagkde {
namespace {

constexpr int kRsThreads = 256;
constexpr int kRsRounds = 16;  // elements per block = 256 * 16
constexpr int kRsChunk = kRsThreads * kRsRounds;

__device__ __forceinline__ uint32_t float_order_bits(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// path id of tile t after `level` halvings of [0, T)
__device__ __forceinline__ uint32_t seg_id(int64_t t, int64_t T, int level) {
    int64_t a = 0, b = T;
    uint32_t id = 0;
    for (int l = 0; l < level; ++l) {
        const int64_t mid = a + (b - a) / 2;
        if (t < mid) {
            b = mid;
            id <<= 1;
        } else {
            a = mid;
            id = (id << 1) | 1u;
        }
    }
    return id;
}

// ------------------------------------------------------------------ radix sort
// dcount (device, optional): only the first min(n, *dcount) entries take part
__device__ __forceinline__ int64_t rs_count(int64_t n, const int *dcount) {
    return dcount ? min(n, (int64_t)max(0, *dcount)) : n;
}

__global__ void rs_hist_kernel(const uint64_t *__restrict__ keys, int64_t n, const int *__restrict__ dcount, int shift,
                               int nblocks, uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t b0 = (int64_t)blockIdx.x * kRsChunk;
    const int64_t b1 = min(rs_count(n, dcount), b0 + kRsChunk);
    for (int64_t i = b0 + threadIdx.x; i < b1; i += kRsThreads) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of the histogram, in two levels: every block scans one chunk of
// kScanChunk entries in place and writes the chunk's total to part[chunk]; one block then
// scans the chunk totals (rs_scan_kernel), and the scatter adds part[entry / kScanChunk].
constexpr int kScanThreads = 1024;
constexpr int kScanChunk = 4 * kScanThreads;

__global__ void __launch_bounds__(kScanThreads)
rs_scan_chunks_kernel(uint32_t *__restrict__ a, int64_t count, uint32_t *__restrict__ part) {
    __shared__ uint32_t wsum[32];
    const int64_t i0 = (int64_t)blockIdx.x * kScanChunk + 4 * threadIdx.x;
    uint32_t v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = i0 + e < count ? a[i0 + e] : 0u;
    const uint32_t t0 = v[0], t1 = t0 + v[1], t2 = t1 + v[2], t3 = t2 + v[3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = t3;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = wsum[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        wsum[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const uint32_t excl = (warp ? wsum[warp - 1] : 0u) + inc - t3;
    const uint32_t out[4] = {excl, excl + t0, excl + t1, excl + t2};
#pragma unroll
    for (int e = 0; e < 4; ++e)
        if (i0 + e < count) a[i0 + e] = out[e];
    if (threadIdx.x == kScanThreads - 1) part[blockIdx.x] = wsum[31];
}

// exclusive scan of `count` entries in place (single block of 1024 threads)
__global__ void rs_scan_kernel(uint32_t *__restrict__ a, int64_t count) {
    __shared__ uint32_t s[1024];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < count; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const uint32_t v = i < count ? a[i] : 0u;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            const uint32_t t = threadIdx.x >= off ? s[threadIdx.x - off] : 0u;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < count) a[i] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += s[1023];
        __syncthreads();
    }
}

// Stable scatter: rounds of 256 consecutive elements; rank inside a round from warp
// match masks and per-warp digit counts.
__global__ void __launch_bounds__(kRsThreads)
rs_scatter_kernel(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
                  uint32_t *__restrict__ vout, int64_t n, const int *__restrict__ dcount, int shift, int nblocks,
                  const uint32_t *__restrict__ hist, const uint32_t *__restrict__ part) {
    __shared__ uint32_t base[256];
    __shared__ uint32_t cnt[kRsThreads / 32][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t hidx = (int64_t)threadIdx.x * nblocks + blockIdx.x;
    base[threadIdx.x] = hist[hidx] + part[hidx / kScanChunk];
    for (int w = 0; w < kRsThreads / 32; ++w) cnt[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t b0 = (int64_t)blockIdx.x * kRsChunk;
    const int64_t b1 = min(rs_count(n, dcount), b0 + kRsChunk);
    for (int64_t r0 = b0; r0 < b1; r0 += kRsThreads) {
        const int64_t i = r0 + threadIdx.x;
        const bool valid = i < b1;
        uint64_t k = 0;
        uint32_t v = 0, dg = 0;
        if (valid) {
            k = kin[i];
            v = vin[i];
            dg = (uint32_t)((k >> shift) & 255u);
        }
        const uint32_t active = __ballot_sync(0xffffffffu, valid);
        uint32_t peers = 0, rank = 0;
        if (valid) {
            peers = __match_any_sync(active, dg);
            rank = __popc(peers & ((1u << lane) - 1u));
            if (rank == 0) cnt[warp][dg] = __popc(peers);
        }
        __syncthreads();
        if (valid) {
            uint32_t off = base[dg] + rank;
            for (int w = 0; w < warp; ++w) off += cnt[w][dg];
            kout[off] = k;
            vout[off] = v;
        }
        __syncthreads();
        uint32_t tot = 0;
        for (int w = 0; w < kRsThreads / 32; ++w) {
            tot += cnt[w][threadIdx.x];
            cnt[w][threadIdx.x] = 0;
        }
        base[threadIdx.x] += tot;
        __syncthreads();
    }
}

// ------------------------------------------------------------------ k-d levels
__global__ void kd_init_kernel(uint32_t *perm, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        perm[i] = (uint32_t)i;
}

__global__ void kd_fill_minmax_kernel(uint32_t *mn, uint32_t *mx, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        mn[i] = 0xffffffffu;
        mx[i] = 0u;
    }
}

// one block per tile: min/max of every coordinate over the tile's points (in the
// current order), folded into the tile's segment with one atomic per coordinate
__global__ void kd_minmax_kernel(const float *__restrict__ X, int64_t n, int64_t d, int BN, int64_t T, int level,
                                 const uint32_t *__restrict__ perm, uint32_t *mn, uint32_t *mx) {
    const int64_t t = blockIdx.x;
    const uint32_t sid = seg_id(t, T, level);
    const int64_t p0 = t * BN, p1 = min(n, p0 + BN);
    for (int64_t k = threadIdx.x; k < d; k += blockDim.x) {
        uint32_t lo = 0xffffffffu, hi = 0u;
        for (int64_t p = p0; p < p1; ++p) {
            const uint32_t o = float_order_bits(X[(int64_t)perm[p] * d + k]);
            lo = min(lo, o);
            hi = max(hi, o);
        }
        atomicMin(&mn[(int64_t)sid * d + k], lo);
        atomicMax(&mx[(int64_t)sid * d + k], hi);
    }
}

__device__ __forceinline__ float order_bits_to_float(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

__global__ void kd_choose_dim_kernel(const uint32_t *__restrict__ mn, const uint32_t *__restrict__ mx, int64_t nseg,
                                     int64_t d, int *__restrict__ dim) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg; s += (int64_t)gridDim.x * blockDim.x) {
        int best = 0;
        float spread = -1.f;
        for (int64_t k = 0; k < d; ++k) {
            const uint32_t a = mn[s * d + k], b = mx[s * d + k];
            if (a > b) continue;  // empty segment
            const float sp = order_bits_to_float(b) - order_bits_to_float(a);
            if (sp > spread) {
                spread = sp;
                best = (int)k;
            }
        }
        dim[s] = best;
    }
}

__global__ void kd_keys_kernel(const float *__restrict__ X, int64_t n, int64_t d, int BN, int64_t T, int level,
                               const uint32_t *__restrict__ perm, const int *__restrict__ dim, uint64_t *__restrict__ keys,
                               uint32_t *__restrict__ vals) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t sid = seg_id(p / BN, T, level);
        const uint32_t idx = perm[p];
        const float x = X[(int64_t)idx * d + dim[sid]];
        keys[p] = ((uint64_t)sid << 32) | float_order_bits(x);
        vals[p] = idx;
    }
}

__global__ void kd_gather_kernel(const float *__restrict__ X, const uint32_t *__restrict__ perm, int64_t n, int64_t d,
                                 float *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * d; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = X[(int64_t)perm[i / d] * d + (i % d)];
}

int grid_of(int64_t total, int threads) { return (int)std::min<int64_t>(ceil_div(total, threads), 152 * 16); }

}  // namespace

// Stable sort of (keys, vals) by key bits [0, bits), ping-ponging with the tmp buffers;
// the result ends in (keys, vals). hist needs radix_sort_hist_entries(n) entries.
int radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *ktmp, uint32_t *vtmp, uint32_t *hist, int64_t n,
                     int bits, cudaStream_t s, const int *dcount) {
    const int nblocks = (int)ceil_div(n, kRsChunk);
    const int64_t entries = (int64_t)256 * nblocks;
    const int64_t chunks = ceil_div(entries, kScanChunk);
    uint32_t *part = hist + entries;  // chunk totals, scanned in place
    uint64_t *ka = keys, *kb = ktmp;
    uint32_t *va = vals, *vb = vtmp;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += 8, ++passes) {
        count_launch(4);
        rs_hist_kernel<<<nblocks, 256, 0, s>>>(ka, n, dcount, shift, nblocks, hist);
        rs_scan_chunks_kernel<<<(unsigned)chunks, kScanThreads, 0, s>>>(hist, entries, part);
        rs_scan_kernel<<<1, 1024, 0, s>>>(part, chunks);
        rs_scatter_kernel<<<nblocks, kRsThreads, 0, s>>>(ka, va, kb, vb, n, dcount, shift, nblocks, hist, part);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    STAG_CUDA_TRY(cudaGetLastError());
    if (passes & 1) {
        STAG_CUDA_TRY(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        STAG_CUDA_TRY(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
    return 0;
}

// Writes into dXs (n x d, device) the points of dX reordered so that every block of BN
// consecutive points is a leaf of the k-d tree described above.
int kd_reorder(const float *dX, int64_t n, int64_t d, int BN, float *dXs, cudaStream_t s) {
    if (n > 0xffffffffll) return fail(STAG_KDE_EUNSUPPORTED, "k-d ordering: n >= 2^32");
    const int64_t T = ceil_div(n, BN);
    int levels = 0;
    while (((int64_t)1 << levels) < T) ++levels;
    const int64_t max_seg = (int64_t)1 << levels;
    const int nblocks = (int)ceil_div(n, kRsChunk);
    uint32_t *perm = nullptr, *vtmp = nullptr, *mn = nullptr, *mx = nullptr, *hist = nullptr;
    uint64_t *keys = nullptr, *ktmp = nullptr;
    int *dim = nullptr;
    auto cleanup = [&]() {
        cudaStreamSynchronize(s);
        cudaFree(perm);
        cudaFree(vtmp);
        cudaFree(mn);
        cudaFree(mx);
        cudaFree(hist);
        cudaFree(keys);
        cudaFree(ktmp);
        cudaFree(dim);
    };
    cudaError_t e = cudaSuccess;
    if ((e = dev_malloc(&perm, n * 4)) || (e = dev_malloc(&vtmp, n * 4)) || (e = dev_malloc(&keys, n * 8)) ||
        (e = dev_malloc(&ktmp, n * 8)) || (e = dev_malloc(&mn, max_seg * d * 4)) ||
        (e = dev_malloc(&mx, max_seg * d * 4)) || (e = dev_malloc(&hist, radix_sort_hist_entries(n) * 4)) ||
        (e = dev_malloc(&dim, max_seg * sizeof(int)))) {
        cleanup();
        return cuda_fail(e, "dev_malloc(k-d ordering)");
    }
    count_launch();
    kd_init_kernel<<<grid_of(n, 256), 256, 0, s>>>(perm, n);
    int rc = 0;
    for (int level = 0; level < levels && !rc; ++level) {
        const int64_t nseg = (int64_t)1 << level;
        count_launch(4);
        kd_fill_minmax_kernel<<<grid_of(nseg * d, 256), 256, 0, s>>>(mn, mx, nseg * d);
        kd_minmax_kernel<<<(unsigned)T, (unsigned)std::min<int64_t>(d, 128), 0, s>>>(dX, n, d, BN, T, level, perm,
                                                                                      mn, mx);
        kd_choose_dim_kernel<<<grid_of(nseg, 128), 128, 0, s>>>(mn, mx, nseg, d, dim);
        kd_keys_kernel<<<grid_of(n, 256), 256, 0, s>>>(dX, n, d, BN, T, level, perm, dim, keys, vtmp);
        // sort (segment, coordinate) keys; the values are the point indices
        uint32_t *vals = vtmp;
        rc = radix_sort_pairs(keys, vals, ktmp, perm, hist, n, 32 + level, s);
        if (!rc) {
            // sorted point indices are now in `vtmp`; make them the current order
            std::swap(perm, vtmp);
        }
    }
    if (!rc) {
        count_launch();
        kd_gather_kernel<<<grid_of(n * d, 256), 256, 0, s>>>(dX, perm, n, d, dXs);
        cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) rc = cuda_fail(le, "kd_gather_kernel");
    }
    cleanup();
    return rc;
}

}  // namespace stagkde
