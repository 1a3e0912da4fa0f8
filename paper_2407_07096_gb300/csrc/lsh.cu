// Euclidean LSH tables (E2LSH, Sec. 2) on the GPU: they supply the candidate lists that
// the weighted subset sums (kde_subset.cu) evaluate in the LSH-based estimators (Sec. 3.1).
//
// Hash function: h_{a,b}(x) = floor((<x, a> + b) / 4), a ~ N(0, I), b ~ U(0, 4). The
// caller supplies the L*K functions (the library draws no random numbers). The integer is
// decided in FP32 with a fixed order (s = 0; s = fma(x_k, a_k, s) for k = 0..d-1, then
// (s + b) * 1/4, floor, saturated to int32), so the values are exactly reproducible and
// equal those of any implementation that takes the decision the same way.
//
// Tables: for table l, point i's K values (functions l*K .. l*K+K-1) are mixed into a
// 58-bit key (a salted hash); (l << 58 | key, i) pairs of all tables are sorted together
// by one stable radix sort, so table l is the contiguous, key-sorted range
// [l*n, (l+1)*n) and each bucket a run of equal keys with its point indices in
// increasing order. Membership is exact, not probabilistic: after the sort every pair
// of neighbours with equal keys is checked to have equal K-tuples, and if two different
// tuples share a key the keys are rebuilt with another salt (a run therefore always
// holds one tuple); a query's lookup then recomputes the K values of the first point of
// the run it found and keeps the run only if they equal the query's own (Sec. 2: a
// collision needs all K values equal).
//
// Query: hash the queries, binary-search each table for the query's key (one thread per
// (query, table)), then remove repeats across tables so that every query gets its
// distinct candidates in increasing index order. Up to 2^22 points, a block takes one
// (query, slice of at most 1572864 points) at a time, sets a bit per bucket member in a
// shared-memory bitmap of the slice and walks it in index order (a counting pass, a
// prefix sum over the items, a writing pass). Beyond that, every bucket member is listed
// (one warp per query) and repeats are removed by a radix sort of (query << 32 | index)
// keys and a per-query unique pass.
#include <stdint.h>
#include <stdlib.h>

#include <algorithm>
#include <new>
#include <vector>

#include "internal.h"

struct stag_lsh {
    int device = 0;
    int64_t n = 0, d = 0;
    int K = 0, L = 0;
    cudaStream_t stream = nullptr;
    float *A = nullptr, *B = nullptr;  // functions: L*K x d, L*K
    uint64_t *keys = nullptr;          // n*L sorted keys (table id in bits 58..63)
    uint32_t *ids = nullptr;           // n*L point indices in key order
    float *X = nullptr;                // n x d points (the lookup recomputes a member's K values)
    uint64_t salt = 0;                 // salt of the bucket keys
    int key_bits = 58;                 // bits of a bucket key
    // query scratch (grown on demand)
    void *scratch = nullptr;
    int64_t scratch_cap = 0;
    void *cand = nullptr;  // the last query's deduplicated candidates (int64)
    int64_t cand_cap = 0;
    void *host_q = nullptr;  // host API: device copies of Q and the offsets
    int64_t host_q_cap = 0;
    int64_t last_total = 0;  // size of the kept candidate lists (device query)
    void *sort_buf = nullptr;  // raw candidate keys and radix-sort buffers (grown on demand)
    int64_t sort_cap = 0;
};

namespace stagkde {
namespace {

constexpr int kHashFns = 32;   // functions per block (one warp's lanes)
constexpr int kHashRows = 8;   // rows per block
constexpr int kKeyShift = 58;  // table id above the 58-bit bucket key

// h = floor((<x, a> + b) / 4) in FP32, fixed order, saturated to int32 (the conversion
// with rounding toward -inf saturates). One function of one row, the same operations as
// the tiled kernel below.
__device__ __forceinline__ int32_t hash_one(const float *__restrict__ x, const float *__restrict__ a, float b, int d) {
    float s = 0.f;
    for (int k = 0; k < d; ++k) s = __fmaf_rn(x[k], a[k], s);
    return __float2int_rd(__fmul_rn(__fadd_rn(s, b), 0.25f));
}

__global__ void __launch_bounds__(kHashFns * kHashRows)
lsh_hash_kernel(const float *__restrict__ X, int64_t n, int d, const float *__restrict__ A,
                const float *__restrict__ B, int nf, int32_t *__restrict__ H) {
    extern __shared__ float sa[];  // [d][kHashFns]: function f0 + lane's coordinate k at [k][lane]
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int f0 = blockIdx.x * kHashFns;
    const int nfb = min(kHashFns, nf - f0);
    for (int e = ty * kHashFns + lane; e < d * kHashFns; e += kHashFns * kHashRows) {
        const int k = e / kHashFns, f = e % kHashFns;
        sa[e] = f < nfb ? A[(int64_t)(f0 + f) * d + k] : 0.f;
    }
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.y * kHashRows + ty;
    if (i >= n || lane >= nfb) return;
    const float *x = X + i * d;
    float s = 0.f;
    for (int k = 0; k < d; ++k) s = __fmaf_rn(x[k], sa[k * kHashFns + lane], s);
    const float v = __fmul_rn(__fadd_rn(s, B[f0 + lane]), 0.25f);
    H[i * nf + f0 + lane] = __float2int_rd(v);
}

// key_bits-bit key (at most 58) of K hash values: a SplitMix64-style mix of each value
// into a salted state.
__device__ __forceinline__ uint64_t bucket_key(const int32_t *h, int K, uint64_t salt, int key_bits) {
    uint64_t z = 0x9E3779B97F4A7C15ull ^ salt;
    for (int k = 0; k < K; ++k) {
        z ^= (uint64_t)(uint32_t)h[k] + 0x9E3779B97F4A7C15ull + (z << 6) + (z >> 2);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
    }
    return z >> (64 - key_bits);
}

__global__ void lsh_keys_kernel(const int32_t *__restrict__ H, int64_t n, int K, int L, uint64_t salt, int key_bits,
                                uint64_t *__restrict__ keys, uint32_t *__restrict__ ids) {
    const int64_t total = n * L;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = e / n, i = e % n;
        keys[e] = ((uint64_t)l << kKeyShift) | bucket_key(H + i * (int64_t)K * L + l * K, K, salt, key_bits);
        ids[e] = (uint32_t)i;
    }
}

// After the sort: flags (*bad = 1) a pair of neighbours in one table whose keys are
// equal but whose K-tuples differ (two buckets merged by the key).
__global__ void lsh_collision_kernel(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ ids,
                                     const int32_t *__restrict__ H, int64_t n, int K, int L, int *__restrict__ bad) {
    const int64_t total = n * L;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x + 1; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (keys[e] != keys[e - 1]) continue;  // (the table id is part of the key)
        const int64_t l = (int64_t)(keys[e] >> kKeyShift);
        const int32_t *a = H + (int64_t)ids[e] * K * L + l * K;
        const int32_t *b = H + (int64_t)ids[e - 1] * K * L + l * K;
        for (int k = 0; k < K; ++k)
            if (a[k] != b[k]) {
                *bad = 1;
                break;
            }
    }
}

__device__ __forceinline__ int64_t lower_bound(const uint64_t *a, int64_t lo, int64_t hi, uint64_t v) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// The table view the lookup needs.
struct LshTables {
    const uint64_t *keys;
    const uint32_t *ids;
    const float *X, *A, *B;  // points and functions (L*K x d), offsets
    int64_t n;
    int d, K, L, key_bits;
    uint64_t salt;
};

// Per (query, table): the bucket's range in the sorted arrays (empty unless the first
// member's K values equal the query's: exact membership); per query: the total.
__global__ void lsh_lookup_kernel(const int32_t *__restrict__ HQ, int64_t m, LshTables t, int64_t *__restrict__ range,
                                  unsigned long long *__restrict__ count) {
    const int K = t.K, L = t.L;
    const int64_t n = t.n;
    const int64_t total = m * L;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / L, l = e % L;
        const int32_t *hq = HQ + j * (int64_t)K * L + l * K;
        const uint64_t key = ((uint64_t)l << kKeyShift) | bucket_key(hq, K, t.salt, t.key_bits);
        const int64_t lo = lower_bound(t.keys, l * n, (l + 1) * n, key);
        int64_t hi = lower_bound(t.keys, lo, (l + 1) * n, key + 1);
        if (hi > lo) {
            const float *x = t.X + (int64_t)t.ids[lo] * t.d;
            for (int k = 0; k < K; ++k) {
                const int64_t f = l * K + k;
                if (hash_one(x, t.A + f * t.d, t.B[f], t.d) != hq[k]) {
                    hi = lo;  // another tuple with the same key: not this query's bucket
                    break;
                }
            }
        }
        range[2 * e] = lo;
        range[2 * e + 1] = hi;
        if (count && hi > lo) atomicAdd(&count[j], (unsigned long long)(hi - lo));
    }
}

// out[0] = 0, out[j + 1] = sum of in[0..j] (one block; m is modest: one entry per query)
__global__ void scan_i64_kernel(const unsigned long long *__restrict__ in, int64_t m, int64_t *__restrict__ out) {
    __shared__ long long s[1024];
    __shared__ long long carry;
    if (threadIdx.x == 0) {
        carry = 0;
        out[0] = 0;
    }
    __syncthreads();
    for (int64_t base = 0; base < m; base += 1024) {
        const int64_t i = base + threadIdx.x;
        long long v = i < m ? (long long)in[i] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            const long long t = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < m) out[i + 1] = carry + s[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 1023) carry += s[1023];
        __syncthreads();
    }
}

// One warp per query: every bucket member of every table, as (query << 32 | index) keys.
__global__ void lsh_fill_kernel(const int64_t *__restrict__ range, int64_t m, int L, const uint32_t *__restrict__ ids,
                                const int64_t *__restrict__ raw_off, uint64_t *__restrict__ raw) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); j < m; j += warps) {
        int64_t pos = raw_off[j];
        for (int l = 0; l < L; ++l) {
            const int64_t lo = range[2 * (j * L + l)], hi = range[2 * (j * L + l) + 1];
            for (int64_t p = lo + lane; p < hi; p += 32) raw[pos + (p - lo)] = ((uint64_t)j << 32) | ids[p];
            pos += hi - lo;
        }
    }
}

// One warp per query over its sorted raw keys: the number of distinct indices (pass 0)
// or the distinct indices themselves at out_off[j] (pass 1).
template <bool kWrite>
__global__ void lsh_unique_kernel(const uint64_t *__restrict__ raw, const int64_t *__restrict__ raw_off, int64_t m,
                                  unsigned long long *__restrict__ ucount, const int64_t *__restrict__ out_off,
                                  int64_t *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); j < m; j += warps) {
        const int64_t a = raw_off[j], b = raw_off[j + 1];
        int64_t w = kWrite ? out_off[j] : 0;
        unsigned long long cnt = 0;
        for (int64_t p0 = a; p0 < b; p0 += 32) {
            const int64_t p = p0 + lane;
            const bool first = p < b && (p == a || raw[p] != raw[p - 1]);
            const unsigned mask = __ballot_sync(0xffffffffu, first);
            if (kWrite && first) out[w + __popc(mask & ((1u << lane) - 1u))] = (int64_t)(raw[p] & 0xffffffffull);
            w += __popc(mask);
            cnt += __popc(mask);
        }
        if (!kWrite && lane == 0) ucount[j] = cnt;
    }
}

constexpr int kBmThreads = 1024;
constexpr int64_t kMaxSliceWords = 49152;  // bitmap words per work item at most (1572864 points, 192 KB)
// Beyond 2^22 points (16 slices, each re-reading the query's bucket members) the sort
// path is used.
constexpr int64_t kBmMaxPoints = (int64_t)1 << 22;

// Words of the bitmap over n points, the number of slices it is cut into (as few as fit
// in shared memory: every slice re-reads the query's bucket members) and their size.
int64_t bitmap_words(int64_t n) { return (n + 31) / 32; }
int64_t bitmap_slices(int64_t n) { return (bitmap_words(n) + kMaxSliceWords - 1) / kMaxSliceWords; }
int64_t bitmap_slice_words(int64_t n) { return (bitmap_words(n) + bitmap_slices(n) - 1) / bitmap_slices(n); }
bool bitmap_fits(int64_t n) { return n <= kBmMaxPoints; }

// Exclusive prefix sum of c over the block's threads (thread order); *total gets the sum.
__device__ __forceinline__ int block_exclusive_scan(int c, int *warp_sums, int *total) {
    constexpr int kWarps = kBmThreads >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int v = lane < kWarps ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane < kWarps) warp_sums[lane] = v;  // inclusive prefix over warps
    }
    __syncthreads();
    const int before = (warp > 0 ? warp_sums[warp - 1] : 0) + inc - c;
    *total = warp_sums[kWarps - 1];
    return before;
}

// Distinct candidates of each query from its L bucket ranges, through a bitmap of the
// points in shared memory. A work item is (query j, slice s): the points
// [s * 32 * sw, (s + 1) * 32 * sw) (sw words per slice; one slice up to 1572864 points);
// items are taken grid-stride, slice fastest, so that the slices of one query read its
// bucket members while they are in L2. Every bucket member inside the slice sets its bit (one warp per table), then each
// thread walks a contiguous run of words in index order. Pass kWrite = false writes the
// number of distinct candidates per item to ucount; kWrite = true writes them, increasing,
// at out[item_off[item] ..], so a query's list is its slices' lists in slice order.
template <bool kWrite, bool kSliced>
__global__ void __launch_bounds__(kBmThreads)
lsh_bitmap_kernel(const int64_t *__restrict__ range, int64_t m, int L, const uint32_t *__restrict__ ids,
                  int64_t words, int64_t slices, int64_t sw, unsigned long long *__restrict__ ucount,
                  const int64_t *__restrict__ item_off, int64_t *__restrict__ out) {
    extern __shared__ uint32_t bm[];  // [sw] bitmap words, then 32 ints of scan scratch
    int *warp_sums = reinterpret_cast<int *>(bm + sw);
    const int tid = threadIdx.x;
    // an odd run length keeps the 32 lanes' words in 32 different banks
    const int64_t per = ((sw + kBmThreads - 1) / kBmThreads) | 1;
    const int64_t items = m * slices;
    for (int64_t w = tid; w < sw; w += kBmThreads) bm[w] = 0u;
    __syncthreads();
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        // (one slice: the item is the query, every member's bit is in the bitmap)
        const int64_t j = kSliced ? it / slices : it;
        const int64_t wbase = kSliced ? (it % slices) * sw : 0;
        const int64_t wn = kSliced ? min(sw, words - wbase) : words;  // words of this slice
        const uint32_t ilo = (uint32_t)(wbase * 32), ihi = (uint32_t)((wbase + wn) * 32);
        // one warp per table (the tables' loads are in flight together), lanes over members,
        // four loads issued before their bits are set (indices are below n < 2^32 - 1, so
        // the all-ones word marks an empty slot)
        for (int l = tid >> 5; l < L; l += kBmThreads >> 5) {
            const int64_t lo = range[2 * (j * L + l)], hi = range[2 * (j * L + l) + 1];
            for (int64_t p = lo + (tid & 31); p < hi; p += 128) {
                uint32_t iv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) iv[u] = p + 32 * u < hi ? ids[p + 32 * u] : 0xffffffffu;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t i = iv[u];
                    if (i != 0xffffffffu && (!kSliced || (i >= ilo && i < ihi)))
                        atomicOr(&bm[(i - ilo) >> 5], 1u << (i & 31));
                }
            }
        }
        __syncthreads();
        const int64_t w0 = min(wn, (int64_t)tid * per), w1 = min(wn, w0 + per);
        int c = 0;
        for (int64_t w = w0; w < w1; ++w) c += __popc(bm[w]);
        int total = 0;
        const int before = block_exclusive_scan(c, warp_sums, &total);
        if (kWrite) {
            int64_t pos = item_off[it] + before;
            for (int64_t w = w0; w < w1; ++w) {
                uint32_t v = bm[w];
                while (v) {
                    out[pos++] = (int64_t)ilo + w * 32 + (__ffs(v) - 1);
                    v &= v - 1u;
                }
            }
        } else if (tid == 0) {
            ucount[it] = (unsigned long long)total;
        }
        for (int64_t w = w0; w < w1; ++w) bm[w] = 0u;
        __syncthreads();  // cleared, and the scan scratch is free again
    }
}

// dOff[j] = item_off[j * slices] for j = 0..m (a query's list starts at its first slice).
__global__ void lsh_item_to_query_off_kernel(const int64_t *__restrict__ item_off, int64_t m, int64_t slices,
                                             int64_t *__restrict__ dOff) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j <= m; j += (int64_t)gridDim.x * blockDim.x)
        dOff[j] = item_off[j * slices];
}

int grow(void **p, int64_t *cap, int64_t bytes) {
    if (*cap >= bytes) return 0;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    STAG_CUDA_TRY(dev_malloc(p, bytes));
    *cap = bytes;
    return 0;
}

unsigned hash_grid_y(int64_t rows) { return (unsigned)ceil_div(rows, kHashRows); }

int launch_hash(const stag_lsh *h, const float *X, int64_t rows, int32_t *H, cudaStream_t s) {
    const int nf = h->K * h->L;
    if (rows == 0) return 0;
    if (hash_grid_y(rows) > 65535u * 1024u) return fail(STAG_KDE_EINVAL, "too many rows");
    const size_t smem = (size_t)h->d * kHashFns * sizeof(float);
    // grid.y is limited to 65535: walk the rows in slices
    const int64_t slice = (int64_t)65535 * kHashRows;
    for (int64_t r0 = 0; r0 < rows; r0 += slice) {
        const int64_t r = std::min(slice, rows - r0);
        dim3 grid((unsigned)ceil_div(nf, kHashFns), hash_grid_y(r));
        count_launch();
        lsh_hash_kernel<<<grid, dim3(kHashFns, kHashRows), smem, s>>>(X + r0 * h->d, r, (int)h->d, h->A, h->B, nf,
                                                                       H + r0 * nf);
    }
    STAG_CUDA_TRY(cudaGetLastError());
    return 0;
}

unsigned grid_for_elems(int64_t total, int threads) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, threads), 152 * 32));
}

int bits_for(int64_t v) {
    int b = 0;
    while (b < 63 && ((int64_t)1 << b) <= v) ++b;
    return b;
}

LshTables tables_of(const stag_lsh *h) {
    return LshTables{h->keys, h->ids, h->X, h->A, h->B, h->n, (int)h->d, h->K, h->L, h->key_bits, h->salt};
}

// The bitmap path of lsh_run: bucket ranges, distinct counts per (query, slice), their
// prefix sum, the lists, and the per-query offsets. Synchronises the stream.
int lsh_run_bitmap(stag_lsh *h, const int32_t *HQ, int64_t *range, int64_t m, int64_t *dOff, cudaStream_t s,
                   int64_t *total) {
    const int64_t words = bitmap_words(h->n), slices = bitmap_slices(h->n), items = m * slices;
    const int64_t sw = bitmap_slice_words(h->n);
    const size_t smem = (size_t)(sw + 32) * 4;
    constexpr int kMaxSmem = (int)((kMaxSliceWords + 32) * 4);
    static const cudaError_t attr = [] {
        cudaError_t e = cudaFuncSetAttribute(lsh_bitmap_kernel<false, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(lsh_bitmap_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kMaxSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(lsh_bitmap_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kMaxSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(lsh_bitmap_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kMaxSmem);
        return e;
    }();
    STAG_CUDA_TRY(attr);
    auto count_k = slices > 1 ? lsh_bitmap_kernel<false, true> : lsh_bitmap_kernel<false, false>;
    auto write_k = slices > 1 ? lsh_bitmap_kernel<true, true> : lsh_bitmap_kernel<true, false>;
    const int64_t b_cnt = round_up(items * 8, 256), b_off = round_up((items + 1) * 8, 256);
    int rc = grow(&h->sort_buf, &h->sort_cap, b_cnt + b_off);
    if (rc) return rc;
    unsigned long long *ucount = (unsigned long long *)h->sort_buf;
    int64_t *item_off = (int64_t *)((char *)h->sort_buf + b_cnt);
    int dev_sms = 0;
    STAG_CUDA_TRY(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, h->device));
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)dev_sms * 2));
    count_launch(4);
    lsh_lookup_kernel<<<grid_for_elems(m * h->L, 256), 256, 0, s>>>(HQ, m, tables_of(h), range, nullptr);
    count_k<<<grid, kBmThreads, smem, s>>>(range, m, h->L, h->ids, words, slices, sw, ucount, nullptr, nullptr);
    scan_i64_kernel<<<1, 1024, 0, s>>>(ucount, items, item_off);
    lsh_item_to_query_off_kernel<<<grid_for_elems(m + 1, 256), 256, 0, s>>>(item_off, m, slices, dOff);
    STAG_CUDA_TRY(cudaGetLastError());
    int64_t U = 0;
    STAG_CUDA_TRY(cudaMemcpyAsync(&U, dOff + m, 8, cudaMemcpyDeviceToHost, s));
    STAG_CUDA_TRY(cudaStreamSynchronize(s));
    rc = grow(&h->cand, &h->cand_cap, std::max<int64_t>(U, 1) * 8);
    if (rc) return rc;
    count_launch();
    write_k<<<grid, kBmThreads, smem, s>>>(range, m, h->L, h->ids, words, slices, sw, nullptr, item_off,
                                           (int64_t *)h->cand);
    STAG_CUDA_TRY(cudaGetLastError());
    STAG_CUDA_TRY(cudaStreamSynchronize(s));
    *total = U;
    return 0;
}

// Candidate lists of the device queries dQ into dOff (m + 1, device) and the handle's
// candidate buffer; *total = number of candidates. Synchronises the stream.
int lsh_run(stag_lsh *h, const float *dQ, int64_t m, int64_t *dOff, cudaStream_t s, int64_t *total) {
    const int L = h->L, K = h->K;
    const int64_t nf = (int64_t)K * L;
    // scratch: HQ (m * nf int32) | range (m * L * 2 int64) | count (m u64) | raw_off (m + 1 int64)
    const int64_t b_hq = round_up(m * nf * 4, 256), b_rng = round_up(m * L * 16, 256);
    const int64_t b_cnt = round_up(m * 8, 256), b_off = round_up((m + 1) * 8, 256);
    int rc = grow(&h->scratch, &h->scratch_cap, b_hq + b_rng + b_cnt + b_off);
    if (rc) return rc;
    char *base = (char *)h->scratch;
    int32_t *HQ = (int32_t *)base;
    int64_t *range = (int64_t *)(base + b_hq);
    unsigned long long *count = (unsigned long long *)(base + b_hq + b_rng);
    int64_t *raw_off = (int64_t *)(base + b_hq + b_rng + b_cnt);
    rc = launch_hash(h, dQ, m, HQ, s);
    if (rc) return rc;
    if (bitmap_fits(h->n)) return lsh_run_bitmap(h, HQ, range, m, dOff, s, total);
    STAG_CUDA_TRY(cudaMemsetAsync(count, 0, m * 8, s));
    count_launch(2);
    lsh_lookup_kernel<<<grid_for_elems(m * L, 256), 256, 0, s>>>(HQ, m, tables_of(h), range, count);
    scan_i64_kernel<<<1, 1024, 0, s>>>(count, m, raw_off);
    STAG_CUDA_TRY(cudaGetLastError());
    int64_t R = 0;
    STAG_CUDA_TRY(cudaMemcpyAsync(&R, raw_off + m, 8, cudaMemcpyDeviceToHost, s));
    STAG_CUDA_TRY(cudaStreamSynchronize(s));
    // raw keys + sort buffers: keys, ktmp (R u64 each), vals, vtmp (R u32 each), hist
    const int64_t b_k = round_up(std::max<int64_t>(R, 1) * 8, 256), b_v = round_up(std::max<int64_t>(R, 1) * 4, 256);
    const int64_t b_h = round_up(radix_sort_hist_entries(std::max<int64_t>(R, 1)) * 4, 256), b_u = round_up(m * 8, 256);
    int rcs = grow(&h->sort_buf, &h->sort_cap, 2 * b_k + 2 * b_v + b_h + b_u);
    if (rcs) return rcs;
    char *sb = (char *)h->sort_buf;
    uint64_t *raw = (uint64_t *)sb, *ktmp = (uint64_t *)(sb + b_k);
    uint32_t *vals = (uint32_t *)(sb + 2 * b_k), *vtmp = (uint32_t *)(sb + 2 * b_k + b_v);
    uint32_t *hist = (uint32_t *)(sb + 2 * b_k + 2 * b_v);
    unsigned long long *ucount = (unsigned long long *)(sb + 2 * b_k + 2 * b_v + b_h);
    const unsigned wgrid = grid_for_elems(m * 32, 256);
    count_launch();
    lsh_fill_kernel<<<wgrid, 256, 0, s>>>(range, m, L, h->ids, raw_off, raw);
    if (R > 0 && L > 1) {
        // one table's buckets list each index once, in increasing order; across tables repeats occur
        STAG_CUDA_TRY(cudaMemsetAsync(vals, 0, R * 4, s));
        rc = radix_sort_pairs(raw, vals, ktmp, vtmp, hist, R, 32 + bits_for(m - 1), s);
    }
    if (!rc) {
        count_launch(2);
        lsh_unique_kernel<false><<<wgrid, 256, 0, s>>>(raw, raw_off, m, ucount, nullptr, nullptr);
        scan_i64_kernel<<<1, 1024, 0, s>>>(ucount, m, dOff);
        int64_t U = 0;
        cudaError_t e = cudaMemcpyAsync(&U, dOff + m, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "candidate count");
        } else {
            rc = grow(&h->cand, &h->cand_cap, std::max<int64_t>(U, 1) * 8);
            if (!rc) {
                count_launch();
                lsh_unique_kernel<true><<<wgrid, 256, 0, s>>>(raw, raw_off, m, nullptr, dOff, (int64_t *)h->cand);
                e = cudaGetLastError();
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) rc = cuda_fail(e, "candidate lists");
                *total = U;
            }
        }
    }
    cudaStreamSynchronize(s);
    return rc;
}

struct Guard {
    int prev = 0;
    bool ok = false;
    explicit Guard(int dev) {
        ok = cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess;
    }
    ~Guard() { cudaSetDevice(prev); }
};

bool finite_all(const float *p, int64_t count) {
    for (int64_t i = 0; i < count; ++i)
        if (!(p[i] == p[i]) || p[i] > 1e15f || p[i] < -1e15f) return false;
    return true;
}

void free_lsh(stag_lsh *h) {
    if (!h) return;
    Guard g(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    cudaFree(h->A);
    cudaFree(h->B);
    cudaFree(h->keys);
    cudaFree(h->ids);
    cudaFree(h->X);
    cudaFree(h->scratch);
    cudaFree(h->cand);
    cudaFree(h->sort_buf);
    cudaFree(h->host_q);
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // namespace
}  // namespace stagkde

using namespace stagkde;

extern "C" {

stag_lsh_t *stag_lsh_create(const float *X, int64_t n, int64_t d, int K, int L, const float *A, const float *B,
                            int device) {
    if (!X || !A || !B) return (set_error("X, A or B is NULL"), nullptr);
    if (n < 1 || d < 1 || K < 1 || L < 1) return (set_error("need n, d, K, L >= 1"), nullptr);
    if (L > 63) return (set_error("at most 63 tables"), nullptr);
    if (n >= ((int64_t)1 << 32) || d > 384 || (int64_t)K * L > 4096)
        return (set_error("need n < 2^32, d <= 384 and K * L <= 4096"), nullptr);
    if (!finite_all(X, n * d) || !finite_all(A, (int64_t)K * L * d) || !finite_all(B, (int64_t)K * L))
        return (set_error("X, A or B has a non-finite value or |value| > 1e15"), nullptr);
    stag_lsh *h = new (std::nothrow) stag_lsh();
    if (!h) return (set_error("out of host memory"), nullptr);
    if (device < 0) {
        if (cudaGetDevice(&h->device) != cudaSuccess) {
            delete h;
            return (set_error("no CUDA device"), nullptr);
        }
    } else {
        h->device = device;
    }
    Guard g(h->device);
    h->n = n;
    h->d = d;
    h->K = K;
    h->L = L;
    const int64_t nf = (int64_t)K * L;
    auto bail = [&](int rc) -> stag_lsh_t * {
        (void)rc;
        free_lsh(h);
        return nullptr;
    };
    cudaError_t e;
    if (!g.ok) return (cuda_fail(cudaErrorInvalidDevice, "cudaSetDevice"), bail(0));
    if ((e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)) != cudaSuccess)
        return (cuda_fail(e, "cudaStreamCreate"), bail(0));
    int32_t *H = nullptr;
    void *sortb = nullptr;
    int *dbad = nullptr;
    auto cleanup = [&]() {
        cudaStreamSynchronize(h->stream);
        cudaFree(H);
        cudaFree(sortb);
        cudaFree(dbad);
    };
    const int64_t nl = n * L;
    if ((e = dev_malloc(&h->A, nf * d * 4)) != cudaSuccess || (e = dev_malloc(&h->B, nf * 4)) != cudaSuccess ||
        (e = dev_malloc(&h->keys, nl * 8)) != cudaSuccess || (e = dev_malloc(&h->ids, nl * 4)) != cudaSuccess ||
        (e = dev_malloc(&h->X, n * d * 4)) != cudaSuccess || (e = dev_malloc(&H, n * nf * 4)) != cudaSuccess ||
        (e = dev_malloc(&sortb, nl * 12 + radix_sort_hist_entries(nl) * 4)) != cudaSuccess ||
        (e = dev_malloc(&dbad, sizeof(int))) != cudaSuccess) {
        cleanup();
        return (cuda_fail(e, "cudaMalloc (LSH tables)"), bail(0));
    }
    float *dX = h->X;
    // test hook: fewer key bits make different tuples share keys, exercising the salt
    // retry and the lookup's tuple check
    if (const char *kb = getenv("STAG_KDE_LSH_KEY_BITS")) h->key_bits = std::min(58, std::max(8, atoi(kb)));
    cudaStream_t s = h->stream;
    if ((e = cudaMemcpyAsync(h->A, A, nf * d * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(h->B, B, nf * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dX, X, n * d * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) {
        cleanup();
        return (cuda_fail(e, "cudaMemcpy (LSH inputs)"), bail(0));
    }
    int rc = launch_hash(h, dX, n, H, s);
    // keys, sort, and the check that no key is shared by two different K-tuples; on a
    // shared key the tables are rebuilt with the next salt
    constexpr int kSalts = 16;
    bool clean = false;
    for (int attempt = 0; attempt < kSalts && !rc && !clean; ++attempt) {
        h->salt = 0xD1B54A32D192ED03ull * (uint64_t)attempt;
        count_launch(2);
        lsh_keys_kernel<<<grid_for_elems(nl, 256), 256, 0, s>>>(H, n, K, L, h->salt, h->key_bits, h->keys, h->ids);
        char *sb = (char *)sortb;
        rc = radix_sort_pairs(h->keys, h->ids, (uint64_t *)sb, (uint32_t *)(sb + nl * 8), (uint32_t *)(sb + nl * 12),
                              nl, 64, s);
        if (rc) break;
        int bad = 0;
        if ((e = cudaMemsetAsync(dbad, 0, sizeof(int), s)) != cudaSuccess) {
            rc = cuda_fail(e, "cudaMemsetAsync");
            break;
        }
        lsh_collision_kernel<<<grid_for_elems(nl, 256), 256, 0, s>>>(h->keys, h->ids, H, n, K, L, dbad);
        if ((e = cudaMemcpyAsync(&bad, dbad, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess) {
            rc = cuda_fail(e, "LSH table build");
            break;
        }
        clean = bad == 0;
    }
    if (!rc && !clean) rc = fail(STAG_KDE_EUNSUPPORTED, "LSH tables: every salt left two K-tuples sharing a key");
    cleanup();
    if (rc) return bail(rc);
    return h;
}

int stag_lsh_hash_dev(stag_lsh_t *h, const float *dQ, int64_t m, int32_t *dH, void *stream) {
    if (!h) return fail(STAG_KDE_EINVAL, "handle is NULL");
    if (m < 0) return fail(STAG_KDE_EINVAL, "m < 0");
    if (m == 0) return 0;
    if (!dQ || !dH) return fail(STAG_KDE_EINVAL, "dQ or dH is NULL");
    Guard g(h->device);
    if (!g.ok) return fail(STAG_KDE_ECUDA, "cudaSetDevice failed");
    return launch_hash(h, dQ, m, dH, (cudaStream_t)stream);
}

int stag_lsh_query_dev(stag_lsh_t *h, const float *dQ, int64_t m, int64_t *dOff, int64_t *dIdx, int64_t cap,
                       int64_t *total, void *stream) {
    if (!h) return fail(STAG_KDE_EINVAL, "handle is NULL");
    if (m < 0 || !total) return fail(STAG_KDE_EINVAL, "m < 0, or total is NULL");
    if (m > 0 && (!dQ || !dOff)) return fail(STAG_KDE_EINVAL, "dQ or dOff is NULL");
    Guard g(h->device);
    if (!g.ok) return fail(STAG_KDE_ECUDA, "cudaSetDevice failed");
    *total = 0;
    h->last_total = 0;
    if (m == 0) return 0;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = lsh_run(h, dQ, m, dOff, s, total);
    if (rc) return rc;
    h->last_total = *total;
    if (dIdx && cap >= *total && *total > 0)
        STAG_CUDA_TRY(cudaMemcpyAsync(dIdx, h->cand, *total * 8, cudaMemcpyDeviceToDevice, s));
    return 0;
}

int stag_lsh_fetch_dev(stag_lsh_t *h, int64_t *dIdx, int64_t cap, void *stream) {
    if (!h) return fail(STAG_KDE_EINVAL, "handle is NULL");
    if (h->last_total == 0) return 0;
    if (!dIdx || cap < h->last_total) return fail(STAG_KDE_EINVAL, "dIdx is NULL or cap is below the list size");
    Guard g(h->device);
    if (!g.ok) return fail(STAG_KDE_ECUDA, "cudaSetDevice failed");
    STAG_CUDA_TRY(cudaMemcpyAsync(dIdx, h->cand, h->last_total * 8, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return 0;
}

int stag_lsh_query(stag_lsh_t *h, const float *Q, int64_t m, int64_t *off, int64_t *idx, int64_t cap,
                   int64_t *total) {
    if (!h) return fail(STAG_KDE_EINVAL, "handle is NULL");
    if (m < 0 || !total || !off) return fail(STAG_KDE_EINVAL, "m < 0, or total / off is NULL");
    *total = 0;
    off[0] = 0;
    if (m == 0) return 0;
    if (!Q) return fail(STAG_KDE_EINVAL, "Q is NULL");
    if (!finite_all(Q, m * h->d)) return fail(STAG_KDE_EINVAL, "Q has a non-finite value or |q| > 1e15");
    Guard g(h->device);
    if (!g.ok) return fail(STAG_KDE_ECUDA, "cudaSetDevice failed");
    const int64_t b_q = round_up(m * h->d * 4, 256);
    int rc = grow(&h->host_q, &h->host_q_cap, b_q + (m + 1) * 8);
    if (rc) return rc;
    float *dQ = (float *)h->host_q;
    int64_t *dOff = (int64_t *)((char *)h->host_q + b_q);
    cudaStream_t s = h->stream;
    STAG_CUDA_TRY(cudaMemcpyAsync(dQ, Q, m * h->d * 4, cudaMemcpyHostToDevice, s));
    h->last_total = 0;
    rc = lsh_run(h, dQ, m, dOff, s, total);
    if (rc) return rc;
    h->last_total = *total;
    STAG_CUDA_TRY(cudaMemcpyAsync(off, dOff, (m + 1) * 8, cudaMemcpyDeviceToHost, s));
    if (idx && cap >= *total && *total > 0)
        STAG_CUDA_TRY(cudaMemcpyAsync(idx, h->cand, *total * 8, cudaMemcpyDeviceToHost, s));
    STAG_CUDA_TRY(cudaStreamSynchronize(s));
    return 0;
}

int stag_lsh_fetch(stag_lsh_t *h, int64_t *idx, int64_t cap) {
    if (!h) return fail(STAG_KDE_EINVAL, "handle is NULL");
    if (h->last_total == 0) return 0;
    if (!idx || cap < h->last_total) return fail(STAG_KDE_EINVAL, "idx is NULL or cap is below the list size");
    Guard g(h->device);
    if (!g.ok) return fail(STAG_KDE_ECUDA, "cudaSetDevice failed");
    STAG_CUDA_TRY(cudaMemcpyAsync(idx, h->cand, h->last_total * 8, cudaMemcpyDeviceToHost, h->stream));
    STAG_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return 0;
}

int stag_lsh_info(const stag_lsh_t *h, int64_t *n, int64_t *d, int *K, int *L) {
    if (!h) return fail(STAG_KDE_EINVAL, "handle is NULL");
    if (n) *n = h->n;
    if (d) *d = h->d;
    if (K) *K = h->K;
    if (L) *L = h->L;
    return 0;
}

void stag_lsh_destroy(stag_lsh_t *h) { free_lsh(h); }

}  // extern "C"
