// Tensor-core form of exact Gaussian KDE (Sec. 3: K(q) = sum_i exp(-a ||q - x_i||^2)) on
// sm_103a: tcgen05.mma into TMEM, operands fed by TMA, exp and row sum fused into the
// epilogue, so the m x n matrix of kernel values never exists in memory.
//
// Arithmetic. The point set is cut into tiles of BN points (spatially coherent, k-d
// order); tile t has a centre c_t (the FP64 mean of its points, stored as FP32) and the
// queries are centred on the global mean c_g. With v = x - c_t, u = q - c_g and
// D_t = c_t - c_g,
//     ||q - x||^2 = ||q - c_t||^2 + ( ||v||^2 + 2 D_t . v ) - 2 u . v        (exact)
//                 =  R(q, t)     +        g(x)             - 2 u . v
// R is computed by direct differences in FP32 (rowterm kernel, one value per query and
// tile), g in FP64 at create time (one value per point), and u . v on the tensor cores
// with FP16 hi/lo splits of u and v (power-of-two scaled into FP16 range):
//     u . v ~ u_hi . v_hi + u_hi . v_lo + u_lo . v_hi        (three MMAs, FP32 accumulate)
// which represents both operands to ~2^-22 and drops only the u_lo . v_lo term (~2^-22).
// The point term g rides along as a fourth MMA of K = 16: the A side is the constant
// column [s_a, s_a, s_a, 0, ...] and the B side holds -g / (2 scale) split into three
// FP16 pieces (~2^-33), so the accumulator already holds u.v - g/2 in scaled units and
// the epilogue needs no per-column data. Per pair it evaluates
//     e = 2^( kk * D - (c R + s_row) ),   c = a log2(e), kk = 2c / (scale_u scale_v)
// with the same integer per-row shift s as the plain form (see kde_simt.cu) so that
// rows whose every term is below FP32's range are still represented.
//
// Kernel structure (persistent, one CTA per SM, warp-specialised):
//   warp 0      TMA producer: per work unit the query tile's A planes (u_hi, u_lo, the
//               constant column), per point tile the B planes (v_hi, v_lo, -g pieces)
//               and a metadata block (R of the unit's 128 queries, the tile's
//               radius) into rings of stages;
//   warp 1      allocates TMEM; one thread issues 3 * K/16 + 1 MMAs per accumulator
//               and commits. K = 16 ("ring"): four accumulators of 128 lanes x BN/2
//               FP32 columns, half tile k into accumulator k mod 4; K >= 32: two
//               accumulators of BN columns, tile t into accumulator t mod 2;
//   4*EG warps  epilogue, EG groups of 4 warps (one per TMEM lane quadrant), each
//               thread one query row (its TMEM lane): tcgen05.ld, packed FMA, ex2,
//               packed add. Ring: group g takes the half tiles k with k mod EG = g and
//               waits only for its own accumulators, so the groups drift apart by up to
//               a tile without stalling one another; K >= 32: group g takes BN/EG
//               columns of every tile, so an accumulator is drained by all warps at once.
// A work unit is (query tile of 128 rows, contiguous range of point tiles); the partial
// sums per (range, query) are combined in FP64, together with a per-query error
// estimate, by tc_combine_kernel; queries whose estimate is too large are recomputed by
// the plain FP32 form.
// Every mbarrier wait is bounded (%globaltimer); on expiry the kernel records an error
// code, makes the other roles stop, waits for its own copies and MMAs, frees TMEM and
// returns, and the host reports STAG_KDE_ETIMEDOUT.
#include <cuda.h>
#include <cuda_fp16.h>
#include <math.h>

#include <stdlib.h>

#include <algorithm>
#include <climits>
#include <type_traits>
#include <mutex>

#include "f32x2.cuh"
#include "internal.h"
#include "kernel_fn.cuh"
#include "sm100_ptx.cuh"

namespace stagkde {

// --------------------------------------------------------------------------------------
// Host-side data of the tensor-core form.
// --------------------------------------------------------------------------------------
struct TcData {
    int Kp = 0;          // per-split operand width in FP16 elements (16, 32, 64 or 128)
    int BN = 0;          // points per tile (MMA N)
    int64_t T = 0;       // number of point tiles
    int64_t n_pad = 0;   // T * BN
    __half *b_hi = nullptr, *b_lo = nullptr;  // [n_pad][Kp]
    __half *b_aug = nullptr;                  // [n_pad][16]: -g / (2 scale) in 3 FP16 pieces, then 0
    __half *a_aug = nullptr;                  // [128][16]: s_a, s_a, s_a, 0, ...
    float *tinfo = nullptr;                   // [T][4]: RMS radius (the error estimate's split
                                              //         term), max radius rounded up so that it bounds
                                              //         FP32 distances (exponent bounds, pruning), max
                                              //         radius, the estimate's accumulation weight
    float *cent = nullptr;                    // [T][Kp]: tile centres c_t (FP32)
    float *centT = nullptr;                   // [Kp][T]: the same, coordinate-major (row terms)
    float *cg = nullptr;                      // [Kp]: global centre c_g
    double *tsum = nullptr;                   // [T][Kp]: FP64 per-tile coordinate sums
    unsigned *vmax_bits = nullptr;            // max |x_k - c_t,k| (float bits)
    unsigned *xmax_bits = nullptr;            // max |x_k - c_g,k| (float bits)
    float *scales = nullptr;                  // [4]: scale_v, scale_u, kk, s_a
    CUtensorMap map_bhi, map_blo, map_baug, map_aaug;
    // query-side scratch
    __half *a_hi = nullptr, *a_lo = nullptr;  // [m_cap][Kp]
    int64_t a_rows_cap = 0;
    CUtensorMap map_ahi, map_alo;
    float *rowterm = nullptr;  // [T][m_pad]
    int64_t rt_cap = 0;        // floats
    float *unorm = nullptr;    // [m_cap]: ||q - c_g|| per query
    int *qbad = nullptr;       // [m_cap]: query outside the FP16 range of the split
    unsigned *ub = nullptr;    // [m_cap]: per-query exponent bound (order bits)
    int64_t unorm_cap = 0;
    double *part_w = nullptr;  // [splits][m]: contribution-weighted tile radius sums
    int64_t part_w_cap = 0;
    float *xkt = nullptr;      // k-d ordered points in the plain form's tile-transposed layout
                               // (the recompute of flagged queries)
    void *gbuf = nullptr;      // grouped-recompute scratch (GroupScratch), sized for gbuf_m rows
    int64_t gbuf_m = 0;
    int *fix_idx = nullptr;    // [m_cap]: queries handed to the plain form
    int *fix_count = nullptr;  // device counter
    int *err = nullptr;        // device error code (timeouts)
    int *err_host = nullptr;   // pinned mirror
};

namespace {

constexpr int kErrTimeout = 1;
constexpr int BM = 128;  // queries per tile (MMA M, TMEM lanes)
// Queries whose estimated tensor-core error exceeds this are recomputed with the plain
// FP32 form; the estimate bounds the measured error from above (ratio <= ~0.96), so the
// queries kept stay below ~7.2e-5 against the 1e-4 tolerance.
constexpr double kTcErrThreshold = 7.5e-5;
}  // namespace

// Epilogue warps per TMEM lane quadrant (2 or 4); STAG_KDE_TC_EG overrides the default.
int tc_epilogue_groups() {
    static int eg = []() {
        const char *e = getenv("STAG_KDE_TC_EG");
        const int v = e ? atoi(e) : 4;
        return v == 2 ? 2 : 4;
    }();
    return eg;
}

namespace {

// ------------------------------------------------------------------ layout helpers
template <int KP>
struct Geo {
    static constexpr int CW = KP < 64 ? KP : 64;       // elements per TMA box row / swizzle span
    static constexpr int CH = KP / CW;                 // chunks along K
    static constexpr int SPC = CW / 16;                // MMA K-steps per chunk
    static constexpr uint32_t SW = CW == 16 ? ptx::kSw32 : (CW == 32 ? ptx::kSw64 : ptx::kSw128);
    static constexpr uint32_t SBO = 8 * CW * 2;        // bytes between 8-row core-matrix groups
    // byte offset of MMA K-step s inside a plane of `rows` rows
    __host__ __device__ static constexpr uint32_t koff(int s, int rows) {
        return (uint32_t)((s / SPC) * rows * CW * 2 + (s % SPC) * 32);
    }
};

template <int KP, int BN, int SB, int SMETA, int AB, int EG>
struct Cfg {
    static constexpr int THREADS = 64 + 128 * EG;  // TMA warp, MMA warp, 4 * EG epilogue warps
    static constexpr int A_PLANE = BM * KP * 2;
    static constexpr int B_PLANE = BN * KP * 2;
    static constexpr int A_AUG = BM * 16 * 2;
    static constexpr int B_AUG = BN * 16 * 2;
    static constexpr int A_BYTES = 2 * A_PLANE + A_AUG;
    static constexpr int B_BYTES = 2 * B_PLANE + B_AUG;
    static constexpr int META_BYTES = BM * 4 + 16;  // R of 128 queries, tile info
    static constexpr int META_STRIDE = (META_BYTES + 127) / 128 * 128;
    static constexpr int OFF_A = 0;
    static constexpr int OFF_B = OFF_A + AB * A_BYTES;
    static constexpr int OFF_META = OFF_B + SB * B_BYTES;
    static constexpr int OFF_MERGE = OFF_META + SMETA * META_STRIDE;
    static constexpr int OFF_BAR = OFF_MERGE + BM * 24 * (EG - 1);
    static constexpr int NBAR = 2 * SB + 2 * SMETA + 2 * AB + 2 * 4 + 3;  // 4: accumulators, at most
    static constexpr int OFF_MISC = OFF_BAR + NBAR * 8;
    static constexpr int BYTES = OFF_MISC + 64;
    static constexpr int SMEM = BYTES + 1024;  // + alignment slack
    // Accumulator layout. RING (K = 16, where the epilogue's ex2 rate is the bound): four
    // TMEM accumulators of BN/2 columns, one per half tile, each owned by one epilogue
    // group, so the groups run up to a tile apart without waiting for one another.
    // Otherwise (K >= 32, where the tensor pipe has less slack and the N = BN MMAs are
    // more efficient): two accumulators of BN columns shared by all groups, each group
    // taking BN/EG columns of every tile, which hands an accumulator back sooner.
    static constexpr bool RING = KP <= 16;
    static constexpr int NACC = RING ? 4 : 2;
    static constexpr int ACC_COLS = RING ? BN / 2 : BN;
    static constexpr int WCOLS = RING ? BN / 2 : BN / EG;     // columns one warp reads per visit
    static constexpr int ACC_READERS = RING ? 4 : 4 * EG;     // warps reading one accumulator
    static constexpr int META_READERS = RING ? 8 : 4 * EG;    // warps reading one tile's row terms
    static constexpr uint32_t TMEM_COLS = NACC * ACC_COLS;
    static constexpr uint32_t IDESC = ptx::idesc_f16_f32(BM, ACC_COLS);
    static_assert(!RING || NACC % EG == 0, "every accumulator belongs to one epilogue group");
    static_assert(A_PLANE % 1024 == 0 && B_PLANE % 1024 == 0 && A_AUG % 1024 == 0 && B_AUG % 1024 == 0,
                  "planes must keep 1024-byte alignment");
};

// One KDE instance as the tensor-core kernel sees it. A launch processes a table of
// instances of the same operand width; the units of instance i are the global unit
// indices [unit_begin, unit_begin + q_tiles * splits). The tensor maps sit in this
// struct, in kernel-parameter space (one instance) or global memory (a batch table).
struct TcInst {
    CUtensorMap map_ahi, map_alo, map_aaug, map_bhi, map_blo, map_baug;
    const float *tinfo;    // [T][4]
    const float *rowterm;  // [T][m_pad]
    const float *scales;   // device: scale_v, scale_u, kk, s_a
    const unsigned *ub;    // [m_pad]: per-query upper bound on every exponent (order bits)
    const float *unorm;    // [m_pad]: ||q - c_g|| (the error estimate's split term)
    double *part_sum;      // [splits][m]
    float *part_shift;
    double *part_w;
    int64_t m, m_pad, n, T, q_tiles, tiles_per_split, unit_begin, units;
};

// The instance owning global unit u (binary search over unit_begin).
__device__ __forceinline__ const TcInst *find_inst(const TcInst *insts, int n_inst, int64_t u) {
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (insts[mid].unit_begin <= u)
            lo = mid;
        else
            hi = mid - 1;
    }
    return insts + lo;
}

__device__ __forceinline__ int64_t ceil_div_dev(int64_t a, int64_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ int cexp(float e) { return (int)fminf(fmaxf(e, -4000.f), 4000.f); }

__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(uint64_t v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ uint32_t float_order_bits(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float order_bits_to_float(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// A row's running sums in units of 2^shift. Each tile's sum is folded into a compensated
// FP32 sum (ksum, kc; Kahan), which keeps ~2^-24 relative accuracy over thousands of
// tiles without touching the slow FP64 pipe in the loop; FP64 is used once per work unit.
struct RowState {
    float shift;
    float ksum;  // compensated sum of the tiles so far
    float kc;    // its compensation term
    float w32;   // sum over tiles of (tile sum) * (tile's error weight), same units as ksum
};

__device__ __forceinline__ void kahan_add(float &sum, float &comp, float x) {
    const float y = x - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// Adds 2^(kk*D[j] + nb) for the 32 columns of one TMEM chunk into two packed accumulators
// (four independent FP32 chains). nb = -(c R + s) with the row's fixed shift s, which bounds
// every exponent from above, so no term exceeds ~1 and no rescaling is needed. kMasked:
// only the first `valid` columns hold real points (the point set's last, padded tile).
template <bool kMasked>
__device__ __forceinline__ void epi_chunk(uint64_t &acc_a, uint64_t &acc_b, const uint32_t (&D)[32], uint64_t kk2,
                                          uint64_t nb2, int valid) {
#pragma unroll
    for (int j = 0; j < 32; j += 4) {
        const uint64_t x01 = fma2(kk2, pack2(__uint_as_float(D[j]), __uint_as_float(D[j + 1])), nb2);
        const uint64_t x23 = fma2(kk2, pack2(__uint_as_float(D[j + 2]), __uint_as_float(D[j + 3])), nb2);
        float a0, a1, a2, a3;
        unpack2(x01, a0, a1);
        unpack2(x23, a2, a3);
        float e0 = ptx::ex2_approx(a0), e1 = ptx::ex2_approx(a1);
        float e2 = ptx::ex2_approx(a2), e3 = ptx::ex2_approx(a3);
        if constexpr (kMasked) {
            e0 = j < valid ? e0 : 0.f;
            e1 = j + 1 < valid ? e1 : 0.f;
            e2 = j + 2 < valid ? e2 : 0.f;
            e3 = j + 3 < valid ? e3 : 0.f;
        }
        acc_a = add2(acc_a, pack2(e0, e1));
        acc_b = add2(acc_b, pack2(e2, e3));
    }
}

// The persistent tensor-core kernel's work, for one CTA of `ncta` serving the units of a
// table of instances of one operand width: CTA number `cta` takes units cta, cta + ncta,
// ... . `insts` points at kernel-parameter space when in_params (one instance; its tensor
// maps are prefetched) or at a table in global memory.
template <int KP, int BN, int SB, int SMETA, int AB, int EG>
__device__ __forceinline__ void tc_body(const TcInst *__restrict__ insts, bool in_params, int n_inst,
                                        int64_t total_units, int *err, uint64_t wait_ns, uint64_t stall_ns,
                                        int cta, int ncta) {
    using C = Cfg<KP, BN, SB, SMETA, AB, EG>;
    using G = Geo<KP>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + C::OFF_BAR);
    uint64_t *full_b = bars;
    uint64_t *empty_b = full_b + SB;
    uint64_t *full_m = empty_b + SB;
    uint64_t *empty_m = full_m + SMETA;
    uint64_t *a_full = empty_m + SMETA;
    uint64_t *a_empty = a_full + AB;
    uint64_t *acc_full = a_empty + AB;
    uint64_t *acc_empty = acc_full + 4;
    uint64_t *merge_full = acc_empty + 4;
    uint64_t *merge_empty = merge_full + 1;
    uint64_t *drain = merge_empty + 1;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(smem + C::OFF_MISC);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + C::OFF_MISC + 16);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < SB; ++i) {
            ptx::mbar_init(&full_b[i], 1);
            ptx::mbar_init(&empty_b[i], 1);
        }
        for (int i = 0; i < SMETA; ++i) {
            ptx::mbar_init(&full_m[i], 1);
            ptx::mbar_init(&empty_m[i], C::META_READERS);
        }
        for (int i = 0; i < AB; ++i) {
            ptx::mbar_init(&a_full[i], 1);
            ptx::mbar_init(&a_empty[i], 1);
        }
        for (int i = 0; i < C::NACC; ++i) {
            ptx::mbar_init(&acc_full[i], 1);
            ptx::mbar_init(&acc_empty[i], C::ACC_READERS);
        }
        ptx::mbar_init(merge_full, 4 * (EG - 1));
        ptx::mbar_init(merge_empty, 4);
        ptx::mbar_init(drain, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
        ptx::fence_proxy_async();
    }
    if (warp == 0 && lane == 0) {
        if (in_params) {
            ptx::prefetch_tensormap(&insts->map_ahi);
            ptx::prefetch_tensormap(&insts->map_alo);
            ptx::prefetch_tensormap(&insts->map_aaug);
            ptx::prefetch_tensormap(&insts->map_bhi);
            ptx::prefetch_tensormap(&insts->map_blo);
            ptx::prefetch_tensormap(&insts->map_baug);
        }
    }
    if (warp == 1) {
        ptx::tmem_alloc(tmem_holder, C::TMEM_COLS);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;

    auto timed_out = [&]() {
        atomicExch(err, kErrTimeout);
        *abort_flag = 1;
    };

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t ucount = 0, tcount = 0;
            uint32_t issued_a = 0, issued_b = 0, issued_m = 0;
            bool ok = true;
            if (stall_ns) {
                // injected delay (tests of the bounded waits): the consumers find nothing
                // arriving for stall_ns; ends early once another role has given up
                const uint64_t t0 = ptx::globaltimer();
                while (ptx::globaltimer() - t0 < stall_ns && !*abort_flag) __nanosleep(1000);
            }
            for (int64_t u = cta; u < total_units && ok; u += ncta, ++ucount) {
                if (*abort_flag) {  // another role gave up: issue nothing more
                    ok = false;
                    break;
                }
                const TcInst &I = *find_inst(insts, n_inst, u);
                const int64_t lu = u - I.unit_begin;
                const int64_t split = lu / I.q_tiles, qt = lu % I.q_tiles;
                const int64_t t0 = split * I.tiles_per_split;
                const int64_t t1 = min(I.T, t0 + I.tiles_per_split);
                const int ab = ucount % AB;
                if (!ptx::mbar_wait_bounded(&a_empty[ab], ((ucount / AB) & 1) ^ 1, wait_ns, abort_flag)) {
                    timed_out();
                    ok = false;
                    break;
                }
                uint8_t *abuf = smem + C::OFF_A + ab * C::A_BYTES;
                ptx::mbar_arrive_expect_tx(&a_full[ab], C::A_BYTES);
#pragma unroll
                for (int ch = 0; ch < G::CH; ++ch) {
                    ptx::tma_load_2d(abuf + ch * BM * G::CW * 2, &I.map_ahi, ch * G::CW, (int)(qt * BM), &a_full[ab]);
                    ptx::tma_load_2d(abuf + C::A_PLANE + ch * BM * G::CW * 2, &I.map_alo, ch * G::CW, (int)(qt * BM),
                                     &a_full[ab]);
                }
                ptx::tma_load_2d(abuf + 2 * C::A_PLANE, &I.map_aaug, 0, 0, &a_full[ab]);
                ++issued_a;
                for (int64_t t = t0; t < t1; ++t, ++tcount) {
                    const int sb = tcount % SB;
                    if (!ptx::mbar_wait_bounded(&empty_b[sb], ((tcount / SB) & 1) ^ 1, wait_ns, abort_flag)) {
                        timed_out();
                        ok = false;
                        break;
                    }
                    uint8_t *bbuf = smem + C::OFF_B + sb * C::B_BYTES;
                    ptx::mbar_arrive_expect_tx(&full_b[sb], C::B_BYTES);
#pragma unroll
                    for (int ch = 0; ch < G::CH; ++ch) {
                        ptx::tma_load_2d(bbuf + ch * BN * G::CW * 2, &I.map_bhi, ch * G::CW, (int)(t * BN), &full_b[sb]);
                        ptx::tma_load_2d(bbuf + C::B_PLANE + ch * BN * G::CW * 2, &I.map_blo, ch * G::CW, (int)(t * BN),
                                         &full_b[sb]);
                    }
                    ptx::tma_load_2d(bbuf + 2 * C::B_PLANE, &I.map_baug, 0, (int)(t * BN), &full_b[sb]);
                    ++issued_b;
                    const int ms = tcount % SMETA;
                    if (!ptx::mbar_wait_bounded(&empty_m[ms], ((tcount / SMETA) & 1) ^ 1, wait_ns, abort_flag)) {
                        timed_out();
                        ok = false;
                        break;
                    }
                    uint8_t *mbuf = smem + C::OFF_META + ms * C::META_STRIDE;
                    ptx::mbar_arrive_expect_tx(&full_m[ms], C::META_BYTES);
                    ptx::bulk_load(mbuf, I.rowterm + t * I.m_pad + qt * BM, BM * 4, &full_m[ms]);
                    ptx::bulk_load(mbuf + BM * 4, I.tinfo + t * 4, 16, &full_m[ms]);
                    ++issued_m;
                }
            }
            if (!ok) {
                // Let the copies already issued land before the CTA's shared memory is
                // released: wait for the last armed phase of every stage (bounded).
                volatile int no_abort = 0;
                auto drain_ring = [&](uint64_t *full, uint32_t issued, uint32_t depth) {
                    for (uint32_t i = 0; i < depth && i < issued; ++i) {
                        const uint32_t j = i + ((issued - 1 - i) / depth) * depth;
                        ptx::mbar_wait_bounded(&full[i], (j / depth) & 1, 100000000ull, &no_abort);
                    }
                };
                drain_ring(full_b, issued_b, SB);
                drain_ring(full_m, issued_m, SMETA);
                drain_ring(a_full, issued_a, AB);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t ucount = 0, tcount = 0;
            bool ok = true;
            const uint32_t a0 = ptx::smem_u32(smem + C::OFF_A);
            const uint32_t b0 = ptx::smem_u32(smem + C::OFF_B);
            for (int64_t u = cta; u < total_units && ok; u += ncta, ++ucount) {
                const TcInst &I = *find_inst(insts, n_inst, u);
                const int64_t split = (u - I.unit_begin) / I.q_tiles;
                const int64_t t0 = split * I.tiles_per_split;
                const int64_t t1 = min(I.T, t0 + I.tiles_per_split);
                const int ab = ucount % AB;
                if (!ptx::mbar_wait_bounded(&a_full[ab], (ucount / AB) & 1, wait_ns, abort_flag)) {
                    timed_out();
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t abase = a0 + ab * C::A_BYTES;
                const uint32_t alo = ptx::smem_desc_lo(abase, 16);
                const uint32_t alo_aug = ptx::smem_desc_lo(abase + 2 * C::A_PLANE, 16);
                for (int64_t t = t0; t < t1 && ok; ++t, ++tcount) {
                    const int sb = tcount % SB;
                    if (!ptx::mbar_wait_bounded(&full_b[sb], (tcount / SB) & 1, wait_ns, abort_flag)) {
                        timed_out();
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint32_t bbase = b0 + sb * C::B_BYTES;
                    // 3 * K/16 + 1 MMAs: the split products, then the point term. Each operand's
                    // descriptor is the stage's base low word plus a compile-time constant and a
                    // constant high word, so the single issuing thread (which shares its
                    // scheduler with epilogue warps) spends one add per operand: at K = 16 the
                    // MMAs of a half tile are short and issue cost decides the pipe's rate.
                    const uint32_t blo = ptx::smem_desc_lo(bbase, 16);
                    const uint32_t blo_aug = ptx::smem_desc_lo(bbase + 2 * C::B_PLANE, 16);
                    constexpr uint32_t HI = ptx::smem_desc_hi(G::SBO, G::SW);
                    constexpr uint32_t HI_AUG = ptx::smem_desc_hi(256, ptx::kSw32);
                    auto issue = [&](uint32_t d_tmem, uint32_t row0) {
                        uint32_t accumulate = 0;
#pragma unroll
                        for (int prod = 0; prod < 3; ++prod) {
                            // (u_hi, v_hi), (u_hi, v_lo), (u_lo, v_hi); B rows row0..
#pragma unroll
                            for (int s = 0; s < KP / 16; ++s) {
                                const uint32_t aoff = (prod == 2 ? C::A_PLANE : 0) + G::koff(s, BM);
                                const uint32_t boff =
                                    (prod == 1 ? C::B_PLANE : 0) + row0 * G::CW * 2 + G::koff(s, BN);
                                ptx::mma_f16_w(d_tmem, alo + (aoff >> 4), HI, blo + (boff >> 4), HI, C::IDESC,
                                               accumulate);
                                accumulate = 1;
                            }
                        }
                        // constant A column x (-g/2) pieces, one K = 16 step
                        ptx::mma_f16_w(d_tmem, alo_aug, HI_AUG, blo_aug + ((row0 * 32) >> 4), HI_AUG, C::IDESC, 1);
                    };
                    if constexpr (C::RING) {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const uint32_t k = 2 * tcount + h;  // half tile index, CTA-wide
                            const int acc = k % C::NACC;
                            if (!ptx::mbar_wait_bounded(&acc_empty[acc], ((k / C::NACC) & 1) ^ 1, wait_ns,
                                                        abort_flag)) {
                                timed_out();
                                ok = false;
                                break;
                            }
                            ptx::tc_fence_after();
                            issue(tmem_base + acc * C::ACC_COLS, h * C::ACC_COLS);
                            ptx::mma_commit(&acc_full[acc]);
                        }
                    } else {
                        const int acc = tcount % C::NACC;
                        if (!ptx::mbar_wait_bounded(&acc_empty[acc], ((tcount / C::NACC) & 1) ^ 1, wait_ns,
                                                    abort_flag)) {
                            timed_out();
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        issue(tmem_base + acc * C::ACC_COLS, 0);
                        ptx::mma_commit(&acc_full[acc]);
                    }
                    if (!ok) break;
                    // the stage's operands are free once the tile's MMAs are done
                    ptx::mma_commit(&empty_b[sb]);
                }
                if (ok) ptx::mma_commit(&a_empty[ab]);
            }
            // every MMA issued by this thread must finish before TMEM is released
            volatile int no_abort = 0;
            ptx::mma_commit(drain);
            ptx::mbar_wait_bounded(drain, 0, 100000000ull, &no_abort);
        }
    } else {
        // ------------------------------------------------------------ epilogue (4 * EG warps)
        const int ew = warp - 2;             // 0 .. 4*EG-1
        const int quad = warp & 3;           // TMEM lane quadrant this warp may access
        const int grp = ew >> 2;             // epilogue group
        const int row = quad * 32 + lane;    // query row within the tile
        // RING: the group takes half tiles k with k mod EG = grp, i.e. half (grp & 1) of
        // every STEP-th tile; otherwise columns [grp*WCOLS, (grp+1)*WCOLS) of every tile
        const int half = grp & 1;
        constexpr int STEP = C::RING ? EG / 2 : 1;
        constexpr int WCOLS = C::WCOLS;
        constexpr int NCH = WCOLS / 32;
        const int col0 = C::RING ? half * WCOLS : grp * WCOLS;   // first point column of the visit
        static_assert(WCOLS % 32 == 0 && (EG == 2 || EG == 4), "whole 32-column chunks");
        double *msum = reinterpret_cast<double *>(smem + C::OFF_MERGE);   // [EG-1][BM]
        double *mw = msum + (EG - 1) * BM;                                 // [EG-1][BM]
        float *mshift = reinterpret_cast<float *>(mw + (EG - 1) * BM);     // [EG-1][BM]
        uint32_t tcount = 0, ucount = 0;  // point tiles and units this CTA has passed
        bool ok = true;
        RowState st{0.f, 0.f, 0.f, 0.f};
        float au = 0.f;  // 2^-21 ||q - c_g|| of this row's query (set per unit)
        // This warp's columns of point tile number tc (CTA-wide count): wait for their
        // accumulator and the tile's row terms, sum the exponentials, release both, fold
        // the sum into the row state. Returns false on timeout or abort.
        auto visit = [&](auto masked, uint64_t kk2, uint32_t tc, int vcols) -> bool {
            constexpr bool kMasked = decltype(masked)::value;
            const uint32_t k = C::RING ? 2 * tc + half : tc;   // accumulator use, CTA-wide
            const int acc = k % C::NACC;
            const int ms = tc % SMETA;
            // lane 0 waits (the other lanes do not spend issue slots polling); the outcome
            // is broadcast so that the warp never splits around __syncwarp
            bool got = true;
            if (lane == 0)
                got = ptx::mbar_wait_bounded(&acc_full[acc], (k / C::NACC) & 1, wait_ns, abort_flag) &&
                      ptx::mbar_wait_bounded(&full_m[ms], (tc / SMETA) & 1, wait_ns, abort_flag);
            if (!__shfl_sync(0xffffffffu, (int)got, 0)) return false;
            ptx::tc_fence_after();
            const float *meta = reinterpret_cast<const float *>(smem + C::OFF_META + ms * C::META_STRIDE);
            const float nb = -(meta[row] + st.shift);
            // the tile's error-estimate weight for this row: the split term (RMS radius times
            // 2^-21 ||u||) or, where larger, the accumulation term beta_K rho_t^2 (slot 3)
            const float vw = fmaxf(au * meta[BM], meta[BM + 3]);
            const uint64_t nb2 = pack2(nb, nb);
            const uint32_t taddr =
                tmem_base + ((uint32_t)(quad * 32) << 16) + acc * C::ACC_COLS + (C::RING ? 0 : grp * WCOLS);
            uint64_t acc_a = 0, acc_b = 0;  // {0.f, 0.f}
            auto release_acc = [&]() {
                // every TMEM column of this accumulator has been read: hand it back
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&acc_empty[acc]);
            };
            if constexpr (EG >= 4 || NCH == 1) {
                // enough warps per scheduler to hide the TMEM load latency: one buffer
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    uint32_t Da[32];
                    ptx::tmem_ld_32x32b_x32(taddr + c * 32, Da);
                    ptx::tmem_ld_wait();
                    ptx::reg_fence32(Da);
                    if (c + 1 == NCH) release_acc();
                    epi_chunk<kMasked>(acc_a, acc_b, Da, kk2, nb2, vcols - c * 32);
                }
            } else {
                // software pipeline: the TMEM load of chunk c+1 is in flight while chunk c
                // is processed (tcgen05.wait::ld waits for every load issued before it)
                uint32_t Da[32], Db[32];
                ptx::tmem_ld_32x32b_x32(taddr, Da);
                ptx::tmem_ld_wait();
                ptx::reg_fence32(Da);
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    if (c + 1 < NCH) {
                        if (c & 1)
                            ptx::tmem_ld_32x32b_x32(taddr + (c + 1) * 32, Da);
                        else
                            ptx::tmem_ld_32x32b_x32(taddr + (c + 1) * 32, Db);
                    } else {
                        release_acc();
                    }
                    if (c & 1)
                        epi_chunk<kMasked>(acc_a, acc_b, Db, kk2, nb2, vcols - c * 32);
                    else
                        epi_chunk<kMasked>(acc_a, acc_b, Da, kk2, nb2, vcols - c * 32);
                    if (c + 1 < NCH) {
                        ptx::tmem_ld_wait();
                        if (c & 1)
                            ptx::reg_fence32(Da);
                        else
                            ptx::reg_fence32(Db);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&empty_m[ms]);
            float s0, s1, s2, s3;
            unpack2(acc_a, s0, s1);
            unpack2(acc_b, s2, s3);
            const float ts = (s0 + s1) + (s2 + s3);
            kahan_add(st.ksum, st.kc, ts);
            st.w32 = fmaf(ts, vw, st.w32);
            return true;
        };
        for (int64_t u = cta; u < total_units && ok; u += ncta) {
            // everything the tile loop needs is read once per unit, into registers
            const TcInst &I = *find_inst(insts, n_inst, u);
            const int64_t lu = u - I.unit_begin;
            const int64_t q_tiles = I.q_tiles, T = I.T;
            const int64_t split = lu / q_tiles, qt = lu - split * q_tiles;
            const int64_t t0 = split * I.tiles_per_split;
            const int64_t t1 = min(T, t0 + I.tiles_per_split);
            const float kk = I.scales[2];
            const uint64_t kk2 = pack2(kk, kk);
            const int ntiles = (int)(t1 - t0);
            // this warp's tiles of the unit: i0, i0 + STEP, ... (by CTA-wide tile parity)
            const uint32_t tbase = tcount;
            const int i0 = (int)(((uint32_t)(grp >> 1) - tbase) & (uint32_t)(STEP - 1));
            // real points among this warp's columns of the point set's last (padded) tile
            const int vlast = (int)max((int64_t)0, min((int64_t)WCOLS, I.n - (T - 1) * BN - col0));
            const bool mine_last = ntiles - 1 >= i0 && (ntiles - 1 - i0) % STEP == 0;
            const bool masked_end = t1 == T && vlast < WCOLS && mine_last;
            const int i_end = masked_end ? ntiles - 1 : ntiles;
            // the row's fixed shift: ceil of an upper bound on every exponent of the row
            st = RowState{ceilf(order_bits_to_float(I.ub[qt * BM + row])), 0.f, 0.f, 0.f};
            au = 0x1p-21f * I.unorm[qt * BM + row];
            for (int i = i0; i < i_end && ok; i += STEP) ok = visit(std::false_type{}, kk2, tbase + i, WCOLS);
            if (ok && masked_end) ok = visit(std::true_type{}, kk2, tbase + ntiles - 1, vlast);
            tcount = tbase + ntiles;
            if (!ok) {
                timed_out();
                break;
            }
            const double acc64 = (double)st.ksum - (double)st.kc;
            const double w64 = (double)st.w32;
            // merge the column groups of each row (groups 1.. hand their sums to group 0
            // through shared memory; group 0 adds them in group order), then store the
            // unit's partials
            if (grp > 0) {
                const bool got = ptx::mbar_wait_bounded(merge_empty, (ucount & 1) ^ 1, wait_ns, abort_flag);
                if (!__all_sync(0xffffffffu, got)) {
                    timed_out();
                    break;
                }
                msum[(grp - 1) * BM + row] = acc64;
                mw[(grp - 1) * BM + row] = w64;
                mshift[(grp - 1) * BM + row] = st.shift;
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(merge_full);
            } else {
                const bool got = ptx::mbar_wait_bounded(merge_full, ucount & 1, wait_ns, abort_flag);
                if (!__all_sync(0xffffffffu, got)) {
                    timed_out();
                    break;
                }
                float os[EG - 1];
                double oa[EG - 1], ow[EG - 1];
                float sm = st.shift;
#pragma unroll
                for (int g = 0; g < EG - 1; ++g) {
                    oa[g] = msum[g * BM + row];
                    ow[g] = mw[g * BM + row];
                    os[g] = mshift[g * BM + row];
                    sm = fmaxf(sm, os[g]);
                }
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(merge_empty);
                const int e0 = cexp(st.shift - sm);
                double tot = ldexp(acc64, e0), wt = ldexp(w64, e0);
#pragma unroll
                for (int g = 0; g < EG - 1; ++g) {
                    const int e = cexp(os[g] - sm);
                    tot += ldexp(oa[g], e);
                    wt += ldexp(ow[g], e);
                }
                const int64_t q = qt * BM + row;
                if (q < I.m) {
                    I.part_sum[split * I.m + q] = tot;
                    I.part_shift[split * I.m + q] = sm;
                    I.part_w[split * I.m + q] = wt;
                }
            }
            ++ucount;
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem_base, C::TMEM_COLS);
    }
}

template <int KP, int BN, int SB, int SMETA, int AB, int EG>
__global__ void __launch_bounds__(64 + 128 * EG, 1) __maxnreg__(EG >= 4 ? 112 : 200)
kde_tc_kernel(const __grid_constant__ TcInst inst0, const TcInst *__restrict__ table, int n_inst,
              int64_t total_units, int *err, uint64_t wait_ns, uint64_t stall_ns) {
    tc_body<KP, BN, SB, SMETA, AB, EG>(table ? table : &inst0, table == nullptr, n_inst, total_units, err, wait_ns,
                                       stall_ns, blockIdx.x, gridDim.x);
}

// Every operand width in one persistent launch (the batched path): the CTAs are split
// into one contiguous range per width, sized by the width's share of the work; a range
// serves its width's table of instances like a launch of its own.
struct TcMulti {
    const TcInst *table[4];  // widths 16, 32, 64, 128 (device tables; unused where n_inst = 0)
    int n_inst[4];
    int64_t units[4];
    int cta_begin[5];        // CTA range of width c: [cta_begin[c], cta_begin[c + 1])
};

template <int EG>
__global__ void __launch_bounds__(64 + 128 * EG, 1) __maxnreg__(EG >= 4 ? 112 : 200)
kde_tc_multi_kernel(const __grid_constant__ TcMulti mp, int *err, uint64_t wait_ns, uint64_t stall_ns) {
    const int b = blockIdx.x;
    if (b < mp.cta_begin[1])
        tc_body<16, 256, 4, 8, 2, EG>(mp.table[0], false, mp.n_inst[0], mp.units[0], err, wait_ns, stall_ns,
                                      b - mp.cta_begin[0], mp.cta_begin[1] - mp.cta_begin[0]);
    else if (b < mp.cta_begin[2])
        tc_body<32, 256, 4, 8, 2, EG>(mp.table[1], false, mp.n_inst[1], mp.units[1], err, wait_ns, stall_ns,
                                      b - mp.cta_begin[1], mp.cta_begin[2] - mp.cta_begin[1]);
    else if (b < mp.cta_begin[3])
        tc_body<64, 256, 2, 8, 1, EG>(mp.table[2], false, mp.n_inst[2], mp.units[2], err, wait_ns, stall_ns,
                                      b - mp.cta_begin[2], mp.cta_begin[3] - mp.cta_begin[2]);
    else if (b < mp.cta_begin[4])
        tc_body<128, 128, 2, 8, 1, EG>(mp.table[3], false, mp.n_inst[3], mp.units[3], err, wait_ns, stall_ns,
                                       b - mp.cta_begin[3], mp.cta_begin[4] - mp.cta_begin[3]);
}

// ------------------------------------------------------------------ prep kernels
// The tile centres coordinate-major, centT[k][t] = cent[t][k] (the row-term kernel reads
// 64 tiles' coordinate k with one coalesced load).
__global__ void tc_transpose_centres_kernel(const float *__restrict__ cent, int64_t T, int Kp,
                                            float *__restrict__ centT) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < T * Kp; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i / T, t = i % T;
        centT[i] = cent[t * Kp + k];
    }
}

// Per-tile FP64 coordinate sums and FP32 centres (mean of the tile's real points).
__global__ void tc_centres_kernel(const float *__restrict__ X, int64_t n, int64_t d, int BN, int Kp,
                                  double *__restrict__ tsum, float *__restrict__ cent) {
    const int64_t t = blockIdx.x;
    const int64_t r0 = t * BN;
    const int64_t cnt = min((int64_t)BN, n - r0);
    for (int k = threadIdx.x; k < Kp; k += blockDim.x) {
        double s = 0.0;
        if (k < d)
            for (int64_t r = 0; r < cnt; ++r) s += (double)X[(r0 + r) * d + k];
        tsum[t * Kp + k] = s;
        cent[t * Kp + k] = (k < d && cnt > 0) ? (float)(s / (double)cnt) : 0.f;
    }
}

// Global centre c_g = (sum over tiles of the tile sums) / n, in FP64, fixed order.
__global__ void tc_global_centre_kernel(const double *__restrict__ tsum, int64_t T, int Kp, int64_t n, int64_t d,
                                        float *__restrict__ cg) {
    for (int k = threadIdx.x; k < Kp; k += blockDim.x) {
        double s = 0.0;
        for (int64_t t = 0; t < T; ++t) s += tsum[t * Kp + k];
        cg[k] = k < d ? (float)(s / (double)n) : 0.f;
    }
}

__device__ __forceinline__ void atomic_max_pos(unsigned *bits, float v) {
    atomicMax(bits, __float_as_uint(fabsf(v)));
}

// max over points and coordinates of |x_k - c_k|, with c = the point's tile centre
// (per_tile = true) or the global centre
__global__ void tc_maxabs_kernel(const float *__restrict__ X, int64_t n, int64_t d, int BN, int Kp,
                                 const float *__restrict__ cent, const float *__restrict__ cg, bool per_tile,
                                 unsigned *out) {
    float mx = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * d; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / d, k = i % d;
        const float c = per_tile ? cent[(r / BN) * Kp + k] : cg[k];
        mx = fmaxf(mx, fabsf(X[i] - c));
    }
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomic_max_pos(out, mx);
}

__device__ __forceinline__ double pow2_at_or_above(double x) {
    int e;
    frexp(x, &e);  // x in [2^(e-1), 2^e)
    return ldexp(1.0, e);
}

// Power-of-two scales of the split (one thread):
//   scale_v: max |v_k| * scale_v < 2^10          (v = x - c_t)
//   scale_u: max |x_k - c_g| * scale_u < 2^9    (queries up to 64x farther still fit FP16)
//   kk = 2c / (scale_u scale_v)
//   s_a: the point-term pieces g * scale_u * scale_v / (2 s_a) stay below 2^14, using
//        |g| <= d vmax^2 + 2 d xmax vmax; for d <= 128 this keeps s_a <= 2^13
// and the constant A column [s_a, s_a, s_a, 0, ...] of every query row. FP16 keeps 11
// significant bits at any magnitude, so the modest ranges cost no precision and leave
// room for the u . v sums and the point term in the same FP32 accumulator.
__global__ void tc_scales_kernel(const unsigned *__restrict__ vmax, const unsigned *__restrict__ xmax, int64_t d,
                                 double c, float *__restrict__ scales, __half *__restrict__ a_aug) {
    __shared__ float sa_sh;
    if (threadIdx.x == 0) {
        const double vm = (double)__uint_as_float(*vmax), xm = (double)__uint_as_float(*xmax);
        const double sv = vm > 0.0 && isfinite(vm) ? 0x1p10 / pow2_at_or_above(vm) : 1.0;
        const double su = xm > 0.0 && isfinite(xm) ? 0x1p9 / pow2_at_or_above(xm) : 1.0;
        const double gmax = (double)d * vm * vm + 2.0 * (double)d * xm * vm;
        double sa = gmax > 0.0 ? pow2_at_or_above(gmax * su * sv * 0.5) * 0x1p-14 : 1.0;
        sa = fmin(fmax(sa, 0x1p-14), 0x1p15);
        scales[0] = (float)sv;
        scales[1] = (float)su;
        scales[2] = (float)(2.0 * c / (su * sv));
        scales[3] = (float)sa;
        sa_sh = (float)sa;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < BM * 16; i += blockDim.x) a_aug[i] = __float2half_rn((i % 16) < 3 ? sa_sh : 0.f);
}

// Splits x - c_t into FP16 hi/lo (scaled by scale_v) and the point term
// g = |v~|^2 + 2 D_t . v~ (FP64, from the represented v~ = (hi + lo) / scale_v) into three
// FP16 pieces of -g * scale_u * scale_v / (2 s_a). Padding points are all zero (the
// epilogue masks them).
__global__ void tc_split_points_kernel(const float *__restrict__ X, int64_t n, int64_t d, int BN, int Kp, int64_t n_pad,
                                       const float *__restrict__ cent, const float *__restrict__ cg,
                                       const float *__restrict__ scales, __half *__restrict__ bhi,
                                       __half *__restrict__ blo, __half *__restrict__ baug) {
    const double sv = scales[0], su = scales[1], sa = scales[3];
    const double inv = 1.0 / sv;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_pad; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / BN;
        double nv2 = 0.0, dv = 0.0;
        for (int k = 0; k < Kp; ++k) {
            __half h = __float2half_rn(0.f), l = __float2half_rn(0.f);
            if (i < n && k < d) {
                const float ct = cent[t * Kp + k];
                const double v = ((double)X[i * d + k] - (double)ct) * sv;
                h = __double2half(v);
                l = __double2half(v - (double)__half2float(h));
                const double vr = ((double)__half2float(h) + (double)__half2float(l)) * inv;
                nv2 += vr * vr;
                dv += ((double)ct - (double)cg[k]) * vr;
            }
            bhi[i * Kp + k] = h;
            blo[i * Kp + k] = l;
        }
        double y = i < n ? -(nv2 + 2.0 * dv) * su * sv / (2.0 * sa) : 0.0;
        for (int k = 0; k < 16; ++k) {
            __half pc = __float2half_rn(0.f);
            if (k < 3) {
                pc = __double2half(y);
                y -= (double)__half2float(pc);
            }
            baug[i * 16 + k] = pc;
        }
    }
}

// Per tile: the RMS and the largest distance of its points from the tile centre (the
// per-query error estimate and the exponent bounds).
__global__ void tc_tile_radius_kernel(const float *__restrict__ X, int64_t n, int64_t d, int BN, int Kp,
                                      const float *__restrict__ cent, float *__restrict__ tinfo) {
    __shared__ double red[128];
    __shared__ double redm[128];
    const int64_t t = blockIdx.x;
    const int64_t r0 = t * BN, cnt = min((int64_t)BN, n - r0);
    double acc = 0.0, mx = 0.0;
    for (int64_t r = threadIdx.x; r < cnt; r += blockDim.x) {
        double s2 = 0.0;
        for (int64_t k = 0; k < d; ++k) {
            const double v = (double)X[(r0 + r) * d + k] - (double)cent[t * Kp + k];
            s2 += v * v;
        }
        acc += s2;
        mx = fmax(mx, s2);
    }
    red[threadIdx.x] = acc;
    redm[threadIdx.x] = mx;
    __syncthreads();
    for (int o = 64; o; o >>= 1) {
        if (threadIdx.x < o) {
            red[threadIdx.x] += red[threadIdx.x + o];
            redm[threadIdx.x] = fmax(redm[threadIdx.x], redm[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // RMS radius: the error estimate's split term (the typical |v| of the tile)
        tinfo[t * 4 + 0] = cnt > 0 ? (float)sqrt(red[0] / (double)cnt) : 0.f;
        // max radius, rounded up so that it bounds the FP32 distances too
        tinfo[t * 4 + 1] = cnt > 0 ? (float)(sqrt(redm[0]) * (1.0 + 1e-6)) : 0.f;
        tinfo[t * 4 + 2] = cnt > 0 ? (float)sqrt(redm[0]) : 0.f;  // max radius
        // the estimate's accumulation term: for a point near the query the FP32 accumulator
        // carries about ||v||^2 + D_t . v before the point term cancels it, so its rounding
        // error grows with the tile's largest ||v||^2 (large for a tile holding a few points
        // of another cluster): 2^-23 sqrt(MMA steps) rho^2
        const double steps = 3.0 * Kp / 16.0 + 1.0;
        tinfo[t * 4 + 3] = cnt > 0 ? (float)(0x1p-23 * sqrt(steps) * redm[0]) : 0.f;
    }
}

// R[t][q] = c * ||q - c_t||^2 by direct differences in FP32 (padding queries: 0), the
// per-query upper bound on every exponent, and ||q - c_g||. The first column of blocks
// also writes the query's scaled, centred coordinates u = (q - c_g) * scale_u as FP16
// hi/lo pairs (the MMA's A operand; the difference and scale in FP64, u_lo = u - u_hi)
// and flags, in qbad, a query farther from the data than that range (its row is zeroed and
// the combine hands it to the plain FP32 form).
// Register tiling: a block takes 128 queries and walks its range of point tiles 64 at a
// time; a thread computes 8 queries (four packed pairs) x 4 tiles. The block's queries are
// staged once, transposed ([k][query], dynamic shared memory); the centres of a chunk come
// 16 coordinates at a time from their coordinate-major copy (coalesced), each stored twice
// (c, c) so that one 64-bit operand serves a packed query pair. Per coordinate a thread
// reads its queries' values and its four centres (four 16-byte loads) and spends 16 packed
// subtractions and 16 packed FMAs: eight operations per shared-memory load. The sums run
// in blocks of 16 coordinates (a fresh chain per block, added to the total), like the
// plain form. Lane l of warp w: queries 32 (w % 4) + 8 (l % 4) .. +8, tiles 32 (w / 4) +
// 4 (l / 4) .. +4 of the chunk, so a warp's query loads touch 128 bytes and its centre
// loads 128 bytes (one wavefront each).
struct RowTermGeo {
    static constexpr int THREADS = 256;
    static constexpr int TG = 64;       // tiles per chunk
    static constexpr int KC = 16;       // coordinates per staged block of centres
    static constexpr int QS = 128 + 4;  // row stride of the transposed queries (floats)
    static constexpr int smem_bytes(int kp) { return kp * QS * 4; }
};

template <int KP>
__global__ void __launch_bounds__(RowTermGeo::THREADS, KP <= 16 ? 3 : 2)
tc_rowterm_kernel(const float *__restrict__ Q, int64_t m, int64_t d, int64_t m_pad, const float *__restrict__ cent,
                  int64_t T, int tiles_per_block, float c, float *__restrict__ R, const float *__restrict__ cg,
                  float *__restrict__ unorm, const float *__restrict__ tinfo, unsigned *__restrict__ ub,
                  const float *__restrict__ scales, __half *__restrict__ ahi, __half *__restrict__ alo,
                  int *__restrict__ qbad, const float *__restrict__ centT) {
    using RG = RowTermGeo;
    constexpr int TG = RG::TG, KC = RG::KC, QS = RG::QS;
    extern __shared__ __align__(16) float sq[];              // [KP][QS]: the block's queries
    __shared__ __align__(16) uint64_t sc[KC * TG];           // [k][tile slot]: (c, c)
    __shared__ float srad[TG];
    const int64_t q0 = (int64_t)blockIdx.x * 128;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (blockIdx.y == 0) {
        // ||q - c_g|| and the A operand: FP16 hi/lo splits of u, zero for padding rows and
        // coordinates, stored eight coordinates (16 bytes) at a time; two threads per query
        const int r = tid >> 1, part = tid & 1;
        const int64_t q = q0 + r;
        const bool real = q < m;
        const int k0 = part * (KP / 2);
        const double su = scales[1];
        float s2 = 0.f;
        int bad = 0;
        uint4 *dh = reinterpret_cast<uint4 *>(ahi + q * KP + k0);
        uint4 *dl = reinterpret_cast<uint4 *>(alo + q * KP + k0);
#pragma unroll 1
        for (int k8 = 0; k8 < KP / 16; ++k8) {
            __align__(16) __half hv[8], lv[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = k0 + k8 * 8 + j;
                __half hh = __float2half_rn(0.f), ll = __float2half_rn(0.f);
                if (real && k < d) {
                    const float qk = Q[q * d + k];
                    const float df = qk - cg[k];
                    s2 = fmaf(df, df, s2);
                    const double u = ((double)qk - (double)cg[k]) * su;
                    if (fabs(u) < 0x1p15) {
                        hh = __float2half_rn((float)u);
                        ll = __float2half_rn((float)(u - (double)__half2float(hh)));
                    } else {
                        bad = 1;
                    }
                }
                hv[j] = hh;
                lv[j] = ll;
            }
            dh[k8] = *reinterpret_cast<const uint4 *>(hv);
            dl[k8] = *reinterpret_cast<const uint4 *>(lv);
        }
        s2 += __shfl_xor_sync(0xffffffffu, s2, 1);
        bad |= __shfl_xor_sync(0xffffffffu, bad, 1);
        if (part == 0) {
            unorm[q] = real ? sqrtf(s2) : 0.f;
            if (bad) qbad[q] = 1;
        }
    }
    const int wq = warp & 3, wt = warp >> 2, lq = lane & 3, lt = lane >> 2;
    const int qo = wq * 32 + lq * 8;  // first of the thread's 8 queries (block-relative)
    const int to = wt * 32 + lt * 4;  // first of its 4 tiles (chunk-relative)
    // centre slots: the pairs (to, to+1) of a warp's lanes side by side, then (to+2, to+3)
    const int cs0 = wt * 32 + lt * 2, cs1 = cs0 + 16;
    const int64_t ta = (int64_t)blockIdx.y * tiles_per_block;
    const int64_t tb = min(T, ta + tiles_per_block);
    // upper bound on the exponent -c ||q - x||^2 over the tiles of this block: every x of
    // tile t lies within the tile's max radius rho_t of c_t, so
    //     -c ||q - x||^2 <= -( max(0, sqrt(c R') - sqrt(c) rho_t) )^2,  R' = ||q - c_t||^2
    const float sqc = sqrtf(c);
    float ubest[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) ubest[i] = -INFINITY;
    // the block's queries, transposed (rows read coordinate-fast; padding: 0)
    for (int e = tid; e < KP * 128; e += RG::THREADS) {
        const int r = e / KP, k = e % KP;
        const int64_t q = q0 + r;
        sq[k * QS + r] = (q < m && k < d) ? Q[q * d + k] : 0.f;
    }
    // Stages: (chunk of 64 tiles, block of 16 coordinates). The centres (and, at a chunk's
    // first block, the tiles' radii) of the next stage are loaded into registers while the
    // current stage is computed, so the global-memory latency hides behind the math.
    constexpr int NKB = KP / KC, PER = KC * TG / RG::THREADS;  // values a thread stages
    const int nstages = (int)ceil_div_dev(tb - ta, (int64_t)TG) * NKB;
    float pv[PER], prad = 0.f;
    auto load_stage = [&](int st) {
        const int64_t g0 = ta + (int64_t)(st / NKB) * TG;
        const int kb = (st % NKB) * KC;
        const int gn = (int)min((int64_t)TG, tb - g0);
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int e = tid + i * RG::THREADS;
            const int j = e % TG, k = e / TG;  // tile j of the chunk, coordinate kb + k
            pv[i] = j < gn ? centT[(int64_t)(kb + k) * T + g0 + j] : 0.f;
        }
        prad = (kb == 0 && tid < gn) ? tinfo[(g0 + tid) * 4 + 1] : 0.f;
    };
    if (nstages > 0) load_stage(0);
    uint64_t tot[4][4];  // [tile][query pair], packed (query 2p, 2p+1)
#pragma unroll 1
    for (int st = 0; st < nstages; ++st) {
        const int64_t g0 = ta + (int64_t)(st / NKB) * TG;
        const int kb = (st % NKB) * KC;
        const int gn = (int)min((int64_t)TG, tb - g0);
        __syncthreads();  // the previous stage's centres (and radii) have been read
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int e = tid + i * RG::THREADS;
            const int j = e % TG, k = e / TG;
            const int jw = j >> 5, jj = j & 31;
            const int slot = jw * 32 + ((jj & 3) >> 1) * 16 + (jj >> 2) * 2 + (jj & 1);
            sc[k * TG + slot] = f2::pack(pv[i], pv[i]);
        }
        if (kb == 0 && tid < TG) srad[tid] = prad;
        __syncthreads();
        if (st + 1 < nstages) load_stage(st + 1);
        if (to >= gn) continue;  // all four of this thread's tiles lie past the range's end
        uint64_t acc[4][4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int p = 0; p < 4; ++p) acc[j][p] = 0;
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const ulonglong2 qa = *reinterpret_cast<const ulonglong2 *>(&sq[(kb + k) * QS + qo]);
            const ulonglong2 qb = *reinterpret_cast<const ulonglong2 *>(&sq[(kb + k) * QS + qo + 4]);
            const ulonglong2 ca = *reinterpret_cast<const ulonglong2 *>(&sc[k * TG + cs0]);
            const ulonglong2 cb = *reinterpret_cast<const ulonglong2 *>(&sc[k * TG + cs1]);
            const uint64_t qv[4] = {qa.x, qa.y, qb.x, qb.y};
            const uint64_t cv[4] = {ca.x, ca.y, cb.x, cb.y};
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const uint64_t df = f2::sub(qv[p], cv[j]);
                    acc[j][p] = f2::fma(df, df, acc[j][p]);
                }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int p = 0; p < 4; ++p) tot[j][p] = kb == 0 ? acc[j][p] : f2::add(tot[j][p], acc[j][p]);
        if (kb + KC < KP) continue;
        // the chunk's row terms (padding queries: 0) and the bounds
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int jt = to + j;
            if (jt >= gn) continue;
            float rv[8];
#pragma unroll
            for (int p = 0; p < 4; ++p) f2::unpack(tot[j][p], rv[2 * p], rv[2 * p + 1]);
            const float rr = sqc * srad[jt];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                rv[i] = q0 + qo + i < m ? c * rv[i] : 0.f;
                // slack of 1e-5 relative (far above the approximate square root's ~2^-22
                // error and the FP32 rounding of the exponents) so that the bound holds
                const float g = fmaxf(0.f, ptx::sqrt_approx(rv[i]) * (1.f - 1e-5f) - rr);
                ubest[i] = fmaxf(ubest[i], -g * g);
            }
            float4 *dst = reinterpret_cast<float4 *>(R + (g0 + jt) * m_pad + q0 + qo);
            dst[0] = make_float4(rv[0], rv[1], rv[2], rv[3]);
            dst[1] = make_float4(rv[4], rv[5], rv[6], rv[7]);
        }
    }
    // the lanes holding the same queries (lane bits 2..4) combine their bounds
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        ubest[i] = fmaxf(ubest[i], __shfl_xor_sync(0xffffffffu, ubest[i], 4));
        ubest[i] = fmaxf(ubest[i], __shfl_xor_sync(0xffffffffu, ubest[i], 8));
        ubest[i] = fmaxf(ubest[i], __shfl_xor_sync(0xffffffffu, ubest[i], 16));
    }
    if (tb > ta && lt == 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t q = q0 + qo + i;
            atomicMax(ub + q, float_order_bits(q < m ? ubest[i] : 0.f));
        }
    }
}

// FP32 recompute of the queries the tensor-core estimate flags, over the tiles that can
// matter only. Per query, from the row terms R_t = c ||q - c_t||^2 and the tiles' max
// radii rho_t (c = a log2 e, exponents in log2 units):
//     ub_t = -(max(0, sqrt(R_t) - sqrt(c) rho_t))^2  >= every exponent -c ||q - x||^2 in tile t
//     lb_t = -(sqrt(R_t) + sqrt(c) rho_t)^2          <= the largest exponent in tile t
// (with a 1e-5 relative slack on sqrt(R_t) for rounding), so LB = max_t lb_t bounds the
// row's largest term from below, and a tile with ub_t < LB - 64 holds only terms below
// 2^-64 of it: all of them together change the sum by less than n 2^-64 relative, and
// the tile is skipped. The others are evaluated like the plain FP32 form.
constexpr float kPruneLog2 = 64.f;

// ---------------------------------------------------------------- grouped recompute
// The flagged queries are recomputed in groups of 64 so that every point load serves 64
// queries (the plain form's register-tiled kernel), while the tiles that cannot matter
// are still skipped:
//   (1) the combine kernel flags queries and counts them per block; a scan and an ordered
//       compaction list the flagged queries in query order, each with the bound LB of its
//       largest exponent, its threshold LB - 64 and, as sort key, the tile holding LB;
//   (2) a stable sort by that tile (k-d order: queries near the same points become
//       neighbours; stable on an ordered input, so the groups are deterministic; it visits
//       only the flagged entries) and the gather of the sorted queries, 64 per group;
//   (3) per group, the union of its members' kept tiles (ub_t >= threshold for at least
//       one member);
//   (4) the list kernel (kde_simt.cu) over each group's kept tiles, in segments of `seg`
//       tiles;
//   (5) per query, the FP64 combine of its group's segments.
// A member evaluates the other members' tiles too: more terms than its own bound needs,
// never fewer.
// Exclusive prefix sum (one block): off[0..n] from in[0..n), n = *n_dev if given, else
// the flagged queries' group count ceil(*cnt_dev / 64) if given, else n_host; the total
// also goes to *total_out if given.
__global__ void __launch_bounds__(1024)
tc_scan_kernel(const int *__restrict__ in, const int *__restrict__ cnt_dev, int n_host, int *__restrict__ off,
               int *__restrict__ total_out) {
    __shared__ int sdata[1024];
    __shared__ int carry;
    const int n = cnt_dev ? (*cnt_dev + 63) / 64 : n_host;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 1024) {
        const int i = base + threadIdx.x;
        sdata[threadIdx.x] = i < n ? in[i] : 0;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int v = threadIdx.x >= o ? sdata[threadIdx.x - o] : 0;
            __syncthreads();
            sdata[threadIdx.x] += v;
            __syncthreads();
        }
        if (i < n) off[i + 1] = carry + sdata[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 1023) carry += sdata[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        off[0] = 0;
        if (total_out) *total_out = carry;
    }
}

// The flagged queries in query order (block b's flagged queries start at boff[b]; inside
// a block, by warp, then lane), each with the tile holding the lower bound LB of its
// largest exponent as sort key, and its threshold LB - 64.
__global__ void __launch_bounds__(256)
tc_flag_compact_kernel(const int *__restrict__ qflag, const int *__restrict__ boff, int64_t m, int64_t m_pad,
                       const float *__restrict__ R, const float *__restrict__ tinfo, int64_t T, float c,
                       int *__restrict__ fix_idx, uint64_t *__restrict__ key, uint32_t *__restrict__ val,
                       float *__restrict__ thr) {
    __shared__ int wcnt[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool flag = j < m && qflag[j];
    const unsigned mask = __ballot_sync(0xffffffffu, flag);
    if (lane == 0) wcnt[warp] = __popc(mask);
    __syncthreads();
    if (!mask) return;
    int w0 = boff[blockIdx.x];
    for (int k = 0; k < warp; ++k) w0 += wcnt[k];
    const float sqc = sqrtf(c);
    if (__popc(mask) >= 8) {
        // many flagged queries in the warp: each lane walks the tiles of its own query
        // (eight row terms in flight; the loads of the warp's queries coalesce)
        if (flag) {
            float best = -INFINITY;
            int bt = 0;
            constexpr int U = 8;
            for (int t0 = 0; t0 < (int)T; t0 += U) {
                float rv[U], rho[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int t = min(t0 + u, (int)T - 1);
                    rv[u] = R[(int64_t)t * m_pad + j];
                    rho[u] = tinfo[(int64_t)t * 4 + 1];
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const float h2 = sqrtf(rv[u]) * (1.f + 1e-5f) + sqc * rho[u];
                    const float lb = -h2 * h2;
                    if (t0 + u < (int)T && lb > best) {  // ties keep the smaller tile
                        best = lb;
                        bt = t0 + u;
                    }
                }
            }
            const int w = w0 + __popc(mask & ((1u << lane) - 1u));
            fix_idx[w] = (int)j;
            key[w] = (uint64_t)bt;
            val[w] = (uint32_t)j;
            thr[j] = best - kPruneLog2;
        }
        return;
    }
    // few: the warp takes its flagged queries one at a time, its lanes striding over the
    // tiles (four row terms in flight per lane), then a warp arg-max (ties keep the
    // smaller tile)
    unsigned rem = mask;
    while (rem) {
        const int src = __ffs(rem) - 1;
        rem &= rem - 1u;
        const int64_t jq = blockIdx.x * (int64_t)blockDim.x + warp * 32 + src;
        float best = -INFINITY;
        int bt = INT_MAX;
        for (int t0 = lane; t0 < (int)T; t0 += 4 * 32) {
            float rv[4], rho[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = min(t0 + 32 * u, (int)T - 1);
                rv[u] = R[(int64_t)t * m_pad + jq];
                rho[u] = tinfo[(int64_t)t * 4 + 1];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float h2 = sqrtf(rv[u]) * (1.f + 1e-5f) + sqc * rho[u];
                const float lb = -h2 * h2;
                if (t0 + 32 * u < (int)T && lb > best) {  // a lane's tiles ascend
                    best = lb;
                    bt = t0 + 32 * u;
                }
            }
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, off);
            const int ot = __shfl_xor_sync(0xffffffffu, bt, off);
            if (ob > best || (ob == best && ot < bt)) {
                best = ob;
                bt = ot;
            }
        }
        if (lane == src) {
            const int w = w0 + __popc(mask & ((1u << src) - 1u));
            fix_idx[w] = (int)jq;
            key[w] = (uint64_t)bt;
            val[w] = (uint32_t)jq;
            thr[jq] = best - kPruneLog2;
        }
    }
}

// Per group (one block of 256 threads, grid-stride): the tiles some member may need, in
// increasing order, into kept[g * T ..]; their number and the group's segment count.
__global__ void __launch_bounds__(256)
tc_group_keep_kernel(const uint32_t *__restrict__ order, const float *__restrict__ thr,
                     const int *__restrict__ fix_count, int *__restrict__ n_groups, int64_t m_pad,
                     const float *__restrict__ R, const float *__restrict__ tinfo, int64_t T, float c, int seg,
                     int *__restrict__ kept, int *__restrict__ kcount, int *__restrict__ items) {
    __shared__ int sq[64];
    __shared__ float sthr[64];
    __shared__ int wcnt[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cnt = *fix_count, G = (cnt + 63) / 64;
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_groups = G;
    const float sqc = sqrtf(c);
    for (int g = blockIdx.x; g < G; g += gridDim.x) {
        const int rows = min(64, cnt - g * 64);
        __syncthreads();
        if (threadIdx.x < rows) {
            const int q = (int)order[g * 64 + threadIdx.x];
            sq[threadIdx.x] = q;
            sthr[threadIdx.x] = thr[q];
        }
        __syncthreads();
        int base = 0;
        for (int64_t t0 = 0; t0 < T; t0 += 256) {
            const int64_t t = t0 + threadIdx.x;
            bool keep = false;
            if (t < T) {
                const float rho = sqc * tinfo[t * 4 + 1];
                // eight members' row terms in flight at a time
                for (int r0 = 0; r0 < rows && !keep; r0 += 8) {
                    float rv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) rv[u] = R[t * m_pad + sq[min(r0 + u, rows - 1)]];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const float gap = fmaxf(0.f, sqrtf(rv[u]) * (1.f - 1e-5f) - rho);
                        keep = keep || (r0 + u < rows && -gap * gap >= sthr[r0 + u]);
                    }
                }
            }
            const unsigned mask = __ballot_sync(0xffffffffu, keep);
            if (lane == 0) wcnt[warp] = __popc(mask);
            __syncthreads();
            int off = base;
            for (int w = 0; w < warp; ++w) off += wcnt[w];
            if (keep) kept[(int64_t)g * T + off + __popc(mask & ((1u << lane) - 1u))] = (int)t;
            for (int w = 0; w < 8; ++w) base += wcnt[w];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            kcount[g] = base;
            items[g] = (base + seg - 1) / seg;
        }
    }
}

// Per flagged query (sorted position j): the FP64 sum of its group's segment partials.
__global__ void tc_group_combine_kernel(const double *__restrict__ part_sum, const float *__restrict__ part_shift,
                                        const int *__restrict__ item_off, const uint32_t *__restrict__ order,
                                        const int *__restrict__ fix_count, double scale, double *__restrict__ out) {
    const int cnt = *fix_count;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cnt; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = j / 64, r = j % 64;
        const int w0 = item_off[g], w1 = item_off[g + 1];
        float smax = -INFINITY;
        for (int w = w0; w < w1; ++w) smax = fmaxf(smax, part_shift[(int64_t)w * 64 + r]);
        double tot = 0.0;
        for (int w = w0; w < w1; ++w) tot += ldexp(part_sum[(int64_t)w * 64 + r], cexp(part_shift[(int64_t)w * 64 + r] - smax));
        out[order[j]] = w1 > w0 ? ldexp(tot, cexp(smax)) * scale : 0.0;
    }
}

// FP64 combine of the per-split partials (as kde_combine.cu) plus the per-query error
// estimate of the tensor-core form,
//     est = a * (sum_t S_t w_t) / (sum_t S_t),   w_t = max(2^-21 ||q - c_g|| r_t, beta rho_t^2),
// S_t the query's sum over tile t, r_t that tile's RMS radius, rho_t its largest radius
// and beta = 2^-23 sqrt(MMA steps). The first term (the split products' error grows with
// ||q - c_g|| |x - c_t|) was calibrated on the whole arithmetic over spatially coherent
// tiles, so it covers their FP32 accumulation error too; the second takes over where the
// accumulation error of a tile's outlying points (it grows with ||x - c_t||^2; see
// tc_tile_radius) exceeds it. The epilogue accumulates sum_t S_t w_t. Queries with
// est > thr (or an empty sum) are appended to fix_idx for the plain FP32 form.
__global__ void __launch_bounds__(256)
tc_combine_kernel(const double *__restrict__ part_sum, const float *__restrict__ part_shift,
                  const double *__restrict__ part_w, int64_t m, int splits, double scale, const int *__restrict__ qbad,
                  double a, double thr, double *__restrict__ out, int *__restrict__ qflag, int *__restrict__ bcnt) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // one query per thread
    bool flag = false;
    if (j < m) {
        float smax = -INFINITY;
        for (int k = 0; k < splits; ++k) smax = fmaxf(smax, part_shift[(int64_t)k * m + j]);
        double tot = 0.0, wt = 0.0;
        for (int k = 0; k < splits; ++k) {
            const int e = cexp(part_shift[(int64_t)k * m + j] - smax);
            tot += ldexp(part_sum[(int64_t)k * m + j], e);
            wt += ldexp(part_w[(int64_t)k * m + j], e);
        }
        out[j] = ldexp(tot, cexp(smax)) * scale;
        // tot is in units of 2^smax, a bound on every term: below 2^-40 the bound was too
        // loose for the fixed shift (terms under 2^-126 of it were flushed)
        const double est = (tot >= 0x1p-40 && !qbad[j]) ? a * (wt / tot) : INFINITY;
        flag = est > thr && qflag;
        if (qflag) qflag[j] = flag ? 1 : 0;
    }
    const int c = __syncthreads_count(flag);
    if (bcnt && threadIdx.x == 0) bcnt[blockIdx.x] = c;
}

// ------------------------------------------------------------------ host helpers
typedef CUresult (*PFN_encodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                    const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

PFN_encodeTiled get_encode() {
    static PFN_encodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_encodeTiled>(p);
    });
    return fn;
}

// 2-D FP16 tensor map over a [rows][width] plane with box {min(width,64), box_rows}.
int make_map(CUtensorMap *map, void *base, int64_t rows, int width, int box_rows) {
    PFN_encodeTiled enc = get_encode();
    if (!enc) return fail(STAG_KDE_ECUDA, "cuTensorMapEncodeTiled unavailable");
    const int cw = width < 64 ? width : 64;
    cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)width * 2};
    cuuint32_t box[2] = {(cuuint32_t)cw, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    const CUtensorMapSwizzle sw = cw == 16 ? CU_TENSOR_MAP_SWIZZLE_32B
                                           : (cw == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B);
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(STAG_KDE_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return 0;
}

// Test hook: STAG_KDE_INJECT_PRODUCER_STALL_NS (at most 1 s) delays the start of the
// tensor-core kernel's TMA producer, so that the other warps' bounded waits expire.
uint64_t injected_stall_ns() {
    const char *v = getenv("STAG_KDE_INJECT_PRODUCER_STALL_NS");
    if (!v) return 0;
    const long long ns = atoll(v);
    return ns <= 0 ? 0 : (uint64_t)std::min(ns, 1000000000ll);
}

int kp_for(int64_t d) {
    if (d <= 16) return 16;
    if (d <= 32) return 32;
    if (d <= 64) return 64;
    if (d <= 128) return 128;
    return 0;
}

int bn_for(int Kp) { return Kp >= 128 ? 128 : 256; }

int grid_for(int64_t total, int threads) { return (int)std::min<int64_t>(ceil_div(total, threads), 152 * 16); }

template <int KP, int BN, int SB, int SMETA, int AB, int EG>
int launch_tc(const TcInst &inst0, const TcInst *table, int n_inst, int64_t total_units, int *err, int sm_count,
              uint64_t wait_ns, cudaStream_t s) {
    const uint64_t stall_ns = injected_stall_ns();
    using C = Cfg<KP, BN, SB, SMETA, AB, EG>;
    auto kern = kde_tc_kernel<KP, BN, SB, SMETA, AB, EG>;
    static_assert(C::SMEM <= 232448, "shared memory budget");
    // at least 116 KB so that no two CTAs share an SM (each holds up to 512 TMEM columns)
    const int smem = std::max(C::SMEM, 118 * 1024);
    // set once per instantiation (before any stream capture can be in progress)
    static cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    STAG_CUDA_TRY(attr);
    const int grid = (int)std::min<int64_t>(total_units, sm_count);
    count_launch();
    kern<<<grid, C::THREADS, smem, s>>>(inst0, table, n_inst, total_units, err, wait_ns, stall_ns);
    STAG_CUDA_TRY(cudaGetLastError());
    return 0;
}

// Dispatch on the operand width and the number of epilogue warp groups.
int launch_tc_any(int Kp, int eg, const TcInst &inst0, const TcInst *table, int n_inst, int64_t total_units,
                  int *err, int sm_count, uint64_t wait_ns, cudaStream_t s) {
    switch (Kp * 10 + eg) {
        case 162: return launch_tc<16, 256, 4, 8, 2, 2>(inst0, table, n_inst, total_units, err, sm_count, wait_ns, s);
        case 164: return launch_tc<16, 256, 4, 8, 2, 4>(inst0, table, n_inst, total_units, err, sm_count, wait_ns, s);
        case 322: return launch_tc<32, 256, 4, 8, 2, 2>(inst0, table, n_inst, total_units, err, sm_count, wait_ns, s);
        case 324: return launch_tc<32, 256, 4, 8, 2, 4>(inst0, table, n_inst, total_units, err, sm_count, wait_ns, s);
        case 642: return launch_tc<64, 256, 2, 8, 1, 2>(inst0, table, n_inst, total_units, err, sm_count, wait_ns, s);
        case 644: return launch_tc<64, 256, 2, 8, 1, 4>(inst0, table, n_inst, total_units, err, sm_count, wait_ns, s);
        case 1282: return launch_tc<128, 128, 2, 8, 1, 2>(inst0, table, n_inst, total_units, err, sm_count, wait_ns, s);
        case 1284: return launch_tc<128, 128, 2, 8, 1, 4>(inst0, table, n_inst, total_units, err, sm_count, wait_ns, s);
    }
    return fail(STAG_KDE_EUNSUPPORTED, "tensor-core form: unsupported operand width");
}

template <int EG>
int launch_multi_eg(const TcMulti &mp, int grid, int *err, uint64_t wait_ns, cudaStream_t s) {
    const uint64_t stall_ns = injected_stall_ns();
    // the largest shared-memory layout of the four widths (and one CTA per SM at most)
    constexpr int smem = std::max({Cfg<16, 256, 4, 8, 2, EG>::SMEM, Cfg<32, 256, 4, 8, 2, EG>::SMEM,
                                   Cfg<64, 256, 2, 8, 1, EG>::SMEM, Cfg<128, 128, 2, 8, 1, EG>::SMEM, 118 * 1024});
    static_assert(smem <= 232448, "shared memory budget");
    auto kern = kde_tc_multi_kernel<EG>;
    // set once per instantiation (before any stream capture can be in progress)
    static cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    STAG_CUDA_TRY(attr);
    count_launch();
    kern<<<grid, 64 + 128 * EG, smem, s>>>(mp, err, wait_ns, stall_ns);
    STAG_CUDA_TRY(cudaGetLastError());
    return 0;
}

}  // namespace

int tc_launch_multi(int eg, const void *const tables[4], const int n_inst[4], const int64_t units[4],
                    const double work[4], int *err, int sm_count, uint64_t wait_ns, cudaStream_t s) {
    // CTAs per width in proportion to its work, at least one for a width with units and
    // never more than its units
    TcMulti mp{};
    int cta[4] = {0, 0, 0, 0};
    double wsum = 0.0;
    for (int c = 0; c < 4; ++c)
        if (n_inst[c] > 0 && units[c] > 0) wsum += std::max(work[c], 1e-30);
    if (wsum <= 0.0) return 0;
    int total = 0;
    for (int c = 0; c < 4; ++c) {
        if (n_inst[c] <= 0 || units[c] <= 0) continue;
        const double share = sm_count * std::max(work[c], 1e-30) / wsum;
        cta[c] = (int)std::min<int64_t>(units[c], std::max<int64_t>(1, (int64_t)share));
        total += cta[c];
    }
    while (total > sm_count) {  // more widths than SMs would need: trim the largest
        int big = 0;
        for (int c = 1; c < 4; ++c)
            if (cta[c] > cta[big]) big = c;
        if (cta[big] <= 1) break;
        --cta[big];
        --total;
    }
    while (total < sm_count) {  // hand the rest to the width with the most work per CTA
        int best = -1;
        double bw = 0.0;
        for (int c = 0; c < 4; ++c) {
            if (cta[c] == 0 || cta[c] >= units[c]) continue;
            const double w = std::max(work[c], 1e-30) / cta[c];
            if (w > bw) {
                bw = w;
                best = c;
            }
        }
        if (best < 0) break;
        ++cta[best];
        ++total;
    }
    mp.cta_begin[0] = 0;
    for (int c = 0; c < 4; ++c) {
        mp.table[c] = reinterpret_cast<const TcInst *>(tables[c]);
        mp.n_inst[c] = cta[c] > 0 ? n_inst[c] : 0;
        mp.units[c] = cta[c] > 0 ? units[c] : 0;
        mp.cta_begin[c + 1] = mp.cta_begin[c] + cta[c];
    }
    if (total <= 0) return 0;
    return eg == 2 ? launch_multi_eg<2>(mp, total, err, wait_ns, s) : launch_multi_eg<4>(mp, total, err, wait_ns, s);
}

bool tc_supported(int64_t d) { return kp_for(d) != 0; }

int tc_tile_points(int64_t d) { return kp_for(d) ? bn_for(kp_for(d)) : 0; }

void tc_free(stag_kde *h) {
    TcData *tc = h->tc;
    if (!tc) return;
    if (!h->is_view) {
        // the point set's data (shared with views)
        cudaFree(tc->b_hi);
        cudaFree(tc->b_lo);
        cudaFree(tc->b_aug);
        cudaFree(tc->a_aug);
        cudaFree(tc->tinfo);
        cudaFree(tc->cent);
        cudaFree(tc->centT);
        cudaFree(tc->cg);
        cudaFree(tc->xkt);
        cudaFree(tc->tsum);
        cudaFree(tc->vmax_bits);
        cudaFree(tc->xmax_bits);
        cudaFree(tc->scales);
    }
    // per-handle scratch
    cudaFree(tc->a_hi);
    cudaFree(tc->a_lo);
    cudaFree(tc->rowterm);
    cudaFree(tc->unorm);
    cudaFree(tc->qbad);
    cudaFree(tc->ub);
    cudaFree(tc->part_w);
    cudaFree(tc->fix_idx);
    cudaFree(tc->gbuf);
    cudaFree(tc->fix_count);
    cudaFree(tc->err);
    if (tc->err_host) cudaFreeHost(tc->err_host);
    delete tc;
    h->tc = nullptr;
}

// A view of the tensor-core data of `base`: shares the point set's arrays and tensor
// maps, owns empty scratch of its own.
int tc_make_view(const stag_kde *base, stag_kde *view) {
    const TcData *b = base->tc;
    if (!b) return 0;
    TcData *tc = new (std::nothrow) TcData();
    if (!tc) return fail(STAG_KDE_ENOMEM, "out of host memory");
    view->tc = tc;
    tc->Kp = b->Kp;
    tc->BN = b->BN;
    tc->T = b->T;
    tc->n_pad = b->n_pad;
    tc->b_hi = b->b_hi;
    tc->b_lo = b->b_lo;
    tc->b_aug = b->b_aug;
    tc->a_aug = b->a_aug;
    tc->tinfo = b->tinfo;
    tc->cent = b->cent;
    tc->centT = b->centT;
    tc->cg = b->cg;
    tc->xkt = b->xkt;
    tc->tsum = b->tsum;
    tc->vmax_bits = b->vmax_bits;
    tc->xmax_bits = b->xmax_bits;
    tc->scales = b->scales;
    tc->map_bhi = b->map_bhi;
    tc->map_blo = b->map_blo;
    tc->map_baug = b->map_baug;
    tc->map_aaug = b->map_aaug;
    STAG_CUDA_TRY(dev_malloc(&tc->err, sizeof(int)));
    STAG_CUDA_TRY(cudaMemset(tc->err, 0, sizeof(int)));
    STAG_CUDA_TRY(cudaMallocHost(&tc->err_host, sizeof(int)));
    return 0;
}

int tc_prepare_points(stag_kde *h, const float *dX) {
    TcData *tc = new (std::nothrow) TcData();
    if (!tc) return fail(STAG_KDE_ENOMEM, "out of host memory");
    h->tc = tc;
    cudaStream_t s = h->stream;
    tc->Kp = kp_for(h->d);
    tc->BN = bn_for(tc->Kp);
    tc->T = ceil_div(h->n, tc->BN);
    tc->n_pad = tc->T * tc->BN;
    const int Kp = tc->Kp;
    STAG_CUDA_TRY(dev_malloc(&tc->b_hi, tc->n_pad * Kp * sizeof(__half)));
    STAG_CUDA_TRY(dev_malloc(&tc->b_lo, tc->n_pad * Kp * sizeof(__half)));
    STAG_CUDA_TRY(dev_malloc(&tc->b_aug, tc->n_pad * 16 * sizeof(__half)));
    STAG_CUDA_TRY(dev_malloc(&tc->a_aug, BM * 16 * sizeof(__half)));
    STAG_CUDA_TRY(dev_malloc(&tc->tinfo, tc->T * 4 * sizeof(float)));
    STAG_CUDA_TRY(dev_malloc(&tc->cent, tc->T * Kp * sizeof(float)));
    STAG_CUDA_TRY(dev_malloc(&tc->cg, Kp * sizeof(float)));
    STAG_CUDA_TRY(dev_malloc(&tc->centT, tc->T * Kp * sizeof(float)));
    // the recompute of flagged queries reads the points in tile (k-d) order, in the plain
    // form's tile-transposed layout
    if (h->tc_check) {
        STAG_CUDA_TRY(dev_malloc(&tc->xkt, h->n_tiles * h->d_pad * kSimtTile * sizeof(float)));
        int rc0 = simt_tiles_from_rows(h, dX, tc->xkt, s);
        if (rc0) return rc0;
    }
    STAG_CUDA_TRY(dev_malloc(&tc->tsum, tc->T * Kp * sizeof(double)));
    STAG_CUDA_TRY(dev_malloc(&tc->vmax_bits, sizeof(unsigned)));
    STAG_CUDA_TRY(dev_malloc(&tc->xmax_bits, sizeof(unsigned)));
    STAG_CUDA_TRY(dev_malloc(&tc->scales, 4 * sizeof(float)));
    STAG_CUDA_TRY(dev_malloc(&tc->err, sizeof(int)));
    STAG_CUDA_TRY(cudaMallocHost(&tc->err_host, sizeof(int)));
    STAG_CUDA_TRY(cudaMemsetAsync(tc->err, 0, sizeof(int), s));
    STAG_CUDA_TRY(cudaMemsetAsync(tc->vmax_bits, 0, sizeof(unsigned), s));
    STAG_CUDA_TRY(cudaMemsetAsync(tc->xmax_bits, 0, sizeof(unsigned), s));

    const double c = h->a * 1.4426950408889634;
    count_launch(7);
    tc_centres_kernel<<<(unsigned)tc->T, 128, 0, s>>>(dX, h->n, h->d, tc->BN, Kp, tc->tsum, tc->cent);
    tc_global_centre_kernel<<<1, 128, 0, s>>>(tc->tsum, tc->T, Kp, h->n, h->d, tc->cg);
    tc_maxabs_kernel<<<grid_for(h->n * h->d, 256), 256, 0, s>>>(dX, h->n, h->d, tc->BN, Kp, tc->cent, tc->cg, true,
                                                               tc->vmax_bits);
    tc_maxabs_kernel<<<grid_for(h->n * h->d, 256), 256, 0, s>>>(dX, h->n, h->d, tc->BN, Kp, tc->cent, tc->cg, false,
                                                               tc->xmax_bits);
    tc_scales_kernel<<<1, 256, 0, s>>>(tc->vmax_bits, tc->xmax_bits, h->d, c, tc->scales, tc->a_aug);
    tc_split_points_kernel<<<grid_for(tc->n_pad, 128), 128, 0, s>>>(dX, h->n, h->d, tc->BN, Kp, tc->n_pad, tc->cent,
                                                                    tc->cg, tc->scales, tc->b_hi, tc->b_lo, tc->b_aug);
    tc_tile_radius_kernel<<<(unsigned)tc->T, 128, 0, s>>>(dX, h->n, h->d, tc->BN, Kp, tc->cent, tc->tinfo);
    count_launch();
    tc_transpose_centres_kernel<<<grid_for(tc->T * Kp, 256), 256, 0, s>>>(tc->cent, tc->T, Kp, tc->centT);
    STAG_CUDA_TRY(cudaGetLastError());
    int rc = make_map(&tc->map_bhi, tc->b_hi, tc->n_pad, Kp, tc->BN);
    if (!rc) rc = make_map(&tc->map_blo, tc->b_lo, tc->n_pad, Kp, tc->BN);
    if (!rc) rc = make_map(&tc->map_baug, tc->b_aug, tc->n_pad, 16, tc->BN);
    if (!rc) rc = make_map(&tc->map_aaug, tc->a_aug, BM, 16, BM);
    return rc;
}

// Carving of the grouped-recompute scratch for up to m query rows.
struct GroupScratch {
    uint64_t *key, *ktmp;
    uint32_t *val, *vtmp, *hist;
    float *thr;
    int *qflag, *bcnt, *boff, *kept, *kcount, *items, *item_off, *n_groups;
    double *psum;
    float *pshift;
};

// Kept point tiles per work item: at least eight 64-point tiles (the per-item set-up is
// then amortised), and at most 64 items per group.
static int group_seg(int64_t T, int BN) { return (int)std::max<int64_t>(8 * 64 / BN, ceil_div(T, 64)); }

static int64_t group_scratch_bytes(int64_t m, int64_t T, int BN, GroupScratch *gs, void *base) {
    const int64_t G = ceil_div(std::max<int64_t>(m, 1), 64);
    const int64_t B = ceil_div(std::max<int64_t>(m, 1), 256);  // blocks of the combine kernel
    const int64_t items = G * ceil_div(T, group_seg(T, BN));  // at most 64 segments per group
    int64_t off = 0;
    auto take = [&](int64_t bytes) {
        const int64_t o = off;
        off += round_up(bytes, 256);
        return static_cast<char *>(base) + o;
    };
    const int64_t mm = std::max<int64_t>(m, 1);
    GroupScratch g;
    g.key = (uint64_t *)take(mm * 8);
    g.ktmp = (uint64_t *)take(mm * 8);
    g.val = (uint32_t *)take(mm * 4);
    g.vtmp = (uint32_t *)take(mm * 4);
    g.hist = (uint32_t *)take(radix_sort_hist_entries(mm) * 4);
    g.thr = (float *)take(mm * 4);
    g.qflag = (int *)take(mm * 4);
    g.bcnt = (int *)take(B * 4);
    g.boff = (int *)take((B + 1) * 4);
    g.kept = (int *)take(G * T * 4);
    g.kcount = (int *)take(G * 4);
    g.items = (int *)take(G * 4);
    g.item_off = (int *)take((G + 1) * 4);
    g.n_groups = (int *)take(4);
    g.psum = (double *)take(items * 64 * 8);
    g.pshift = (float *)take(items * 64 * 4);
    if (gs) *gs = g;
    return off;
}

static int ensure_query_scratch(stag_kde *h, int64_t m_pad) {
    TcData *tc = h->tc;
    const int Kp = tc->Kp;
    if (tc->a_rows_cap < m_pad || tc->unorm_cap < m_pad || tc->rt_cap < tc->T * m_pad) ++h->scratch_epoch;
    if (tc->a_rows_cap < m_pad) {
        cudaFree(tc->a_hi);
        cudaFree(tc->a_lo);
        tc->a_hi = tc->a_lo = nullptr;
        tc->a_rows_cap = 0;
        STAG_CUDA_TRY(dev_malloc(&tc->a_hi, m_pad * Kp * sizeof(__half)));
        STAG_CUDA_TRY(dev_malloc(&tc->a_lo, m_pad * Kp * sizeof(__half)));
        tc->a_rows_cap = m_pad;
        int rc = make_map(&tc->map_ahi, tc->a_hi, m_pad, Kp, BM);
        if (!rc) rc = make_map(&tc->map_alo, tc->a_lo, m_pad, Kp, BM);
        if (rc) return rc;
    }
    if (tc->unorm_cap < m_pad) {
        cudaFree(tc->unorm);
        cudaFree(tc->qbad);
        cudaFree(tc->ub);
        cudaFree(tc->fix_idx);
        tc->unorm = nullptr;
        tc->qbad = nullptr;
        tc->ub = nullptr;
        tc->fix_idx = nullptr;
        tc->unorm_cap = 0;
        STAG_CUDA_TRY(dev_malloc(&tc->unorm, m_pad * sizeof(float)));
        STAG_CUDA_TRY(dev_malloc(&tc->qbad, m_pad * sizeof(int)));
        STAG_CUDA_TRY(dev_malloc(&tc->ub, m_pad * sizeof(unsigned)));
        STAG_CUDA_TRY(dev_malloc(&tc->fix_idx, m_pad * sizeof(int)));
        tc->unorm_cap = m_pad;
    }
    if (!tc->fix_count) STAG_CUDA_TRY(dev_malloc(&tc->fix_count, sizeof(int)));
    const int64_t need = tc->T * m_pad;
    if (tc->rt_cap < need) {
        cudaFree(tc->rowterm);
        tc->rowterm = nullptr;
        tc->rt_cap = 0;
        STAG_CUDA_TRY(dev_malloc(&tc->rowterm, need * sizeof(float)));
        tc->rt_cap = need;
    }
    return 0;
}

// Work split of one query call: units of (query tile, range of point tiles). With
// tiles_per_unit = 0 the ranges are chosen for ~8 units per SM; otherwise each range has
// about tiles_per_unit tiles (the batched path uses this to even out unit sizes).
static void plan_units(const stag_kde *h, int64_t m, int tiles_per_unit, int64_t *q_tiles, int64_t *splits,
                       int64_t *tps) {
    const TcData *tc = h->tc;
    const int64_t m_pad = round_up(m, BM);
    *q_tiles = m_pad / BM;
    int64_t sp;
    if (tiles_per_unit > 0) {
        sp = std::max<int64_t>(1, ceil_div(tc->T, tiles_per_unit));
    } else {
        sp = std::max<int64_t>(1, ceil_div((int64_t)h->sm_count * 8, *q_tiles));
        sp = std::min<int64_t>(sp, std::max<int64_t>(1, tc->T / 4));
    }
    *tps = ceil_div(tc->T, sp);
    *splits = ceil_div(tc->T, *tps);
}

int tc_reserve(stag_kde *h, int64_t m, int tiles_per_unit) {
    TcData *tc = h->tc;
    const int64_t m_pad = round_up(std::max<int64_t>(m, 1), BM);
    int rc = ensure_query_scratch(h, m_pad);
    if (rc) return rc;
    int64_t qt, sp, tps;
    plan_units(h, m, tiles_per_unit, &qt, &sp, &tps);
    // the grouped recompute needs its scratch and gathered query tiles
    if (h->tc_check) {
        if (tc->gbuf_m < m) {
            ++h->scratch_epoch;
            cudaFree(tc->gbuf);
            tc->gbuf = nullptr;
            tc->gbuf_m = 0;
            STAG_CUDA_TRY(dev_malloc(&tc->gbuf, group_scratch_bytes(m, tc->T, tc->BN, nullptr, nullptr)));
            tc->gbuf_m = m;
        }
        rc = ensure_qt(h, ceil_div(m, kSimtTile) * h->d_pad * kSimtTile);
    }
    if (!rc) rc = ensure_partials(h, sp * m);
    if (rc) return rc;
    if (tc->part_w_cap < sp * m) {
        ++h->scratch_epoch;
        cudaFree(tc->part_w);
        tc->part_w = nullptr;
        tc->part_w_cap = 0;
        STAG_CUDA_TRY(dev_malloc(&tc->part_w, sp * m * sizeof(double)));
        tc->part_w_cap = sp * m;
    }
    return 0;
}

// Query-side preparation: FP16 splits of the queries, the row terms and bounds (one launch).
static int tc_prep(stag_kde *h, const float *dQ, int64_t m, cudaStream_t s) {
    TcData *tc = h->tc;
    const int Kp = tc->Kp;
    const int64_t m_pad = round_up(m, BM);
    const double c = h->a * 1.4426950408889634;
    STAG_CUDA_TRY(cudaMemsetAsync(tc->qbad, 0, m_pad * sizeof(int), s));
    STAG_CUDA_TRY(cudaMemsetAsync(tc->ub, 0, m_pad * sizeof(unsigned), s));
    count_launch(1);
    // tiles per block: 256, fewer when that leaves under ~4 blocks per SM (small batches)
    int tpb = 256;
    while (tpb > RowTermGeo::TG && (m_pad / BM) * ceil_div(tc->T, tpb) < 4 * (int64_t)h->sm_count) tpb /= 2;
    dim3 grid((unsigned)(m_pad / BM), (unsigned)ceil_div(tc->T, tpb));
    switch (Kp) {
#define STAG_ROWTERM(KPV)                                                                                          \
    case KPV: {                                                                                                    \
        /* set once per instantiation (before any stream capture can be in progress) */                           \
        static cudaError_t attr = cudaFuncSetAttribute(tc_rowterm_kernel<KPV>,                                    \
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize,               \
                                                       RowTermGeo::smem_bytes(KPV));                              \
        STAG_CUDA_TRY(attr);                                                                                       \
        tc_rowterm_kernel<KPV><<<grid, RowTermGeo::THREADS, RowTermGeo::smem_bytes(KPV), s>>>(                     \
            dQ, m, h->d, m_pad, tc->cent, tc->T, tpb, (float)c, tc->rowterm, tc->cg, tc->unorm, tc->tinfo, tc->ub,  \
            tc->scales, tc->a_hi, tc->a_lo, tc->qbad, tc->centT);                                                  \
        break;                                                                                                     \
    }
        STAG_ROWTERM(16)
        STAG_ROWTERM(32)
        STAG_ROWTERM(64)
        STAG_ROWTERM(128)
#undef STAG_ROWTERM
    }
    STAG_CUDA_TRY(cudaGetLastError());
    return 0;
}

// Fills the kernel's view of one instance (units numbered from unit_begin).
static void fill_inst(const stag_kde *h, int64_t m, int64_t q_tiles, int64_t splits, int64_t tps, int64_t unit_begin,
                      TcInst *I) {
    const TcData *tc = h->tc;
    I->map_ahi = tc->map_ahi;
    I->map_alo = tc->map_alo;
    I->map_aaug = tc->map_aaug;
    I->map_bhi = tc->map_bhi;
    I->map_blo = tc->map_blo;
    I->map_baug = tc->map_baug;
    I->tinfo = tc->tinfo;
    I->rowterm = tc->rowterm;
    I->scales = tc->scales;
    I->ub = tc->ub;
    I->unorm = tc->unorm;
    I->part_sum = h->part.sum;
    I->part_shift = h->part.shift;
    I->part_w = tc->part_w;
    I->m = m;
    I->m_pad = round_up(m, BM);
    I->n = h->n;
    I->T = tc->T;
    I->q_tiles = q_tiles;
    I->tiles_per_split = tps;
    I->unit_begin = unit_begin;
    I->units = q_tiles * splits;
}

// Grouped recompute of the flagged queries, all on stream s (after tc_combine_kernel has
// written the per-query flags and per-block counts into the scratch).
static int tc_fixup_grouped(stag_kde *h, const float *dQ, int64_t m, double *dOut, cudaStream_t s) {
    TcData *tc = h->tc;
    GroupScratch g;
    group_scratch_bytes(m, tc->T, tc->BN, &g, tc->gbuf);
    const int64_t m_pad = round_up(m, BM);
    const int64_t B = ceil_div(m, 256);
    const float c = (float)(h->a * 1.4426950408889634);
    const int seg = group_seg(tc->T, tc->BN);
    const int per = tc->BN / kSimtTile;
    count_launch(2);
    // the flagged queries in query order (their count into fix_count), with sort keys
    tc_scan_kernel<<<1, 1024, 0, s>>>(g.bcnt, nullptr, (int)B, g.boff, tc->fix_count);
    tc_flag_compact_kernel<<<(unsigned)B, 256, 0, s>>>(g.qflag, g.boff, m, m_pad, tc->rowterm, tc->tinfo, tc->T, c,
                                                       tc->fix_idx, g.key, g.val, g.thr);
    STAG_CUDA_TRY(cudaGetLastError());
    // stable sort by leading tile of the flagged entries only (device count): the input
    // is in query order, so the groups are deterministic
    int bits = 1;
    while (((int64_t)1 << bits) < tc->T) ++bits;
    int rc = radix_sort_pairs(g.key, g.val, g.ktmp, g.vtmp, g.hist, m, bits, s, tc->fix_count);
    if (rc) return rc;
    rc = simt_gather_rows(h, dQ, reinterpret_cast<const int *>(g.val), tc->fix_count, m, h->qt, s);
    if (rc) return rc;
    count_launch(2);
    tc_group_keep_kernel<<<(unsigned)(h->sm_count * 4), 256, 0, s>>>(g.val, g.thr, tc->fix_count, g.n_groups, m_pad,
                                                                      tc->rowterm, tc->tinfo, tc->T, c, seg, g.kept,
                                                                      g.kcount, g.items);
    tc_scan_kernel<<<1, 1024, 0, s>>>(g.items, tc->fix_count, 0, g.item_off, nullptr);
    STAG_CUDA_TRY(cudaGetLastError());
    rc = simt_list_launch(h, tc->xkt, h->qt, g.kept, tc->T, g.kcount, g.item_off, g.n_groups, seg, per, g.psum,
                          g.pshift, s);
    if (rc) return rc;
    count_launch();
    tc_group_combine_kernel<<<(unsigned)std::min<int64_t>(ceil_div(m, 256), 1024), 256, 0, s>>>(
        g.psum, g.pshift, g.item_off, g.val, tc->fix_count, h->normalise ? 1.0 / (double)h->n : 1.0, dOut);
    STAG_CUDA_TRY(cudaGetLastError());
    return 0;
}

// FP64 combine with the per-query error estimate, then the FP32 recompute of the flagged
// queries over the tiles that can matter (tc_fixup_grouped).
static int tc_finish(stag_kde *h, const float *dQ, int64_t m, int64_t splits, double *dOut, cudaStream_t s) {
    TcData *tc = h->tc;
    const bool check = h->tc_check;
    GroupScratch g{};
    if (check) group_scratch_bytes(m, tc->T, tc->BN, &g, tc->gbuf);
    count_launch();
    tc_combine_kernel<<<(unsigned)ceil_div(m, 256), 256, 0, s>>>(
        h->part.sum, h->part.shift, tc->part_w, m, (int)splits, h->normalise ? 1.0 / (double)h->n : 1.0, tc->qbad,
        h->a, kTcErrThreshold, dOut, check ? g.qflag : nullptr, check ? g.bcnt : nullptr);
    STAG_CUDA_TRY(cudaGetLastError());
    if (!check) return 0;
    // groups of 64 flagged queries share every point load (a per-query pass would re-read
    // its kept tiles once per query)
    return tc_fixup_grouped(h, dQ, m, dOut, s);
}

int tc_operand_width(const stag_kde *h) { return h->tc ? h->tc->Kp : 0; }

size_t tc_inst_size() { return sizeof(TcInst); }

int tc_prep_public(stag_kde *h, const float *dQ, int64_t m, cudaStream_t s) { return tc_prep(h, dQ, m, s); }

int64_t tc_fill_inst(const stag_kde *h, int64_t m, int tiles_per_unit, int64_t unit_begin, void *inst,
                     int64_t *splits) {
    int64_t q_tiles, tps;
    plan_units(h, m, tiles_per_unit, &q_tiles, splits, &tps);
    TcInst *I = reinterpret_cast<TcInst *>(inst);
    fill_inst(h, m, q_tiles, *splits, tps, unit_begin, I);
    return I->units;
}

int tc_finish_public(stag_kde *h, const float *dQ, int64_t m, int64_t splits, double *dOut, cudaStream_t s) {
    return tc_finish(h, dQ, m, splits, dOut, s);
}

int tc_query(stag_kde *h, const float *dQ, int64_t m, double *dOut, cudaStream_t s, int *dflag) {
    TcData *tc = h->tc;
    int rc = tc_reserve(h, m, h->tune_tiles_per_unit);
    if (rc) return rc;
    if (dflag) {
        rc = launch_check_finite_f32(dQ, m * h->d, dflag, s);
        if (rc) return rc;
    }
    rc = tc_prep(h, dQ, m, s);
    if (rc) return rc;
    int64_t q_tiles, splits, tps;
    plan_units(h, m, h->tune_tiles_per_unit, &q_tiles, &splits, &tps);
    TcInst inst;
    fill_inst(h, m, q_tiles, splits, tps, 0, &inst);
    prof_start(h, s);
    rc = launch_tc_any(tc->Kp, h->tune_eg ? h->tune_eg : tc_epilogue_groups(), inst, nullptr, 1, inst.units,
                       tc->err, h->sm_count, h->wait_ns, s);
    prof_stop(h, s, (double)m * (double)h->n);
    if (rc) return rc;
    return tc_finish(h, dQ, m, splits, dOut, s);
}

int tc_fixed_rows(stag_kde *h, int64_t *count) {
    TcData *tc = h->tc;
    int v = 0;
    if (tc && tc->fix_count && h->tc_check) STAG_CUDA_TRY(cudaMemcpy(&v, tc->fix_count, sizeof(int), cudaMemcpyDeviceToHost));
    *count = v;
    return 0;
}

int tc_error_enqueue(stag_kde *h, cudaStream_t s) {
    TcData *tc = h->tc;
    if (!tc) return 0;
    STAG_CUDA_TRY(cudaMemcpyAsync(tc->err_host, tc->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    return 0;
}

int tc_error_take(stag_kde *h, cudaStream_t s) {
    TcData *tc = h->tc;
    if (!tc) return 0;
    if (*tc->err_host) {
        STAG_CUDA_TRY(cudaMemsetAsync(tc->err, 0, sizeof(int), s));
        return fail(STAG_KDE_ETIMEDOUT, "tensor-core kernel: a bounded wait expired");
    }
    return 0;
}

}  // namespace stagkde
