/*
 * CPU oracle for the Euclidean LSH of Sec. 2 (E2LSH).
 *
 * TEST INFRASTRUCTURE ONLY, like kde_oracle.c: only the tests, the package's smoke check
 * and the benchmark's CPU legs call it; it shares no code with the CUDA path.
 *
 * Hash function (Sec. 2, "Random Projection"): for a in R^d and b in [0, 4),
 *     h_{a,b}(x) = floor((<x, a> + b) / 4).
 * The random a ~ N(0, I) and b ~ U(0, 4) are inputs (the caller draws them). The decision
 * is an integer taken from floating point, so it is taken in one stated precision, the
 * one the GPU path uses: FP32, with the dot product accumulated by fused multiply-adds
 * in coordinate order (s = 0; s = fma(x_k, a_k, s) for k = 0..d-1), then (s + b) / 4
 * (an exact scaling) and floor, clamped to the int32 range.
 *
 * Tables (Sec. 2, "Boosting the Probability"): L tables of K functions each; x and q share
 * table l's bucket when all K values of functions l*K .. l*K+K-1 agree. The near
 * neighbours of q are the distinct points that share q's bucket in at least one table;
 * they are listed in increasing index order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

static int32_t clamp_floor(float v) {
    float f = floorf(v);
    if (f >= 2147483648.0f) return INT32_MAX;
    if (f < -2147483648.0f) return INT32_MIN;
    return (int32_t)f;
}

/* H (n x nf, row-major) = hash values of the rows of X (n x d) under the nf functions
 * (rows of A, nf x d, and the offsets B). */
int oracle_lsh_hash(const float *X, int64_t n, int64_t d, int64_t nf, const float *A, const float *B, int32_t *H) {
    if (n < 0 || d < 1 || nf < 1 || !X || !A || !B || !H) return -1;
    for (int64_t i = 0; i < n; ++i) {
        const float *x = X + i * d;
        for (int64_t f = 0; f < nf; ++f) {
            const float *a = A + f * d;
            float s = 0.0f;
            for (int64_t k = 0; k < d; ++k) s = fmaf(x[k], a[k], s);
            const float v = (s + B[f]) * 0.25f;
            H[i * nf + f] = clamp_floor(v);
        }
    }
    return 0;
}

/* Near-neighbour candidates of the queries from hash values HX (n x K*L) and HQ
 * (m x K*L): off (m + 1 entries) and, when idx is not NULL and cap is large enough, the
 * candidate indices. Returns the total count, or -1 on a bad argument. */
int64_t oracle_lsh_candidates(const int32_t *HX, int64_t n, const int32_t *HQ, int64_t m, int K, int L,
                              int64_t *off, int64_t *idx, int64_t cap) {
    if (n < 0 || m < 0 || K < 1 || L < 1 || !off) return -1;
    const int64_t nf = (int64_t)K * L;
    int64_t total = 0;
    off[0] = 0;
    for (int64_t j = 0; j < m; ++j) {
        const int32_t *hq = HQ + j * nf;
        for (int64_t i = 0; i < n; ++i) {
            const int32_t *hx = HX + i * nf;
            int hit = 0;
            for (int l = 0; l < L && !hit; ++l) {
                int same = 1;
                for (int k = 0; k < K && same; ++k) same = hx[l * K + k] == hq[l * K + k];
                hit = same;
            }
            if (hit) {
                if (idx && total < cap) idx[total] = i;
                ++total;
            }
        }
        off[j + 1] = total;
    }
    return total;
}
