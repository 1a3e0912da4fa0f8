// Cross-block combine of per-split partial sums (Sec. 3: K(q) = sum_i k(||q - x_i||) is a
// sum over the whole point set; the kernels split the point set into contiguous ranges).
// Partial k of query j is part_sum[k*m + j] * 2^part_shift[k*m + j] with an integer
// shift. The combine takes the largest shift S, adds sum_k * 2^(shift_k - S) in FP64 in
// split order (fixed, so the result is reproducible), then scales by 2^S and by `scale`
// (1, or 1/n for the normalised density).
#include <math.h>

#include "internal.h"

namespace stagkde {
namespace {

__device__ __forceinline__ int clamp_exp_c(float e) { return (int)fminf(fmaxf(e, -4000.f), 4000.f); }

__global__ void combine_kernel(const double *__restrict__ part_sum, const float *__restrict__ part_shift,
                               int64_t m, int splits, double scale, double *__restrict__ out) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m;
         j += (int64_t)gridDim.x * blockDim.x) {
        float smax = -INFINITY;
        for (int k = 0; k < splits; ++k) smax = fmaxf(smax, part_shift[(int64_t)k * m + j]);
        double tot = 0.0;
        for (int k = 0; k < splits; ++k)
            tot += ldexp(part_sum[(int64_t)k * m + j], clamp_exp_c(part_shift[(int64_t)k * m + j] - smax));
        out[j] = ldexp(tot, clamp_exp_c(smax)) * scale;
    }
}

}  // namespace

int launch_combine(const double *part_sum, const float *part_shift, int64_t m, int splits, double scale,
                   double *out, cudaStream_t s) {
    if (m <= 0) return 0;
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>(ceil_div(m, threads), 4096);
    count_launch();
    combine_kernel<<<blocks, threads, 0, s>>>(part_sum, part_shift, m, splits, scale, out);
    STAG_CUDA_TRY(cudaGetLastError());
    return 0;
}

}  // namespace stagkde
