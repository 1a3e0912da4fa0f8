// The kernel functions of Sec. 3 in the log2-shifted form the plain kernels evaluate:
// with negc = -a log2(e) and a per-row integer shift s, one term is k(r) 2^-s, where
//   Gaussian     k = exp(-a r^2)                      -> 2^(negc d2 - s)
//   exponential  k = exp(-a r)                        -> 2^(negc r - s)
//   logistic     k = 4 / (2 + e^{ar} + e^{-ar})       -> 4 t' / (1 + t)^2,
//                t = 2^(negc r) <= 1, t' = 2^(negc r - s)
// (the logistic form in the bounded variable t equals the definition and cannot
// overflow). d2 is the squared distance, r = sqrt(d2).
#pragma once
#include "stag_kde.h"

namespace stagkde {
namespace kfn {

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// sqrt with the hardware approximation (relative error ~2^-23, 0 at 0): r enters the
// exponent, where this adds ~a r 2^-23 to a term's relative error, below the squared
// distance's own rounding error for d >= 4 and within the plain form's bound for all d.
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int KERN>
__device__ __forceinline__ float term(float negc, float d2, float shift) {
    if constexpr (KERN == STAG_KDE_KERNEL_GAUSSIAN) {
        return ex2_approx(fmaf(negc, d2, -shift));
    } else {
        const float x = negc * sqrt_approx(d2);  // log2 of exp(-a r)
        const float ts = ex2_approx(x - shift);
        if constexpr (KERN == STAG_KDE_KERNEL_EXPONENTIAL) {
            return ts;
        } else {
            const float t = ex2_approx(x);
            const float den = (1.f + t) * (1.f + t);
            return __fdividef(4.f * ts, den);
        }
    }
}

// Upper bound (log2) of a term before the shift, used to choose a new shift.
template <int KERN>
__device__ __forceinline__ float term_log2(float negc, float d2) {
    if constexpr (KERN == STAG_KDE_KERNEL_GAUSSIAN)
        return negc * d2;
    else
        return negc * sqrt_approx(d2);  // the logistic factor 4 / (1 + t)^2 is at most 4
}

}  // namespace kfn
}  // namespace stagkde
