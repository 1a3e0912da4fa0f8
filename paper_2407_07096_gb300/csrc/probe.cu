// Throughput probe of the MUFU ex2 unit (stag_kde_probe_ex2): the peak behind the
// roofline of the kernels whose bound is one ex2.approx per (query, point) pair.
//
// Every thread runs 8 independent chains x <- ex2(x) - 0.5 (one MUFU op and one FP32 add
// per step; the FP32 pipe has four times the MUFU rate, so MUFU sets the pace) on a grid
// of 8 blocks of 256 threads per SM; the chains keep values in [-0.5, 0.5] and their sum
// is stored so that no step can be removed.
#include "internal.h"

namespace stagkde {
namespace {

__device__ __forceinline__ float ex2a(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void __launch_bounds__(256) ex2_probe_kernel(int iters, float seed, float *out) {
    float x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = seed * (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) x[c] = ex2a(x[c]) - 0.5f;
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += x[c];
    out[blockIdx.x * 256 + threadIdx.x] = s;
}

}  // namespace
}  // namespace stagkde

using namespace stagkde;

extern "C" int stag_kde_probe_ex2(int64_t iters, double *ms, double *ex2_per_s) {
    if (iters < 1 || iters > (1 << 24) || !ms || !ex2_per_s) return fail(STAG_KDE_EINVAL, "bad probe arguments");
    int dev = 0, sms = 0;
    STAG_CUDA_TRY(cudaGetDevice(&dev));
    STAG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8;
    float *out = nullptr;
    STAG_CUDA_TRY(dev_malloc(&out, (size_t)blocks * 256 * sizeof(float)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = 0;
    auto run = [&]() -> int {
        STAG_CUDA_TRY(cudaEventCreate(&e0));
        STAG_CUDA_TRY(cudaEventCreate(&e1));
        count_launch(2);
        ex2_probe_kernel<<<blocks, 256>>>((int)std::min<int64_t>(iters, 4096), 0.37f, out);  // warm-up
        STAG_CUDA_TRY(cudaEventRecord(e0));
        ex2_probe_kernel<<<blocks, 256>>>((int)iters, 0.37f, out);
        STAG_CUDA_TRY(cudaEventRecord(e1));
        STAG_CUDA_TRY(cudaEventSynchronize(e1));
        float t = 0.f;
        STAG_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
        *ms = t;
        *ex2_per_s = (double)blocks * 256.0 * 8.0 * (double)iters / ((double)t * 1e-3);
        return 0;
    };
    rc = run();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}
