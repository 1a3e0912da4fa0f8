// C-ABI of the exact Gaussian KDE library (declared in include/stag_kde.h).
//
// The life cycle follows the paper's ExactGaussianKDE (Sec. 5.3): a constructor that
// takes the data matrix and the bandwidth a, and a query of a matrix of points that
// returns one density per row. Everything numerical runs in the CUDA kernels of this
// library; this file validates arguments, owns device memory and streams, and moves
// data across the host/device boundary.
#include <math.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <stdlib.h>
#include <cstdio>
#include <new>
#include <string>

#include "internal.h"

namespace stagkde {

static thread_local std::string g_last_error;
static thread_local int g_last_code = STAG_KDE_OK;
static std::atomic<uint64_t> g_launches{0};

void count_launch(int k) { g_launches.fetch_add((uint64_t)k, std::memory_order_relaxed); }
void uncount_launches(uint64_t k) { g_launches.fetch_sub(k, std::memory_order_relaxed); }

void set_error(const std::string &msg) {
    g_last_error = msg;
    g_last_code = STAG_KDE_EINVAL;
}

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    g_last_code = code;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    // an allocation the device could not satisfy is reported as out of memory
    g_last_code = e == cudaErrorMemoryAllocation ? STAG_KDE_ENOMEM : STAG_KDE_ECUDA;
    return g_last_code;
}

cudaError_t dev_malloc_bytes(void **p, size_t bytes) {
    static std::mutex mu;
    static std::string armed;  // the variable's value the count started from
    static long long count = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        const char *v = getenv("STAG_KDE_INJECT_ALLOC_FAIL");
        const std::string now = v ? v : "";
        if (now != armed) {
            armed = now;
            count = 0;
        }
        const long long k = now.empty() ? 0 : atoll(now.c_str());
        if (k > 0 && ++count == k) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    return cudaMalloc(p, bytes);
}

static cudaEvent_t prof_event(stag_kde *h) {
    if (!h->prof_pool.empty()) {
        cudaEvent_t e = h->prof_pool.back();
        h->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

void prof_start(stag_kde *h, cudaStream_t s) {
    if (!h->profiling) return;
    cudaEvent_t e = prof_event(h);
    if (!e) return;
    cudaEventRecord(e, s);
    h->prof_events.push_back(e);
}

void prof_stop(stag_kde *h, cudaStream_t s, double pairs) {
    if (!h->profiling || h->prof_events.size() % 2 == 0) return;
    cudaEvent_t e = prof_event(h);
    if (!e) {
        h->prof_pool.push_back(h->prof_events.back());
        h->prof_events.pop_back();
        return;
    }
    cudaEventRecord(e, s);
    h->prof_events.push_back(e);
    h->prof_launches += 1;
    h->prof_pairs += pairs;
}

namespace {

constexpr double kMaxAbs = 1e15;

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (dev >= 0 && dev != prev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

template <typename T>
bool host_values_ok(const T *p, int64_t count) {
    for (int64_t i = 0; i < count; ++i) {
        const double v = (double)p[i];
        if (!(fabs(v) <= kMaxAbs)) return false;
    }
    return true;
}

int check_a(double a) {
    if (!(a >= 0.0) || !isfinite(a)) return fail(STAG_KDE_EINVAL, "bandwidth a must be finite and >= 0");
    return 0;
}

void free_handle(stag_kde *h) {
    if (!h) return;
    batch_forget_handle(h);
    DeviceGuard g(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    tc_free(h);
    if (!h->is_view) {
        cudaFree(h->xt);
        cudaFree(h->x64);
    }
    cudaFree(h->q_dev);
    cudaFree(h->xrow);
    cudaFree(h->sub_dev);
    cudaFree(h->qt);
    cudaFree(h->out_dev);
    cudaFree(h->part.sum);
    cudaFree(h->part.shift);
    cudaFree(h->flag_dev);
    if (h->flag_host) cudaFreeHost(h->flag_host);
    for (int i = 0; i < 2; ++i) {
        if (h->copy_done[i]) cudaEventDestroy(h->copy_done[i]);
        if (h->copy_stream[i]) cudaStreamDestroy(h->copy_stream[i]);
    }
    for (cudaEvent_t e : h->prof_events) cudaEventDestroy(e);
    for (cudaEvent_t e : h->prof_pool) cudaEventDestroy(e);
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // namespace

stag_kde *make_view(stag_kde *base) {
    stag_kde *v = new (std::nothrow) stag_kde();
    if (!v) return (set_error("out of host memory"), nullptr);
    DeviceGuard g(base->device);
    v->device = base->device;
    v->n = base->n;
    v->d = base->d;
    v->a = base->a;
    v->dtype = base->dtype;
    v->form = base->form;
    v->normalise = base->normalise;
    v->kernel = base->kernel;
    v->tc_check = base->tc_check;
    v->tune_eg = base->tune_eg;
    v->tune_tiles_per_unit = base->tune_tiles_per_unit;
    v->wait_ns = base->wait_ns;
    v->is_view = true;
    v->xt = base->xt;
    v->n_tiles = base->n_tiles;
    v->d_pad = base->d_pad;
    v->x64 = base->x64;
    v->sm_count = base->sm_count;
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&v->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = dev_malloc(&v->flag_dev, sizeof(int))) != cudaSuccess ||
        (e = cudaMallocHost(&v->flag_host, sizeof(int))) != cudaSuccess) {
        cuda_fail(e, "view set-up");
        free_handle(v);
        return nullptr;
    }
    if (tc_make_view(base, v)) {
        free_handle(v);
        return nullptr;
    }
    return v;
}

void free_view(stag_kde *view) { free_handle(view); }

namespace {

int resolve_form(int requested, int dtype, int64_t d, int kernel, int *form) {
    if (kernel != STAG_KDE_KERNEL_GAUSSIAN && kernel != STAG_KDE_KERNEL_EXPONENTIAL &&
        kernel != STAG_KDE_KERNEL_LOGISTIC)
        return fail(STAG_KDE_EINVAL, "unknown kernel function");
    if (dtype == STAG_KDE_F64) {
        if (requested != STAG_KDE_FORM_AUTO && requested != STAG_KDE_FORM_SIMT_F64)
            return fail(STAG_KDE_EUNSUPPORTED, "FP64 data supports only the FP64 form");
        *form = STAG_KDE_FORM_SIMT_F64;
        return 0;
    }
    switch (requested) {
        case STAG_KDE_FORM_AUTO:
            *form = kernel == STAG_KDE_KERNEL_GAUSSIAN && tc_supported(d) ? STAG_KDE_FORM_TC : STAG_KDE_FORM_SIMT_F32;
            return 0;
        case STAG_KDE_FORM_SIMT_F32:
            *form = requested;
            return 0;
        case STAG_KDE_FORM_TC:
            if (kernel != STAG_KDE_KERNEL_GAUSSIAN)
                return fail(STAG_KDE_EUNSUPPORTED, "tensor-core form serves only the Gaussian kernel");
            if (!tc_supported(d)) return fail(STAG_KDE_EUNSUPPORTED, "tensor-core form does not support this d");
            *form = requested;
            return 0;
        default:
            return fail(STAG_KDE_EINVAL, "unknown form");
    }
}

int ensure_bytes(void **p, int64_t *cap, int64_t bytes) {
    if (*cap >= bytes) return 0;
    // (callers bump the handle's scratch epoch)
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    STAG_CUDA_TRY(dev_malloc(p, bytes));
    *cap = bytes;
    return 0;
}

int run_query(stag_kde *h, const void *dQ, int64_t m, double *dOut, cudaStream_t s, int *dflag) {
    switch (h->form) {
        case STAG_KDE_FORM_SIMT_F32:
            return simt_query_f32(h, (const float *)dQ, m, dOut, s, dflag);
        case STAG_KDE_FORM_SIMT_F64:
            return simt_query_f64(h, (const double *)dQ, m, dOut, s, dflag);
        case STAG_KDE_FORM_TC:
            return tc_query(h, (const float *)dQ, m, dOut, s, dflag);
    }
    return fail(STAG_KDE_EINVAL, "handle has an unknown form");
}

size_t elem_size(int dtype) { return dtype == STAG_KDE_F64 ? sizeof(double) : sizeof(float); }

}  // namespace
}  // namespace stagkde

using namespace stagkde;

extern "C" {

void stag_kde_opts_init(stag_kde_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->form = STAG_KDE_FORM_AUTO;
    o->normalise = 0;
    o->device = -1;
}

stag_kde_t *stag_kde_create_ex(const void *X, int dtype, int64_t n, int64_t d, double a,
                               const stag_kde_opts *opts) {
    stag_kde_opts o;
    stag_kde_opts_init(&o);
    if (opts) o = *opts;
    if (!X) return (set_error("X is NULL"), nullptr);
    if (n < 1 || d < 1) return (set_error("need n >= 1 and d >= 1"), nullptr);
    if (d > (1 << 20) || n > ((int64_t)1 << 40)) return (set_error("n or d too large"), nullptr);
    if (dtype != STAG_KDE_F32 && dtype != STAG_KDE_F64) return (set_error("unknown dtype"), nullptr);
    if (check_a(a)) return nullptr;
    const bool ok = dtype == STAG_KDE_F32 ? host_values_ok((const float *)X, n * d)
                                          : host_values_ok((const double *)X, n * d);
    if (!ok) return (set_error("X has a non-finite value or |x| > 1e15"), nullptr);
    int form = 0;
    for (int r : o.reserved)
        if (r != 0) return (set_error("stag_kde_opts.reserved must be zero"), nullptr);
    if (resolve_form(o.form, dtype, d, o.kernel, &form)) return nullptr;

    stag_kde *h = new (std::nothrow) stag_kde();
    if (!h) return (set_error("out of host memory"), nullptr);
    if (o.device < 0) {
        if (cudaGetDevice(&h->device) != cudaSuccess) {
            set_error("no CUDA device");
            delete h;
            return nullptr;
        }
    } else {
        h->device = o.device;
    }
    DeviceGuard g(h->device);
    h->n = n;
    h->d = d;
    h->a = a;
    h->dtype = dtype;
    h->form = form;
    h->normalise = o.normalise ? 1 : 0;
    h->kernel = o.kernel;
    h->tc_check = o.tc_no_check == 0;
    auto bail = [&](const char *what, cudaError_t e) -> stag_kde_t * {
        if (e != cudaSuccess) cuda_fail(e, what);
        free_handle(h);
        return nullptr;
    };
    cudaError_t e;
    if (!g.ok) return bail("cudaSetDevice", cudaErrorInvalidDevice);
    if ((e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device)) != cudaSuccess)
        return bail("cudaDeviceGetAttribute", e);
    if ((e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)) != cudaSuccess)
        return bail("cudaStreamCreate", e);
    if ((e = dev_malloc(&h->flag_dev, sizeof(int))) != cudaSuccess) return bail("dev_malloc(flag)", e);
    if ((e = cudaMallocHost(&h->flag_host, sizeof(int))) != cudaSuccess) return bail("cudaMallocHost", e);

    const size_t bytes = (size_t)(n * d) * elem_size(dtype);
    if (dtype == STAG_KDE_F64) {
        if ((e = dev_malloc(&h->x64, bytes)) != cudaSuccess) return bail("dev_malloc(X)", e);
        if ((e = cudaMemcpyAsync(h->x64, X, bytes, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess)
            return bail("cudaMemcpy(X)", e);
    } else {
        float *dX = nullptr;
        if ((e = dev_malloc(&dX, bytes)) != cudaSuccess) return bail("dev_malloc(X)", e);
        int rc = 0;
        if ((e = cudaMemcpyAsync(dX, X, bytes, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess) {
            cudaFree(dX);
            return bail("cudaMemcpy(X)", e);
        }
        // the plain form's layout is always built: it is also the fallback and the
        // reference used by the tensor-core form's tests
        rc = simt_prepare_points(h, dX);
        if (!rc && form == STAG_KDE_FORM_TC) {
            // tensor-core form: tiles of spatially coherent points (k-d order)
            float *dXs = nullptr;
            if ((e = dev_malloc(&dXs, bytes)) != cudaSuccess) {
                rc = cuda_fail(e, "dev_malloc(ordered X)");
            } else {
                rc = kd_reorder(dX, n, d, tc_tile_points(d), dXs, h->stream);
                if (!rc) rc = tc_prepare_points(h, dXs);
                cudaStreamSynchronize(h->stream);
                cudaFree(dXs);
            }
        }
        cudaStreamSynchronize(h->stream);
        cudaFree(dX);
        if (rc) return bail("prepare", cudaSuccess);
    }
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return bail("create", e);
    return h;
}

stag_kde_t *stag_kde_create(const float *X, int64_t n, int64_t d, double a) {
    return stag_kde_create_ex(X, STAG_KDE_F32, n, d, a, nullptr);
}

int stag_kde_reserve(stag_kde_t *h, int64_t m) {
    if (!h) return fail(STAG_KDE_EINVAL, "handle is NULL");
    if (m < 0) return fail(STAG_KDE_EINVAL, "m < 0");
    DeviceGuard g(h->device);
    int rc = ensure_bytes(&h->q_dev, &h->q_dev_cap, std::max<int64_t>(1, m * h->d) * elem_size(h->dtype));
    if (!rc) rc = ensure_bytes((void **)&h->out_dev, &h->out_cap, std::max<int64_t>(1, m) * 8);
    if (rc) return rc;
    if (h->form == STAG_KDE_FORM_SIMT_F32) rc = simt_reserve(h, std::max<int64_t>(m, 1));
    if (h->form == STAG_KDE_FORM_TC) rc = tc_reserve(h, std::max<int64_t>(m, 1), h->tune_tiles_per_unit);
    if (h->form == STAG_KDE_FORM_SIMT_F64 && h->normalise) rc = ensure_partials(h, std::max<int64_t>(m, 1));
    return rc;
}

int stag_kde_query(stag_kde_t *h, const void *Q, int64_t m, double *out) {
    if (!h) return fail(STAG_KDE_EINVAL, "handle is NULL");
    if (m < 0) return fail(STAG_KDE_EINVAL, "m < 0");
    if (m == 0) return 0;
    if (!Q || !out) return fail(STAG_KDE_EINVAL, "Q or out is NULL");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(STAG_KDE_ECUDA, "cudaSetDevice failed");
    const int64_t qbytes = m * h->d * (int64_t)elem_size(h->dtype);
    int rc = ensure_bytes(&h->q_dev, &h->q_dev_cap, qbytes);
    if (rc) return rc;
    rc = ensure_bytes((void **)&h->out_dev, &h->out_cap, m * 8);
    if (rc) return rc;
    STAG_CUDA_TRY(cudaMemsetAsync(h->flag_dev, 0, sizeof(int), h->stream));
    STAG_CUDA_TRY(cudaMemcpyAsync(h->q_dev, Q, qbytes, cudaMemcpyHostToDevice, h->stream));
    rc = run_query(h, h->q_dev, m, h->out_dev, h->stream, h->flag_dev);
    if (rc) {
        cudaStreamSynchronize(h->stream);
        return rc;
    }
    // one synchronisation for both checks: the input flag and the kernel's error code
    STAG_CUDA_TRY(cudaMemcpyAsync(h->flag_host, h->flag_dev, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    if (h->form == STAG_KDE_FORM_TC) {
        rc = tc_error_enqueue(h, h->stream);
        if (rc) {
            cudaStreamSynchronize(h->stream);
            return rc;
        }
    }
    STAG_CUDA_TRY(cudaStreamSynchronize(h->stream));
    // (a set error code is cleared either way; the input error is the one reported)
    const int terr = h->form == STAG_KDE_FORM_TC ? tc_error_take(h, h->stream) : 0;
    if (*h->flag_host) return fail(STAG_KDE_EINVAL, "Q has a non-finite value or |q| > 1e15");
    if (terr) return terr;
    STAG_CUDA_TRY(cudaMemcpyAsync(out, h->out_dev, m * 8, cudaMemcpyDeviceToHost, h->stream));
    STAG_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return 0;
}

int stag_kde_query_dev(stag_kde_t *h, const void *dQ, int64_t m, double *dOut, void *stream) {
    if (!h) return fail(STAG_KDE_EINVAL, "handle is NULL");
    if (m < 0) return fail(STAG_KDE_EINVAL, "m < 0");
    if (m == 0) return 0;
    if (!dQ || !dOut) return fail(STAG_KDE_EINVAL, "dQ or dOut is NULL");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(STAG_KDE_ECUDA, "cudaSetDevice failed");
    return run_query(h, dQ, m, dOut, (cudaStream_t)stream, nullptr);
}

int stag_kde_query_subset_dev(stag_kde_t *h, const float *dQ, int64_t m, const int64_t *dOff, const int64_t *dIdx,
                              const float *dW, double *dOut, void *stream) {
    if (!h) return fail(STAG_KDE_EINVAL, "handle is NULL");
    if (m < 0) return fail(STAG_KDE_EINVAL, "m < 0");
    if (m == 0) return 0;
    if (!dQ || !dOff || !dIdx || !dOut) return fail(STAG_KDE_EINVAL, "dQ, dOff, dIdx or dOut is NULL");
    if (h->dtype != STAG_KDE_F32) return fail(STAG_KDE_EUNSUPPORTED, "subset sums: FP32 handles only");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(STAG_KDE_ECUDA, "cudaSetDevice failed");
    return subset_query(h, dQ, m, dOff, dIdx, dW, dOut, (cudaStream_t)stream, 0.0);
}

int stag_kde_query_subset(stag_kde_t *h, const float *Q, int64_t m, const int64_t *off, const int64_t *idx,
                          const float *W, double *out) {
    if (!h) return fail(STAG_KDE_EINVAL, "handle is NULL");
    if (m < 0) return fail(STAG_KDE_EINVAL, "m < 0");
    if (m == 0) return 0;
    if (!Q || !off || !out) return fail(STAG_KDE_EINVAL, "Q, off or out is NULL");
    if (h->dtype != STAG_KDE_F32) return fail(STAG_KDE_EUNSUPPORTED, "subset sums: FP32 handles only");
    if (off[0] != 0) return fail(STAG_KDE_EINVAL, "off[0] must be 0");
    for (int64_t j = 0; j < m; ++j)
        if (off[j + 1] < off[j]) return fail(STAG_KDE_EINVAL, "offsets must be non-decreasing");
    const int64_t nnz = off[m];
    if (nnz > 0 && !idx) return fail(STAG_KDE_EINVAL, "idx is NULL");
    // (the offsets are checked here because the kernel's reads depend on them; Q, the
    // indices and the weights are checked on the device, beside the sum, before out is
    // written)
    DeviceGuard g(h->device);
    if (!g.ok) return fail(STAG_KDE_ECUDA, "cudaSetDevice failed");
    // one device buffer: offsets | indices | weights | queries (16-byte aligned parts)
    const int64_t b_off = round_up((m + 1) * 8, 16), b_idx = round_up(std::max<int64_t>(nnz, 1) * 8, 16);
    const int64_t b_w = round_up(std::max<int64_t>(nnz, 1) * 4, 16), b_q = round_up(m * h->d * 4, 16);
    int rc = ensure_bytes(&h->sub_dev, &h->sub_dev_cap, b_off + b_idx + b_w + b_q);
    if (rc) return rc;
    rc = ensure_bytes((void **)&h->out_dev, &h->out_cap, m * 8);
    if (rc) return rc;
    char *base = (char *)h->sub_dev;
    int64_t *dOff = (int64_t *)base, *dIdx = (int64_t *)(base + b_off);
    float *dW = (float *)(base + b_off + b_idx), *dQ = (float *)(base + b_off + b_idx + b_w);
    cudaStream_t s = h->stream;
    // the index list goes up in two halves on two more streams, beside the rest on the
    // handle's stream, so that several copy engines move the lists
    for (int i = 0; i < 2; ++i) {
        if (!h->copy_stream[i]) STAG_CUDA_TRY(cudaStreamCreateWithFlags(&h->copy_stream[i], cudaStreamNonBlocking));
        if (!h->copy_done[i]) STAG_CUDA_TRY(cudaEventCreateWithFlags(&h->copy_done[i], cudaEventDisableTiming));
    }
    // Everything from the first copy on reports through rc: on any failure the copy streams
    // and the handle's stream are drained before the return, so that no queued copy reads
    // the caller's buffers afterwards.
    auto enqueue = [&]() -> int {
        const int64_t half = nnz / 2;
        if (half > 0) STAG_CUDA_TRY(cudaMemcpyAsync(dIdx, idx, half * 8, cudaMemcpyHostToDevice, h->copy_stream[0]));
        if (nnz > half)
            STAG_CUDA_TRY(cudaMemcpyAsync(dIdx + half, idx + half, (nnz - half) * 8, cudaMemcpyHostToDevice,
                                          h->copy_stream[1]));
        for (int i = 0; i < 2; ++i) STAG_CUDA_TRY(cudaEventRecord(h->copy_done[i], h->copy_stream[i]));
        STAG_CUDA_TRY(cudaMemcpyAsync(dOff, off, (m + 1) * 8, cudaMemcpyHostToDevice, s));
        if (W && nnz > 0) STAG_CUDA_TRY(cudaMemcpyAsync(dW, W, nnz * 4, cudaMemcpyHostToDevice, s));
        STAG_CUDA_TRY(cudaMemcpyAsync(dQ, Q, m * h->d * 4, cudaMemcpyHostToDevice, s));
        STAG_CUDA_TRY(cudaMemsetAsync(h->flag_dev, 0, sizeof(int), s));
        int r = launch_check_finite_f32(dQ, m * h->d, h->flag_dev, s, 4);
        if (r) return r;
        for (int i = 0; i < 2; ++i) STAG_CUDA_TRY(cudaStreamWaitEvent(s, h->copy_done[i], 0));
        r = subset_check_entries(dIdx, W ? dW : nullptr, nnz, h->n, h->flag_dev, s);
        if (r) return r;
        r = subset_query(h, dQ, m, dOff, dIdx, W ? dW : nullptr, h->out_dev, s, (double)nnz);
        if (r) return r;
        STAG_CUDA_TRY(cudaMemcpyAsync(h->flag_host, h->flag_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
        return 0;
    };
    rc = enqueue();
    if (rc) {
        cudaStreamSynchronize(h->copy_stream[0]);
        cudaStreamSynchronize(h->copy_stream[1]);
        cudaStreamSynchronize(s);
        return rc;
    }
    STAG_CUDA_TRY(cudaStreamSynchronize(s));
    if (*h->flag_host & 4) return fail(STAG_KDE_EINVAL, "Q has a non-finite value or |q| > 1e15");
    if (*h->flag_host & 1) return fail(STAG_KDE_EINVAL, "an index is outside [0, n)");
    if (*h->flag_host & 2) return fail(STAG_KDE_EINVAL, "weights must be finite and >= 0");
    STAG_CUDA_TRY(cudaMemcpyAsync(out, h->out_dev, m * 8, cudaMemcpyDeviceToHost, s));
    STAG_CUDA_TRY(cudaStreamSynchronize(s));
    return 0;
}

int stag_kde_degrees(stag_kde_t *h, int exclude_self, double *dOut, void *stream) {
    if (!h || !dOut) return fail(STAG_KDE_EINVAL, "handle or dOut is NULL");
    if (h->dtype != STAG_KDE_F32) return fail(STAG_KDE_EUNSUPPORTED, "degrees: FP32 handles only");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(STAG_KDE_ECUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    // the point set in original order, as a query batch against itself
    int rc = ensure_bytes(&h->q_dev, &h->q_dev_cap, h->n * h->d * (int64_t)sizeof(float));
    if (rc) return rc;
    rc = simt_points_rows(h, (float *)h->q_dev, s);
    if (rc) return rc;
    rc = run_query(h, h->q_dev, h->n, dOut, s, nullptr);
    if (rc) return rc;
    if (exclude_self) rc = launch_subtract(dOut, h->n, h->normalise ? 1.0 / (double)h->n : 1.0, s);
    return rc;
}

int stag_kde_info(const stag_kde_t *h, int64_t *n, int64_t *d, double *a, int *dtype, int *form) {
    if (!h) return fail(STAG_KDE_EINVAL, "handle is NULL");
    if (n) *n = h->n;
    if (d) *d = h->d;
    if (a) *a = h->a;
    if (dtype) *dtype = h->dtype;
    if (form) *form = h->form;
    return 0;
}

void stag_kde_destroy(stag_kde_t *h) { free_handle(h); }

int stag_kde_set_wait_limit(stag_kde_t *h, int64_t limit_ns) {
    if (!h) return fail(STAG_KDE_EINVAL, "handle is NULL");
    if (limit_ns < 0 || limit_ns > 60000000000ll) return fail(STAG_KDE_EINVAL, "wait limit must be in [0, 60 s]");
    h->wait_ns = limit_ns == 0 ? 2000000000ull : (uint64_t)limit_ns;
    return 0;
}

int stag_kde_last_recomputed(stag_kde_t *h, int64_t *count) {
    if (!h || !count) return fail(STAG_KDE_EINVAL, "handle or count is NULL");
    *count = 0;
    if (h->form != STAG_KDE_FORM_TC) return 0;
    DeviceGuard g(h->device);
    return tc_fixed_rows(h, count);
}

int stag_kde_profile_begin(stag_kde_t *h) {
    if (!h) return fail(STAG_KDE_EINVAL, "handle is NULL");
    for (cudaEvent_t e : h->prof_events) h->prof_pool.push_back(e);
    h->prof_events.clear();
    h->prof_launches = 0;
    h->prof_pairs = 0.0;
    h->profiling = true;
    return 0;
}

int stag_kde_profile_end(stag_kde_t *h, double *ms, int64_t *launches, double *pairs) {
    if (!h) return fail(STAG_KDE_EINVAL, "handle is NULL");
    DeviceGuard g(h->device);
    double total = 0.0;
    for (size_t i = 0; i + 1 < h->prof_events.size(); i += 2) {
        STAG_CUDA_TRY(cudaEventSynchronize(h->prof_events[i + 1]));
        float t = 0.f;
        STAG_CUDA_TRY(cudaEventElapsedTime(&t, h->prof_events[i], h->prof_events[i + 1]));
        total += t;
    }
    if (ms) *ms = total;
    if (launches) *launches = h->prof_launches;
    if (pairs) *pairs = h->prof_pairs;
    for (cudaEvent_t e : h->prof_events) h->prof_pool.push_back(e);
    h->prof_events.clear();
    h->profiling = false;
    return 0;
}

const char *stag_kde_last_error(void) { return g_last_error.c_str(); }

int stag_kde_last_error_code(void) { return g_last_code; }

const char *stag_kde_version(void) { return "stag-kde-gb300 0.1 (sm_103a)"; }

uint64_t stag_kde_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
