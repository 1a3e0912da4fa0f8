// Batched exact KDE (stag_kde_query_batch) and the tensor-core autotuner.
//
// Many independent instances (each a handle with its own point set, d and a, and a query
// batch of its own size) are evaluated together:
//   * query-side preparation of every instance;
//   * ONE persistent tensor-core launch for every operand width (16/32/64/128): its CTAs
//     are split into one range per width, sized by the width's share of the work, and each
//     range walks the units (query tile, range of point tiles) of every instance of its
//     width, read from a device table of instances (kde_tc.cu, TcInst, TcMulti);
//   * per instance: FP64 combine with the error estimate and the FP32 recompute of flagged
//     queries; instances on the plain forms run their usual path.
// The whole sequence is captured once into a CUDA graph and replayed on later calls with
// the same handles, pointers and sizes. Before the first capture the autotuner times the
// candidate (epilogue warp groups, tiles per unit) settings on the batch itself.
//
// A query's result does not depend on the batch around it: every instance keeps its own
// units, partials and combine, and a unit's arithmetic depends only on its own rows.
#include <string.h>

#include <algorithm>
#include <list>
#include <map>
#include <mutex>
#include <vector>

#include "internal.h"

namespace stagkde {
namespace {

struct ClassLaunch {
    int Kp = 0;
    int n_inst = 0;
    int64_t total_units = 0;
    double work = 0.0;        // SM time of the width's pairs, in units of one ex2 per pair
    void *d_table = nullptr;  // device copy of the instance table
};

// Relative SM time of one pair at operand width Kp: the slower of one ex2 (32 per SM per
// clock) and the form's 2 (3 Kp + 16) MMA flops (8192 per SM per clock).
double pair_cost(int Kp) { return std::max(1.0, (3.0 * Kp + 16.0) / 128.0); }

struct BatchPlan {
    std::vector<uintptr_t> key;
    int device = 0;
    std::vector<stag_kde *> hs;
    std::vector<const void *> qs;
    std::vector<int64_t> ms;
    std::vector<double *> outs;
    std::vector<uint64_t> epochs;
    std::vector<int64_t> splits;  // tensor-core instances: splits of their work
    std::vector<ClassLaunch> classes;
    int eg = 4;
    int tiles_per_unit = 32;
    int *d_err = nullptr;
    int *h_err = nullptr;  // pinned copy written at the end of every replay
    cudaStream_t cap = nullptr;
    // side streams: the instances' preparation and finish chains are spread over them so
    // that the small kernels of different instances overlap on the device (in the graph
    // they become parallel branches between a fork and a join event)
    static constexpr int kSide = 32;
    cudaStream_t side[kSide] = {};
    cudaEvent_t fork = nullptr, joined[kSide] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t launches_per_run = 0;
    uint64_t wait_ns = 0;  // the longest wait limit of the batch's handles
};

std::mutex g_mu;
std::list<BatchPlan *> g_plans;  // most recently used first
constexpr size_t kMaxPlans = 16;
// settings chosen by the tuner per batch signature: a plan rebuilt after a scratch change
// reuses them, so the work split (and hence every result bit) stays the same
std::map<std::vector<uintptr_t>, std::pair<int, int>> g_tuned;

void free_plan(BatchPlan *p) {
    if (!p) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(p->device);
    if (p->cap) cudaStreamSynchronize(p->cap);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (auto &c : p->classes) cudaFree(c.d_table);
    cudaFree(p->d_err);
    if (p->h_err) cudaFreeHost(p->h_err);
    if (p->cap) cudaStreamDestroy(p->cap);
    for (int i = 0; i < BatchPlan::kSide; ++i) {
        if (p->side[i]) cudaStreamDestroy(p->side[i]);
        if (p->joined[i]) cudaEventDestroy(p->joined[i]);
    }
    if (p->fork) cudaEventDestroy(p->fork);
    if (prev >= 0) cudaSetDevice(prev);
    delete p;
}

bool is_tc(const stag_kde *h) { return h->form == STAG_KDE_FORM_TC; }

// Reserves every instance's scratch for its m (nothing is allocated while capturing).
int reserve_all(BatchPlan *p) {
    for (size_t i = 0; i < p->hs.size(); ++i) {
        stag_kde *h = p->hs[i];
        const int64_t m = std::max<int64_t>(p->ms[i], 1);
        int rc = 0;
        if (is_tc(h)) {
            rc = tc_reserve(h, m, p->tiles_per_unit);
        } else if (h->form == STAG_KDE_FORM_SIMT_F32) {
            rc = simt_reserve(h, m);
        } else if (h->normalise) {
            rc = ensure_partials(h, m);
        }
        if (rc) return rc;
    }
    return 0;
}

// Instance tables per operand width (device copies), from the current scratch.
int build_tables(BatchPlan *p) {
    for (auto &c : p->classes) cudaFree(c.d_table);
    p->classes.clear();
    p->splits.assign(p->hs.size(), 0);
    const size_t isz = tc_inst_size();
    for (int Kp : {16, 32, 64, 128}) {
        std::vector<unsigned char> host;
        ClassLaunch cl;
        cl.Kp = Kp;
        for (size_t i = 0; i < p->hs.size(); ++i) {
            stag_kde *h = p->hs[i];
            if (!is_tc(h) || tc_operand_width(h) != Kp || p->ms[i] == 0) continue;
            host.resize(host.size() + isz);
            const int64_t units = tc_fill_inst(h, p->ms[i], p->tiles_per_unit, cl.total_units,
                                               host.data() + host.size() - isz, &p->splits[i]);
            cl.total_units += units;
            cl.work += (double)p->ms[i] * (double)h->n * pair_cost(Kp);
            ++cl.n_inst;
        }
        if (!cl.n_inst) continue;
        STAG_CUDA_TRY(dev_malloc(&cl.d_table, host.size()));
        STAG_CUDA_TRY(cudaMemcpy(cl.d_table, host.data(), host.size(), cudaMemcpyHostToDevice));
        p->classes.push_back(cl);
    }
    return 0;
}

// Queues the whole batch on stream s: the instances' query preparation spread over the
// side streams, one persistent tensor-core launch for every operand width on s, then the
// instances' combine and recompute chains spread over the side streams again; s waits
// for every side stream at the end (fork/join with events, so the order holds both when
// run directly and when captured into the graph).
int enqueue(BatchPlan *p, cudaStream_t s) {
    int rc = 0;
    auto fork = [&]() -> int {
        STAG_CUDA_TRY(cudaEventRecord(p->fork, s));
        for (int k = 0; k < BatchPlan::kSide; ++k) STAG_CUDA_TRY(cudaStreamWaitEvent(p->side[k], p->fork, 0));
        return 0;
    };
    auto join = [&]() -> int {
        for (int k = 0; k < BatchPlan::kSide; ++k) {
            STAG_CUDA_TRY(cudaEventRecord(p->joined[k], p->side[k]));
            STAG_CUDA_TRY(cudaStreamWaitEvent(s, p->joined[k], 0));
        }
        return 0;
    };
    auto side_of = [&](size_t i) { return p->side[i % BatchPlan::kSide]; };
    rc = fork();
    for (size_t i = 0; i < p->hs.size() && !rc; ++i) {
        stag_kde *h = p->hs[i];
        if (p->ms[i] == 0) continue;
        if (is_tc(h)) rc = tc_prep_public(h, (const float *)p->qs[i], p->ms[i], side_of(i));
    }
    if (!rc) rc = join();
    if (!rc && !p->classes.empty()) {
        // one persistent launch for every width: each width's CTAs serve its table
        const void *tables[4] = {nullptr, nullptr, nullptr, nullptr};
        int n_inst[4] = {0, 0, 0, 0};
        int64_t units[4] = {0, 0, 0, 0};
        double work[4] = {0.0, 0.0, 0.0, 0.0};
        for (auto &c : p->classes) {
            const int w = c.Kp == 16 ? 0 : c.Kp == 32 ? 1 : c.Kp == 64 ? 2 : 3;
            tables[w] = c.d_table;
            n_inst[w] = c.n_inst;
            units[w] = c.total_units;
            work[w] = c.work;
        }
        rc = tc_launch_multi(p->eg, tables, n_inst, units, work, p->d_err, p->hs[0]->sm_count, p->wait_ns, s);
    }
    if (!rc) rc = fork();
    for (size_t i = 0; i < p->hs.size() && !rc; ++i) {
        stag_kde *h = p->hs[i];
        if (p->ms[i] == 0) continue;
        cudaStream_t si = side_of(i);
        if (is_tc(h))
            rc = tc_finish_public(h, (const float *)p->qs[i], p->ms[i], p->splits[i], p->outs[i], si);
        else if (h->form == STAG_KDE_FORM_SIMT_F32)
            rc = simt_query_f32(h, (const float *)p->qs[i], p->ms[i], p->outs[i], si, nullptr);
        else
            rc = simt_query_f64(h, (const double *)p->qs[i], p->ms[i], p->outs[i], si, nullptr);
    }
    if (!rc) rc = join();
    return rc;
}

// Times the candidate settings on the batch itself (uncaptured runs) and keeps the best.
int autotune(BatchPlan *p) {
    bool any_tc = false;
    for (auto *h : p->hs) any_tc |= is_tc(h);
    if (!any_tc) return 0;
    const int egs[] = {2, 4};
    const int tpus[] = {16, 32, 64};
    cudaEvent_t e0, e1;
    STAG_CUDA_TRY(cudaEventCreate(&e0));
    STAG_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_eg = 4, best_tpu = 32;
    int rc = 0;
    for (int eg : egs) {
        for (int tpu : tpus) {
            p->eg = eg;
            p->tiles_per_unit = tpu;
            if ((rc = reserve_all(p)) || (rc = build_tables(p))) break;
            if ((rc = enqueue(p, p->cap))) break;  // warm-up
            cudaEventRecord(e0, p->cap);
            if ((rc = enqueue(p, p->cap))) break;
            cudaEventRecord(e1, p->cap);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "autotune");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_eg = eg;
                best_tpu = tpu;
            }
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    p->eg = best_eg;
    p->tiles_per_unit = best_tpu;
    return 0;
}

int build_plan(BatchPlan *p) {
    // the tuning runs read the queries and write the outputs on a stream of their own:
    // let every earlier piece of work on the device finish first
    STAG_CUDA_TRY(cudaDeviceSynchronize());
    STAG_CUDA_TRY(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));
    for (int k = 0; k < BatchPlan::kSide; ++k) {
        STAG_CUDA_TRY(cudaStreamCreateWithFlags(&p->side[k], cudaStreamNonBlocking));
        STAG_CUDA_TRY(cudaEventCreateWithFlags(&p->joined[k], cudaEventDisableTiming));
    }
    STAG_CUDA_TRY(cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming));
    STAG_CUDA_TRY(dev_malloc(&p->d_err, sizeof(int)));
    STAG_CUDA_TRY(cudaMemset(p->d_err, 0, sizeof(int)));
    STAG_CUDA_TRY(cudaMallocHost(&p->h_err, sizeof(int)));
    *p->h_err = 0;
    const uint64_t before = stag_kde_launch_count();
    int rc = 0;
    auto tuned = g_tuned.find(p->key);
    if (tuned != g_tuned.end()) {
        p->eg = tuned->second.first;
        p->tiles_per_unit = tuned->second.second;
    } else {
        rc = autotune(p);
        if (!rc) g_tuned[p->key] = {p->eg, p->tiles_per_unit};
    }
    if (!rc) rc = reserve_all(p);
    if (!rc) rc = build_tables(p);
    uncount_launches(stag_kde_launch_count() - before);  // tuning runs are not the caller's work
    if (rc) return rc;
    STAG_CUDA_TRY(cudaStreamSynchronize(p->cap));
    p->epochs.clear();
    for (auto *h : p->hs) p->epochs.push_back(h->scratch_epoch);
    // capture
    const uint64_t c0 = stag_kde_launch_count();
    STAG_CUDA_TRY(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
    rc = enqueue(p, p->cap);
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(p->h_err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, p->cap);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync(batch status)");
    }
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(p->cap, &g);
    const uint64_t c1 = stag_kde_launch_count();
    uncount_launches(c1 - c0);
    p->launches_per_run = c1 - c0;
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (ee != cudaSuccess) return cuda_fail(ee, "cudaStreamEndCapture");
    p->graph = g;
    STAG_CUDA_TRY(cudaGraphInstantiate(&p->exec, p->graph, 0));
    return 0;
}

}  // namespace

void batch_forget_handle(stag_kde *h) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto it = g_plans.begin(); it != g_plans.end();) {
        BatchPlan *p = *it;
        if (std::find(p->hs.begin(), p->hs.end(), h) != p->hs.end()) {
            free_plan(p);
            it = g_plans.erase(it);
        } else {
            ++it;
        }
    }
}

}  // namespace stagkde

using namespace stagkde;

extern "C" int stag_kde_autotune(stag_kde_t *h, const void *dQ, int64_t m) {
    if (!h || !dQ || m < 1) return fail(STAG_KDE_EINVAL, "autotune needs a handle and a non-empty query batch");
    if (h->form != STAG_KDE_FORM_TC) return 0;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != h->device) cudaSetDevice(h->device);
    const int egs[] = {2, 4};
    const int tpus[] = {0, 16, 32, 64, 128};
    double *dout = nullptr;
    cudaError_t e = dev_malloc(&dout, m * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(e, "dev_malloc(autotune)");
    const uint64_t before = stag_kde_launch_count();
    const int keep_eg = h->tune_eg, keep_tpu = h->tune_tiles_per_unit;
    double best = 1e300;
    int best_eg = keep_eg, best_tpu = keep_tpu, rc = 0;
    for (int eg : egs) {
        for (int tpu : tpus) {
            h->tune_eg = eg;
            h->tune_tiles_per_unit = tpu;
            if ((rc = stag_kde_query_dev(h, dQ, m, dout, h->stream))) break;  // warm-up
            stag_kde_profile_begin(h);
            if ((rc = stag_kde_query_dev(h, dQ, m, dout, h->stream))) break;
            double ms = 0.0;
            if ((rc = stag_kde_profile_end(h, &ms, nullptr, nullptr))) break;
            if (ms < best) {
                best = ms;
                best_eg = eg;
                best_tpu = tpu;
            }
        }
        if (rc) break;
    }
    cudaStreamSynchronize(h->stream);
    cudaFree(dout);
    uncount_launches(stag_kde_launch_count() - before);
    h->tune_eg = rc ? keep_eg : best_eg;
    h->tune_tiles_per_unit = rc ? keep_tpu : best_tpu;
    if (prev != h->device && prev >= 0) cudaSetDevice(prev);
    return rc;
}

extern "C" int stag_kde_query_batch(stag_kde_t *const *hs, const void *const *dQs, const int64_t *ms,
                                    double *const *dOuts, int64_t count, void *stream) {
    if (count < 0) return fail(STAG_KDE_EINVAL, "count < 0");
    if (count == 0) return 0;
    if (!hs || !dQs || !ms || !dOuts) return fail(STAG_KDE_EINVAL, "NULL array argument");
    const int device = hs[0] ? hs[0]->device : -1;
    std::vector<uintptr_t> key;
    for (int64_t i = 0; i < count; ++i) {
        if (!hs[i]) return fail(STAG_KDE_EINVAL, "NULL handle in batch");
        if (hs[i]->device != device) return fail(STAG_KDE_EINVAL, "batch handles must share one device");
        if (ms[i] < 0) return fail(STAG_KDE_EINVAL, "m < 0 in batch");
        if (ms[i] > 0 && (!dQs[i] || !dOuts[i])) return fail(STAG_KDE_EINVAL, "NULL query or output in batch");
        for (int64_t j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return fail(STAG_KDE_EINVAL, "a handle may appear once per batch");
        key.push_back((uintptr_t)hs[i]);
        key.push_back((uintptr_t)dQs[i]);
        key.push_back((uintptr_t)ms[i]);
        key.push_back((uintptr_t)dOuts[i]);
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return fail(STAG_KDE_ECUDA, "cudaSetDevice failed");
    struct Restore {
        int dev;
        ~Restore() {
            if (dev >= 0) cudaSetDevice(dev);
        }
    } restore{prev != device ? prev : -1};

    std::lock_guard<std::mutex> lk(g_mu);
    BatchPlan *plan = nullptr;
    for (auto it = g_plans.begin(); it != g_plans.end(); ++it) {
        if ((*it)->key == key) {
            plan = *it;
            g_plans.erase(it);
            break;
        }
    }
    if (plan) {
        // a handle whose scratch moved since the capture invalidates the graph
        bool stale = false;
        for (size_t i = 0; i < plan->hs.size(); ++i) stale |= plan->hs[i]->scratch_epoch != plan->epochs[i];
        if (*plan->h_err) {
            *plan->h_err = 0;
            cudaMemset(plan->d_err, 0, sizeof(int));
            g_plans.push_front(plan);
            return fail(STAG_KDE_ETIMEDOUT, "a bounded wait expired in the previous run of this batch");
        }
        if (stale) {
            free_plan(plan);
            plan = nullptr;
        }
    }
    if (!plan) {
        plan = new BatchPlan();
        plan->key = key;
        plan->device = device;
        for (int64_t i = 0; i < count; ++i) {
            plan->wait_ns = std::max<uint64_t>(plan->wait_ns, hs[i]->wait_ns);
            plan->hs.push_back(hs[i]);
            plan->qs.push_back(dQs[i]);
            plan->ms.push_back(ms[i]);
            plan->outs.push_back(dOuts[i]);
        }
        int rc = build_plan(plan);
        if (rc) {
            free_plan(plan);
            return rc;
        }
        while (g_plans.size() >= kMaxPlans) {
            free_plan(g_plans.back());
            g_plans.pop_back();
        }
    }
    g_plans.push_front(plan);
    cudaError_t e = cudaGraphLaunch(plan->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    count_launch((int)plan->launches_per_run);
    return 0;
}
