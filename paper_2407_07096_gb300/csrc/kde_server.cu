// Serving: exact KDE queries against resident datasets with continuous batching.
//
// The caller registers datasets (handles it created) and submits query batches from any
// thread. A dispatcher thread forms launch groups: it takes the oldest pending request,
// then every other pending request for the same dataset, in arrival order, while the
// rows stay within `max_rows`. A group is admitted when a slot is free and the device
// memory budget of the groups in flight allows it. Each slot owns a CUDA stream, pinned
// staging buffers and a view of every dataset (same resident data, separate scratch), so
// groups in different slots run concurrently on the device while new requests keep
// arriving. A host callback at the end of each group's stream work copies the results
// out, records each request's latency (submit to completion) and frees the slot.
//
// Every query row is computed independently of the other rows of its group, so a
// request's result is the same alone or coalesced with others (to the form's tolerance;
// bitwise when the work split does not change).
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace stagkde {
namespace {

using Clock = std::chrono::steady_clock;

struct SrvRequest {
    uint64_t ticket = 0;
    int dataset = 0;
    const void *Q = nullptr;
    int64_t m = 0;
    double *out = nullptr;
    Clock::time_point t_submit, t_done;
    int status = 1;  // 1 pending/running, 0 done, < 0 error code
    bool done = false;
};

struct Slot {
    cudaStream_t stream = nullptr;
    std::vector<stag_kde *> views;  // per dataset, created on first use
    void *dq = nullptr;             // device queries of the group
    double *dout = nullptr;         // device results of the group
    void *hq = nullptr;             // pinned staging
    double *hout = nullptr;
    std::vector<SrvRequest *> group;
    int64_t mem = 0;
    bool busy = false;
    void *srv = nullptr;  // owning server
};

}  // namespace
}  // namespace stagkde

struct stag_srv {
    std::vector<stag_kde *> datasets;
    int device = 0;
    int64_t max_rows = 8192;
    int64_t mem_budget = 1ll << 30;
    size_t max_elem = 4;
    int64_t max_d = 1;
    std::vector<stagkde::Slot> slots;
    std::mutex mu;
    std::condition_variable cv;        // dispatcher wake-up
    std::condition_variable done_cv;   // waiters
    std::deque<stagkde::SrvRequest *> pending;
    std::unordered_map<uint64_t, stagkde::SrvRequest *> reqs;
    uint64_t next_ticket = 1;
    int64_t inflight_mem = 0;
    bool stopping = false;
    std::thread worker;
    std::vector<double> latencies_us;  // completed requests
    int64_t rows_done = 0;
};

namespace stagkde {
namespace {

size_t elem_bytes(const stag_kde *h) { return h->dtype == STAG_KDE_F64 ? 8 : 4; }

// Device bytes a group of `rows` queries keeps busy: its queries and results plus the
// per-row scratch of the query path (row terms for the tensor-core form).
int64_t group_bytes(const stag_kde *h, int64_t rows) {
    int64_t per_row = h->d * (int64_t)elem_bytes(h) + 8;
    if (h->form == STAG_KDE_FORM_TC) per_row += ceil_div(h->n, tc_tile_points(h->d)) * 4 + 2 * 128 * 2 + 40;
    else per_row += 12 * std::max<int64_t>(1, h->n_tiles / 8);
    return rows * per_row;
}

void CUDART_CB on_group_done(void *arg);

// Launches one admitted group on its slot (called without the server lock held).
int launch_group(stag_srv *srv, Slot &sl) {
    const int ds = sl.group.front()->dataset;
    stag_kde *base = srv->datasets[ds];
    if (!sl.views[ds]) {
        stag_kde *v = make_view(base);
        if (!v) return STAG_KDE_ENOMEM;
        int rc = stag_kde_reserve(v, srv->max_rows);
        if (rc) {
            free_view(v);
            return rc;
        }
        sl.views[ds] = v;
    }
    stag_kde *v = sl.views[ds];
    const size_t eb = elem_bytes(base);
    int64_t rows = 0;
    for (SrvRequest *r : sl.group) {
        memcpy((char *)sl.hq + rows * base->d * eb, r->Q, r->m * base->d * eb);
        rows += r->m;
    }
    STAG_CUDA_TRY(cudaMemcpyAsync(sl.dq, sl.hq, rows * base->d * eb, cudaMemcpyHostToDevice, sl.stream));
    int rc = stag_kde_query_dev(v, sl.dq, rows, sl.dout, sl.stream);
    if (rc) return rc;
    STAG_CUDA_TRY(cudaMemcpyAsync(sl.hout, sl.dout, rows * 8, cudaMemcpyDeviceToHost, sl.stream));
    STAG_CUDA_TRY(cudaLaunchHostFunc(sl.stream, on_group_done, &sl));
    return 0;
}

void finish_group(stag_srv *srv, Slot &sl, int status) {
    // called with srv->mu held
    const Clock::time_point now = Clock::now();
    int64_t off = 0;
    for (SrvRequest *r : sl.group) {
        if (status == 0) memcpy(r->out, sl.hout + off, r->m * 8);
        off += r->m;
        r->status = status;
        r->done = true;
        r->t_done = now;
        if (status == 0) {
            srv->latencies_us.push_back(std::chrono::duration<double, std::micro>(now - r->t_submit).count());
            srv->rows_done += r->m;
        }
    }
    sl.group.clear();
    sl.busy = false;
    srv->inflight_mem -= sl.mem;
    sl.mem = 0;
    srv->done_cv.notify_all();
    srv->cv.notify_all();
}

void CUDART_CB on_group_done(void *arg) {
    Slot *sl = static_cast<Slot *>(arg);
    stag_srv *srv = static_cast<stag_srv *>(sl->srv);
    std::lock_guard<std::mutex> lk(srv->mu);
    finish_group(srv, *sl, 0);
}

void dispatcher(stag_srv *srv) {
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    while (true) {
        Slot *free_slot = nullptr;
        for (auto &s : srv->slots)
            if (!s.busy) {
                free_slot = &s;
                break;
            }
        if (srv->stopping && srv->pending.empty()) break;
        if (srv->pending.empty() || !free_slot) {
            srv->cv.wait(lk);
            continue;
        }
        // group: the oldest request, then later ones for the same dataset
        const int ds = srv->pending.front()->dataset;
        stag_kde *h = srv->datasets[ds];
        std::vector<SrvRequest *> group;
        int64_t rows = 0;
        for (SrvRequest *r : srv->pending) {
            if (r->dataset != ds) continue;
            if (!group.empty() && rows + r->m > srv->max_rows) break;
            group.push_back(r);
            rows += r->m;
        }
        const int64_t need = group_bytes(h, rows);
        if (srv->inflight_mem > 0 && srv->inflight_mem + need > srv->mem_budget) {
            srv->cv.wait(lk);  // wait for memory to be released by a finishing group
            continue;
        }
        for (SrvRequest *r : group) srv->pending.erase(std::find(srv->pending.begin(), srv->pending.end(), r));
        free_slot->busy = true;
        free_slot->group = group;
        free_slot->mem = need;
        srv->inflight_mem += need;
        lk.unlock();
        const int rc = launch_group(srv, *free_slot);
        lk.lock();
        if (rc) finish_group(srv, *free_slot, rc);
    }
    // drain: wait until every slot is idle
    srv->done_cv.wait(lk, [&] {
        for (auto &s : srv->slots)
            if (s.busy) return false;
        return true;
    });
}

void destroy_server(stag_srv *srv) {
    cudaSetDevice(srv->device);
    for (auto &s : srv->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        for (stag_kde *v : s.views)
            if (v) free_view(v);
        cudaFree(s.dq);
        cudaFree(s.dout);
        if (s.hq) cudaFreeHost(s.hq);
        if (s.hout) cudaFreeHost(s.hout);
        if (s.stream) cudaStreamDestroy(s.stream);
    }
    for (auto &kv : srv->reqs) delete kv.second;
    delete srv;
}

}  // namespace
}  // namespace stagkde

using namespace stagkde;

extern "C" {

void stag_srv_opts_init(stag_srv_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->slots = 4;
    o->max_rows = 8192;
    o->mem_budget_bytes = 1ll << 30;
}

stag_srv_t *stag_srv_start(const stag_srv_opts *o) {
    if (!o || !o->datasets || o->n_datasets < 1) return (set_error("need at least one dataset"), nullptr);
    if (o->slots < 1 || o->slots > 64) return (set_error("slots must be in 1..64"), nullptr);
    if (o->max_rows < 1 || o->mem_budget_bytes < 1) return (set_error("max_rows and mem_budget_bytes must be > 0"), nullptr);
    stag_srv *srv = new (std::nothrow) stag_srv();
    if (!srv) return (set_error("out of host memory"), nullptr);
    srv->max_rows = o->max_rows;
    srv->mem_budget = o->mem_budget_bytes;
    for (int i = 0; i < o->n_datasets; ++i) {
        stag_kde *h = o->datasets[i];
        if (!h) {
            delete srv;
            return (set_error("NULL dataset handle"), nullptr);
        }
        if (i > 0 && h->device != o->datasets[0]->device) {
            delete srv;
            return (set_error("datasets must share one device"), nullptr);
        }
        srv->datasets.push_back(h);
        srv->max_elem = std::max(srv->max_elem, elem_bytes(h));
        srv->max_d = std::max(srv->max_d, h->d);
    }
    srv->device = srv->datasets[0]->device;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(srv->device);
    srv->slots.resize(o->slots);
    const int64_t qbytes = srv->max_rows * srv->max_d * (int64_t)srv->max_elem;
    for (auto &s : srv->slots) {
        s.srv = srv;
        s.views.assign(srv->datasets.size(), nullptr);
        cudaError_t e;
        if ((e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = dev_malloc(&s.dq, qbytes)) != cudaSuccess ||
            (e = dev_malloc(&s.dout, srv->max_rows * 8)) != cudaSuccess ||
            (e = cudaMallocHost(&s.hq, qbytes)) != cudaSuccess ||
            (e = cudaMallocHost(&s.hout, srv->max_rows * 8)) != cudaSuccess) {
            cuda_fail(e, "server slot set-up");
            destroy_server(srv);
            if (prev >= 0) cudaSetDevice(prev);
            return nullptr;
        }
    }
    if (prev >= 0) cudaSetDevice(prev);
    srv->worker = std::thread(dispatcher, srv);
    return srv;
}

int stag_srv_submit(stag_srv_t *srv, int dataset, const void *Q, int64_t m, double *out, uint64_t *ticket) {
    if (!srv || !ticket) return fail(STAG_KDE_EINVAL, "server or ticket is NULL");
    if (dataset < 0 || dataset >= (int)srv->datasets.size()) return fail(STAG_KDE_EINVAL, "unknown dataset");
    if (m < 1 || m > srv->max_rows) return fail(STAG_KDE_EINVAL, "m must be in 1..max_rows");
    if (!Q || !out) return fail(STAG_KDE_EINVAL, "Q or out is NULL");
    SrvRequest *r = new (std::nothrow) SrvRequest();
    if (!r) return fail(STAG_KDE_ENOMEM, "out of host memory");
    r->dataset = dataset;
    r->Q = Q;
    r->m = m;
    r->out = out;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stopping) {
            delete r;
            return fail(STAG_KDE_ECANCELED, "server is stopping");
        }
        r->ticket = srv->next_ticket++;
        srv->reqs[r->ticket] = r;
        srv->pending.push_back(r);
        *ticket = r->ticket;
    }
    srv->cv.notify_all();
    return 0;
}

int stag_srv_cancel(stag_srv_t *srv, uint64_t ticket) {
    if (!srv) return fail(STAG_KDE_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return fail(STAG_KDE_EINVAL, "unknown ticket");
    SrvRequest *r = it->second;
    auto p = std::find(srv->pending.begin(), srv->pending.end(), r);
    if (p == srv->pending.end()) return fail(STAG_KDE_EINVAL, "request already running or done");
    srv->pending.erase(p);
    r->status = STAG_KDE_ECANCELED;
    r->done = true;
    srv->done_cv.notify_all();
    return 0;
}

int stag_srv_wait(stag_srv_t *srv, uint64_t ticket, int64_t timeout_us) {
    if (!srv) return fail(STAG_KDE_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return fail(STAG_KDE_EINVAL, "unknown ticket");
    SrvRequest *r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_us < 0)
        srv->done_cv.wait(lk, ready);
    else if (!srv->done_cv.wait_for(lk, std::chrono::microseconds(timeout_us), ready))
        return fail(STAG_KDE_ETIMEDOUT, "request not finished within the timeout");
    const int st = r->status;
    srv->reqs.erase(it);
    delete r;
    if (st < 0) return fail(st, "request failed or was cancelled");
    return 0;
}

int stag_srv_stats(stag_srv_t *srv, int64_t *completed, int64_t *rows, double *p50_us, double *p99_us) {
    if (!srv) return fail(STAG_KDE_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(srv->mu);
    std::vector<double> v = srv->latencies_us;
    if (completed) *completed = (int64_t)v.size();
    if (rows) *rows = srv->rows_done;
    double p50 = 0.0, p99 = 0.0;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        p50 = v[(size_t)(0.50 * (v.size() - 1))];
        p99 = v[(size_t)(0.99 * (v.size() - 1))];
    }
    if (p50_us) *p50_us = p50;
    if (p99_us) *p99_us = p99;
    return 0;
}

int stag_srv_reset_stats(stag_srv_t *srv) {
    if (!srv) return fail(STAG_KDE_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->latencies_us.clear();
    srv->rows_done = 0;
    return 0;
}

int stag_srv_stop(stag_srv_t *srv) {
    if (!srv) return 0;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stopping = true;
        // requests not yet dispatched are cancelled
        for (SrvRequest *r : srv->pending) {
            r->status = STAG_KDE_ECANCELED;
            r->done = true;
        }
        srv->pending.clear();
    }
    srv->cv.notify_all();
    srv->done_cv.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    destroy_server(srv);
    return 0;
}

}  // extern "C"
