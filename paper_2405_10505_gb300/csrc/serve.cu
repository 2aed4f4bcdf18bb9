// Serving loop (fblts_server_*).  Scenario requests arrive over time, each on
// a resident mesh (shared between requests) with its own parameters, initial
// state and duration in coarse steps.  The server admits them first come,
// first served while their device states fit a byte budget, keeps every
// admitted state resident, and advances each on its own stream with its
// captured coarse step, so the work of all running requests overlaps on the
// GPU.  Batching is continuous at coarse-step granularity: a request that
// arrives while others run starts as soon as memory allows, without waiting
// for a round to end, and a finished one frees its memory for the queue.
// fblts_server_progress never blocks: it polls each running request's event,
// issues its next steps, retires finished requests and admits queued ones.
// Oldest first: each progress call ranks the running requests by admission
// and issues request r's steps on a stream of the r-th highest priority (the
// request's work stays ordered through its own event), so the GPU's block
// scheduler favours the oldest requests' kernels and the younger ones fill
// the remaining capacity: time-to-result stays close to first come, first
// served, while the overlap still raises throughput.
#include <algorithm>
#include <chrono>
#include <deque>
#include <new>
#include <unordered_map>
#include <vector>

#include "handles.h"

using namespace fblts;

namespace {

enum ReqStatus : int32_t { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2, RQ_FAILED = 3, RQ_TAKEN = 4 };

struct Request {
    fblts_request_desc d{};
    size_t bytes = 0;
    int64_t cu_per_step = 0;
    fblts_state *st = nullptr;
    cudaEvent_t ev = nullptr;
    int64_t done = 0, inflight = 0;
    int32_t status = RQ_QUEUED;
    fblts_status err = FBLTS_OK;
    double t_submit = 0, t_admit = 0, t_done = 0;
};

}  // namespace

struct fblts_server {
    fblts_server_opts o{};
    // issue streams by rank of age (rank 0 = oldest running request = the
    // highest priority the device offers), created on demand
    std::vector<cudaStream_t> rank_st;
    int prio_least = 0, prio_greatest = 0;
    std::chrono::steady_clock::time_point t0;
    std::unordered_map<int64_t, Request> reqs;
    std::deque<int64_t> queue;
    std::vector<int64_t> running;
    size_t in_use = 0, peak = 0;
    int64_t next_id = 1, finished = 0, cell_updates = 0, max_running = 0;

    double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

// frees the request's device state (its memory returns to the budget) and
// its hold on the mesh
static void release(fblts_server *srv, Request &r) {
    if (r.d.mesh) r.d.mesh->holds.fetch_sub(1);
    r.d.mesh = nullptr;
    if (r.ev) cudaEventDestroy(r.ev);
    r.ev = nullptr;
    if (r.st) {
        fblts_state_destroy(r.st);
        srv->in_use -= r.bytes;
    }
    r.st = nullptr;
}

extern "C" fblts_status fblts_server_create(const fblts_server_opts *opts, fblts_server **out) {
    if (!out) { set_error("server_create: out is NULL"); return FBLTS_E_ARG; }
    *out = nullptr;
    fblts_server *srv = new (std::nothrow) fblts_server();
    if (!srv) { set_error("server_create: host allocation failed"); return FBLTS_E_OOM; }
    if (opts) srv->o = *opts;
    if (srv->o.steps_per_issue <= 0) srv->o.steps_per_issue = 1;
    if (srv->o.max_active < 0) { delete srv; set_error("server_create: max_active < 0"); return FBLTS_E_ARG; }
    if (cudaDeviceGetStreamPriorityRange(&srv->prio_least, &srv->prio_greatest) != cudaSuccess) {
        cudaGetLastError();
        srv->prio_least = srv->prio_greatest = 0;
    }
    srv->t0 = std::chrono::steady_clock::now();
    *out = srv;
    return FBLTS_OK;
}

// the issue stream of age rank k (priority greatest + k, clamped to least)
static cudaStream_t rank_stream(fblts_server *srv, size_t k) {
    while (srv->rank_st.size() <= k) {
        const int r = (int)srv->rank_st.size();
        const int prio = std::min(srv->prio_least, srv->prio_greatest + r);
        cudaStream_t x = nullptr;
        if (cudaStreamCreateWithPriority(&x, cudaStreamNonBlocking, prio) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        srv->rank_st.push_back(x);
    }
    return srv->rank_st[k];
}

// issues n coarse steps of request r on stream x after its earlier work, then
// the state check, and records r.ev; the state's own stream waits for r.ev
// so that later calls on the state (read, synchronize) see the steps
static fblts_status issue(fblts_server *srv, Request &r, cudaStream_t x, int64_t n) {
    fblts_state *s = r.st;
    if (!x || !s->gexec) {
        fblts_status st = fblts_lts_advance(s, n);
        if (st == FBLTS_OK && cudaEventRecord(r.ev, s->st) != cudaSuccess) st = FBLTS_E_CUDA;
        return st;
    }
    CK(cudaStreamWaitEvent(x, r.ev, 0));
    for (int64_t i = 0; i < n; ++i) CK(cudaGraphLaunch(s->gexec, x));
    CK(launch_check(s->arr.a[A_H], s->dm.bottom, s->mesh->hm.nC, s->arr.a[A_U], s->mesh->hm.nE, s->d_flag, x));
    s->steps += n;
    CK(cudaEventRecord(r.ev, x));
    CK(cudaStreamWaitEvent(s->st, r.ev, 0));
    (void)srv;
    return FBLTS_OK;
}

extern "C" fblts_status fblts_server_destroy(fblts_server *srv) {
    if (!srv) return FBLTS_OK;
    for (auto &kv : srv->reqs) {
        if (kv.second.ev) cudaEventSynchronize(kv.second.ev);   // work issued on the rank streams
        release(srv, kv.second);
    }
    for (cudaStream_t x : srv->rank_st) cudaStreamDestroy(x);
    delete srv;
    return FBLTS_OK;
}

extern "C" fblts_status fblts_server_submit(fblts_server *srv, const fblts_request_desc *req, int64_t *id) {
    if (!srv || !req || !id) { set_error("server_submit: NULL argument"); return FBLTS_E_ARG; }
    if (!req->mesh || !req->h0 || !req->u0 || !req->bottom || req->n_steps < 0) {
        set_error("server_submit: request needs a mesh, h0, u0, bottom and n_steps >= 0");
        return FBLTS_E_ARG;
    }
    if (req->params.stream) {
        set_error("server_submit: params.stream must be NULL (each request gets a stream of its own)");
        return FBLTS_E_ARG;
    }
    Request r;
    r.d = *req;
    r.d.params.use_graph = 1;
    fblts_status st = fblts_state_device_bytes(req->mesh, req->params.precision, &r.bytes);
    if (st != FBLTS_OK) return st;
    if (srv->o.hbm_budget && r.bytes > srv->o.hbm_budget) {
        set_error("server_submit: the request needs %zu bytes, more than the budget of %llu", r.bytes,
                  (unsigned long long)srv->o.hbm_budget);
        return FBLTS_E_OOM;
    }
    r.cu_per_step = req->mesh->hm.cell_updates_per_step;
    r.t_submit = srv->now();
    req->mesh->holds.fetch_add(1);
    const int64_t k = srv->next_id++;
    srv->reqs.emplace(k, r);
    srv->queue.push_back(k);
    *id = k;
    return FBLTS_OK;
}

extern "C" fblts_status fblts_server_progress(fblts_server *srv, int32_t *n_finished) {
    if (!srv) { set_error("server_progress: NULL server"); return FBLTS_E_ARG; }
    int32_t fin = 0;
    // running requests, oldest first: account the steps that completed, retire or issue more
    std::vector<int64_t> still;
    size_t rank = 0;
    for (int64_t k : srv->running) {
        Request &r = srv->reqs[k];
        bool active = true;
        if (r.inflight > 0) {
            const cudaError_t q = cudaEventQuery(r.ev);
            if (q == cudaErrorNotReady) {
                still.push_back(k);
                ++rank;
                continue;
            }
            if (q != cudaSuccess) {
                r.status = RQ_FAILED;
                r.err = FBLTS_E_CUDA;
                r.t_done = srv->now();
                active = false;
            } else {
                r.done += r.inflight;
                srv->cell_updates += r.inflight * r.cu_per_step;
                r.inflight = 0;
            }
        }
        if (active && r.done >= r.d.n_steps) {
            r.err = fblts_synchronize(r.st);           // the stream is idle: checks the state
            r.status = r.err == FBLTS_OK ? RQ_DONE : RQ_FAILED;
            r.t_done = srv->now();
            active = false;
        }
        if (active) {
            const int64_t n = std::min<int64_t>(r.d.n_steps - r.done, srv->o.steps_per_issue);
            fblts_status st = issue(srv, r, rank_stream(srv, rank), n);
            if (st != FBLTS_OK) {
                r.status = RQ_FAILED;
                r.err = st;
                r.t_done = srv->now();
                active = false;
            } else {
                r.inflight = n;
            }
        }
        if (active) {
            still.push_back(k);
            ++rank;
        } else {
            ++fin;
        }
    }
    srv->running.swap(still);
    // admission, first come first served, while memory and the active cap allow
    while (!srv->queue.empty()) {
        const int64_t k = srv->queue.front();
        Request &r = srv->reqs[k];
        if (srv->o.hbm_budget && srv->in_use + r.bytes > srv->o.hbm_budget) break;
        if (srv->o.max_active && (int64_t)srv->running.size() >= srv->o.max_active) break;
        srv->queue.pop_front();
        r.t_admit = srv->now();
        fblts_status st = fblts_state_init(r.d.mesh, &r.d.params, r.d.h0, r.d.u0, r.d.bottom, &r.st);
        if (st == FBLTS_OK && cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming) != cudaSuccess) {
            fblts_state_destroy(r.st);
            r.st = nullptr;
            st = FBLTS_E_CUDA;
        }
        if (st != FBLTS_OK) {
            r.status = RQ_FAILED;
            r.err = st;
            r.t_done = srv->now();
            ++fin;
            continue;
        }
        srv->in_use += r.bytes;
        srv->peak = std::max(srv->peak, srv->in_use);
        r.status = RQ_RUNNING;
        if (r.d.n_steps == 0) {
            r.status = RQ_DONE;
            r.t_done = srv->now();
            ++fin;
            continue;
        }
        const int64_t n = std::min<int64_t>(r.d.n_steps, srv->o.steps_per_issue);
        // the first issue follows the state's initialisation on its own stream
        if (cudaEventRecord(r.ev, r.st->st) != cudaSuccess) st = FBLTS_E_CUDA;
        if (st == FBLTS_OK) st = issue(srv, r, rank_stream(srv, srv->running.size()), n);
        if (st != FBLTS_OK) {
            r.status = RQ_FAILED;
            r.err = st;
            r.t_done = srv->now();
            ++fin;
            continue;
        }
        r.inflight = n;
        srv->running.push_back(k);
    }
    srv->max_running = std::max<int64_t>(srv->max_running, (int64_t)srv->running.size());
    srv->finished += fin;
    if (n_finished) *n_finished = fin;
    return FBLTS_OK;
}

extern "C" fblts_status fblts_server_request_info(const fblts_server *srv, int64_t id, fblts_request_info *info) {
    if (!srv || !info) { set_error("server_request_info: NULL argument"); return FBLTS_E_ARG; }
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) { set_error("server_request_info: unknown request %lld", (long long)id); return FBLTS_E_ARG; }
    const Request &r = it->second;
    info->status = r.status;
    info->error = r.err;
    info->steps_done = r.done;
    info->n_steps = r.d.n_steps;
    info->device_bytes = r.bytes;
    info->t_submit = r.t_submit;
    info->t_admit = r.t_admit;
    info->t_done = r.t_done;
    return FBLTS_OK;
}

extern "C" fblts_status fblts_server_take(fblts_server *srv, int64_t id, double *h_out, double *u_out) {
    if (!srv) { set_error("server_take: NULL server"); return FBLTS_E_ARG; }
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) { set_error("server_take: unknown request %lld", (long long)id); return FBLTS_E_ARG; }
    Request &r = it->second;
    if (r.status == RQ_FAILED) {
        release(srv, r);
        r.status = RQ_TAKEN;
        set_error("server_take: request %lld failed", (long long)id);
        return r.err != FBLTS_OK ? r.err : FBLTS_E_STATE;
    }
    if (r.status != RQ_DONE) { set_error("server_take: request %lld is not finished", (long long)id); return FBLTS_E_STATE; }
    fblts_status st = FBLTS_OK;
    if (h_out || u_out) st = fblts_state_read(r.st, h_out, u_out);
    release(srv, r);
    r.status = RQ_TAKEN;
    return st;
}

extern "C" fblts_status fblts_server_get_stats(const fblts_server *srv, fblts_server_stats *s) {
    if (!srv || !s) { set_error("server_get_stats: NULL argument"); return FBLTS_E_ARG; }
    s->queued = (int64_t)srv->queue.size();
    s->running = (int64_t)srv->running.size();
    s->finished = srv->finished;
    s->max_running = srv->max_running;
    s->device_bytes_in_use = srv->in_use;
    s->device_bytes_peak = srv->peak;
    s->cell_updates = srv->cell_updates;
    s->t_now = srv->now();
    return FBLTS_OK;
}
