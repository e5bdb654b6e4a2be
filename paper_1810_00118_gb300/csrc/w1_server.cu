// w1_server.cu -- continuous-batching request loop for W1 solves.
//
// Requests (one density pair each, any grid size, either norm) are submitted
// from any host thread and polled by ticket.  A worker thread owns the GPU
// side:
//   * Requests are grouped by size class (grid, spacing, levels, norm, tol).
//   * A slot is one plan (device-resident multilevel state for up to
//     max_batch pairs of one class), its own stream and its input staging.
//     Slots are created on demand while the device memory they hold stays
//     within the HBM budget; idle slots of other classes are evicted (least
//     recently used) to make room.
//   * Whenever a slot is free, the oldest queued requests of its class are
//     copied into its staging buffer and solved asynchronously on its stream.
//     Several slots are in flight at once, so requests that arrive while
//     others run start as soon as a slot and memory free up, and their work
//     overlaps on the device.
//   * A host callback at the end of each slot's stream work wakes the worker,
//     which moves the results to the finished table.
// A pair is solved by the same kernels with the same per-pair reduction order
// whatever else is in flight, so its result does not depend on the mix.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "w1_internal.h"

namespace {

thread_local std::string g_srv_err;

w1_status srv_fail(w1_status s, const std::string& m)
{
    g_srv_err = m;
    return s;
}

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Key {
    int nx, ny, levels, norm;
    double h, tol;
    bool operator==(const Key& o) const
    {
        return nx == o.nx && ny == o.ny && levels == o.levels && norm == o.norm && h == o.h && tol == o.tol;
    }
};

struct Request {
    uint64_t ticket;
    Key key;
    const float* rho0;
    const float* rho1;
    double t_submit;
};

struct Result {
    w1_status status;
    double dist;
    w1_stats stats;
    double t_submit, t_done;
};

struct Slot {
    w1_server* srv = nullptr;
    Key key{};
    int flavour = 0;  // 0: the configured options; 1: kernels autotuned for one solve alone
    w1_plan* plan = nullptr;
    cudaStream_t stream = nullptr;
    float* in0 = nullptr;
    float* in1 = nullptr;
    size_t bytes = 0;
    bool busy = false;
    std::atomic<bool> done{false};
    std::vector<Request> reqs;
    double last_used = 0.0;
    nvtxRangeId_t nvtx = 0;  // the in-flight batch on the host timeline
};

}  // namespace

struct w1_server {
    int device = 0;
    size_t budget = 0;
    size_t in_use = 0;
    int max_slots = 0;
    int max_batch = 1;
    int latency_below = 0;
    w1_options opt{};
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> queue;
    std::vector<std::unique_ptr<Slot>> slots;
    std::unordered_map<uint64_t, Result> finished;
    std::unordered_map<uint64_t, int> pending;  // ticket -> 1 while queued or in flight
    uint64_t next_ticket = 1;
    uint64_t generation = 0;  // bumped by every submission
    bool stop = false;
    std::thread worker;
    long long submitted = 0, completed = 0, rejected = 0, evictions = 0;
    std::string worker_error;
};

namespace {

void CUDART_CB on_slot_done(void* arg)
{
    Slot* s = static_cast<Slot*>(arg);
    s->done.store(true);
    // Wake the worker.  No CUDA call is allowed here, and the server mutex is
    // not taken: the worker may hold it while it synchronises this very stream
    // (slot eviction), which would deadlock.  A wake-up lost to the race is
    // picked up by the worker's 1 ms wait timeout.
    s->srv->cv.notify_all();
}

// Plan options of a slot flavour: flavour 1 lets the autotuner pick each level's
// kernel for one solve with the GPU otherwise idle (w1_options.tune = 1), where
// the configured options leave that choice open.
w1_options slot_options(const w1_server* srv, int flavour)
{
    w1_options o = srv->opt;
    if (flavour == 1 && o.path == 0 && o.algorithm != 4) o.tune = 1;
    return o;
}

size_t slot_bytes(const w1_server* srv, const Key& k, int flavour)
{
    const w1_options o = slot_options(srv, flavour);
    const size_t plan = w1_plan_bytes(k.nx, k.ny, k.h, k.levels, k.norm, k.tol, srv->max_batch, &o);
    if (plan == 0) return 0;
    return plan + 2 * (size_t)k.nx * k.ny * sizeof(float) * srv->max_batch;
}

void destroy_slot(Slot* s)
{
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->plan) w1_plan_destroy(s->plan);
    if (s->in0) cudaFree(s->in0);
    if (s->in1) cudaFree(s->in1);
    if (s->stream) cudaStreamDestroy(s->stream);
    cudaGetLastError();
}

// Creates a slot for key k within the budget (evicting idle slots of other
// classes if needed); nullptr when the budget or the slot count is exhausted.
Slot* make_slot(w1_server* srv, const Key& k, int flavour)
{
    const size_t need = slot_bytes(srv, k, flavour);
    if (need == 0) return nullptr;
    for (;;) {
        const bool fits = srv->in_use + need <= srv->budget && (int)srv->slots.size() < srv->max_slots;
        if (fits) break;
        // evict the least recently used idle slot
        int victim = -1;
        for (int i = 0; i < (int)srv->slots.size(); ++i) {
            Slot* s = srv->slots[i].get();
            if (s->busy) continue;
            if (victim < 0 || s->last_used < srv->slots[victim]->last_used) victim = i;
        }
        if (victim < 0) return nullptr;
        Slot* v = srv->slots[victim].get();
        srv->in_use -= v->bytes;
        destroy_slot(v);
        srv->slots.erase(srv->slots.begin() + victim);
        ++srv->evictions;
    }
    auto s = std::make_unique<Slot>();
    s->srv = srv;
    s->key = k;
    s->flavour = flavour;
    s->bytes = need;
    const size_t nb = (size_t)k.nx * k.ny * sizeof(float) * srv->max_batch;
    const w1_options o = slot_options(srv, flavour);
    if (w1_plan_create_batch(k.nx, k.ny, k.h, k.levels, k.norm, k.tol, srv->max_batch, &o, &s->plan) != W1_OK ||
        cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&s->in0, nb) != cudaSuccess || cudaMalloc(&s->in1, nb) != cudaSuccess) {
        srv->worker_error = std::string("slot creation failed: ") + w1_last_error();
        destroy_slot(s.get());
        cudaGetLastError();
        return nullptr;
    }
    srv->in_use += need;
    srv->slots.push_back(std::move(s));
    return srv->slots.back().get();
}

void finish_slot(w1_server* srv, Slot* s)
{
    const int nb = (int)s->reqs.size();
    std::vector<double> dist(nb);
    std::vector<w1_stats> st(nb);
    std::vector<int> status(nb);
    w1_plan_results(s->plan, dist.data(), st.data(), status.data());
    const double t = now_s();
    for (int b = 0; b < nb; ++b) {
        const Request& r = s->reqs[b];
        Result res;
        res.status = (w1_status)status[b];
        res.dist = dist[b];
        res.stats = st[b];
        res.t_submit = r.t_submit;
        res.t_done = t;
        srv->finished[r.ticket] = res;
        srv->pending.erase(r.ticket);
        ++srv->completed;
    }
    nvtxRangeEnd(s->nvtx);
    s->reqs.clear();
    s->busy = false;
    s->done.store(false);
    s->last_used = t;
}

void fail_requests(w1_server* srv, std::vector<Request>& reqs, w1_status why)
{
    const double t = now_s();
    for (const Request& r : reqs) {
        Result res{};
        res.status = why;
        res.dist = 0.0;
        res.t_submit = r.t_submit;
        res.t_done = t;
        srv->finished[r.ticket] = res;
        srv->pending.erase(r.ticket);
    }
    reqs.clear();
}

// Starts as many queued requests as free or creatable slots allow.
void dispatch(w1_server* srv)
{
    std::vector<Key> blocked;
    auto is_blocked = [&](const Key& k) {
        for (const Key& b : blocked)
            if (b == k) return true;
        return false;
    };
    size_t i = 0;
    while (i < srv->queue.size()) {
        const Key k = srv->queue[i].key;
        if (is_blocked(k)) {
            ++i;
            continue;
        }
        // a lightly loaded GPU gets the latency-tuned flavour of the class
        int in_flight = 0;
        for (auto& s : srv->slots) in_flight += s->busy ? 1 : 0;
        const int flavour = in_flight < srv->latency_below ? 1 : 0;
        auto free_slot = [&](int f) -> Slot* {
            for (auto& s : srv->slots)
                if (!s->busy && s->key == k && s->flavour == f) return s.get();
            return nullptr;
        };
        Slot* slot = free_slot(flavour);
        if (!slot) slot = make_slot(srv, k, flavour);
        if (!slot && flavour == 1) {  // no room for a latency-tuned slot: the configured kind
            slot = free_slot(0);
            if (!slot) slot = make_slot(srv, k, 0);
        }
        if (!slot) {
            blocked.push_back(k);
            ++i;
            continue;
        }
        // the oldest requests of this class, up to max_batch
        slot->reqs.clear();
        for (size_t j = i; j < srv->queue.size() && (int)slot->reqs.size() < srv->max_batch;) {
            if (srv->queue[j].key == k) {
                slot->reqs.push_back(srv->queue[j]);
                srv->queue.erase(srv->queue.begin() + j);
            } else {
                ++j;
            }
        }
        const size_t n = (size_t)k.nx * k.ny;
        cudaError_t e = cudaSuccess;
        for (size_t b = 0; b < slot->reqs.size() && e == cudaSuccess; ++b) {
            e = cudaMemcpyAsync(slot->in0 + b * n, slot->reqs[b].rho0, n * sizeof(float), cudaMemcpyDeviceToDevice,
                                slot->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(slot->in1 + b * n, slot->reqs[b].rho1, n * sizeof(float),
                                    cudaMemcpyDeviceToDevice, slot->stream);
        }
        w1_status st = W1_ERR_CUDA;
        if (e == cudaSuccess)
            st = w1_solve_async(slot->plan, (int)slot->reqs.size(), slot->in0, slot->in1, slot->stream, nullptr);
        if (st == W1_OK) e = cudaLaunchHostFunc(slot->stream, on_slot_done, slot);
        if (st != W1_OK || e != cudaSuccess) {
            cudaGetLastError();
            srv->worker_error = std::string("dispatch failed: ") + w1_last_error();
            fail_requests(srv, slot->reqs, W1_ERR_CUDA);
            continue;
        }
        slot->busy = true;
        slot->last_used = now_s();
        {
            char name[96];
            std::snprintf(name, sizeof(name), "w1 request %llu %dx%d p%d x%d", (unsigned long long)slot->reqs[0].ticket,
                          k.nx, k.ny, k.norm, (int)slot->reqs.size());
            slot->nvtx = nvtxRangeStartA(name);
        }
    }
}

void worker_main(w1_server* srv)
{
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    uint64_t seen = 0;
    for (;;) {
        for (auto& s : srv->slots)
            if (s->busy && s->done.load()) finish_slot(srv, s.get());
        seen = srv->generation;
        if (!srv->queue.empty()) dispatch(srv);
        bool any_busy = false;
        for (auto& s : srv->slots) any_busy |= s->busy;
        if (srv->stop && srv->queue.empty() && !any_busy) break;
        // sleep until a slot finishes, a request arrives, or shutdown (1 ms at most)
        srv->cv.wait_for(lk, std::chrono::milliseconds(1), [&] {
            if (srv->stop || srv->generation != seen) return true;
            for (auto& s : srv->slots)
                if (s->busy && s->done.load()) return true;
            return false;
        });
        if (srv->stop) {
            // drop what has not started; finish what is in flight
            std::vector<Request> rest(srv->queue.begin(), srv->queue.end());
            srv->queue.clear();
            fail_requests(srv, rest, W1_ERR_INVALID_ARG);
        }
    }
    lk.unlock();
    for (auto& s : srv->slots) destroy_slot(s.get());
    srv->slots.clear();
}

}  // namespace

extern "C" void w1_server_default_config(w1_server_config* c)
{
    if (!c) return;
    c->hbm_budget_bytes = (size_t)40 << 30;
    c->max_slots = 32;
    c->max_batch = 1;
    w1_default_options(&c->opt);
    c->latency_below = 0;
}

extern "C" w1_status w1_server_create_ex(const w1_server_config* cfg, w1_server** out)
{
    if (!out) return srv_fail(W1_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    w1_server_config c;
    w1_server_default_config(&c);
    if (cfg) c = *cfg;
    if (c.max_slots < 1 || c.max_batch < 1 || c.hbm_budget_bytes == 0 || c.latency_below < 0)
        return srv_fail(W1_ERR_INVALID_ARG, "max_slots, max_batch and the budget must be positive");
    auto* srv = new (std::nothrow) w1_server();
    if (!srv) return srv_fail(W1_ERR_NOMEM, "host allocation failed");
    if (cudaGetDevice(&srv->device) != cudaSuccess) {
        cudaGetLastError();
        delete srv;
        return srv_fail(W1_ERR_CUDA, "cudaGetDevice failed");
    }
    srv->budget = c.hbm_budget_bytes;
    srv->max_slots = c.max_slots;
    srv->max_batch = c.max_batch;
    srv->latency_below = c.latency_below;
    srv->opt = c.opt;
    try {
        srv->worker = std::thread(worker_main, srv);
    } catch (...) {
        delete srv;
        return srv_fail(W1_ERR_NOMEM, "could not start the worker thread");
    }
    *out = srv;
    return W1_OK;
}

extern "C" w1_status w1_server_create(size_t hbm_budget_bytes, int max_slots, w1_server** out)
{
    w1_server_config c;
    w1_server_default_config(&c);
    if (hbm_budget_bytes) c.hbm_budget_bytes = hbm_budget_bytes;
    if (max_slots > 0) c.max_slots = max_slots;
    return w1_server_create_ex(&c, out);
}

extern "C" w1_status w1_submit(w1_server* srv, int nx, int ny, double h, int levels, int norm, double tol,
                               const float* rho0, const float* rho1, uint64_t* ticket)
{
    if (!srv || !rho0 || !rho1 || !ticket) return srv_fail(W1_ERR_INVALID_ARG, "NULL server, density or ticket");
    if (nx < 1 || ny < 1) return srv_fail(W1_ERR_INVALID_ARG, "nx and ny must be >= 1");
    if (norm != W1_NORM_L1 && norm != W1_NORM_L2 && norm != W1_NORM_LINF) return srv_fail(W1_ERR_INVALID_ARG, "norm must be 1, 2 or 3");
    if (!(h > 0.0)) h = 1.0 / (double)(nx > ny ? nx : ny);
    Key k{nx, ny, levels, norm, h, tol};
    const size_t need = slot_bytes(srv, k, 0);
    if (need == 0) return srv_fail(W1_ERR_SHAPE, std::string("request rejected: ") + w1_last_error());
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) return srv_fail(W1_ERR_INVALID_ARG, "server is shutting down");
    if (need > srv->budget) {
        ++srv->rejected;
        return srv_fail(W1_ERR_BUDGET, "request needs more device memory than the server's budget");
    }
    Request r{srv->next_ticket++, k, rho0, rho1, now_s()};
    srv->queue.push_back(r);
    srv->pending[r.ticket] = 1;
    ++srv->submitted;
    ++srv->generation;
    *ticket = r.ticket;
    srv->cv.notify_all();
    return W1_OK;
}

static w1_status take_result(w1_server* srv, uint64_t ticket, double* dist, w1_stats* stats, double* latency)
{
    auto it = srv->finished.find(ticket);
    if (it == srv->finished.end()) {
        if (srv->pending.count(ticket)) return W1_PENDING;
        return srv_fail(W1_ERR_INVALID_ARG, "unknown or already collected ticket");
    }
    const Result r = it->second;
    srv->finished.erase(it);
    if (dist) *dist = r.dist;
    if (stats) *stats = r.stats;
    if (latency) *latency = r.t_done - r.t_submit;
    return r.status;
}

extern "C" w1_status w1_poll(w1_server* srv, uint64_t ticket, double* dist, w1_stats* stats)
{
    if (!srv) return srv_fail(W1_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(srv->mu);
    return take_result(srv, ticket, dist, stats, nullptr);
}

extern "C" w1_status w1_poll_latency(w1_server* srv, uint64_t ticket, double* dist, w1_stats* stats,
                                     double* latency_s)
{
    if (!srv) return srv_fail(W1_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(srv->mu);
    return take_result(srv, ticket, dist, stats, latency_s);
}

extern "C" w1_status w1_wait(w1_server* srv, uint64_t ticket, double timeout_s, double* dist, w1_stats* stats)
{
    if (!srv) return srv_fail(W1_ERR_INVALID_ARG, "NULL server");
    const double end = now_s() + (timeout_s > 0 ? timeout_s : 1e30);
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        w1_status st = take_result(srv, ticket, dist, stats, nullptr);
        if (st != W1_PENDING) return st;
        if (now_s() >= end) return W1_PENDING;
        srv->cv.wait_for(lk, std::chrono::milliseconds(1));
    }
}

extern "C" w1_status w1_server_query(w1_server* srv, w1_server_info* info)
{
    if (!srv || !info) return srv_fail(W1_ERR_INVALID_ARG, "NULL server or info");
    std::lock_guard<std::mutex> lk(srv->mu);
    std::memset(info, 0, sizeof(*info));
    info->submitted = srv->submitted;
    info->completed = srv->completed;
    info->rejected = srv->rejected;
    info->queued = (long long)srv->queue.size();
    long long busy = 0;
    for (auto& s : srv->slots) busy += s->busy ? (long long)s->reqs.size() : 0;
    info->in_flight = busy;
    info->slots = (long long)srv->slots.size();
    info->evictions = srv->evictions;
    info->bytes_in_use = srv->in_use;
    return W1_OK;
}

extern "C" w1_status w1_server_destroy(w1_server* srv)
{
    if (!srv) return W1_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        srv->cv.notify_all();
    }
    if (srv->worker.joinable()) srv->worker.join();
    delete srv;
    return W1_OK;
}

extern "C" const char* w1_server_last_error(void) { return g_srv_err.c_str(); }
