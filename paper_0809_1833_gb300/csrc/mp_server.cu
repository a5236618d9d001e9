// Continuous-batching decode server.
//
// Requests (one signal y for one of the resident dictionaries) arrive at any
// time.  Per dictionary the server keeps a table of decode slots on the
// device (sized from the HBM budget), a CUDA stream and a captured graph of
// k batched MP steps (Sec. 3, Eqs. 9-12) followed by a retire kernel.  A
// scheduler thread loops over the dictionaries: when a dictionary's last
// chunk has finished it hands the finished signals' results (written by the
// retire kernel straight into host-mapped memory) to their requests, admits
// queued requests into the freed slots, and launches the next chunk.  So
// requests join and leave the batch between steps while others are
// mid-decode, and the dictionaries' chunks overlap on the device.  A
// signal's arithmetic does not depend on its batch row or on the other
// signals, so every result is the same as when decoded alone.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/mpgb_server.h"
#include "mp_batch.cuh"
#include "mp_internal.h"

namespace mpgb {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    int dict = 0;
    std::vector<float> y;
    double eps = 0.0;
    int T = 0;
    std::vector<float> x;
    mp_result res{};
    bool done = false;
    Clock::time_point t_submit, t_done;
};

struct Dict {
    mp_plan_t plan = nullptr;
    PlanImpl* p = nullptr;
    int prec = 0;
    int cap = 0;
    BatchEngine eng;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    bool inflight = false;
    float* X = nullptr;          // device, cap x M (decode outputs)
    float* d_y = nullptr;        // device admission staging, cap x N
    int* d_slots = nullptr;
    float* h_y = nullptr;        // pinned admission staging
    int* h_slots = nullptr;
    float* h_out_x = nullptr;    // host-mapped outbox, cap x M
    SlotState* h_out_st = nullptr;
    int* h_out_list = nullptr;
    int* h_out_count = nullptr;
    std::vector<int> free_slots;
    std::vector<Request*> slot_req;
    std::deque<Request*> pending;
    int in_use = 0;
    size_t bytes = 0;
};

}  // namespace mpgb

struct mp_server_s {
    size_t budget = 0;
    size_t used = 0;
    int max_slots = 0;
    int max_queue = 0;
    // batched steps per chunk graph (even, for the operand halves): longer
    // chunks cut the scheduler's round trips between chunks, shorter ones
    // admit and hand off sooner; of 8, 16 and 32, 16 sustained the most requests
    int steps = 16;
    int device = 0;
    std::vector<mpgb::Dict*> dicts;
    std::mutex mu;
    std::condition_variable cv;
    std::unordered_map<uint64_t, mpgb::Request*> reqs;
    uint64_t next_ticket = 1;
    std::thread th;
    bool started = false;
    std::atomic<bool> stop{false};
    std::atomic<int> fault{0};
    long long submitted = 0, rejected = 0, admitted = 0, completed = 0;
    std::atomic<long long> chunks{0}, retired{0};
    std::vector<double> lat;     // completed requests, submit -> completion, seconds
};

namespace mpgb {

static void dict_free(Dict* d) {
    if (!d) return;
    if (d->stream) cudaStreamSynchronize(d->stream);
    engine_free(&d->eng);
    cudaFree(d->X);
    cudaFree(d->d_y);
    cudaFree(d->d_slots);
    cudaFreeHost(d->h_y);
    cudaFreeHost(d->h_slots);
    cudaFreeHost(d->h_out_x);
    cudaFreeHost(d->h_out_st);
    cudaFreeHost(d->h_out_list);
    cudaFreeHost(d->h_out_count);
    if (d->ev) cudaEventDestroy(d->ev);
    if (d->stream) cudaStreamDestroy(d->stream);
    delete d;   // its requests are owned by the server's ticket map
}

template <typename T>
static cudaError_t mapped(T** host, T** dev, size_t n) {
    cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(host), sizeof(T) * n, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(dev), *host, 0);
    return e;
}

// Retire the finished signals of a completed chunk (caller holds srv->mu).
static void retire(mp_server_s* srv, Dict* d) {
    const int n = *reinterpret_cast<volatile int*>(d->h_out_count);
    srv->retired += n;
    const int M = d->p->M;
    const Clock::time_point now = Clock::now();
    for (int k = 0; k < n; ++k) {
        const int slot = d->h_out_list[k];
        if (slot < 0 || slot >= d->cap) continue;
        Request* r = d->slot_req[slot];
        if (!r) continue;
        const SlotState& s = d->h_out_st[slot];
        r->x.assign(d->h_out_x + static_cast<size_t>(slot) * M, d->h_out_x + static_cast<size_t>(slot + 1) * M);
        std::memset(&r->res, 0, sizeof(r->res));
        r->res.iters = s.t;
        r->res.stop_reason = s.stop_reason;
        r->res.status = s.status;
        r->res.rel_residual = s.e0 > 0.0 ? std::sqrt(s.e / s.e0) : 0.0;
        r->res.energy_audit_max = s.e0 > 0.0 ? s.audit / s.e0 : 0.0;
        r->done = true;
        r->t_done = now;
        srv->completed++;
        srv->lat.push_back(std::chrono::duration<double>(now - r->t_submit).count());
        d->slot_req[slot] = nullptr;
        d->free_slots.push_back(slot);
        d->in_use--;
    }
}

static cudaError_t admit(mp_server_s* srv, Dict* d, std::vector<Request*>& adm) {
    const int n = static_cast<int>(adm.size());
    const int N = d->p->N;
    for (int k = 0; k < n; ++k) {
        Request* r = adm[k];
        std::memcpy(d->h_y + static_cast<size_t>(k) * N, r->y.data(), sizeof(float) * N);
        d->eng.h_eps2[k] = r->eps * r->eps;
        d->eng.h_T[k] = r->T;
    }
    cudaStream_t st = d->stream;
    cudaError_t e = cudaMemcpyAsync(d->d_y, d->h_y, sizeof(float) * N * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d->d_slots, d->h_slots, sizeof(int) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d->eng.eps2, d->eng.h_eps2, sizeof(double) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d->eng.T, d->eng.h_T, sizeof(int) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = engine_admit(d->p, &d->eng, d->d_y, n, d->d_slots, st);
    (void)srv;
    return e;
}

static void scheduler(mp_server_s* srv) {
    cudaSetDevice(srv->device);
    while (!srv->stop.load()) {
        bool busy = false;
        for (Dict* d : srv->dicts) {
            if (d->inflight) {
                const cudaError_t q = cudaEventQuery(d->ev);
                if (q == cudaErrorNotReady) {
                    busy = true;
                    continue;
                }
                d->inflight = false;
                if (q != cudaSuccess) {
                    srv->fault.store(static_cast<int>(MP_ERR_CUDA));
                    continue;
                }
                if (*d->eng.h_err != 0) srv->fault.store(*d->eng.h_err);   // a device wait timed out
                std::lock_guard<std::mutex> lk(srv->mu);
                retire(srv, d);
                srv->cv.notify_all();
            }
            std::vector<Request*> adm;
            {
                std::lock_guard<std::mutex> lk(srv->mu);
                while (!d->pending.empty() && !d->free_slots.empty()) {
                    Request* r = d->pending.front();
                    d->pending.pop_front();
                    const int slot = d->free_slots.back();
                    d->free_slots.pop_back();
                    d->slot_req[slot] = r;
                    d->h_slots[adm.size()] = slot;
                    adm.push_back(r);
                    d->in_use++;
                    srv->admitted++;
                }
            }
            if (!adm.empty() && admit(srv, d, adm) != cudaSuccess) srv->fault.store(static_cast<int>(MP_ERR_CUDA));
            if (d->in_use > 0) {
                if (cudaGraphLaunch(d->eng.graph, d->stream) != cudaSuccess ||
                    cudaMemcpyAsync(d->eng.h_err, d->eng.err, sizeof(int), cudaMemcpyDeviceToHost, d->stream) !=
                        cudaSuccess ||
                    cudaEventRecord(d->ev, d->stream) != cudaSuccess) {
                    srv->fault.store(static_cast<int>(MP_ERR_CUDA));
                    continue;
                }
                d->p->launches += d->eng.graph_kernels;   // the steps' kernels and the retire kernel
                srv->chunks++;
                d->inflight = true;
                busy = true;
            }
        }
        if (!busy) {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv.wait_for(lk, std::chrono::microseconds(200), [&] {
                if (srv->stop.load()) return true;
                for (Dict* d : srv->dicts)
                    if (!d->pending.empty()) return true;
                return false;
            });
        } else {
            std::this_thread::yield();
        }
    }
}

}  // namespace mpgb

using namespace mpgb;

extern "C" {

mp_status mp_server_create(mp_server_t* out, size_t hbm_budget_bytes, int max_slots, int max_queue) {
    clear_error();
    if (!out) return fail(MP_ERR_INVALID, "mp_server_create: out is NULL");
    *out = nullptr;
    if (max_slots < 1 || max_queue < 0) return fail(MP_ERR_INVALID, "mp_server_create: max_slots >= 1, max_queue >= 0");
    mp_server_s* s = new (std::nothrow) mp_server_s();
    if (!s) return fail(MP_ERR_NOMEM, "mp_server_create: host allocation failed");
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    s->max_queue = max_queue;
    cudaGetDevice(&s->device);
    *out = s;
    return MP_OK;
}

mp_status mp_server_add_dictionary(mp_server_t srv, mp_plan_t plan, int prec, int* dict_id) {
    clear_error();
    if (!srv || !plan || !dict_id) return fail(MP_ERR_INVALID, "mp_server_add_dictionary: NULL argument");
    if (srv->started) return fail(MP_ERR_INVALID, "mp_server_add_dictionary: add dictionaries before the first submit");
    PlanImpl* p = &plan->impl;
    if (prec != MP_PREC_BF16 && prec != MP_PREC_FP8E4M3)
        return fail(MP_ERR_INVALID, "mp_server_add_dictionary: precision must be BF16 or FP8");
    if (!(p->prec_mask & (1u << prec)))
        return fail(MP_ERR_UNSUPPORTED, "mp_server_add_dictionary: the plan holds no copy for this precision");
    // the Gram mode keeps the plan's Gram matrix (built here, counted in the
    // plan's bytes) and a correlation row per slot
    const int gram_R = p->batch_gram;
    if (gram_R > 0) {
        if (prec != MP_PREC_BF16)
            return fail(MP_ERR_UNSUPPORTED, "mp_server_add_dictionary: the Gram mode runs with BF16 correlations");
        if (gram_R % srv->steps)
            return fail(MP_ERR_INVALID, "mp_server_add_dictionary: the Gram period must be a multiple of 16");
        mp_status gs = gram_prepare(p, nullptr);
        if (gs != MP_OK) return gs;
    }
    // HBM admission: the plan, then as many slots as the budget allows
    const size_t slot_bytes = engine_slot_bytes(p, prec, true, gram_R) + sizeof(float) * p->N;
    const size_t fixed = p->device_bytes + (1u << 20);
    if (srv->used + fixed + slot_bytes > srv->budget)
        return fail(MP_ERR_BUSY, "mp_server_add_dictionary: HBM budget exhausted (" + std::to_string(srv->used) + " of " +
                                     std::to_string(srv->budget) + " bytes used)");
    const int cap = static_cast<int>(std::min<size_t>(srv->max_slots, (srv->budget - srv->used - fixed) / slot_bytes));
    Dict* d = new (std::nothrow) Dict();
    if (!d) return fail(MP_ERR_NOMEM, "mp_server_add_dictionary: host allocation failed");
    d->plan = plan;
    d->p = p;
    d->prec = prec;
    d->cap = cap;
    const int N = p->N, M = p->M;
    GemmShape g;
    mp_status st = batch_shape(p, prec, cap, nullptr, nullptr, &g);
    if (st == MP_OK) st = engine_alloc(&d->eng, p, prec, cap, g, gram_R);
    cudaError_t e = cudaSuccess;
    if (st == MP_OK) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&d->stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d->ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&d->X, sizeof(float) * static_cast<size_t>(cap) * M);
        if (e == cudaSuccess) e = cudaMalloc(&d->d_y, sizeof(float) * static_cast<size_t>(cap) * N);
        if (e == cudaSuccess) e = cudaMalloc(&d->d_slots, sizeof(int) * cap);
        if (e == cudaSuccess) e = cudaMallocHost(&d->h_y, sizeof(float) * static_cast<size_t>(cap) * N);
        if (e == cudaSuccess) e = cudaMallocHost(&d->h_slots, sizeof(int) * cap);
        float* dx = nullptr;
        SlotState* dst = nullptr;
        int *dl = nullptr, *dc = nullptr;
        if (e == cudaSuccess) e = mapped(&d->h_out_x, &dx, static_cast<size_t>(cap) * M);
        if (e == cudaSuccess) e = mapped(&d->h_out_st, &dst, cap);
        if (e == cudaSuccess) e = mapped(&d->h_out_list, &dl, cap);
        if (e == cudaSuccess) e = mapped(&d->h_out_count, &dc, 1);
        if (e == cudaSuccess) {
            BatchIO io;
            std::memset(&io, 0, sizeof(io));
            io.X = d->X;
            io.ldx = M;
            *d->eng.h_io = io;
            e = cudaMemcpy(d->eng.io, d->eng.h_io, sizeof(BatchIO), cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess) e = cudaMemset(d->eng.counters, 0, sizeof(int) * 8);
        if (e == cudaSuccess) e = cudaMemset(d->eng.err, 0, sizeof(int));
        if (e == cudaSuccess) st = engine_build_graph(p, &d->eng, srv->steps, true, dx, dst, dl, dc);
    }
    if (st == MP_OK && e != cudaSuccess) st = cuda_fail(e, "mp_server_add_dictionary");
    if (st != MP_OK) {
        dict_free(d);
        return st;
    }
    d->slot_req.assign(cap, nullptr);
    for (int s = cap - 1; s >= 0; --s) d->free_slots.push_back(s);
    d->bytes = fixed + static_cast<size_t>(cap) * slot_bytes;
    srv->used += d->bytes;
    *dict_id = static_cast<int>(srv->dicts.size());
    srv->dicts.push_back(d);
    return MP_OK;
}

mp_status mp_server_dictionary_slots(mp_server_t srv, int dict_id, int* slots) {
    if (!srv || !slots || dict_id < 0 || dict_id >= static_cast<int>(srv->dicts.size()))
        return fail(MP_ERR_INVALID, "mp_server_dictionary_slots: bad argument");
    *slots = srv->dicts[dict_id]->cap;
    return MP_OK;
}

mp_status mp_server_submit(mp_server_t srv, int dict_id, const float* y_host, const mp_stop* stop, uint64_t* ticket) {
    clear_error();
    if (!srv || !y_host || !stop || !ticket) return fail(MP_ERR_INVALID, "mp_server_submit: NULL argument");
    if (dict_id < 0 || dict_id >= static_cast<int>(srv->dicts.size()))
        return fail(MP_ERR_NOT_FOUND, "mp_server_submit: unknown dictionary");
    if (!(stop->eps >= 0.0) || !std::isfinite(stop->eps) || stop->max_iters < 0 || stop->reserved != 0)
        return fail(MP_ERR_INVALID, "mp_server_submit: bad stop parameters");
    if (int f = srv->fault.load()) return fail(static_cast<mp_status>(f), "mp_server_submit: the server hit a CUDA error");
    Dict* d = srv->dicts[dict_id];
    Request* r = new (std::nothrow) Request();
    if (!r) return fail(MP_ERR_NOMEM, "mp_server_submit: host allocation failed");
    r->dict = dict_id;
    r->y.assign(y_host, y_host + d->p->N);
    r->eps = stop->eps;
    r->T = stop->max_iters;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (static_cast<int>(d->pending.size()) >= srv->max_queue) {
            srv->rejected++;
            delete r;
            return fail(MP_ERR_BUSY, "mp_server_submit: queue full");
        }
        r->ticket = srv->next_ticket++;
        srv->reqs[r->ticket] = r;
        d->pending.push_back(r);
        srv->submitted++;
        *ticket = r->ticket;
        if (!srv->started) {
            srv->started = true;
            srv->th = std::thread(scheduler, srv);
        }
    }
    srv->cv.notify_all();
    return MP_OK;
}

mp_status mp_server_poll(mp_server_t srv, uint64_t ticket, float* x_host_out, mp_result* out) {
    if (!srv) return fail(MP_ERR_INVALID, "mp_server_poll: server is NULL");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return fail(MP_ERR_NOT_FOUND, "mp_server_poll: unknown ticket");
    Request* r = it->second;
    if (!r->done) {
        if (int f = srv->fault.load()) return fail(static_cast<mp_status>(f), "mp_server_poll: the server hit a CUDA error");
        return MP_PENDING;
    }
    if (x_host_out) std::memcpy(x_host_out, r->x.data(), sizeof(float) * r->x.size());
    if (out) *out = r->res;
    srv->reqs.erase(it);
    delete r;
    return MP_OK;
}

mp_status mp_server_get_stats(mp_server_t srv, mp_server_stats* out) {
    if (!srv || !out) return fail(MP_ERR_INVALID, "mp_server_get_stats: NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = srv->submitted;
    out->rejected = srv->rejected;
    out->admitted = srv->admitted;
    out->completed = srv->completed;
    long long queued = 0, active = 0;
    for (Dict* d : srv->dicts) {
        queued += static_cast<long long>(d->pending.size());
        active += d->in_use;
    }
    out->queued = queued;
    out->active = active;
    if (!srv->lat.empty()) {
        std::vector<double> v = srv->lat;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) { return v[std::min(v.size() - 1, static_cast<size_t>(q * (v.size() - 1) + 0.5))]; };
        out->latency_p50_s = pct(0.50);
        out->latency_p99_s = pct(0.99);
        double sum = 0.0;
        for (double x : v) sum += x;
        out->latency_mean_s = sum / v.size();
        out->latency_max_s = v.back();
    }
    out->hbm_bytes = srv->used;
    out->chunks = srv->chunks.load();
    out->retired = srv->retired.load();
    return MP_OK;
}

mp_status mp_server_reset_stats(mp_server_t srv) {
    if (!srv) return fail(MP_ERR_INVALID, "mp_server_reset_stats: NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->submitted = srv->rejected = srv->admitted = srv->completed = 0;
    srv->lat.clear();
    return MP_OK;
}

mp_status mp_server_destroy(mp_server_t srv) {
    if (!srv) return MP_OK;
    srv->stop.store(true);
    srv->cv.notify_all();
    if (srv->th.joinable()) srv->th.join();
    for (Dict* d : srv->dicts) dict_free(d);
    for (auto& kv : srv->reqs) delete kv.second;   // queued, in flight, or finished but not polled
    delete srv;
    return MP_OK;
}

}  // extern "C"
