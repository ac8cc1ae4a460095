// server.cu -- the serving loop of the library: sort requests arrive at any
// time, are admitted by HBM footprint, and run on a few CUDA streams
// ("lanes") while others are in flight.
//
// Admission.  A request of n elements of type t needs n * sizeof(t) bytes
// of device memory for its data and nothing more, because the sort is in
// place (Sec. 3 of Axtmann et al.); the server's own scratch is the fixed
// scratch of one sorter per (lane, type), allocated at creation.  A request
// is admitted while the admitted data plus that scratch stays within the
// budget; otherwise the caller gets IPSGPU_E_BUSY and retries once earlier
// requests are released.  A slice of the budget (small_reserve_bytes) is
// open to small requests only (at most batch_max_elems elements), so a large
// request waiting for memory never keeps small ones out.
//
// Scheduling.  Started requests wait in one FIFO queue.  A scheduler thread
// hands them to free lanes (one run per lane at a time): a request larger
// than batch_max_elems runs alone (ipsgpu_sort) on any free lane but the
// last, which is kept for small requests; smaller ones are batched, oldest
// first and one type per batch, into one ipsgpu_sort_batch run, preferably
// on the last lane.  Each lane has a low-priority stream for large runs and
// a high-priority one for batches, so the blocks of a batch are scheduled
// ahead of a large sort's whenever SMs free up, and large sorts share the
// GPU instead of queueing behind one another.  A run that holds at least
// half the memory budget also takes the high-priority stream: requests
// waiting for admission wait for its memory.  The queue is scanned past
// requests that cannot run yet, so a large request waiting for a lane does
// not hold back small ones, nor the reverse.  A host callback after each run
// wakes the scheduler, which reads the run's status and marks its requests
// done.
//
// Locking.  One mutex guards the queue, the request table and the lanes.
// No CUDA call is made while it is held: a host callback takes the mutex,
// so a CUDA call that waited for a callback under the mutex could deadlock.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "ipsgpu.h"

namespace {

constexpr int kTypes = 6;

int elem_bytes(int dtype) {
    switch (dtype) {
    case IPSGPU_U32: return 4;
    case IPSGPU_U64: return 8;
    case IPSGPU_F64: return 8;
    case IPSGPU_PAIR_U64: return 16;
    case IPSGPU_REC100: return 100;
    case IPSGPU_QUARTET: return 32;
    default: return 0;
    }
}
uint64_t elem_align(int dtype) {
    const int d = elem_bytes(dtype);
    return d == 100 ? 4 : (uint64_t)(d < 16 ? d : 16);
}

double now_us() {
    using namespace std::chrono;
    return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}

enum ReqState { RS_RESERVED = 0, RS_QUEUED, RS_RUNNING, RS_DONE };

struct Req {
    int dtype = 0;
    uint64_t n = 0, bytes = 0;
    void *d = nullptr;
    cudaEvent_t ready = nullptr;  // recorded on the caller's stream at start, or null
    int state = RS_RESERVED;
    int status = IPSGPU_OK;
    double t_submit = 0, t_launch = 0, t_done = 0;
};

struct Lane {
    ipsgpu_server *srv = nullptr;
    int idx = 0;
    bool small_only = false;  // kept for batches of small requests
    bool busy = false;
    cudaStream_t st_lo = nullptr, st_hi = nullptr;  // large runs / batches
    cudaStream_t st = nullptr;                      // stream of the current run
    ipsgpu_sorter *sorter[kTypes] = {};
    uint64_t *h_segs = nullptr;  // pinned (address, n) pairs of the running batch
    uint64_t *d_segs = nullptr;
    int dtype = 0;
    std::vector<uint64_t> tickets;
};

// One launch decided by the scheduler.
struct Plan {
    Lane *lane = nullptr;
    int dtype = 0;
    std::vector<uint64_t> tickets;
    std::vector<void *> ptrs;
    std::vector<uint64_t> ns;
    std::vector<cudaEvent_t> ready;
};

}  // namespace

struct ipsgpu_server {
    ipsgpu_server_config cfg;
    int device = 0;
    uint64_t scratch = 0;
    uint64_t used = 0;  // scratch + admitted request bytes
    uint64_t next_ticket = 1;
    bool stop = false;
    std::mutex mu;
    std::condition_variable cv;       // scheduler: start, completion, stop
    std::condition_variable cv_done;  // callers of wait / drain
    std::unordered_map<uint64_t, Req> reqs;
    std::deque<uint64_t> queue;
    std::vector<Lane *> lanes;
    std::vector<int> completed;  // lanes whose run has finished (host callback)
    std::vector<cudaEvent_t> events;  // free events for ready streams
    std::thread th;
};

namespace {

void CUDART_CB lane_done(void *p) {
    Lane *l = static_cast<Lane *>(p);
    ipsgpu_server *s = l->srv;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->completed.push_back(l->idx);
    }
    s->cv.notify_all();
}

// Next launch, or false.  Called with the mutex held.
bool choose(ipsgpu_server *s, Plan &plan) {
    Lane *large = nullptr, *small = nullptr;
    for (Lane *l : s->lanes) {
        if (l->busy) continue;
        if (!l->small_only && !large) large = l;
        if (l->small_only || !small) small = l;  // prefer the small-only lane
    }
    if (!large && !small) return false;
    const uint64_t lim = s->cfg.batch_max_elems;
    int batch_type = -1;
    uint64_t batch_elems = 0;
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        const Req &r = s->reqs[*it];
        if (r.n > lim) {
            if (large && batch_type < 0) {
                plan.lane = large;
                plan.dtype = r.dtype;
                plan.tickets.push_back(*it);
                break;
            }
            continue;
        }
        if (!small) continue;
        if (batch_type < 0) batch_type = r.dtype;
        if (r.dtype != batch_type) continue;
        if (!plan.tickets.empty() &&
            (plan.tickets.size() >= s->cfg.batch_max_requests || batch_elems + r.n > 8 * lim))
            break;
        plan.lane = small;
        plan.dtype = r.dtype;
        plan.tickets.push_back(*it);
        batch_elems += r.n;
    }
    if (plan.tickets.empty()) return false;
    // take the planned requests out of the queue
    std::deque<uint64_t> rest;
    size_t q = 0;
    for (uint64_t t : s->queue) {
        if (q < plan.tickets.size() && plan.tickets[q] == t) {
            q++;
            continue;
        }
        rest.push_back(t);
    }
    s->queue.swap(rest);
    const double t = now_us();
    for (uint64_t tk : plan.tickets) {
        Req &r = s->reqs[tk];
        r.state = RS_RUNNING;
        r.t_launch = t;
        plan.ptrs.push_back(r.d);
        plan.ns.push_back(r.n);
        plan.ready.push_back(r.ready);
    }
    plan.lane->busy = true;
    plan.lane->dtype = plan.dtype;
    plan.lane->tickets = plan.tickets;
    const bool alone = plan.tickets.size() == 1 && plan.ns[0] > lim;
    // a run holding at least half the memory budget goes at high priority
    // too: every request waiting for admission waits for its memory
    const bool holds_half =
        alone && 2 * plan.ns[0] * (uint64_t)elem_bytes(plan.dtype) >= s->cfg.hbm_budget_bytes;
    plan.lane->st = alone && !holds_half ? plan.lane->st_lo : plan.lane->st_hi;
    return true;
}

// Enqueues a planned run on its lane (no mutex held).
int launch(ipsgpu_server *s, Plan &plan) {
    Lane *l = plan.lane;
    ipsgpu_sorter *so = l->sorter[plan.dtype];
    if (!so) return IPSGPU_E_UNSUPPORTED;
    for (cudaEvent_t e : plan.ready)
        if (e && cudaStreamWaitEvent(l->st, e, 0) != cudaSuccess) return IPSGPU_E_CUDA;
    int rc;
    if (plan.tickets.size() == 1 && plan.ns[0] > s->cfg.batch_max_elems) {
        rc = ipsgpu_sort(so, plan.ptrs[0], plan.ns[0], l->st);
    } else {
        const size_t m = plan.tickets.size();
        for (size_t i = 0; i < m; i++) {
            l->h_segs[2 * i] = (uint64_t)(uintptr_t)plan.ptrs[i];
            l->h_segs[2 * i + 1] = plan.ns[i];
        }
        if (cudaMemcpyAsync(l->d_segs, l->h_segs, 16 * m, cudaMemcpyHostToDevice, l->st) !=
            cudaSuccess)
            return IPSGPU_E_CUDA;
        rc = ipsgpu_sort_batch(so, l->d_segs, m, l->st);
    }
    if (rc) return rc;
    return cudaLaunchHostFunc(l->st, lane_done, l) == cudaSuccess ? IPSGPU_OK : IPSGPU_E_CUDA;
}

void finish(ipsgpu_server *s, Lane *l, int status) {
    const double t = now_us();
    for (uint64_t tk : l->tickets) {
        auto it = s->reqs.find(tk);
        if (it == s->reqs.end()) continue;
        it->second.state = RS_DONE;
        it->second.status = status;
        it->second.t_done = t;
    }
    l->tickets.clear();
    l->busy = false;
    s->cv_done.notify_all();
}

void scheduler(ipsgpu_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        bool progress = false;
        while (!s->completed.empty()) {
            Lane *l = s->lanes[s->completed.back()];
            s->completed.pop_back();
            ipsgpu_sorter *so = l->sorter[l->dtype];
            lk.unlock();
            // the run has finished, so this synchronization returns at once
            int st = so ? ipsgpu_status(so, l->st) : IPSGPU_E_INTERNAL;
            lk.lock();
            finish(s, l, st);
            progress = true;
        }
        Plan plan;
        if (choose(s, plan)) {
            lk.unlock();
            const int rc = launch(s, plan);
            lk.lock();
            if (rc) {
                // nothing of the run may still be pending: drain the lane first
                Lane *l = plan.lane;
                lk.unlock();
                cudaStreamSynchronize(l->st);
                if (l->sorter[plan.dtype]) ipsgpu_status(l->sorter[plan.dtype], l->st);
                lk.lock();
                finish(s, l, rc);
            }
            continue;
        }
        if (progress) continue;
        bool busy = false;
        for (Lane *l : s->lanes) busy |= l->busy;
        if (s->stop && !busy && s->queue.empty()) break;
        s->cv.wait(lk);
    }
}

void destroy_lanes(ipsgpu_server *s) {
    for (Lane *l : s->lanes) {
        for (cudaStream_t x : {l->st_lo, l->st_hi})
            if (x) cudaStreamSynchronize(x);
        for (int t = 0; t < kTypes; t++)
            if (l->sorter[t]) ipsgpu_sorter_destroy(l->sorter[t]);
        if (l->h_segs) cudaFreeHost(l->h_segs);
        if (l->d_segs) cudaFree(l->d_segs);
        for (cudaStream_t x : {l->st_lo, l->st_hi})
            if (x) cudaStreamDestroy(x);
        delete l;
    }
    s->lanes.clear();
    for (cudaEvent_t e : s->events) cudaEventDestroy(e);
    s->events.clear();
}

}  // namespace

extern "C" {

int ipsgpu_server_create(const ipsgpu_server_config *cfg, const ipsgpu_params *params,
                         ipsgpu_server **out) {
    if (!cfg || !out || cfg->hbm_budget_bytes == 0) return IPSGPU_E_INVAL;
    *out = nullptr;
    ipsgpu_server *s = new (std::nothrow) ipsgpu_server;
    if (!s) return IPSGPU_E_NOMEM;
    s->cfg = *cfg;
    if (s->cfg.lanes == 0) s->cfg.lanes = 4;
    if (s->cfg.dtype_mask == 0)
        s->cfg.dtype_mask = (1u << IPSGPU_U32) | (1u << IPSGPU_U64) | (1u << IPSGPU_PAIR_U64);
    if (s->cfg.batch_max_elems == 0) s->cfg.batch_max_elems = 1ull << 22;
    if (s->cfg.batch_max_requests == 0) s->cfg.batch_max_requests = 4096;
    if (s->cfg.small_reserve_bytes == 0) s->cfg.small_reserve_bytes = s->cfg.hbm_budget_bytes / 32;
    if (s->cfg.lanes > 64 || (s->cfg.dtype_mask >> kTypes) != 0 ||
        s->cfg.small_reserve_bytes >= s->cfg.hbm_budget_bytes) {
        delete s;
        return IPSGPU_E_INVAL;
    }
    // scratch: one sorter per (lane, type) and the batch descriptors
    uint64_t scratch = 0;
    for (int t = 0; t < kTypes; t++) {
        if (!(s->cfg.dtype_mask >> t & 1u)) continue;
        const uint64_t b = ipsgpu_scratch_bytes(params, t);
        if (b == 0) {
            delete s;
            return IPSGPU_E_INVAL;
        }
        scratch += b * s->cfg.lanes;
    }
    scratch += (uint64_t)s->cfg.lanes * 16 * s->cfg.batch_max_requests;
    if (scratch > s->cfg.hbm_budget_bytes) {
        delete s;
        return IPSGPU_E_NOMEM;
    }
    s->scratch = scratch;
    s->used = scratch;
    int rc = IPSGPU_OK;
    int least = 0, greatest = 0;
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess)
        rc = IPSGPU_E_CUDA;
    for (uint32_t i = 0; i < s->cfg.lanes && rc == IPSGPU_OK; i++) {
        Lane *l = new (std::nothrow) Lane;
        if (!l) {
            rc = IPSGPU_E_NOMEM;
            break;
        }
        s->lanes.push_back(l);
        l->srv = s;
        l->idx = (int)i;
        l->small_only = s->cfg.lanes > 1 && i + 1 == s->cfg.lanes;
        if (cudaStreamCreateWithPriority(&l->st_lo, cudaStreamNonBlocking, least) != cudaSuccess ||
            cudaStreamCreateWithPriority(&l->st_hi, cudaStreamNonBlocking, greatest) !=
                cudaSuccess ||
            cudaMallocHost((void **)&l->h_segs, 16ull * s->cfg.batch_max_requests) != cudaSuccess ||
            cudaMalloc((void **)&l->d_segs, 16ull * s->cfg.batch_max_requests) != cudaSuccess) {
            rc = IPSGPU_E_NOMEM;
            break;
        }
        for (int t = 0; t < kTypes && rc == IPSGPU_OK; t++) {
            if (!(s->cfg.dtype_mask >> t & 1u)) continue;
            rc = ipsgpu_sorter_create(params, t, &l->sorter[t]);
            if (rc == IPSGPU_OK) rc = ipsgpu_sorter_prepare(l->sorter[t]);
        }
    }
    if (rc) {
        destroy_lanes(s);
        cudaGetLastError();
        delete s;
        return rc;
    }
    s->th = std::thread(scheduler, s);
    *out = s;
    return IPSGPU_OK;
}

int ipsgpu_server_reserve(ipsgpu_server *s, uint64_t n, int dtype, uint64_t *ticket) {
    if (!s || !ticket || dtype < 0 || dtype >= kTypes) return IPSGPU_E_INVAL;
    if (!(s->cfg.dtype_mask >> dtype & 1u)) return IPSGPU_E_UNSUPPORTED;
    if (n > (1ull << 40)) return IPSGPU_E_INVAL;
    const uint64_t bytes = n * (uint64_t)elem_bytes(dtype);
    const bool small = n <= s->cfg.batch_max_elems;
    const uint64_t limit =
        small ? s->cfg.hbm_budget_bytes : s->cfg.hbm_budget_bytes - s->cfg.small_reserve_bytes;
    if (s->scratch + bytes > limit) return IPSGPU_E_NOMEM;
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop) return IPSGPU_E_INVAL;
    if (s->used + bytes > limit) return IPSGPU_E_BUSY;
    s->used += bytes;
    const uint64_t t = s->next_ticket++;
    Req &r = s->reqs[t];
    r.dtype = dtype;
    r.n = n;
    r.bytes = bytes;
    r.state = RS_RESERVED;
    *ticket = t;
    return IPSGPU_OK;
}

int ipsgpu_server_start(ipsgpu_server *s, uint64_t ticket, void *d_data, void *ready_stream) {
    if (!s) return IPSGPU_E_INVAL;
    cudaEvent_t ev = nullptr;
    if (ready_stream) {
        {
            std::lock_guard<std::mutex> g(s->mu);
            if (!s->events.empty()) {
                ev = s->events.back();
                s->events.pop_back();
            }
        }
        if (!ev && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
            return IPSGPU_E_CUDA;
        if (cudaEventRecord(ev, (cudaStream_t)ready_stream) != cudaSuccess) {
            cudaEventDestroy(ev);
            return IPSGPU_E_CUDA;
        }
    }
    int rc = IPSGPU_OK;
    {
        std::lock_guard<std::mutex> g(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end() || it->second.state != RS_RESERVED) {
            rc = IPSGPU_E_INVAL;
        } else {
            Req &r = it->second;
            if (r.n > 0 && (!d_data || (uintptr_t)d_data % elem_align(r.dtype))) {
                rc = IPSGPU_E_INVAL;
            } else {
                r.d = d_data;
                r.ready = ev;
                r.t_submit = now_us();
                if (r.n < 2) {
                    r.state = RS_DONE;  // nothing to sort
                    r.t_launch = r.t_done = r.t_submit;
                    s->cv_done.notify_all();
                } else {
                    r.state = RS_QUEUED;
                    s->queue.push_back(ticket);
                }
                ev = nullptr;
            }
        }
        if (ev) s->events.push_back(ev);
    }
    if (rc == IPSGPU_OK) s->cv.notify_all();
    return rc;
}

int ipsgpu_server_submit(ipsgpu_server *s, void *d_data, uint64_t n, int dtype, uint64_t *ticket) {
    int rc = ipsgpu_server_reserve(s, n, dtype, ticket);
    if (rc) return rc;
    rc = ipsgpu_server_start(s, *ticket, d_data, nullptr);
    if (rc) ipsgpu_server_release(s, *ticket);
    return rc;
}

int ipsgpu_server_poll(ipsgpu_server *s, uint64_t ticket, int *done, int *status) {
    if (!s || !done) return IPSGPU_E_INVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return IPSGPU_E_INVAL;
    *done = it->second.state == RS_DONE ? 1 : 0;
    if (status) *status = it->second.status;
    return IPSGPU_OK;
}

int ipsgpu_server_wait(ipsgpu_server *s, uint64_t ticket) {
    if (!s) return IPSGPU_E_INVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end() || it->second.state == RS_RESERVED) return IPSGPU_E_INVAL;
    s->cv_done.wait(lk, [&] { return s->reqs[ticket].state == RS_DONE; });
    return s->reqs[ticket].status;
}

int ipsgpu_server_times(ipsgpu_server *s, uint64_t ticket, double *t_submit_us,
                        double *t_launch_us, double *t_done_us) {
    if (!s) return IPSGPU_E_INVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return IPSGPU_E_INVAL;
    if (t_submit_us) *t_submit_us = it->second.t_submit;
    if (t_launch_us) *t_launch_us = it->second.t_launch;
    if (t_done_us) *t_done_us = it->second.t_done;
    return IPSGPU_OK;
}

double ipsgpu_server_now_us(void) { return now_us(); }

int ipsgpu_server_release(ipsgpu_server *s, uint64_t ticket) {
    if (!s) return IPSGPU_E_INVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return IPSGPU_E_INVAL;
    if (it->second.state == RS_QUEUED || it->second.state == RS_RUNNING) return IPSGPU_E_BUSY;
    s->used -= it->second.bytes;
    if (it->second.ready) s->events.push_back(it->second.ready);
    s->reqs.erase(it);
    return IPSGPU_OK;
}

int ipsgpu_server_cancel(ipsgpu_server *s, uint64_t ticket) {
    if (!s) return IPSGPU_E_INVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end() || it->second.state == RS_DONE) return IPSGPU_E_INVAL;
    Req &r = it->second;
    if (r.state == RS_RUNNING) return IPSGPU_E_BUSY;
    if (r.state == RS_QUEUED) {
        for (auto q = s->queue.begin(); q != s->queue.end(); ++q) {
            if (*q == ticket) {
                s->queue.erase(q);
                break;
            }
        }
    }
    const double t = now_us();
    if (r.state == RS_RESERVED) r.t_submit = r.t_launch = t;
    r.state = RS_DONE;
    r.status = IPSGPU_E_CANCELED;
    r.t_done = t;
    s->cv_done.notify_all();
    return IPSGPU_OK;
}

int ipsgpu_server_drain(ipsgpu_server *s) {
    if (!s) return IPSGPU_E_INVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] {
        if (!s->queue.empty()) return false;
        for (Lane *l : s->lanes)
            if (l->busy) return false;
        return true;
    });
    return IPSGPU_OK;
}

int ipsgpu_server_usage(ipsgpu_server *s, uint64_t *used, uint64_t *budget, uint64_t *scratch) {
    if (!s) return IPSGPU_E_INVAL;
    std::lock_guard<std::mutex> g(s->mu);
    if (used) *used = s->used;
    if (budget) *budget = s->cfg.hbm_budget_bytes;
    if (scratch) *scratch = s->scratch;
    return IPSGPU_OK;
}

int ipsgpu_server_destroy(ipsgpu_server *s) {
    if (!s) return IPSGPU_E_INVAL;
    ipsgpu_server_drain(s);
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->th.joinable()) s->th.join();
    destroy_lanes(s);
    for (auto &kv : s->reqs)
        if (kv.second.ready) cudaEventDestroy(kv.second.ready);
    delete s;
    return IPSGPU_OK;
}

}  // extern "C"
