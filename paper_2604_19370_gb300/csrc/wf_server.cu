// Serving: a request loop over batch handles with continuous batching.
//
// Requests (one fire scenario each: grid, degree, time step, step count, model parameters,
// initial state and wind) are grouped into classes that can share a launch: same nx, ny, p, dt
// and parameters apart from the mean wind.  A class owns pools: batch handles (wf_batch_create)
// of growing capacity, each with its own stream and event.  The worker thread never waits on
// the GPU:
//   - a pool is idle or runs one quantum (wf_step of at most kQuantum steps, an event recorded
//     behind it); completion is polled with cudaEventQuery, so pools of every class run side by
//     side on the device and a slow class delays no other;
//   - every slot carries its request's step count as its budget (wf_batch_set_budget), so a
//     quantum advances each slot by min(quantum, its remaining steps): a request with few steps
//     left no longer shortens the quantum of the others;
//   - queued requests are admitted (first come, first served) into free slots of idle pools of
//     their class; a class with no free slot gets a new pool when the memory budget allows it,
//     its capacity set by the class's queued demand (at least kMinPoolSlots) and checked with
//     wf_batch_bytes before anything is allocated; a class that did not fit is not retried until
//     memory is freed;
//   - a pool's finished slots are retired as soon as its quantum completes: the state is copied
//     into the request's arrays, the slot freed and the latency recorded.
// New requests therefore join running work at quantum boundaries of their own class, and a
// slot's result does not depend on which other slots ran beside it (each slot is computed
// independently inside every launch).
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "wf.h"
#include "wf_internal.h"

namespace {

constexpr int kQuantum = 25;  // steps per quantum of a pool
// Slots of a new pool at least (within max_slots and the budget): under a thin stream of arrivals
// a class's queued demand is one request at a time, and pools sized by it alone came one slot
// each -- a pool per request, each created (allocation, factorisation) on the worker thread and
// stepped by launches over a single slot.  Later requests of the class join a pool's free slots
// at its next quantum instead.
constexpr int kMinPoolSlots = 8;

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t ticket = 0;
    wf_request r{};
    std::vector<double> T0, fuel0, wind;
    Clock::time_point t_submit, t_admit, t_done;
    int remaining = 0;
    int status = WF_PENDING;
    bool done = false;
};

struct ClassKey {
    int nx, ny, p;
    double dt;
    wf_params prm;  // wind_x = wind_y = 0
    bool operator<(const ClassKey& o) const { return memcmp(this, &o, sizeof(ClassKey)) < 0; }
};

struct Pool {
    wf_handle* h = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    size_t bytes = 0;
    std::vector<std::shared_ptr<Req>> slot;  // nullptr: free
    bool running = false;
    int quantum = 0;
    int used() const {
        int n = 0;
        for (auto& q : slot) n += q != nullptr;
        return n;
    }
    int free_slot() const {
        for (int k = 0; k < (int)slot.size(); ++k)
            if (!slot[k]) return k;
        return -1;
    }
};

struct Class {
    std::vector<std::unique_ptr<Pool>> pools;
};

ClassKey key_of(const wf_request& r) {
    ClassKey k;
    memset(&k, 0, sizeof(k));
    k.nx = r.nx;
    k.ny = r.ny;
    k.p = r.p;
    k.dt = r.dt;
    k.prm = r.params;
    k.prm.wind_x = 0.0;
    k.prm.wind_y = 0.0;
    return k;
}

}  // namespace

struct wf_server {
    size_t budget = 0;
    int max_slots = 1;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Req>> incoming;
    std::map<uint64_t, std::shared_ptr<Req>> all;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    // worker-owned
    std::deque<std::shared_ptr<Req>> queue;
    std::map<ClassKey, Class> classes;
    std::set<ClassKey> blocked;  // classes that did not fit; retried once memory is freed
    std::atomic<size_t> used{0};  // device bytes of every pool (read by wf_server_stats)
    // statistics
    double dof_steps = 0.0;
    uint64_t completed = 0;
};

namespace {

void finish(wf_server* s, const std::shared_ptr<Req>& q, int status) {
    std::lock_guard<std::mutex> lock(s->mu);
    q->status = status;
    q->t_done = Clock::now();
    q->done = true;
    if (status == WF_OK) {
        s->dof_steps += (double)(q->r.nx + q->r.p) * (q->r.ny + q->r.p) * q->r.steps;
        s->completed += 1;
    }
}

int pow2ceil(int n) {
    int c = 1;
    while (c < n) c <<= 1;
    return c;
}

// A new pool for `key` of capacity at most `want` (halved until its computed size fits the free
// budget; nothing is allocated before it does); nullptr if not even one slot fits.
std::unique_ptr<Pool> make_pool(wf_server* s, const wf_request& r, int want) {
    for (int cap = std::min(want, s->max_slots); cap >= 1; cap /= 2) {
        size_t need = 0;
        if (wf_batch_bytes(r.nx, r.ny, r.p, r.dt, &r.params, cap, &need) != WF_OK) return nullptr;
        if (s->used + need > s->budget) continue;
        wf_handle* h = nullptr;
        if (wf_batch_create(r.nx, r.ny, r.p, r.dt, &r.params, cap, &h) != WF_OK) continue;
        auto pl = std::make_unique<Pool>();
        pl->h = h;
        wf_device_bytes(h, &pl->bytes);
        pl->slot.assign(cap, nullptr);
        if (cudaStreamCreateWithFlags(&pl->stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&pl->ev, cudaEventDisableTiming) != cudaSuccess) {
            if (pl->stream) cudaStreamDestroy(pl->stream);
            wf_destroy(h);
            return nullptr;
        }
        wf_set_stream(h, pl->stream);
        s->used += pl->bytes;
        return pl;
    }
    return nullptr;
}

void drop_pool(wf_server* s, std::unique_ptr<Pool>& pl) {
    s->used -= pl->bytes;
    wf_set_stream(pl->h, nullptr);
    wf_destroy(pl->h);
    if (pl->ev) cudaEventDestroy(pl->ev);
    if (pl->stream) cudaStreamDestroy(pl->stream);
    pl.reset();
    s->blocked.clear();  // memory was freed: classes that did not fit may now
}

// Drop every idle, empty pool (of any class); true if one was dropped.
bool drop_idle_pools(wf_server* s) {
    bool any = false;
    for (auto& kv : s->classes) {
        auto& v = kv.second.pools;
        for (auto& pl : v)
            if (pl && !pl->running && pl->used() == 0) {
                drop_pool(s, pl);
                any = true;
            }
        v.erase(std::remove(v.begin(), v.end(), nullptr), v.end());
    }
    return any;
}

bool any_pool(const wf_server* s) {
    for (auto& kv : s->classes)
        if (!kv.second.pools.empty()) return true;
    return false;
}

// Put request q into slot k of the idle pool pl.
int place(Pool* pl, int k, const std::shared_ptr<Req>& q) {
    int rc = wf_batch_set_slot(pl->h, k, q->T0.data(), q->fuel0.data(), q->r.params.wind_x, q->r.params.wind_y,
                               q->r.wind_rank, q->r.wind_rank > 0 ? q->wind.data() : nullptr);
    if (rc == WF_OK) rc = wf_batch_set_budget(pl->h, k, q->r.steps);
    if (rc == WF_OK) rc = wf_batch_activate(pl->h, k, 1);
    if (rc != WF_OK) return rc;
    pl->slot[k] = q;
    q->t_admit = Clock::now();
    return WF_OK;
}

// Admit queued requests in arrival order into free slots of idle pools; true if any was.
bool admit(wf_server* s) {
    bool progress = false;
    std::map<ClassKey, int> demand;  // queued requests per class
    for (auto& q : s->queue) demand[key_of(q->r)] += 1;
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        std::shared_ptr<Req> q = *it;
        const ClassKey key = key_of(q->r);
        Class& c = s->classes[key];
        Pool* target = nullptr;
        int k = -1;
        bool any_free = false;
        for (auto& pl : c.pools) {
            const int f = pl->free_slot();
            if (f < 0) continue;
            any_free = true;
            if (!pl->running) {
                target = pl.get();
                k = f;
                break;
            }
        }
        if (!target && !any_free && !s->blocked.count(key)) {
            // no free slot in the class: a new pool sized by the class's queued demand (at least
            // kMinPoolSlots)
            const int want = std::max(kMinPoolSlots, pow2ceil(std::max(1, demand[key])));
            auto pl = make_pool(s, q->r, want);
            if (!pl && drop_idle_pools(s)) pl = make_pool(s, q->r, want);
            if (pl) {
                c.pools.push_back(std::move(pl));
                target = c.pools.back().get();
                k = 0;
            } else if (!any_pool(s)) {
                // nothing else holds memory: the request can never fit
                finish(s, q, WF_ENOMEM);
                demand[key] -= 1;
                it = s->queue.erase(it);
                progress = true;
                continue;
            } else {
                s->blocked.insert(key);
            }
        }
        if (!target) {
            ++it;  // waits for a slot of its class (or for memory)
            continue;
        }
        const int rc = place(target, k, q);
        if (rc != WF_OK) finish(s, q, rc);
        demand[key] -= 1;
        it = s->queue.erase(it);
        progress = true;
    }
    return progress;
}

// A pool's quantum completed: read the slots' flags, retire the finished slots.
void complete(wf_server* s, Pool* pl) {
    pl->running = false;
    std::vector<int> st(pl->slot.size(), 0);
    const int rc = wf_batch_status(pl->h, st.data(), (int)st.size());
    bool timeout = false;
    for (int v : st) timeout = timeout || (v & WF_STATUS_TIMEOUT);
    for (int k = 0; k < (int)pl->slot.size(); ++k) {
        std::shared_ptr<Req> q = pl->slot[k];
        if (!q) continue;
        bool release = true;
        if (rc != WF_OK) {
            finish(s, q, WF_ECUDA);
        } else if (timeout) {
            finish(s, q, WF_ETIMEOUT);  // the launch's output is invalid for every slot
        } else if (st[k] & WF_STATUS_UNSTABLE) {
            finish(s, q, WF_EUNSTABLE);
        } else {
            q->remaining -= std::min(pl->quantum, q->remaining);
            if (q->remaining <= 0)
                finish(s, q, wf_batch_get_slot(pl->h, k, q->r.T_out, q->r.fuel_out));
            else
                release = false;
        }
        if (release) {
            wf_batch_activate(pl->h, k, 0);
            pl->slot[k] = nullptr;
        }
    }
}

// Start the next quantum of an idle pool with work; every slot runs its own budget.
// 1: started, 0: nothing to run, -1: the launch failed.
int launch(Pool* pl) {
    int most = 0;
    for (auto& q : pl->slot)
        if (q) most = std::max(most, q->remaining);
    if (most <= 0) return 0;
    const int n = std::min(kQuantum, most);
    if (wf_step(pl->h, n) != WF_OK || cudaEventRecord(pl->ev, pl->stream) != cudaSuccess) return -1;
    pl->quantum = n;
    pl->running = true;
    return 1;
}

void worker_main(wf_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        bool busy = false;
        for (auto& kv : s->classes)
            for (auto& pl : kv.second.pools) busy = busy || pl->running;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            if (!busy && s->queue.empty() && s->incoming.empty() && !s->stop)
                s->cv.wait_for(lock, std::chrono::milliseconds(50));
            if (s->stop) break;
            while (!s->incoming.empty()) {
                s->queue.push_back(s->incoming.front());
                s->incoming.pop_front();
            }
        }
        bool progress = false;
        // 1. quanta that completed
        for (auto& kv : s->classes)
            for (auto& pl : kv.second.pools) {
                if (!pl->running) continue;
                const cudaError_t e = cudaEventQuery(pl->ev);
                if (e == cudaErrorNotReady) continue;
                if (e != cudaSuccess) cudaGetLastError();
                complete(s, pl.get());
                progress = true;
            }
        // 2. admissions into idle pools
        progress = admit(s) || progress;
        // 3. the next quantum of every idle pool with work
        for (auto& kv : s->classes)
            for (auto& pl : kv.second.pools) {
                if (pl->running || pl->used() == 0) continue;
                const int lr = launch(pl.get());
                if (lr > 0) {
                    progress = true;
                } else if (lr < 0) {
                    // the launch failed: fail the pool's requests
                    for (int k = 0; k < (int)pl->slot.size(); ++k)
                        if (pl->slot[k]) {
                            finish(s, pl->slot[k], WF_ECUDA);
                            wf_batch_activate(pl->h, k, 0);
                            pl->slot[k] = nullptr;
                        }
                }
            }
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    // shut down: wait for the device, drop every pool
    for (auto& kv : s->classes)
        for (auto& pl : kv.second.pools) {
            if (pl->running) cudaEventSynchronize(pl->ev);
            drop_pool(s, pl);
        }
    s->classes.clear();
}

}  // namespace

extern "C" {

int wf_server_create(size_t hbm_budget_bytes, int max_slots, wf_server** out) {
    if (!out) return WF_EINVAL;
    *out = nullptr;
    if (hbm_budget_bytes == 0 || max_slots < 1 || max_slots > 4096) return WF_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaFree(0) != cudaSuccess) return WF_ECUDA;
    wf_server* s = new (std::nothrow) wf_server();
    if (!s) return WF_ENOMEM;
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    s->device = dev;
    try {
        s->worker = std::thread(worker_main, s);
    } catch (...) {
        delete s;
        return WF_ENOMEM;
    }
    *out = s;
    return WF_OK;
}

int wf_submit(wf_server* s, const wf_request* r, uint64_t* ticket) {
    if (!s || !r || !ticket) return WF_EINVAL;
    if (r->nx < 1 || r->ny < 1 || r->p < 1 || r->p > wf::kMaxP || !(r->dt > 0.0) || r->steps < 0) return WF_EINVAL;
    if (!r->T0 || !r->fuel0 || !r->T_out || !r->fuel_out) return WF_EINVAL;
    if (r->wind_rank < 0 || r->wind_rank > wf::kMaxRank || (r->wind_rank > 0 && !r->wind_factors)) return WF_EINVAL;
    auto q = std::make_shared<Req>();
    q->r = *r;
    const size_t n = (size_t)(r->nx + r->p) * (r->ny + r->p);
    q->T0.assign(r->T0, r->T0 + n);
    q->fuel0.assign(r->fuel0, r->fuel0 + n);
    if (r->wind_rank > 0) {
        const size_t nw = 2 * (size_t)r->wind_rank * ((r->nx + r->p) + (r->ny + r->p));
        q->wind.assign(r->wind_factors, r->wind_factors + nw);
    }
    q->remaining = r->steps;
    q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        q->ticket = s->next_ticket++;
        s->all[q->ticket] = q;
        if (r->steps == 0) {
            // nothing to advance: the result is the initial state
            memcpy(r->T_out, r->T0, n * sizeof(double));
            memcpy(r->fuel_out, r->fuel0, n * sizeof(double));
            q->status = WF_OK;
            q->done = true;
            q->t_admit = q->t_done = q->t_submit;
        } else {
            s->incoming.push_back(q);
        }
        *ticket = q->ticket;
    }
    s->cv.notify_one();
    return WF_OK;
}

int wf_poll(wf_server* s, uint64_t ticket, wf_result* res) {
    if (!s) return WF_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return WF_ENOTFOUND;
    const std::shared_ptr<Req>& q = it->second;
    if (!q->done) return WF_PENDING;
    if (res) {
        res->status = q->status;
        res->latency_s = std::chrono::duration<double>(q->t_done - q->t_submit).count();
        res->queue_s = std::chrono::duration<double>(q->t_admit - q->t_submit).count();
        res->run_s = std::chrono::duration<double>(q->t_done - q->t_admit).count();
    }
    const int st = q->status;
    s->all.erase(it);
    return st == WF_OK ? WF_OK : st;
}

int wf_server_stats(wf_server* s, double* dof_steps, uint64_t* completed, size_t* hbm_used) {
    if (!s) return WF_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    if (dof_steps) *dof_steps = s->dof_steps;
    if (completed) *completed = s->completed;
    if (hbm_used) *hbm_used = s->used;
    return WF_OK;
}

void wf_server_destroy(wf_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    delete s;
}

}  // extern "C"
