// Serving: a request loop over batch handles with continuous batching.
//
// Requests (one fire scenario each: grid, degree, time step, step count, model
// parameters, initial state and wind) are grouped into classes that can share a
// launch: same nx, ny, p, dt and parameters apart from the mean wind.  Every class
// owns one batch handle (wf_batch_create) with its own stream.  A worker thread:
//   1. admits queued requests into free slots of their class, creating the class's
//      handle when the device-memory budget allows it (first come, first served);
//   2. advances every class with active slots by one quantum of steps (the smallest
//      remaining step count of its slots, at most kQuantum), all classes enqueued
//      before any is waited for, so their kernels overlap on the GPU;
//   3. retires finished slots: copies the state into the request's output arrays,
//      frees the slot and records the latency.
// New requests therefore join running batches at quantum boundaries, and a slot's
// result does not depend on which other slots ran beside it (each slot is computed
// independently inside every launch).
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "wf.h"
#include "wf_internal.h"

namespace {

constexpr int kQuantum = 25;  // steps per scheduling round

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

struct Class {
    ClassKey key;
    wf_handle* h = nullptr;
    cudaStream_t stream = nullptr;
    size_t bytes = 0;
    std::vector<std::shared_ptr<Req>> slot;  // nullptr: free
    Clock::time_point last_used;
    int active() const {
        int n = 0;
        for (auto& s : slot) n += s != nullptr;
        return n;
    }
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
    std::map<ClassKey, std::unique_ptr<Class>> classes;
    size_t used = 0;
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

// Create a class handle sized to the free budget (capacity up to max_slots); nullptr if none fits.
// The capacity is chosen from the handle's computed size before anything is allocated, so the
// budget is never overshot, not even for a moment.
std::unique_ptr<Class> make_class(wf_server* s, const ClassKey& key, const wf_request& r) {
    for (int cap = s->max_slots; cap >= 1; cap /= 2) {
        size_t need = 0;
        if (wf_batch_bytes(r.nx, r.ny, r.p, r.dt, &r.params, cap, &need) != WF_OK) return nullptr;
        if (s->used + need > s->budget) continue;
        wf_handle* h = nullptr;
        if (wf_batch_create(r.nx, r.ny, r.p, r.dt, &r.params, cap, &h) != WF_OK) continue;
        size_t bytes = 0;
        wf_device_bytes(h, &bytes);
        auto c = std::make_unique<Class>();
        c->key = key;
        c->h = h;
        c->bytes = bytes;
        c->slot.assign(cap, nullptr);
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) == cudaSuccess)
            wf_set_stream(h, c->stream);
        c->last_used = Clock::now();
        s->used += bytes;
        return c;
    }
    return nullptr;
}

void drop_class(wf_server* s, std::map<ClassKey, std::unique_ptr<Class>>::iterator it) {
    Class* c = it->second.get();
    s->used -= c->bytes;
    wf_set_stream(c->h, nullptr);
    wf_destroy(c->h);
    if (c->stream) cudaStreamDestroy(c->stream);
    s->classes.erase(it);
}

// Admit queued requests (in arrival order) into free slots.
void admit(wf_server* s) {
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        std::shared_ptr<Req> q = *it;
        const ClassKey key = key_of(q->r);
        auto ci = s->classes.find(key);
        if (ci == s->classes.end()) {
            auto c = make_class(s, key, q->r);
            if (!c) {
                // free idle classes of other shapes, then retry once
                for (auto jt = s->classes.begin(); jt != s->classes.end();) {
                    auto nx = std::next(jt);
                    if (jt->second->active() == 0) drop_class(s, jt);
                    jt = nx;
                }
                c = make_class(s, key, q->r);
            }
            if (!c) {
                if (s->classes.empty()) {  // nothing else holds memory: the request can never fit
                    finish(s, q, WF_ENOMEM);
                    it = s->queue.erase(it);
                    continue;
                }
                ++it;  // wait for running classes to drain
                continue;
            }
            ci = s->classes.emplace(key, std::move(c)).first;
        }
        Class* c = ci->second.get();
        int slot = -1;
        for (int k = 0; k < (int)c->slot.size(); ++k)
            if (!c->slot[k]) {
                slot = k;
                break;
            }
        if (slot < 0) {
            ++it;
            continue;
        }
        const int rc = wf_batch_set_slot(c->h, slot, q->T0.data(), q->fuel0.data(), q->r.params.wind_x,
                                         q->r.params.wind_y, q->r.wind_rank,
                                         q->r.wind_rank > 0 ? q->wind.data() : nullptr);
        if (rc != WF_OK) {
            finish(s, q, rc);
            it = s->queue.erase(it);
            continue;
        }
        wf_batch_activate(c->h, slot, 1);
        c->slot[slot] = q;
        c->last_used = Clock::now();
        q->t_admit = Clock::now();
        it = s->queue.erase(it);
    }
}

// One scheduling round over every class with active slots.
void run_round(wf_server* s) {
    std::vector<std::pair<Class*, int>> stepped;
    for (auto& kv : s->classes) {
        Class* c = kv.second.get();
        int quantum = kQuantum;
        bool any = false;
        for (auto& q : c->slot)
            if (q) {
                quantum = std::min(quantum, q->remaining);
                any = true;
            }
        if (!any) continue;
        if (quantum > 0 && wf_step(c->h, quantum) == WF_OK) stepped.push_back({c, quantum});
        else stepped.push_back({c, -1});
    }
    for (auto& cs : stepped) {
        Class* c = cs.first;
        const int n = cs.second;
        std::vector<int> st(c->slot.size(), 0);
        const int rc = wf_batch_status(c->h, st.data(), (int)st.size());  // waits for the class's stream
        for (int k = 0; k < (int)c->slot.size(); ++k) {
            std::shared_ptr<Req> q = c->slot[k];
            if (!q) continue;
            bool release = false;
            if (n < 0 || rc != WF_OK) {
                finish(s, q, WF_ECUDA);
                release = true;
            } else if (st[k]) {
                finish(s, q, WF_EUNSTABLE);
                release = true;
            } else {
                q->remaining -= n;
                if (q->remaining <= 0) {
                    const int g = wf_batch_get_slot(c->h, k, q->r.T_out, q->r.fuel_out);
                    finish(s, q, g);
                    release = true;
                }
            }
            if (release) {
                wf_batch_activate(c->h, k, 0);
                c->slot[k] = nullptr;
            }
        }
        c->last_used = Clock::now();
    }
}

void worker_main(wf_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lock(s->mu);
            bool idle = s->queue.empty();
            for (auto& kv : s->classes) idle = idle && kv.second->active() == 0;
            if (idle && s->incoming.empty() && !s->stop)
                s->cv.wait_for(lock, std::chrono::milliseconds(50));
            if (s->stop) break;
            while (!s->incoming.empty()) {
                s->queue.push_back(s->incoming.front());
                s->incoming.pop_front();
            }
        }
        const size_t before = s->queue.size();
        admit(s);
        bool any_active = false;
        for (auto& kv : s->classes) any_active = any_active || kv.second->active() > 0;
        if (any_active)
            run_round(s);
        else if (!s->queue.empty() && s->queue.size() == before)
            std::this_thread::sleep_for(std::chrono::milliseconds(1));  // waiting for memory to free up
    }
    // shut down: drop every class
    while (!s->classes.empty()) drop_class(s, s->classes.begin());
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
