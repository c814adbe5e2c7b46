// moff_server.cu -- streaming request loop over many served plans.
//
// The paper describes the correlator as a stream of channelised blocks (Sec. 2,
// Sec. 5); this file is the library's front end for such a stream: blocks from
// sub-arrays of uneven antenna count and grid size arrive at any time and run
// on the GPU concurrently (continuous batching).  A plan created with
// MOFF_SERVED keeps its kernels, gains and partial integrations resident; the
// transient per-block scratch (the row-transformed field, the FP16 voltage
// planes, a host block's copy) is lent from one device pool allocated when the
// server is created, so admission is by memory:
//
//   - a block starts when a slot is free (at most n_slots on the GPU), its
//     plan has no block on the GPU (a plan's blocks run in submission order)
//     and the pool can lend it its scratch;
//   - blocks start in arrival order, except that a later block may pass one
//     that does not fit yet when it leaves at least that block's bytes free;
//   - a block's GPU work goes on its plan's stream, followed by a host
//     callback that stamps the completion time and wakes the dispatcher, which
//     returns the scratch to the pool and admits more.
//
// One dispatcher thread makes every CUDA call of the loop; the callbacks make
// none.  No lock is held across a CUDA call (a host callback may be waiting
// for the lock while the stream it runs on blocks that call).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "moff_internal.h"

using namespace moff;
using Clock = std::chrono::steady_clock;

namespace {

// First-fit allocator over [0, size) with coalescing of freed neighbours.
struct Pool {
    size_t size = 0, free_total = 0;
    std::map<size_t, size_t> free_list;   // offset -> length

    void init(size_t n) {
        size = free_total = n;
        free_list.clear();
        free_list[0] = n;
    }
    bool alloc(size_t n, size_t *off) {
        for (auto it = free_list.begin(); it != free_list.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n, at = it->first + n;
            free_list.erase(it);
            if (rest) free_list[at] = rest;
            free_total -= n;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n) {
        auto it = free_list.emplace(off, n).first;
        free_total += n;
        auto nx = std::next(it);
        if (nx != free_list.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_list.erase(nx);
        }
        if (it != free_list.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_list.erase(it);
            }
        }
    }
};

enum { kQueued = 0, kRunning = 1, kDone = 2 };

struct Req {
    moff_plan *pl = nullptr;
    const uint8_t *volt = nullptr;
    int n_time = 0, on_device = 0;
    size_t bytes = 0, off = 0;
    long long units = 0;
    int state = kQueued;
    moff_status err = MOFF_OK;
    Clock::time_point t_submit, t_start, t_done;
};

// Everything the dispatcher and the host callbacks share.  Held through a
// shared_ptr by the server, the dispatcher and every pending callback, so the
// lock outlives the last callback that touches it.
struct Core {
    int device = 0;
    unsigned char *pool_base = nullptr;
    Pool pool;
    int n_slots = 1;

    std::mutex mu;
    std::condition_variable cv_work;   // dispatcher: submits, completions, stop
    std::condition_variable cv_done;   // waiters: a block finished
    std::map<long long, Req> reqs;     // every ticket not yet trimmed
    std::deque<long long> queue;       // queued tickets in arrival order
    std::deque<long long> finished;    // tickets whose GPU work ended (set by callbacks)
    std::deque<long long> retired;     // done tickets, oldest first (for trimming)
    std::set<const moff_plan *> busy;  // plans with a block on the GPU
    int inflight = 0;
    long long next_id = 1;
    bool stop = false;

    // statistics window
    std::vector<double> lat_ms;
    long long units_done = 0, n_done = 0;
    bool have_first = false;
    Clock::time_point t_first, t_last;
    bool dirty = false;                // something for the dispatcher to look at
};

}  // namespace

struct moff_server {
    std::shared_ptr<Core> core;
    std::thread th;
};

namespace {

constexpr size_t kKeepDone = 1 << 16;   // finished tickets kept for polling

struct CbCtx {
    std::shared_ptr<Core> core;
    long long id;
};

void CUDART_CB on_block_done(void *p) {
    CbCtx *c = static_cast<CbCtx *>(p);
    {
        std::lock_guard<std::mutex> lk(c->core->mu);
        auto it = c->core->reqs.find(c->id);
        if (it != c->core->reqs.end()) it->second.t_done = Clock::now();
        c->core->finished.push_back(c->id);
        c->core->dirty = true;
        c->core->cv_work.notify_one();
    }
    delete c;
}

// Under the lock: return the scratch of a finished or failed block and record it.
void retire(Core *s, long long id, moff_status err) {
    Req &r = s->reqs[id];
    s->pool.release(r.off, r.bytes);
    s->busy.erase(r.pl);
    s->inflight--;
    r.state = kDone;
    r.err = err;
    if (err == MOFF_OK) {
        const double ms = std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
        s->lat_ms.push_back(ms);
        s->units_done += r.units;
        s->n_done++;
        if (s->n_done == 1 || r.t_done > s->t_last) s->t_last = r.t_done;
    }
    s->retired.push_back(id);
    while (s->retired.size() > kKeepDone) {
        s->reqs.erase(s->retired.front());
        s->retired.pop_front();
    }
}

// Under the lock: pick the queued blocks that may start now.
std::vector<long long> admit(Core *s) {
    std::vector<long long> out;
    std::set<const moff_plan *> held;   // plans with an earlier block still queued
    size_t reserve = 0;                 // bytes kept free for the oldest block that did not fit
    bool blocked = false;
    for (auto it = s->queue.begin(); it != s->queue.end() && s->inflight < s->n_slots;) {
        Req &r = s->reqs[*it];
        if (s->busy.count(r.pl) || held.count(r.pl)) {
            held.insert(r.pl);
            ++it;
            continue;
        }
        size_t off = 0;
        const bool room = !blocked || s->pool.free_total >= reserve + r.bytes;
        if (!room || !s->pool.alloc(r.bytes, &off)) {
            if (!blocked) {
                blocked = true;
                reserve = r.bytes;
            }
            held.insert(r.pl);
            ++it;
            continue;
        }
        r.off = off;
        r.state = kRunning;
        r.t_start = Clock::now();
        s->busy.insert(r.pl);
        s->inflight++;
        out.push_back(*it);
        it = s->queue.erase(it);
    }
    return out;
}

void dispatcher(std::shared_ptr<Core> core) {
    Core *s = core.get();
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<long long> go;
        bool any_done = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->dirty; });
            s->dirty = false;
            while (!s->finished.empty()) {
                retire(s, s->finished.front(), MOFF_OK);
                s->finished.pop_front();
                any_done = true;
            }
            if (s->stop) {
                // cancel what has not started; wait for the GPU to drain
                for (long long id : s->queue) {
                    Req &r = s->reqs[id];
                    r.state = kDone;
                    r.err = MOFF_ESTATE;
                    s->retired.push_back(id);
                }
                s->queue.clear();
                if (s->inflight == 0) {
                    lk.unlock();
                    s->cv_done.notify_all();
                    return;
                }
            } else {
                go = admit(s);
            }
        }
        if (any_done) s->cv_done.notify_all();
        for (long long id : go) {
            Req r;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                r = s->reqs[id];
            }
            moff_status st = plan_run_served(r.pl, s->pool_base + r.off, r.volt, r.n_time, r.on_device);
            if (st == MOFF_OK) {
                CbCtx *c = new CbCtx{core, id};
                if (cudaLaunchHostFunc(plan_stream(r.pl), on_block_done, c) != cudaSuccess) {
                    delete c;
                    cudaGetLastError();
                    // the block's work is enqueued but unobservable: wait for it here
                    cudaStreamSynchronize(plan_stream(r.pl));
                    st = MOFF_ECUDA;
                }
            }
            if (st != MOFF_OK) {
                {
                    std::lock_guard<std::mutex> lk(s->mu);
                    retire(s, id, st);
                }
                s->cv_done.notify_all();
            }
        }
    }
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    // nearest rank
    size_t k = (size_t)std::ceil(q * (double)v.size());
    k = std::min(std::max<size_t>(k, 1), v.size());
    return v[k - 1];
}

}  // namespace

extern "C" {

moff_status moff_server_create(moff_server **out, long long hbm_budget_bytes, int n_slots) {
    if (!out) return fail_msg(MOFF_EINVAL, "out is NULL");
    *out = nullptr;
    if (hbm_budget_bytes < 1024) return fail_msg(MOFF_EINVAL, "hbm_budget_bytes must be >= 1024");
    if (n_slots < 1 || n_slots > 64) return fail_msg(MOFF_EINVAL, "n_slots must be in [1, 64]");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail_msg(MOFF_ECUDA, "no CUDA device");
    }
    void *p = nullptr;
    const size_t bytes = align_up((size_t)hbm_budget_bytes, 1024);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail_msg(e == cudaErrorMemoryAllocation ? MOFF_ENOMEM : MOFF_ECUDA, "server pool allocation failed");
    }
    moff_server *srv = new moff_server();
    srv->core = std::make_shared<Core>();
    Core *s = srv->core.get();
    s->device = dev;
    s->pool_base = static_cast<unsigned char *>(p);
    s->pool.init(bytes);
    s->n_slots = n_slots;
    srv->th = std::thread(dispatcher, srv->core);
    *out = srv;
    return MOFF_OK;
}

moff_status moff_server_submit(moff_server *srv, moff_plan *pl, const uint8_t *volt, int n_time, int on_device,
                               long long *ticket) {
    if (!srv || !pl || !volt || !ticket) return fail_msg(MOFF_EINVAL, "server, plan, volt and ticket must not be NULL");
    Core *s = srv->core.get();
    *ticket = 0;
    if (n_time < 1) return fail_msg(MOFF_EINVAL, "n_time must be >= 1");
    if (!plan_is_served(pl)) return fail_msg(MOFF_ESTATE, "plan was not created with MOFF_SERVED");
    if (plan_device(pl) != s->device) return fail_msg(MOFF_ESTATE, "plan and server are on different devices");
    Req r;
    r.pl = pl;
    r.volt = volt;
    r.n_time = n_time;
    r.on_device = on_device ? 1 : 0;
    r.bytes = align_up(plan_scratch_bytes(pl) + (on_device ? 0 : plan_block_bytes(pl, n_time)), 1024);
    r.units = plan_units(pl, n_time);
    r.t_submit = Clock::now();
    if (r.bytes > s->pool.size) return fail_msg(MOFF_ENOMEM, "block needs more scratch than the server pool holds");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return fail_msg(MOFF_ESTATE, "server is shutting down");
        const long long id = s->next_id++;
        s->reqs[id] = r;
        s->queue.push_back(id);
        if (!s->have_first) {
            s->have_first = true;
            s->t_first = r.t_submit;
        }
        *ticket = id;
        s->dirty = true;
    }
    s->cv_work.notify_one();
    return MOFF_OK;
}

moff_status moff_server_poll(moff_server *srv, long long ticket, int *state, double *latency_ms) {
    if (!srv || !state) return fail_msg(MOFF_EINVAL, "server and state must not be NULL");
    Core *s = srv->core.get();
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail_msg(MOFF_EINVAL, "unknown ticket");
    const Req &r = it->second;
    *state = r.state == kDone && r.err != MOFF_OK ? (int)r.err : r.state;
    if (latency_ms)
        *latency_ms = r.state == kDone && r.err == MOFF_OK
                          ? std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count()
                          : 0.0;
    return MOFF_OK;
}

moff_status moff_server_wait(moff_server *srv, long long ticket, int timeout_ms) {
    if (!srv) return fail_msg(MOFF_EINVAL, "server is NULL");
    Core *s = srv->core.get();
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] {
        if (ticket == 0) return s->queue.empty() && s->inflight == 0;
        auto it = s->reqs.find(ticket);
        return it == s->reqs.end() || it->second.state == kDone;
    };
    if (ticket != 0 && s->reqs.find(ticket) == s->reqs.end()) return fail_msg(MOFF_EINVAL, "unknown ticket");
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, ready);
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
        return fail_msg(MOFF_ETIMEDOUT, "blocks not finished within the time limit");
    }
    if (ticket != 0) {
        auto it = s->reqs.find(ticket);
        if (it != s->reqs.end() && it->second.err != MOFF_OK) return fail_msg(it->second.err, "block failed");
    }
    return MOFF_OK;
}

moff_status moff_server_stats(moff_server *srv, double *p50_ms, double *p99_ms, double *throughput, long long *completed,
                              int reset) {
    if (!srv) return fail_msg(MOFF_EINVAL, "server is NULL");
    Core *s = srv->core.get();
    std::lock_guard<std::mutex> lk(s->mu);
    if (p50_ms) *p50_ms = percentile(s->lat_ms, 0.50);
    if (p99_ms) *p99_ms = percentile(s->lat_ms, 0.99);
    if (throughput) {
        const double sec =
            s->n_done ? std::chrono::duration<double>(s->t_last - s->t_first).count() : 0.0;
        *throughput = sec > 0.0 ? (double)s->units_done / sec : 0.0;
    }
    if (completed) *completed = s->n_done;
    if (reset) {
        s->lat_ms.clear();
        s->units_done = 0;
        s->n_done = 0;
        s->have_first = false;
        // the next window starts at the oldest block not yet finished, if any
        for (const auto &kv : s->reqs)
            if (kv.second.state != kDone) {
                s->have_first = true;
                s->t_first = kv.second.t_submit;
                break;
            }
    }
    return MOFF_OK;
}

moff_status moff_server_destroy(moff_server *srv) {
    if (!srv) return MOFF_OK;
    Core *s = srv->core.get();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->dirty = true;
    }
    s->cv_work.notify_one();
    if (srv->th.joinable()) srv->th.join();
    cudaFree(s->pool_base);
    delete srv;   // the shared state goes with the last callback holding it
    return MOFF_OK;
}

}  // extern "C"
