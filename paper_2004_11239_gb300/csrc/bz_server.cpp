// Serving loop: continuous batching of homogeneous relaxation solves (RK4 on the collision
// operator) of mixed N, (gamma, s), data form and precision.
//
// A worker thread owns the device work.  Requests with the same plan geometry, data form,
// precision and dt form a group with its own plan, batch (gamma per slot), stream and
// completion event; a group steps all its active slots with one bz_batch_step_rk call (one
// batched kernel per RK stage on the fused pipeline, the slots one after another on the chunked
// one).  The worker loops over the groups:
//   - admission, in arrival order, while the HBM budget and group slots allow (a request whose
//     own footprint exceeds the whole budget fails with BZ_ERR_OOM; one queued longer than its
//     max_queue_s fails with BZ_ERR_TIMEOUT); a request admitted to a group whose step is in
//     flight joins its next step,
//   - a group whose event has completed (cudaEventQuery, never a blocking wait on another
//     group) retires that step: each participant advances one RK4 step, finished requests copy
//     their result to the host (BZ_ERR_NONFINITE if it holds NaN or Inf, BZ_ERR_CUDA if the
//     step failed) and free their slots,
//   - an idle group with active requests launches its next step and records its event.
// Groups therefore run ahead independently and overlap on the device, except that at most one
// heavy (chunked-pipeline) step is in flight at a time -- concurrent chunked pipelines evict
// each other's L2-resident scratch -- chosen by shortest remaining work (the group that can
// finish a request soonest), aged by the time since the group last stepped so that none waits
// for ever.  (All
// streams keep the default priority: giving light groups a higher one starved the heavy ones
// under load.)  State stays on the
// device from admission to completion; results do not depend on the other requests in flight
// (batched results are per-instance invariant).  Idle plans and batches stay cached until the
// budget needs their memory.
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <vector>

#include "bz_internal.h"

struct bz_plan;

namespace bz {
const Plan *plan_internal(const bz_plan *plan);
}

namespace {

using Clock = std::chrono::steady_clock;

struct Key {
    int N, N_rho, M, kernel, data, precision;
    double L, R, s, dt, gamma_plan;   // gamma_plan is 0 for batched groups (gamma per slot)
    bool operator<(const Key &o) const {
        return std::tie(N, N_rho, M, kernel, data, precision, L, R, s, dt, gamma_plan) <
               std::tie(o.N, o.N_rho, o.M, o.kernel, o.data, o.precision, o.L, o.R, o.s, o.dt, o.gamma_plan);
    }
};

struct Request {
    uint64_t id = 0;
    bz_request req{};
    std::vector<double2> input;        // host copy of fhat0 (FP64)
    std::vector<double2> output;       // host result
    int steps_total = 0, steps_done = 0;
    int status = BZ_ERR_BUSY;          // BZ_ERR_BUSY while queued or running
    int slot = -1;
    struct Group *group = nullptr;
    Clock::time_point t_submit, t_admit, t_done;
};

struct Group {
    Key key{};
    bz_plan *plan = nullptr;
    bz_batch *batch = nullptr;
    double2 *state = nullptr;          // [capacity][N^3] c128
    int capacity = 0;
    std::vector<Request *> slots;      // per slot (nullptr = free)
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;        // recorded after each step's launches
    bool inflight = false;
    bool heavy = false;                // chunked pipeline: its scratch fills L2 (one such step at a time)
    Clock::time_point last_step;       // launch time of its latest step (ages the heavy choice)
    int launch_status = BZ_OK;         // status of the in-flight step's launches
    std::vector<Request *> running;    // participants of the in-flight step
    size_t bytes = 0;
    Clock::time_point last_used;
    int active() const {
        int n = 0;
        for (auto *r : slots) n += r != nullptr;
        return n;
    }
};

}  // namespace

struct bz_server {
    int device = 0;
    size_t budget = 0, used = 0;
    int max_batch = 64;
    int terms_per_item = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request *> queue;
    std::map<uint64_t, std::unique_ptr<Request>> all;
    std::map<Key, std::unique_ptr<Group>> groups;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread worker;
    // statistics
    long completed = 0, steps = 0;
    double busy_s = 0.0;
};

namespace {

// Groups on the fused pipeline (N <= 32; N | 32 for the real-data form) keep per-slot working
// arrays in their batch; on the chunked pipeline the batch holds only the slots' radial scales.
bool fused(const bz_request &r) {
    if (r.N > 32) return false;
    return r.data != BZ_DATA_REAL || 32 % r.N == 0;
}

size_t plan_bytes(const bz_request &r) {
    const size_t n3 = (size_t)r.N * r.N * r.N;
    const size_t P = (size_t)r.N_rho * r.M;
    size_t b = P * n3 * 8 + P * 3 * r.N * 8 + (size_t)(64u << 20) + 6 * n3 * 16;
    if (r.data == BZ_DATA_REAL) b += (P / 2) * (n3 * 8 + (size_t)3 * r.N * r.N * 8) + 2 * n3 * 16;
    return b;
}

size_t batch_bytes(const bz_request &r, int capacity) {
    const size_t n3 = (size_t)r.N * r.N * r.N;
    const size_t P = (size_t)r.N_rho * r.M;
    const size_t nblk_max = (P + 15) / 16;
    if (!fused(r)) return (size_t)capacity * n3 * 16;                       // the slots' state
    return (size_t)capacity * n3 * (8 + 8 * nblk_max + 32 + 16 + 16 + (r.data == BZ_DATA_REAL ? 8 : 0));
}

Key key_of(const bz_request &r) {
    Key k{r.N, r.N_rho, r.M, r.kernel, r.data, r.precision, r.L, r.R, r.s, r.dt, 0.0};
    return k;
}

void destroy_group(bz_server *S, Group *g) {
    if (g->batch) bz_batch_destroy(g->batch);
    if (g->plan) bz_plan_destroy(g->plan);
    cudaFree(g->state);
    if (g->done) cudaEventDestroy(g->done);
    if (g->stream) cudaStreamDestroy(g->stream);
    S->used -= g->bytes;
}

// Frees idle groups (least recently used first) until `need` more bytes fit.
bool make_room(bz_server *S, size_t need) {
    while (S->used + need > S->budget) {
        Group *victim = nullptr;
        for (auto &kv : S->groups) {
            Group *g = kv.second.get();
            if (g->active() == 0 && (!victim || g->last_used < victim->last_used)) victim = g;
        }
        if (!victim) return false;
        destroy_group(S, victim);
        S->groups.erase(victim->key);
    }
    return true;
}

Group *get_group(bz_server *S, const bz_request &r, int *err) {
    Key k = key_of(r);
    auto it = S->groups.find(k);
    if (it != S->groups.end()) return it->second.get();
    const int cap = S->max_batch;
    const size_t need = plan_bytes(r) + batch_bytes(r, cap);
    if (need > S->budget) { *err = BZ_ERR_OOM; return nullptr; }
    if (!make_room(S, need)) { *err = BZ_ERR_BUSY; return nullptr; }
    std::unique_ptr<Group> g(new Group());
    g->key = k;
    bz_plan_desc d;
    std::memset(&d, 0, sizeof(d));
    d.N = r.N; d.L = r.L; d.R = r.R; d.gamma = k.gamma_plan; d.s = r.s; d.N_rho = r.N_rho; d.M = r.M;
    d.kernel = r.kernel; d.precision = r.precision; d.data = r.data;
    int st = bz_plan_create_ex(&g->plan, &d);
    if (st != BZ_OK) { *err = st; return nullptr; }
    if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (g->stream) cudaStreamDestroy(g->stream);
        bz_plan_destroy(g->plan);
        *err = BZ_ERR_CUDA;
        return nullptr;
    }
    {
        st = bz_batch_create(&g->batch, g->plan, cap, S->terms_per_item);
        const size_t n3 = (size_t)r.N * r.N * r.N;
        if (st == BZ_OK && cudaMalloc(&g->state, (size_t)cap * n3 * sizeof(double2)) != cudaSuccess) st = BZ_ERR_OOM;
        if (st != BZ_OK) {
            cudaGetLastError();
            if (g->batch) bz_batch_destroy(g->batch);
            bz_plan_destroy(g->plan);
            cudaEventDestroy(g->done);
            cudaStreamDestroy(g->stream);
            *err = st;
            return nullptr;
        }
        g->capacity = cap;
        g->slots.assign(cap, nullptr);
        g->heavy = !fused(r);
    }
    g->bytes = need;
    g->last_used = Clock::now();
    S->used += need;
    Group *raw = g.get();
    S->groups.emplace(k, std::move(g));
    return raw;
}

// Admission in arrival order; stops at the first request that cannot be placed yet.
void admit(bz_server *S) {
    while (!S->queue.empty()) {
        Request *q = S->queue.front();
        const bz_request &r = q->req;
        if (r.max_queue_s > 0 &&
            std::chrono::duration<double>(Clock::now() - q->t_submit).count() > r.max_queue_s) {
            q->status = BZ_ERR_TIMEOUT;
            q->t_done = Clock::now();
            S->queue.pop_front();
            continue;
        }
        int err = BZ_OK;
        Group *g = get_group(S, r, &err);
        if (!g) {
            if (err == BZ_ERR_BUSY) return;               // wait for memory
            q->status = err;
            q->t_done = Clock::now();
            S->queue.pop_front();
            continue;
        }
        const size_t n3 = (size_t)r.N * r.N * r.N;
        int slot = -1;
        for (int k = 0; k < g->capacity; ++k)
            if (!g->slots[k]) { slot = k; break; }
        if (slot < 0) return;                              // group full: wait for a slot
        if (bz_batch_set_gamma(g->batch, slot, r.gamma) != BZ_OK ||
            cudaMemcpyAsync(g->state + (size_t)slot * n3, q->input.data(), n3 * sizeof(double2),
                            cudaMemcpyHostToDevice, g->stream) != cudaSuccess) {
            q->status = BZ_ERR_CUDA;
            q->t_done = Clock::now();
            S->queue.pop_front();
            continue;
        }
        g->slots[slot] = q;
        q->slot = slot;
        q->group = g;
        q->t_admit = Clock::now();
        g->last_used = q->t_admit;
        S->queue.pop_front();
    }
}

// Retires a request: its result to the host (a finite check on it), its slot or state freed.
// The group's stream is idle here (its step has completed; at most an admission copy follows).
void finish(bz_server *S, Request *q, int status) {
    Group *g = q->group;
    const size_t n3 = (size_t)q->req.N * q->req.N * q->req.N;
    q->output.resize(n3);
    const void *src = g->state + (size_t)q->slot * n3;
    if (status == BZ_OK &&
        (cudaMemcpyAsync(q->output.data(), src, n3 * sizeof(double2), cudaMemcpyDeviceToHost, g->stream) != cudaSuccess ||
         cudaStreamSynchronize(g->stream) != cudaSuccess))
        status = BZ_ERR_CUDA;
    if (status == BZ_OK)
        for (const double2 &v : q->output)
            if (!(std::isfinite(v.x) && std::isfinite(v.y))) {
                status = BZ_ERR_NONFINITE;
                break;
            }
    g->slots[q->slot] = nullptr;
    q->status = status;
    q->t_done = Clock::now();
    g->last_used = q->t_done;
    S->completed++;
}

// Retires the completed step of g (its event has fired or failed).
void retire_step(bz_server *S, Group *g, cudaError_t ev) {
    const int st = ev == cudaSuccess ? g->launch_status : BZ_ERR_CUDA;
    g->inflight = false;
    std::vector<Request *> run;
    run.swap(g->running);
    for (Request *q : run) {
        if (st != BZ_OK) { finish(S, q, st); continue; }
        S->steps++;
        if (++q->steps_done >= q->steps_total) finish(S, q, BZ_OK);
    }
}

// Launches one RK4 step of every active request of g on its stream and records its event.
void launch_step(Group *g) {
    g->running.clear();
    std::vector<int> sl;
    for (int i = 0; i < g->capacity; ++i)
        if (g->slots[i]) {
            sl.push_back(i);
            g->running.push_back(g->slots[i]);
        }
    int st = bz_batch_step_rk(g->batch, (int)sl.size(), sl.data(), g->state, BZ_C128, g->key.dt, 1, g->stream);
    if (cudaEventRecord(g->done, g->stream) != cudaSuccess && st == BZ_OK) st = BZ_ERR_CUDA;
    g->launch_status = st;
    g->inflight = true;
    g->last_step = Clock::now();
}

void worker_main(bz_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        admit(S);
        bool progressed = false, inflight = false, heavy_busy = false;
        auto t0 = Clock::now();
        for (auto &kv : S->groups) {
            Group *g = kv.second.get();
            if (g->inflight) {
                const cudaError_t ev = cudaEventQuery(g->done);
                if (ev == cudaErrorNotReady) {
                    inflight = true;
                    heavy_busy = heavy_busy || g->heavy;
                    continue;
                }
                retire_step(S, g, ev);
                progressed = true;
            }
            if (g->active() > 0 && !g->heavy) {        // light groups: as soon as they are idle
                launch_step(g);
                inflight = true;
                progressed = true;
            }
        }
        if (!heavy_busy) {
            // one heavy step at a time (concurrent chunked pipelines evict each other's scratch
            // from L2): the heavy group that finishes a request soonest first (shortest remaining
            // work: its fewest remaining steps times the work of one of its steps)
            Group *next = nullptr;
            double best = 0.0;
            for (auto &kv : S->groups) {
                Group *g = kv.second.get();
                if (!g->heavy || g->inflight || g->active() == 0) continue;
                int left = 1 << 30;
                for (Request *q : g->slots)
                    if (q && q->steps_total - q->steps_done < left) left = q->steps_total - q->steps_done;
                const double n3 = (double)g->key.N * g->key.N * g->key.N;
                // aged: a group left waiting for seconds comes back into turn
                const double age = std::chrono::duration<double>(Clock::now() - g->last_step).count();
                const double work = (double)left * g->active() * n3 * std::log2((double)g->key.N) *
                                    g->key.N_rho * g->key.M / (1.0 + age * age);
                if (!next || work < best) {
                    next = g;
                    best = work;
                }
            }
            if (next) {
                launch_step(next);
                inflight = true;
                progressed = true;
            }
        }
        if (progressed) {
            S->busy_s += std::chrono::duration<double>(Clock::now() - t0).count();
            S->cv.notify_all();
        } else {
            // nothing completed: poll again shortly (steps in flight) or wait for a request
            S->cv.wait_for(lk, inflight ? std::chrono::microseconds(50) : std::chrono::microseconds(2000));
        }
    }
}

}  // namespace

extern "C" {

bz_status bz_server_create(bz_server **out, size_t hbm_budget_bytes, int max_batch, int terms_per_item) {
    if (!out || hbm_budget_bytes == 0 || max_batch < 1) return BZ_ERR_ARG;
    *out = nullptr;
    bz_server *S = new (std::nothrow) bz_server();
    if (!S) return BZ_ERR_OOM;
    cudaGetDevice(&S->device);
    S->budget = hbm_budget_bytes;
    S->max_batch = max_batch;
    S->terms_per_item = terms_per_item;
    try {
        S->worker = std::thread(worker_main, S);
    } catch (...) {
        delete S;
        return BZ_ERR_OOM;
    }
    *out = S;
    return BZ_OK;
}

bz_status bz_submit(bz_server *S, const bz_request *req, uint64_t *ticket) {
    if (!S || !req || !ticket || !req->fhat0) return BZ_ERR_ARG;
    const bz_request &r = *req;
    if (!bz::supported_N(r.N) || r.N_rho < 1 || r.M < 1 || !(r.dt > 0) || !(r.t_end >= r.t0) ||
        (r.dtype != BZ_C64 && r.dtype != BZ_C128) || r.kernel < BZ_KERNEL_FAMILY || r.kernel > BZ_KERNEL_B8 ||
        (r.data != BZ_DATA_COMPLEX && r.data != BZ_DATA_REAL) ||
        (r.precision != BZ_PREC_FP32 && r.precision != BZ_PREC_BF16X3))
        return BZ_ERR_ARG;
    if ((r.data == BZ_DATA_REAL && (r.M & 1)) ||
        (r.precision == BZ_PREC_BF16X3 && (r.N != 32 || r.data != BZ_DATA_COMPLEX)))
        return BZ_ERR_UNSUPPORTED;
    std::unique_ptr<Request> q(new (std::nothrow) Request());
    if (!q) return BZ_ERR_OOM;
    q->req = r;
    q->req.fhat0 = nullptr;
    const size_t n3 = (size_t)r.N * r.N * r.N;
    q->input.resize(n3);
    if (r.dtype == BZ_C128) {
        std::memcpy(q->input.data(), r.fhat0, n3 * sizeof(double2));
    } else {
        const float2 *f = (const float2 *)r.fhat0;
        for (size_t i = 0; i < n3; ++i) q->input[i] = make_double2(f[i].x, f[i].y);
    }
    q->steps_total = (int)std::llround((r.t_end - r.t0) / r.dt);
    q->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    q->id = S->next_id++;
    *ticket = q->id;
    S->queue.push_back(q.get());
    S->all.emplace(q->id, std::move(q));
    S->cv.notify_all();
    return BZ_OK;
}

bz_status bz_poll(bz_server *S, uint64_t ticket, bz_result *out, void *fhat_out, int dtype) {
    if (!S || !out) return BZ_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return BZ_ERR_ARG;
    Request *q = it->second.get();
    if (q->status == BZ_ERR_BUSY) return BZ_ERR_BUSY;
    out->status = q->status;
    out->steps = q->steps_done;
    out->t = q->req.t0 + q->steps_done * q->req.dt;
    out->latency_s = std::chrono::duration<double>(q->t_done - q->t_submit).count();
    out->queue_s = q->group ? std::chrono::duration<double>(q->t_admit - q->t_submit).count() : out->latency_s;
    if (q->status == BZ_OK && fhat_out) {
        const size_t n3 = q->output.size();
        if (dtype == BZ_C128) std::memcpy(fhat_out, q->output.data(), n3 * sizeof(double2));
        else {
            float2 *f = (float2 *)fhat_out;
            for (size_t i = 0; i < n3; ++i) f[i] = make_float2((float)q->output[i].x, (float)q->output[i].y);
        }
    }
    S->all.erase(it);
    return BZ_OK;
}

bz_status bz_server_stats(bz_server *S, long *completed, long *steps, size_t *hbm_used, int *queued, int *active) {
    if (!S) return BZ_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (completed) *completed = S->completed;
    if (steps) *steps = S->steps;
    if (hbm_used) *hbm_used = S->used;
    if (queued) *queued = (int)S->queue.size();
    if (active) {
        int n = 0;
        for (auto &kv : S->groups) n += kv.second->active();
        *active = n;
    }
    return BZ_OK;
}

void bz_server_destroy(bz_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    for (auto &kv : S->groups) destroy_group(S, kv.second.get());
    delete S;
}

}  // extern "C"
