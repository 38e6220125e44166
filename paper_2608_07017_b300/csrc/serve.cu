// serve.cu -- request server for PDE solves on device-resident toolboxes.
//
// Requests (a toolbox, coefficient fields, 1..k right-hand sides, linear or semilinear) are
// queued in arrival order and admitted to worker slots as slots free up: continuous batching.
// A slot is one host thread, one non-blocking CUDA stream and one solve workspace; the slots'
// streams run concurrently, so requests in different slots overlap on the GPU.  Within a
// request all right-hand sides are refined together, one CUDA-graph launch per sweep (mixed
// mode; semilinear problems by the chord iteration with an exact-Newton fallback).
// Admission by memory: the device memory free when the server starts (minus a reserve) is the
// budget; a slot's workspace is counted against it from the estimate for the toolbox's shape,
// and a request that would exceed it waits until a slot releases memory.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "solve_internal.hpp"
#include "toolbox.hpp"

namespace ewos {

static double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct ServerRequest {
    uint64_t ticket = 0;
    ewos_toolbox* tb = nullptr;
    ewos_problem pb{};
    std::vector<double> A, b, c, f, g, nl;
    std::vector<double> u, s;
    ewos_solve_report rep{};
    ewos_status status = EWOS_OK;
    std::string err;
    bool done = false;
    int slot = -1;
    double t_submit = 0, t_start = 0, t_end = 0;
};

struct ServerSlot {
    int id = 0;
    cudaStream_t st = nullptr;
    SolveWorkspace* ws = nullptr;
    size_t charged = 0;           // bytes of the budget this slot's workspace holds
    // shape of the toolboxes the workspace was made for, by value (the toolbox itself may be
    // destroyed while the workspace stays with the slot)
    bool has_shape = false;
    int64_t n = 0, m = 0, p = 0;
    int dim = 0;
    int64_t cap_rhs = 0;
    bool mixed = false, fp64 = false;
    bool busy = false;
    std::thread th;
};

}  // namespace ewos

struct ewos_server {
    int device = 0;
    ewos_server_opts opts{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ewos::ServerRequest*> queue;
    std::unordered_map<uint64_t, ewos::ServerRequest*> reqs;
    std::vector<ewos::ServerSlot*> slots;
    bool stop = false;
    uint64_t next_ticket = 1;
    size_t budget = 0, charged = 0;
    int active = 0, peak_active = 0;
    uint64_t submitted = 0, completed = 0, failed = 0;
};

namespace ewos {

static void run_request(ewos_server* sv, ServerSlot* sl, ServerRequest* rq) {
    cudaSetDevice(sv->device);
    ewos_problem pb = rq->pb;
    pb.stream = sl->st;
    pb.inputs_on_device = 0;
    SolveOptions opt;
    opt.batched = pb.mode == EWOS_SOLVE_MIXED;
    opt.newton_reuse = pb.newton_refactor == 0;
    rq->u.assign((size_t)rq->tb->n * pb.nrhs, 0.0);
    rq->s.assign((size_t)rq->tb->m * pb.nrhs, 0.0);
    rq->status = solve_on(rq->tb, sl->ws, &pb, rq->u.data(), rq->s.data(), 0, &rq->rep, opt);
    if (rq->status != EWOS_OK) rq->err = ewos_last_error();   // the worker's message, for the waiter
}

static bool same_shape(const ServerSlot* sl, const ewos_toolbox* tb) {
    return sl->ws && sl->has_shape && sl->n == tb->n && sl->m == tb->m && sl->p == tb->p && sl->dim == tb->dim;
}

static bool slot_fits(const ServerSlot* sl, const ServerRequest* rq) {
    const bool mixed = rq->pb.mode == EWOS_SOLVE_MIXED;
    return same_shape(sl, rq->tb) && sl->cap_rhs >= rq->pb.nrhs && (mixed ? sl->mixed : sl->fp64);
}

// Frees the workspace of an idle slot (called with sv->mu held; the slot cannot start work
// without the lock, and its stream has nothing queued).
static void reclaim(ewos_server* sv, ServerSlot* o) {
    if (!o->ws) return;
    cudaStreamSynchronize(o->st);
    {
        AllocStream as(o->st);
        free_workspace(o->ws);
    }
    cudaStreamSynchronize(o->st);
    o->ws = nullptr;
    sv->charged -= o->charged;
    o->charged = 0;
    o->has_shape = false;
    o->cap_rhs = 0;
    o->mixed = o->fp64 = false;
}

// Memory for slot sl to serve rq (called with sv->mu held).  Returns 1 admitted, 0 wait for
// memory, 2 leave it to an idle slot whose workspace fits, -1 never.
static int admit(ewos_server* sv, ServerSlot* sl, ServerRequest* rq) {
    if (slot_fits(sl, rq)) return 1;
    for (ServerSlot* o : sv->slots)
        if (o != sl && !o->busy && slot_fits(o, rq)) return 2;     // an idle slot can take it as it is
    const bool mixed = rq->pb.mode == EWOS_SOLVE_MIXED;
    const ewos_toolbox* tb = rq->tb;
    const bool same = same_shape(sl, tb);
    const int64_t cap = std::max<int64_t>(rq->pb.nrhs, same ? sl->cap_rhs : 0);
    const bool want_mixed = mixed || (same && sl->mixed);
    const bool want_fp64 = !mixed || (same && sl->fp64);
    const size_t need = (want_mixed ? workspace_bytes(tb, cap, true) : 0) + (want_fp64 ? workspace_bytes(tb, cap, false) : 0);
    if (need > sv->budget) return -1;
    // room from the workspaces of idle slots when the budget is short
    for (ServerSlot* o : sv->slots) {
        if (sv->charged - sl->charged + need <= sv->budget) break;
        if (o != sl && !o->busy) reclaim(sv, o);
    }
    if (sv->charged - sl->charged + need <= sv->budget) {
        // the slot's old workspace is released or grown by the solve; the new estimate is charged
        sv->charged = sv->charged - sl->charged + need;
        sl->charged = need;
        sl->has_shape = true;
        sl->n = tb->n; sl->m = tb->m; sl->p = tb->p; sl->dim = tb->dim;
        sl->cap_rhs = cap;
        sl->mixed = want_mixed;
        sl->fp64 = want_fp64;
        return 1;
    }
    return sv->active > 0 ? 0 : -1;
}

static void worker(ewos_server* sv, ServerSlot* sl) {
    cudaSetDevice(sv->device);
    for (;;) {
        ServerRequest* rq = nullptr;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            for (;;) {
                if (sv->stop && sv->queue.empty()) return;
                if (!sv->queue.empty()) {
                    ServerRequest* front = sv->queue.front();
                    const int a = admit(sv, sl, front);
                    if (a == 2) {
                        sv->cv_work.notify_all();
                    } else if (a != 0) {
                        sv->queue.pop_front();
                        if (a < 0) {
                            front->status = EWOS_ENOMEM;
                            front->err = "ewos_server: the request's workspace does not fit in the memory budget";
                            front->done = true;
                            front->t_start = front->t_end = now_ms();
                            ++sv->failed;
                            sv->cv_done.notify_all();
                            continue;
                        }
                        rq = front;
                        break;
                    }
                }
                sv->cv_work.wait(lk);
            }
            ++sv->active;
            sl->busy = true;
            sv->peak_active = std::max(sv->peak_active, sv->active);
            rq->slot = sl->id;
            rq->t_start = now_ms();
        }
        run_request(sv, sl, rq);
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            rq->t_end = now_ms();
            rq->done = true;
            --sv->active;
            sl->busy = false;
            ++sv->completed;
            if (rq->status != EWOS_OK && rq->status != EWOS_ENOCONV) ++sv->failed;
        }
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
}

}  // namespace ewos

using namespace ewos;

extern "C" ewos_status ewos_server_create(const ewos_server_opts* opts, ewos_server** out) {
    if (!out) { set_error("ewos_server_create: out is NULL"); return EWOS_EINVAL; }
    ewos_server* sv = new ewos_server();
    if (opts) sv->opts = *opts;
    if (sv->opts.max_slots <= 0) sv->opts.max_slots = 4;
    if (sv->opts.max_slots > 64) sv->opts.max_slots = 64;
    if (sv->opts.memory_fraction <= 0 || sv->opts.memory_fraction > 1) sv->opts.memory_fraction = 0.8;
    cudaGetDevice(&sv->device);
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) {
        delete sv;
        set_error(std::string("ewos_server_create: ") + cudaGetErrorString(e));
        return EWOS_ECUDA;
    }
    const size_t reserve = sv->opts.reserve_bytes > 0 ? (size_t)sv->opts.reserve_bytes : 0;
    const size_t usable = free_b > reserve ? free_b - reserve : 0;
    sv->budget = (size_t)(sv->opts.memory_fraction * (double)usable);
    if (sv->opts.budget_bytes > 0) sv->budget = std::min(sv->budget, (size_t)sv->opts.budget_bytes);
    for (int i = 0; i < sv->opts.max_slots; ++i) {
        ServerSlot* sl = new ServerSlot();
        sl->id = i;
        e = cudaStreamCreateWithFlags(&sl->st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete sl;
            break;
        }
        sv->slots.push_back(sl);
    }
    if (sv->slots.empty()) {
        delete sv;
        set_error("ewos_server_create: no stream");
        return EWOS_ECUDA;
    }
    for (ServerSlot* sl : sv->slots) sl->th = std::thread(worker, sv, sl);
    *out = sv;
    return EWOS_OK;
}

extern "C" ewos_status ewos_server_submit(ewos_server* sv, ewos_toolbox* tb, const ewos_problem* pb, uint64_t* ticket) {
    if (!sv || !tb || !pb || !ticket || !pb->A || !pb->f || !pb->g || pb->nrhs < 1) {
        set_error("ewos_server_submit: need server, toolbox, problem with A, f, g, nrhs >= 1, ticket");
        return EWOS_EINVAL;
    }
    if (pb->inputs_on_device) { set_error("ewos_server_submit: inputs must be host arrays"); return EWOS_EINVAL; }
    if (pb->mode != EWOS_SOLVE_FP64 && pb->mode != EWOS_SOLVE_MIXED) { set_error("ewos_server_submit: unknown mode"); return EWOS_EINVAL; }
    if (pb->nl_kind != EWOS_NL_NONE && (!pb->nl_coef || pb->nl_ncoef < 1 || pb->nl_ncoef > 64)) {
        set_error("ewos_server_submit: nonlinearity needs 1..64 coefficients");
        return EWOS_EINVAL;
    }
    ServerRequest* rq = new ServerRequest();
    const int64_t n = tb->n, p = tb->p;
    const int D = tb->dim;
    rq->tb = tb;
    rq->A.assign(pb->A, pb->A + n * D * D);
    if (pb->b) rq->b.assign(pb->b, pb->b + n * D);
    if (pb->c) rq->c.assign(pb->c, pb->c + n);
    rq->f.assign(pb->f, pb->f + n * pb->nrhs);
    rq->g.assign(pb->g, pb->g + p * pb->nrhs);
    if (pb->nl_kind != EWOS_NL_NONE) rq->nl.assign(pb->nl_coef, pb->nl_coef + pb->nl_ncoef);
    rq->pb = *pb;
    rq->pb.A = rq->A.data();
    rq->pb.b = pb->b ? rq->b.data() : nullptr;
    rq->pb.c = pb->c ? rq->c.data() : nullptr;
    rq->pb.f = rq->f.data();
    rq->pb.g = rq->g.data();
    rq->pb.nl_coef = rq->nl.empty() ? nullptr : rq->nl.data();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) {
            delete rq;
            set_error("ewos_server_submit: server is stopping");
            return EWOS_EINVAL;
        }
        rq->ticket = sv->next_ticket++;
        rq->t_submit = now_ms();
        sv->reqs[rq->ticket] = rq;
        sv->queue.push_back(rq);
        ++sv->submitted;
        *ticket = rq->ticket;
    }
    sv->cv_work.notify_all();
    return EWOS_OK;
}

extern "C" ewos_status ewos_server_wait(ewos_server* sv, uint64_t ticket, double timeout_s, double* u_out,
                                        double* s_out, ewos_solve_report* rep, ewos_request_timing* tm) {
    if (!sv) { set_error("ewos_server_wait: NULL server"); return EWOS_EINVAL; }
    ServerRequest* rq = nullptr;
    {
        std::unique_lock<std::mutex> lk(sv->mu);
        auto it = sv->reqs.find(ticket);
        if (it == sv->reqs.end()) { set_error("ewos_server_wait: unknown ticket"); return EWOS_EINVAL; }
        rq = it->second;
        auto ready = [&] { return rq->done; };
        if (timeout_s > 0) {
            if (!sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
                set_error("ewos_server_wait: request still running");
                return EWOS_ETIMEOUT;
            }
        } else {
            sv->cv_done.wait(lk, ready);
        }
        sv->reqs.erase(it);
    }
    if (u_out && !rq->u.empty()) std::memcpy(u_out, rq->u.data(), sizeof(double) * rq->u.size());
    if (s_out && !rq->s.empty()) std::memcpy(s_out, rq->s.data(), sizeof(double) * rq->s.size());
    if (rep) *rep = rq->rep;
    if (tm) {
        tm->queue_ms = rq->t_start - rq->t_submit;
        tm->run_ms = rq->t_end - rq->t_start;
        tm->total_ms = rq->t_end - rq->t_submit;
        tm->slot = rq->slot;
    }
    const ewos_status st = rq->status;
    if (st != EWOS_OK) set_error(rq->err);
    delete rq;
    return st;
}

extern "C" ewos_status ewos_server_query(ewos_server* sv, ewos_server_stats* out) {
    if (!sv || !out) { set_error("ewos_server_query: NULL argument"); return EWOS_EINVAL; }
    std::lock_guard<std::mutex> lk(sv->mu);
    out->submitted = sv->submitted;
    out->completed = sv->completed;
    out->failed = sv->failed;
    out->queued = (int)sv->queue.size();
    out->active = sv->active;
    out->peak_active = sv->peak_active;
    out->slots = (int)sv->slots.size();
    out->budget_bytes = (int64_t)sv->budget;
    out->charged_bytes = (int64_t)sv->charged;
    return EWOS_OK;
}

extern "C" void ewos_server_destroy(ewos_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    for (ServerSlot* sl : sv->slots) {
        if (sl->th.joinable()) sl->th.join();
    }
    for (ServerSlot* sl : sv->slots) {
        if (sl->ws) {
            cudaStreamSynchronize(sl->st);
            AllocStream as(sl->st);
            free_workspace(sl->ws);
        }
        cudaStreamSynchronize(sl->st);
        cudaStreamDestroy(sl->st);
        delete sl;
    }
    for (auto& kv : sv->reqs) delete kv.second;
    delete sv;
}
