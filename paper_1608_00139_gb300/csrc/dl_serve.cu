// dl_serve.cu -- asynchronous requests with continuous batching (dl_submit / dl_poll / dl_cancel).
//
// A context that receives its first dl_submit starts `max_slots` worker threads.  Each slot
// owns a CUDA stream and a resident workspace (grow-only device buffers that stay allocated
// between requests).  Requests wait in a queue; a free slot admits the oldest queued
// request whose device footprint (dense n^2-byte operands plus workspace, footprint_bytes)
// fits the remaining HBM budget, so requests arriving while others run are admitted as
// slots and memory free up, and their kernels overlap on the GPU (each slot its own stream).
// A request's result does not depend on what else runs: the kernels are exact and every
// slot has its own scratch.  Latency is measured from dl_submit to completion on the host's
// monotonic clock.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dl_ctx.h"

using namespace dl;

namespace {

using Clock = std::chrono::steady_clock;

enum Phase { QUEUED, RUNNING, DONE, CANCELED };

struct ReqRec {
    uint64_t ticket = 0;
    dl_request req{};
    Phase phase = QUEUED;
    dl_status status = DL_OK;
    std::string err;
    dl_stats stats{};
    Clock::time_point t_submit, t_admit, t_done;
    size_t footprint = 0;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct dl_ctx::Serve {
    struct Slot {
        std::thread th;
        Workspace ws;
        cudaStream_t stream = nullptr;
    };
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<ReqRec>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<ReqRec>> reqs;
    uint64_t next_ticket = 1;
    size_t budget = 0, in_use = 0;
    bool stop = false;
    std::vector<std::unique_ptr<Slot>> slots;
};

namespace {

void worker(dl_ctx *ctx, dl_ctx::Serve *sv, dl_ctx::Serve::Slot *slot) {
    cudaSetDevice(ctx->device);
    for (;;) {
        std::shared_ptr<ReqRec> r;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            for (;;) {
                if (sv->stop) return;
                // the oldest queued request that fits the remaining budget
                for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
                    if (sv->in_use + (*it)->footprint <= sv->budget) {
                        r = *it;
                        sv->queue.erase(it);
                        break;
                    }
                }
                if (r) break;
                sv->cv_work.wait(lk);
            }
            r->phase = RUNNING;
            r->t_admit = Clock::now();
            sv->in_use += r->footprint;
        }
        dl_status rc = DL_OK;
        std::string err;
        dl_stats st{};
        cudaError_t e = slot->ws.init();
        if (e != cudaSuccess) {
            rc = DL_ENOMEM;
            err = std::string("slot workspace: ") + cudaGetErrorString(e);
        } else {
            SolveArgs a;
            a.n = r->req.n;
            a.E = r->req.base;
            a.E2 = r->req.B;
            a.mem = r->req.mem;
            a.path = r->req.path;
            a.out_bits = r->req.out_bits;
            Range trace_(r->req.kind == 0 ? "serve:closure" : "serve:same_generation");
            rc = r->req.kind == 0 ? solve_tc(ctx, slot->ws, slot->stream, a, &st)
                                  : solve_sg(ctx, slot->ws, slot->stream, a, &st);
            if (rc != DL_OK) {
                err = dl_last_error();
                cudaStreamSynchronize(slot->stream);
                for (cudaStream_t x : slot->ws.mx_stream)
                    if (x) cudaStreamSynchronize(x);
                cudaGetLastError();
            }
        }
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->in_use -= r->footprint;
            r->status = rc;
            r->err = err;
            r->stats = st;
            r->t_done = Clock::now();
            r->stats.ms_queue = ms_between(r->t_submit, r->t_admit);
            r->stats.ms_latency = ms_between(r->t_submit, r->t_done);
            r->phase = DONE;
        }
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();  // memory came free
    }
}

dl_status start_serving(dl_ctx *ctx) {
    if (ctx->serve) return DL_OK;
    auto *sv = new dl_ctx::Serve();
    cudaSetDevice(ctx->device);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    sv->budget = ctx->cfg.hbm_budget_bytes ? ctx->cfg.hbm_budget_bytes : free_b / 2;
    const int nslots = ctx->cfg.max_slots > 0 ? ctx->cfg.max_slots : 4;
    for (int i = 0; i < nslots; ++i) {
        auto slot = std::make_unique<dl_ctx::Serve::Slot>();
        if (cudaStreamCreateWithFlags(&slot->stream, cudaStreamNonBlocking) != cudaSuccess) {
            set_error("serving: cudaStreamCreate failed");
            for (auto &s : sv->slots) cudaStreamDestroy(s->stream);
            delete sv;
            return DL_EDEVICE;
        }
        sv->slots.push_back(std::move(slot));
    }
    ctx->serve = sv;
    for (auto &s : sv->slots) s->th = std::thread(worker, ctx, sv, s.get());
    return DL_OK;
}

}  // namespace

void dl_serve_shutdown(dl_ctx *ctx) {
    dl_ctx::Serve *sv = ctx ? ctx->serve : nullptr;
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    for (auto &s : sv->slots)
        if (s->th.joinable()) s->th.join();
    cudaSetDevice(ctx->device);
    for (auto &s : sv->slots) {
        cudaStreamSynchronize(s->stream);
        s->ws.release();
        cudaStreamDestroy(s->stream);
    }
    delete sv;
    ctx->serve = nullptr;
}

extern "C" {

dl_status dl_submit(dl_ctx *ctx, const dl_request *req, uint64_t *ticket) {
    if (!ctx || !req || !ticket) {
        set_error("ctx, req and ticket must not be NULL");
        return DL_EINVAL;
    }
    *ticket = 0;
    if (req->kind != 0 && req->kind != 1) {
        set_error("request kind must be 0 (closure) or 1 (same generation)");
        return DL_EINVAL;
    }
    if (req->n < 0 || (req->mem != DL_MEM_HOST && req->mem != DL_MEM_DEVICE) ||
        (req->n > 0 && (!req->base || !req->out_bits)) || (req->kind == 0 && req->B)) {
        set_error("bad request (n, memory kind, NULL pointer, or B given for a closure)");
        return DL_EINVAL;
    }
    if (req->path != DL_PATH_AUTO && req->path != DL_PATH_BOOL_FP8) {
        set_error("serving runs DL_PATH_AUTO / DL_PATH_BOOL_FP8 requests");
        return DL_ENOTIMPL;
    }
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        dl_status rc = start_serving(ctx);
        if (rc) return rc;
    }
    dl_ctx::Serve *sv = ctx->serve;
    auto r = std::make_shared<ReqRec>();
    r->req = *req;
    r->footprint = req->n > 0 ? footprint_bytes(req->kind, req->n) : 0;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (r->footprint > sv->budget) {
            set_error("request needs %zu bytes, more than the serving budget %zu", r->footprint, sv->budget);
            return DL_ENOMEM;
        }
        r->ticket = sv->next_ticket++;
        *ticket = r->ticket;
        sv->reqs[r->ticket] = r;
        if (req->n == 0) {  // nothing to compute
            r->phase = DONE;
            r->t_admit = r->t_done = r->t_submit;
        } else {
            sv->queue.push_back(r);
        }
    }
    sv->cv_work.notify_one();
    return DL_OK;
}

dl_status dl_poll(dl_ctx *ctx, uint64_t ticket, int64_t timeout_us, dl_stats *stats) {
    if (!ctx || !ctx->serve) {
        set_error("no request was submitted on this context");
        return DL_EINVAL;
    }
    dl_ctx::Serve *sv = ctx->serve;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) {
        set_error("unknown or already collected ticket %llu", static_cast<unsigned long long>(ticket));
        return DL_EINVAL;
    }
    std::shared_ptr<ReqRec> r = it->second;
    auto finished = [&] { return r->phase == DONE || r->phase == CANCELED; };
    if (!finished()) {
        if (timeout_us < 0) sv->cv_done.wait(lk, finished);
        else if (timeout_us > 0) sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), finished);
    }
    if (!finished()) return DL_EBUSY;
    sv->reqs.erase(it);
    if (r->phase == CANCELED) {
        set_error("request %llu was cancelled", static_cast<unsigned long long>(ticket));
        return DL_ECANCELED;
    }
    if (stats) *stats = r->stats;
    if (r->status != DL_OK) set_error("%s", r->err.c_str());
    return r->status;
}

dl_status dl_cancel(dl_ctx *ctx, uint64_t ticket) {
    if (!ctx || !ctx->serve) {
        set_error("no request was submitted on this context");
        return DL_EINVAL;
    }
    dl_ctx::Serve *sv = ctx->serve;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) {
        set_error("unknown ticket %llu", static_cast<unsigned long long>(ticket));
        return DL_EINVAL;
    }
    std::shared_ptr<ReqRec> r = it->second;
    if (r->phase != QUEUED) return DL_EBUSY;
    for (auto q = sv->queue.begin(); q != sv->queue.end(); ++q)
        if (*q == r) {
            sv->queue.erase(q);
            break;
        }
    r->phase = CANCELED;
    sv->cv_done.notify_all();
    return DL_OK;
}

}  // extern "C"
