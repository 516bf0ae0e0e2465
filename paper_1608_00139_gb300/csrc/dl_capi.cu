// dl_capi.cu -- the extern "C" entry points of libdl (declared in include/dl.h): argument
// checks, context management, and dispatch to the drivers in dl_solve.cu / dl_serve.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "dl_ctx.h"
#include "dl_ptx.cuh"

namespace dl {

namespace {
thread_local std::string g_last_error;
}

void set_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

const char *last_error() { return g_last_error.c_str(); }
void clear_error() { g_last_error.clear(); }

int num_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

namespace {
// Waits on an mbarrier that nobody arrives at; the bounded wait must give up.
__global__ void selftest_wait_kernel(int *status, uint64_t budget_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait_bounded(&bar, 0u, budget_ns, status, ST_TIMEOUT_DEP);
    __syncthreads();
}
}  // namespace

}  // namespace dl

using namespace dl;

#define GUARD_CTX(ctx)                                \
    do {                                              \
        if (!(ctx)) {                                 \
            set_error("ctx is NULL");                 \
            return DL_EINVAL;                         \
        }                                             \
    } while (0)

namespace {

dl_status set_device(dl_ctx *ctx) {
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) {
        set_error("cudaSetDevice(%d): %s", ctx->device, cudaGetErrorString(e));
        return DL_EDEVICE;
    }
    return DL_OK;
}

bool valid_mem(dl_mem m) { return m == DL_MEM_HOST || m == DL_MEM_DEVICE; }

template <class F>
dl_status run_sync(dl_ctx *ctx, dl_stats *stats, F &&f) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    dl_status rc = set_device(ctx);
    if (rc) return rc;
    cudaError_t e = ctx->ws.init();
    if (e != cudaSuccess) {
        set_error("workspace init: %s", cudaGetErrorString(e));
        return DL_ENOMEM;
    }
    dl_stats local{};
    rc = f(ctx->ws, ctx->stream, stats ? stats : &local);
    if (rc != DL_OK) {
        // leave the streams idle and usable after a failure (the mixed path's two as well)
        cudaStreamSynchronize(ctx->stream);
        for (cudaStream_t x : ctx->ws.mx_stream)
            if (x) cudaStreamSynchronize(x);
        cudaGetLastError();
    }
    return rc;
}

// With dl_config.autotune, a size bucket met for the first time is tuned before the call.
dl_status maybe_autotune(dl_ctx *ctx, Workspace &ws, cudaStream_t s, int32_t n) {
    if (!ctx->tune.autotune || n <= 0) return DL_OK;
    if (tuned(ctx, (static_cast<int64_t>(n) + 255) / 256 * 256).measured) return DL_OK;
    TuneEntry e;
    std::string src;
    return autotune_bucket(ctx, ws, s, n, false, &e, &src);
}

}  // namespace

extern "C" {

dl_status dl_create(dl_ctx **out, int device, const dl_config *cfg) {
    clear_error();
    Range trace_(__func__);
    if (!out) {
        set_error("out is NULL");
        return DL_EINVAL;
    }
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
        cudaGetLastError();
        set_error("no CUDA device");
        return DL_EDEVICE;
    }
    if (device < 0 || device >= count) {
        set_error("device %d out of range [0, %d)", device, count);
        return DL_EINVAL;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        set_error("cudaGetDeviceProperties failed");
        return DL_EDEVICE;
    }
    if (prop.major != 10 || prop.minor != 3) {
        set_error("device %d is sm_%d%d; this library is built for sm_103a (GB300)", device, prop.major,
                  prop.minor);
        return DL_EDEVICE;
    }
    auto *ctx = new (std::nothrow) dl_ctx();
    if (!ctx) {
        set_error("out of host memory");
        return DL_ENOMEM;
    }
    ctx->device = device;
    if (cfg) ctx->cfg = *cfg;
    if (ctx->cfg.wait_timeout_s > 0) ctx->budget_ns = static_cast<uint64_t>(ctx->cfg.wait_timeout_s * 1e9);
    if (set_device(ctx) != DL_OK) {
        delete ctx;
        return DL_EDEVICE;
    }
    ctx->sms = prop.multiProcessorCount;
    if (cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        set_error("cudaStreamCreate failed");
        delete ctx;
        return DL_EDEVICE;
    }
    ctx->stream = ctx->cfg.stream ? static_cast<cudaStream_t>(ctx->cfg.stream) : ctx->own_stream;
    tune_init(ctx);  // key prefix, flags, and the cache's entries for this GPU and driver
    *out = ctx;
    return DL_OK;
}

dl_status dl_destroy(dl_ctx *ctx) {
    clear_error();
    Range trace_(__func__);
    if (!ctx) return DL_OK;
    dl_serve_shutdown(ctx);
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        cudaSetDevice(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        ctx->ws.release();
        if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    }
    delete ctx;
    return DL_OK;
}

const char *dl_last_error(void) { return last_error(); }

dl_status dl_set_stream(dl_ctx *ctx, void *stream) {
    clear_error();
    Range trace_(__func__);
    GUARD_CTX(ctx);
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->stream = stream ? static_cast<cudaStream_t>(stream) : ctx->own_stream;
    return DL_OK;
}

dl_status dl_tc_closure(dl_ctx *ctx, int32_t n, const uint8_t *E, dl_mem mem, double eps,
                        double thr, dl_path path, uint64_t *out_bits, double *out_rtilde,
                        dl_stats *stats) {
    clear_error();
    Range trace_(__func__);
    GUARD_CTX(ctx);
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (n < 0 || !valid_mem(mem)) {
        set_error("bad n (%d) or memory kind", n);
        return DL_EINVAL;
    }
    if (n == 0) return DL_OK;
    if (!E || !out_bits) {
        set_error("E and out_bits must not be NULL");
        return DL_EINVAL;
    }
    SolveArgs a;
    a.n = n;
    a.E = E;
    a.mem = mem;
    a.eps = eps;
    a.thr = thr;
    a.path = path;
    a.out_bits = out_bits;
    a.out_rtilde = out_rtilde;
    return run_sync(ctx, stats, [&](Workspace &ws, cudaStream_t s, dl_stats *st) {
        dl_status r = maybe_autotune(ctx, ws, s, a.n);
        return r ? r : solve_tc(ctx, ws, s, a, st);
    });
}

dl_status dl_tc_closure_bits(dl_ctx *ctx, int32_t n, const uint64_t *E_bits, dl_mem mem, double eps,
                             double thr, dl_path path, uint64_t *out_bits, double *out_rtilde,
                             dl_stats *stats) {
    clear_error();
    Range trace_(__func__);
    GUARD_CTX(ctx);
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (n < 0 || !valid_mem(mem)) {
        set_error("bad n (%d) or memory kind", n);
        return DL_EINVAL;
    }
    if (n == 0) return DL_OK;
    if (!E_bits || !out_bits) {
        set_error("E_bits and out_bits must not be NULL");
        return DL_EINVAL;
    }
    SolveArgs a;
    a.n = n;
    a.E_bits = E_bits;
    a.mem = mem;
    a.eps = eps;
    a.thr = thr;
    a.path = path;
    a.out_bits = out_bits;
    a.out_rtilde = out_rtilde;
    return run_sync(ctx, stats, [&](Workspace &ws, cudaStream_t s, dl_stats *st) {
        dl_status r = maybe_autotune(ctx, ws, s, a.n);
        return r ? r : solve_tc(ctx, ws, s, a, st);
    });
}

dl_status dl_sg_least_model(dl_ctx *ctx, int32_t n, const uint8_t *P, const uint8_t *B,
                            dl_mem mem, double eps, double thr, dl_path path,
                            uint64_t *out_bits, dl_stats *stats) {
    clear_error();
    Range trace_(__func__);
    GUARD_CTX(ctx);
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (n < 0 || !valid_mem(mem)) {
        set_error("bad n (%d) or memory kind", n);
        return DL_EINVAL;
    }
    if (n == 0) return DL_OK;
    if (!P || !out_bits) {
        set_error("P and out_bits must not be NULL");
        return DL_EINVAL;
    }
    SolveArgs a;
    a.n = n;
    a.E = P;
    a.E2 = B;
    a.mem = mem;
    a.eps = eps;
    a.thr = thr;
    a.path = path;
    a.out_bits = out_bits;
    return run_sync(ctx, stats, [&](Workspace &ws, cudaStream_t s, dl_stats *st) {
        dl_status r = maybe_autotune(ctx, ws, s, a.n);
        return r ? r : solve_sg(ctx, ws, s, a, st);
    });
}

dl_status dl_tail_recursive(dl_ctx *ctx, int32_t n, const uint8_t *B0, const uint8_t *A, dl_mem mem, double eps,
                            double thr, dl_path path, uint64_t *out_bits, double *out_rtilde, dl_stats *stats) {
    clear_error();
    Range trace_(__func__);
    GUARD_CTX(ctx);
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (n < 0 || !valid_mem(mem)) {
        set_error("bad n (%d) or memory kind", n);
        return DL_EINVAL;
    }
    if (n == 0) return DL_OK;
    if (!B0 || !A || !out_bits) {
        set_error("B0, A and out_bits must not be NULL");
        return DL_EINVAL;
    }
    SolveArgs a;
    a.n = n;
    a.E = B0;
    a.E2 = A;
    a.mem = mem;
    a.eps = eps;
    a.thr = thr;
    a.path = path;
    a.out_bits = out_bits;
    a.out_rtilde = out_rtilde;
    return run_sync(ctx, stats, [&](Workspace &ws, cudaStream_t s, dl_stats *st) {
        return solve_tail(ctx, ws, s, a, st);
    });
}

dl_status dl_tail_recursive_real(dl_ctx *ctx, int32_t n, const uint8_t *B0, const uint8_t *A1, int32_t nterms,
                                 const uint8_t *const *B, const double *const *R, dl_mem mem, double eps, dl_path path,
                                 uint64_t *out_bits, double *out_rtilde, dl_stats *stats) {
    clear_error();
    Range trace_(__func__);
    GUARD_CTX(ctx);
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (n < 0 || nterms < 0 || !valid_mem(mem)) {
        set_error("bad n (%d), nterms (%d) or memory kind", n, nterms);
        return DL_EINVAL;
    }
    if (n == 0) return DL_OK;
    if (!out_bits || (nterms > 0 && (!B || !R))) {
        set_error("out_bits, and B and R when nterms > 0, must not be NULL");
        return DL_EINVAL;
    }
    for (int32_t k = 0; k < nterms; ++k)
        if (!B[k] || !R[k]) {
            set_error("B[%d] and R[%d] must not be NULL", k, k);
            return DL_EINVAL;
        }
    return run_sync(ctx, stats, [&](Workspace &ws, cudaStream_t s, dl_stats *st) -> dl_status {
        const size_t nn = static_cast<size_t>(n) * n;
        auto stage = [&](const void *src, size_t bytes, const std::string &name, const void **out) -> dl_status {
            if (!src || mem == DL_MEM_DEVICE) {
                *out = src;
                return DL_OK;
            }
            void *d = ws.get(name, std::max<size_t>(bytes, 16));
            if (!d) {
                set_error("device allocation failed (%s)", name.c_str());
                return DL_ENOMEM;
            }
            if (cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) {
                set_error("copy of %s to the device failed", name.c_str());
                return DL_EDEVICE;
            }
            *out = d;
            return DL_OK;
        };
        const void *b0 = nullptr, *a1 = nullptr;
        dl_status rc;
        if ((rc = stage(B0, nn, "tq_b0", &b0)) || (rc = stage(A1, nn, "tq_a1", &a1))) return rc;
        std::vector<const uint8_t *> bq(static_cast<size_t>(nterms));
        std::vector<const double *> rq(static_cast<size_t>(nterms));
        for (int32_t k = 0; k < nterms; ++k) {
            const void *bd = nullptr, *rd = nullptr;
            if ((rc = stage(B[k], nn, "tq_term_b" + std::to_string(k), &bd)) ||
                (rc = stage(R[k], nn * 8, "tq_term_r" + std::to_string(k), &rd)))
                return rc;
            bq[k] = static_cast<const uint8_t *>(bd);
            rq[k] = static_cast<const double *>(rd);
        }
        return solve_tail_real(ctx, ws, s, n, static_cast<const uint8_t *>(b0), static_cast<const uint8_t *>(a1),
                               nterms, bq.data(), rq.data(), eps, path, mem, out_bits, out_rtilde, st);
    });
}

dl_status dl_tail_system(dl_ctx *ctx, int32_t n, int32_t m, const dl_tail_eq *eqs, dl_mem mem, dl_path path,
                         uint64_t *const *out_bits, double *const *out_rtilde, dl_stats *stats) {
    clear_error();
    Range trace_(__func__);
    GUARD_CTX(ctx);
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (n < 0 || m < 0 || !valid_mem(mem)) {
        set_error("bad n (%d), m (%d) or memory kind", n, m);
        return DL_EINVAL;
    }
    if (n == 0 || m == 0) return DL_OK;
    if (!eqs || !out_bits) {
        set_error("eqs and out_bits must not be NULL");
        return DL_EINVAL;
    }
    return run_sync(ctx, stats, [&](Workspace &ws, cudaStream_t s, dl_stats *st) {
        return solve_tail_system(ctx, ws, s, n, m, eqs, mem, path, out_bits, out_rtilde, st);
    });
}

dl_status dl_autotune(dl_ctx *ctx, int32_t n, int32_t flags, char *report, size_t cap, size_t *len) {
    clear_error();
    Range trace_(__func__);
    GUARD_CTX(ctx);
    if (n < 0 || (cap > 0 && !report) || (flags & ~1)) {
        set_error("bad n (%d), flags (%d) or report buffer", n, flags);
        return DL_EINVAL;
    }
    std::string text;
    dl_status rc = run_sync(ctx, nullptr, [&](Workspace &ws, cudaStream_t s, dl_stats *) {
        TuneEntry e;
        std::string src;
        dl_status r = autotune_bucket(ctx, ws, s, n, (flags & 1) != 0, &e, &src);
        if (r == DL_OK) text = tune_report(ctx, e, src);
        return r;
    });
    if (rc) return rc;
    if (len) *len = text.size();
    if (cap > 0) {
        const size_t k = std::min(cap - 1, text.size());
        std::memcpy(report, text.data(), k);
        report[k] = 0;
    }
    return DL_OK;
}

dl_status dl_program_create(dl_ctx *ctx, const char *text, dl_program **out) {
    clear_error();
    Range trace_(__func__);
    GUARD_CTX(ctx);
    if (!text || !out) {
        set_error("text and out must not be NULL");
        return DL_EINVAL;
    }
    *out = nullptr;
    return program_create(ctx, text, out);
}

dl_status dl_program_destroy(dl_program *prog) {
    clear_error();
    Range trace_(__func__);
    if (!prog) return DL_OK;
    dl_ctx *ctx = program_ctx(prog);
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (set_device(ctx) == DL_OK) program_destroy(prog);
    return DL_OK;
}

dl_status dl_program_set(dl_program *prog, const char *pred, int32_t n, const uint8_t *R, dl_mem mem) {
    clear_error();
    Range trace_(__func__);
    if (!prog || !pred || n < 0 || !valid_mem(mem) || (n > 0 && !R)) {
        set_error("bad program, predicate, n (%d), matrix or memory kind", n);
        return DL_EINVAL;
    }
    dl_ctx *ctx = program_ctx(prog);
    return run_sync(ctx, nullptr, [&](Workspace &, cudaStream_t s, dl_stats *) {
        return program_set(prog, s, pred, n, R, mem);
    });
}

dl_status dl_program_run(dl_program *prog, dl_stats *stats) {
    clear_error();
    Range trace_(__func__);
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (!prog) {
        set_error("prog is NULL");
        return DL_EINVAL;
    }
    dl_ctx *ctx = program_ctx(prog);
    return run_sync(ctx, stats, [&](Workspace &ws, cudaStream_t s, dl_stats *st) {
        return program_run(ctx, ws, s, prog, st);
    });
}

dl_status dl_program_get(dl_program *prog, const char *pred, uint64_t *out_bits, dl_mem mem) {
    clear_error();
    Range trace_(__func__);
    if (!prog || !pred || !out_bits || !valid_mem(mem)) {
        set_error("prog, pred and out_bits must not be NULL, mem must be a memory kind");
        return DL_EINVAL;
    }
    dl_ctx *ctx = program_ctx(prog);
    return run_sync(ctx, nullptr, [&](Workspace &ws, cudaStream_t s, dl_stats *) {
        return program_get(prog, ws, s, pred, out_bits, mem);
    });
}

dl_status dl_program_describe(const dl_program *prog, char *buf, size_t cap, size_t *len) {
    clear_error();
    Range trace_(__func__);
    if (!prog || (cap > 0 && !buf)) {
        set_error("prog is NULL, or buf is NULL with cap > 0");
        return DL_EINVAL;
    }
    const std::string d = program_describe(prog);
    if (len) *len = d.size();
    if (cap > 0) {
        const size_t k = std::min(cap - 1, d.size());
        std::memcpy(buf, d.data(), k);
        buf[k] = 0;
    }
    return DL_OK;
}

dl_status dl_transposed(dl_ctx *ctx, int32_t n, const uint8_t *R1, dl_mem mem, double eps, double thr, dl_path path,
                        uint64_t *out_bits, double *out_rtilde, dl_stats *stats) {
    clear_error();
    Range trace_(__func__);
    GUARD_CTX(ctx);
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (n < 0 || !valid_mem(mem)) {
        set_error("bad n (%d) or memory kind", n);
        return DL_EINVAL;
    }
    if (n == 0) return DL_OK;
    if (!R1 || !out_bits) {
        set_error("R1 and out_bits must not be NULL");
        return DL_EINVAL;
    }
    SolveArgs a;
    a.n = n;
    a.E = R1;
    a.mem = mem;
    a.eps = eps;
    a.thr = thr;
    a.path = path;
    a.out_bits = out_bits;
    a.out_rtilde = out_rtilde;
    return run_sync(ctx, stats, [&](Workspace &ws, cudaStream_t s, dl_stats *st) {
        return solve_transposed(ctx, ws, s, a, st);
    });
}

dl_status dl_sg_real(dl_ctx *ctx, int32_t n, const uint8_t *P, const uint8_t *B, dl_mem mem, double eps,
                     dl_path path, double *out_stilde, uint64_t *out_bits, dl_stats *stats) {
    clear_error();
    Range trace_(__func__);
    GUARD_CTX(ctx);
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (n < 0 || !valid_mem(mem)) {
        set_error("bad n (%d) or memory kind", n);
        return DL_EINVAL;
    }
    if (n == 0) return DL_OK;
    if (!P || !out_stilde) {
        set_error("P and out_stilde must not be NULL");
        return DL_EINVAL;
    }
    SolveArgs a;
    a.n = n;
    a.E = P;
    a.E2 = B;
    a.mem = mem;
    a.eps = eps;
    a.path = path;
    a.out_bits = out_bits;
    a.out_rtilde = out_stilde;
    return run_sync(ctx, stats, [&](Workspace &ws, cudaStream_t s, dl_stats *st) {
        return solve_sg_real(ctx, ws, s, a, st);
    });
}

dl_status dl_compose(dl_ctx *ctx, int32_t n, const uint8_t *R1, const uint8_t *R2, dl_mem mem,
                     uint64_t *out_bits, dl_stats *stats) {
    clear_error();
    Range trace_(__func__);
    GUARD_CTX(ctx);
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (n < 0 || !valid_mem(mem)) {
        set_error("bad n (%d) or memory kind", n);
        return DL_EINVAL;
    }
    if (n == 0) return DL_OK;
    if (!R1 || !R2 || !out_bits) {
        set_error("R1, R2 and out_bits must not be NULL");
        return DL_EINVAL;
    }
    SolveArgs a;
    a.n = n;
    a.E = R1;
    a.E2 = R2;
    a.mem = mem;
    a.out_bits = out_bits;
    return run_sync(ctx, stats, [&](Workspace &ws, cudaStream_t s, dl_stats *st) {
        return solve_compose(ctx, ws, s, a, st);
    });
}

dl_status dl_selftest_wait_timeout(dl_ctx *ctx, double seconds) {
    clear_error();
    Range trace_(__func__);
    GUARD_CTX(ctx);
    if (!(seconds > 0.0 && seconds <= 10.0)) {
        set_error("seconds must be in (0, 10]");
        return DL_EINVAL;
    }
    return run_sync(ctx, nullptr, [&](Workspace &ws, cudaStream_t s, dl_stats *) -> dl_status {
        cudaMemsetAsync(ws.status, 0, sizeof(int), s);
        selftest_wait_kernel<<<1, 32, 0, s>>>(ws.status, static_cast<uint64_t>(seconds * 1e9));
        cudaError_t e = cudaGetLastError();
        int st = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&st, ws.status, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_error("self-test launch failed: %s", cudaGetErrorString(e));
            return DL_EDEVICE;
        }
        if (st & ST_TIMEOUT_DEP) {
            set_error("bounded device wait expired after %.3f s (expected)", seconds);
            return DL_ETIMEOUT;
        }
        set_error("the wait returned without expiring");
        return DL_OK;
    });
}

dl_status dl_tc_batch(dl_ctx *ctx, int32_t count, const int32_t *ns, const uint8_t *const *Es,
                      dl_mem mem, uint64_t *const *out_bits, dl_stats *stats) {
    clear_error();
    Range trace_(__func__);
    GUARD_CTX(ctx);
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (count < 0 || !valid_mem(mem)) {
        set_error("bad count (%d) or memory kind", count);
        return DL_EINVAL;
    }
    if (count == 0) return DL_OK;
    if (!ns || !Es || !out_bits) {
        set_error("ns, Es and out_bits must not be NULL");
        return DL_EINVAL;
    }
    for (int32_t k = 0; k < count; ++k) {
        if (ns[k] < 0 || (ns[k] > 0 && (!Es[k] || !out_bits[k]))) {
            set_error("problem %d: bad n or NULL pointer", k);
            return DL_EINVAL;
        }
    }
    return run_sync(ctx, stats, [&](Workspace &ws, cudaStream_t s, dl_stats *st) {
        return solve_tc_batch(ctx, ws, s, count, ns, Es, mem, out_bits, st);
    });
}

}  // extern "C"
