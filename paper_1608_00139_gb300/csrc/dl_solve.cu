// dl_solve.cu -- per-call drivers: which kernels run, in which order, on which buffers.
//
// Closure on the FP8 tensor cores (DL_PATH_BOOL_FP8): the reflexive closure
// C* = min1(I + E + E^2 + ...) is reached by repeated squaring, C_0 = I + E,
// C_{t+1} = min1(C_t C_t), which covers paths of length up to 2^t after t squarings; every
// squaring is one tcgen05 launch whose epilogue clamps (min1), packs bits and counts ones.
// The least model of eq. matrixeq:trcl is then R2 = min1(E C*) (one step from E, then any
// path), computed on bits by the sweep kernel, which at the same time checks that C_t
// already satisfies C = min1(I + E C): if it does, C_t is the reflexive closure and the
// squarings stop early; if a squaring adds no new one, they stop as well.
//
// Closure in FP64 (DL_PATH_FP64): Proposition 1 literally (dl_fp64.cu), threshold > 0
// (Theorem 1), then the same sweep in its in-place "recheck" mode confirms the model
// satisfies R2 = min1(E + E R2) and adds any fact the rounding lost (e.g. an underflowed
// eps^d, Lemma 2 footnote); the number of corrected rows is reported.
//
// Same generation (Sec. 7.2): the least S = min1(B + P S P^T) by doubling on boolean
// matrices: S_1 = B, Q_1 = P, S_{2m} = min1(S_m + Q_m S_m Q_m^T), Q_{2m} = min1(Q_m Q_m).
// S_m collects the facts derivable through at most m-1 nested applications of the
// recursive clause; when a step adds nothing (S_{2m} = S_m) or Q becomes 0, S is the
// fixpoint.  Each step: one grouped launch {T = Q S, Q' = Q Q} and one launch
// {S' = T Q^T OR S}.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dl_ctx.h"
#include "dl_internal.h"

namespace dl {

namespace {

constexpr size_t kHostPinned = 8u << 20;
constexpr size_t kTableOffset = 4096;

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Events at a solver's phase boundaries (0: start, 1: set-up done, 2: main work done, 3: end);
// with a tag, each phase is also an NVTX range "<tag>:set-up", "<tag>:main", "<tag>:epilogue".
struct Timer {
    cudaEvent_t *ev;
    cudaStream_t s;
    const char *tag = nullptr;
    bool open = false;
    void mark(int i) {
        cudaEventRecord(ev[i], s);
        if (!tag) return;
        if (open) nvtxRangePop();
        static const char *const kPhase[] = {"set-up", "main", "epilogue"};
        open = i >= 0 && i < 3;
        if (open) {
            char name[96];
            std::snprintf(name, sizeof name, "%s:%s", tag, kPhase[i]);
            nvtxRangePushA(name);
        }
    }
    ~Timer() {
        if (open) nvtxRangePop();
    }
    double ms(int a, int b) {
        float t = 0.f;
        cudaEventElapsedTime(&t, ev[a], ev[b]);
        return t;
    }
};

// Start/stop events around each group of sweep launches, on the launching stream.
struct SweepClock {
    Workspace &ws;
    cudaStream_t s;
    int k = 0, launches = 0;
    double bytes = 0.0;
    void start() {
        if (2 * k + 1 < Workspace::kGemmEvents) cudaEventRecord(ws.sev[2 * k], s);
    }
    void stop() {
        if (2 * k + 1 < Workspace::kGemmEvents) {
            cudaEventRecord(ws.sev[2 * k + 1], s);
            ++k;
        }
    }
    void account(int count, double bytes_each) {  // sweeps that did their work
        launches += count;
        bytes += count * bytes_each;
    }
    void fill(dl_stats *st) const {  // valid once the stream has been synchronised
        double t = 0.0;
        for (int i = 0; i < k; ++i) {
            float x = 0.f;
            cudaEventElapsedTime(&x, ws.sev[2 * i], ws.sev[2 * i + 1]);
            t += x;
        }
        st->sweep_launches = launches;
        st->ms_sweep = t;
        st->sweep_bytes = bytes;
    }
};

// Start/stop events around each tensor-core GEMM launch, on the launching stream.
struct GemmClock {
    Workspace &ws;
    cudaStream_t s;
    int k = 0, launches = 0;
    double flops = 0.0, timed_flops = 0.0;  // timed_flops: of the launches that have events
    void start() {
        if (2 * k + 1 < Workspace::kGemmEvents) cudaEventRecord(ws.gev[2 * k], s);
    }
    void stop(double f) {
        if (2 * k + 1 < Workspace::kGemmEvents) {
            cudaEventRecord(ws.gev[2 * k + 1], s);
            ++k;
            timed_flops += f;
        }
        ++launches;
        flops += f;
    }
    // valid once the stream has been synchronised
    double ms() const {
        double t = 0.0;
        for (int i = 0; i < k; ++i) {
            float x = 0.f;
            cudaEventElapsedTime(&x, ws.gev[2 * i], ws.gev[2 * i + 1]);
            t += x;
        }
        return t;
    }
    void fill(dl_stats *st) const {
        st->gemm_launches = launches;
        st->ms_gemm = ms() * (k > 0 ? static_cast<double>(launches) / k : 0.0);
        st->gemm_flops = flops;
    }
};

#define CK(x)                                                                          \
    do {                                                                               \
        cudaError_t e_ = (x);                                                          \
        if (e_ != cudaSuccess) {                                                       \
            set_error("%s failed: %s (%s:%d)", #x, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return DL_EDEVICE;                                                         \
        }                                                                              \
    } while (0)

#define NEED(p)                                                                        \
    do {                                                                               \
        if (!(p)) {                                                                    \
            set_error("device allocation failed (%s)", #p);                            \
            return DL_ENOMEM;                                                          \
        }                                                                              \
    } while (0)

unsigned long long *host_scal(Workspace &ws) {
    return static_cast<unsigned long long *>(ws.host_pinned);
}

dl_status read_scalars(Workspace &ws, cudaStream_t s) {
    CK(cudaMemcpyAsync(ws.host_pinned, ws.scal, kScalars * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return DL_OK;
}

dl_status check_status(Workspace &ws, cudaStream_t s) {
    int st = 0;
    CK(cudaMemcpyAsync(&st, ws.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (st & ST_BAD_INPUT) {
        set_error("input matrix holds a byte that is neither 0 nor 1");
        return DL_EINVAL;
    }
    if (st & ST_BAD_PAD) {
        set_error("bit-packed input has a bit set at a column >= n");
        return DL_EINVAL;
    }
    if (st) {
        set_error("a device-side wait expired (status word 0x%x)", st);
        return DL_ETIMEOUT;
    }
    return DL_OK;
}

// Upload `count` GEMM problems into the workspace table (device) and return it.
dl_status upload_problems(Workspace &ws, cudaStream_t s, const GemmProblem *probs, int count,
                          GemmProblem **out) {
    const size_t bytes = sizeof(GemmProblem) * static_cast<size_t>(count);
    if (kTableOffset + bytes > ws.host_bytes) {
        set_error("GEMM table too large");
        return DL_ENOMEM;
    }
    auto *d = static_cast<GemmProblem *>(ws.get("gemm_table", std::max<size_t>(bytes, 4096)));
    NEED(d);
    std::memcpy(static_cast<char *>(ws.host_pinned) + kTableOffset, probs, bytes);
    CK(cudaMemcpyAsync(d, static_cast<char *>(ws.host_pinned) + kTableOffset, bytes,
                       cudaMemcpyHostToDevice, s));
    *out = d;
    return DL_OK;
}

// Bring an n x n input to the device (copy if it is host memory).
dl_status stage_input(Workspace &ws, cudaStream_t s, const uint8_t *src, int32_t n, dl_mem mem,
                      const char *name, const uint8_t **dev) {
    if (mem == DL_MEM_DEVICE) {
        *dev = src;
        return DL_OK;
    }
    const size_t bytes = static_cast<size_t>(n) * n;
    auto *d = static_cast<uint8_t *>(ws.get(name, std::max<size_t>(bytes, 16)));
    NEED(d);
    CK(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, s));
    *dev = d;
    return DL_OK;
}

// Bring a bit-packed n x n input (n rows of ceil(n/64) words) to the device.
dl_status stage_bits(Workspace &ws, cudaStream_t s, const uint64_t *src, int32_t n, dl_mem mem,
                     const uint64_t **dev) {
    if (mem == DL_MEM_DEVICE) {
        *dev = src;
        return DL_OK;
    }
    const size_t bytes = static_cast<size_t>(n) * ((n + 63) / 64) * sizeof(uint64_t);
    auto *d = static_cast<uint64_t *>(ws.get("in0b", std::max<size_t>(bytes, 16)));
    NEED(d);
    CK(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, s));
    *dev = d;
    return DL_OK;
}

// Memory kind of the closure input E as the paths see it.
dl_mem in_mem(const SolveArgs &a) { return a.e_device ? DL_MEM_DEVICE : a.mem; }

dl_status write_bits(cudaStream_t s, const uint64_t *src, int64_t wp, uint64_t *dst, int32_t n,
                     dl_mem mem) {
    const int64_t w = (n + 63) / 64;
    CK(cudaMemcpy2DAsync(dst, w * 8, src, wp * 8, w * 8, n,
                         mem == DL_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    return DL_OK;
}

Operand square_op(const void *base, int64_t np) { return Operand{base, np, np, np, 0, 0}; }

GemmEpilogue bool_epi(uint8_t *out8, int64_t np, uint64_t *bits, int64_t wp,
                      unsigned long long *count, const uint8_t *add8) {
    GemmEpilogue e{};
    e.out8 = out8;
    e.ld_out8 = np;
    e.add8 = add8;
    e.ld_add8 = np;
    e.bits = reinterpret_cast<uint32_t *>(bits);
    e.ld_bits32 = 2 * wp;
    e.count = count;
    return e;
}

// The FP8 squaring's tile width for np (tuned per size bucket, else 256).
int bool_bn(dl_ctx *ctx, int64_t np) { return tuned(ctx, np).sq_bn; }

// Validate eps against ||E||_inf (Lemma 1) or pick the paper's default.
dl_status choose_eps(double user, double dflt, const char *what, double *out) {
    if (user <= 0.0) {
        *out = dflt;
        return DL_OK;
    }
    if (!(user <= dflt) || !std::isfinite(user)) {
        set_error("eps = %g exceeds the bound %g of %s", user, dflt, what);
        return DL_EINVAL;
    }
    *out = user;
    return DL_OK;
}

// Ingest (validation, row sums, e4m3 operand).  Sets *dmax, *nnz, *count.
dl_status ingest(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const uint8_t *dev, int32_t n,
                 int64_t np, uint8_t *dst, int add_identity, int slot_dmax, int slot_nnz,
                 int slot_count, int *launches) {
    (void)ctx;
    CK(ingest_u8_to_e4m3(dev, n, static_cast<int>(np), dst, add_identity, ws.scal + slot_dmax,
                         ws.scal + slot_nnz, ws.scal + slot_count, ws.status, s));
    ++*launches;
    return DL_OK;
}

dl_status tc_bool(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a, dl_stats *st) {
    const int32_t n = a.n;
    const int64_t np = round_up(std::max<int64_t>(n, 1), 256);
    const int64_t wp = np / 64;
    Timer tm{ws.ev, s, "tc_fp8"};
    int launches = 0;
    tm.mark(0);
    const uint8_t *E = nullptr;
    dl_status rc = stage_input(ws, s, a.E, n, in_mem(a), "in0", &E);
    if (rc) return rc;
    auto *C0 = static_cast<uint8_t *>(ws.get("c0", np * np));
    auto *C1 = static_cast<uint8_t *>(ws.get("c1", np * np));
    auto *rbits = static_cast<uint64_t *>(ws.get("bits0", np * wp * 8));
    auto *mbits = static_cast<uint64_t *>(ws.get("bits1", np * wp * 8));
    NEED(C0 && C1 && rbits && mbits);
    CK(cudaMemsetAsync(ws.scal, 0, kScalars * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(ws.status, 0, sizeof(int), s));
    if ((rc = ingest(ctx, ws, s, E, n, np, C0, 1, SC_DMAX, SC_NNZ, SC_COUNT0, &launches))) return rc;
    if ((rc = read_scalars(ws, s))) return rc;
    if ((rc = check_status(ws, s))) return rc;
    const unsigned long long dmax = host_scal(ws)[SC_DMAX];
    double eps = 0;
    if ((rc = choose_eps(a.eps, 1.0 / (1.0 + static_cast<double>(dmax)), "Lemma 1 (1/(1+||E||))", &eps)))
        return rc;
    unsigned long long prev = host_scal(ws)[SC_COUNT0];
    // successor lists for the certificate (edge-parallel, balanced for heavy-tailed degrees)
    auto *cnt_s = static_cast<int *>(ws.get("g_cnt", (np + 1) * 4));
    auto *ptr = static_cast<int *>(ws.get("g_ptr", (np + 1) * 4));
    auto *uoff = static_cast<int *>(ws.get("g_units", (np + 1) * 4));
    auto *col = static_cast<int *>(
        ws.get("g_col", static_cast<size_t>(std::max<unsigned long long>(host_scal(ws)[SC_NNZ], 1)) * 4));
    NEED(cnt_s && ptr && uoff && col);
    CK(csr_build(E, n, cnt_s, ptr, s));
    CK(csr_fill(E, n, ptr, col, s));
    CK(sweep_units(ptr, n, cnt_s, uoff, s));
    launches += 4;
    tm.mark(1);

    // GEMM tables: squaring C0 -> C1 and C1 -> C0, bits into rbits, count into slot
    GemmProblem probs[2];
    std::string err;
    const int bn = bool_bn(ctx, np);
    for (int p = 0; p < 2; ++p) {
        const uint8_t *src = p == 0 ? C0 : C1;
        uint8_t *dst = p == 0 ? C1 : C0;
        GemmEpilogue epi = bool_epi(dst, np, rbits, wp, ws.scal + SC_STEP0, nullptr);
        if (!gemm_make_problem(&probs[p], KIND_F8, false, bn, static_cast<int>(np), static_cast<int>(np),
                               static_cast<int>(np), square_op(src, np), square_op(src, np), epi, &err)) {
            set_error("%s", err.c_str());
            return DL_EDEVICE;
        }
    }
    GemmProblem *dprobs = nullptr;
    if ((rc = upload_problems(ws, s, probs, 2, &dprobs))) return rc;
    const int tiles = probs[0].tiles_m * probs[0].tiles_n;
    const int grid = std::min(tiles, ctx->sms);

    GemmClock gc{ws, s};
    int t = 0;
    bool have_model = false;
    int sweeps = 0;
    const int max_squarings = 2 + static_cast<int>(std::ceil(std::log2(static_cast<double>(np) + 1.0)));
    for (;;) {
        if (t >= max_squarings) {
            set_error("closure did not converge in %d squarings", t);
            return DL_ENOTCONV;
        }
        CK(cudaMemsetAsync(ws.scal + SC_STEP0, 0, sizeof(unsigned long long), s));
        gc.start();
        CK(gemm_launch(KIND_F8, false, bn, EPI_BOOL, dprobs + (t & 1), 1, tiles, grid, ws.status,
                       ctx->budget_ns, s));
        gc.stop(2.0 * np * np * np);
        ++launches;
        ++t;
        if ((rc = read_scalars(ws, s))) return rc;
        const unsigned long long cnt = host_scal(ws)[SC_STEP0];
        if (cnt == prev) break;  // C_t = C_{t-1}: reflexive closure reached
        prev = cnt;
        // certificate: does C_t satisfy C = min1(I + E C)?  (stops at the first violation)
        CK(cudaMemsetAsync(ws.scal + SC_VIOL, 0, 2 * sizeof(unsigned long long), s));
        CK(bits_sweep_csr(ptr, col, uoff, n, rbits, mbits, wp, 0, ws.scal + SC_VIOL, ws.scal + SC_ONES, &launches, s, static_cast<int>(dmax)));
        ++sweeps;
        if ((rc = read_scalars(ws, s))) return rc;
        if (host_scal(ws)[SC_VIOL] == 0) {
            have_model = true;
            break;
        }
    }
    tm.mark(2);
    if (!have_model) {
        CK(cudaMemsetAsync(ws.scal + SC_VIOL, 0, 2 * sizeof(unsigned long long), s));
        CK(bits_sweep_csr(ptr, col, uoff, n, rbits, mbits, wp, 0, ws.scal + SC_VIOL, ws.scal + SC_ONES, &launches, s, static_cast<int>(dmax)));
        ++sweeps;
        if ((rc = read_scalars(ws, s))) return rc;
        if (host_scal(ws)[SC_VIOL] != 0) {
            set_error("internal: converged closure failed its certificate");
            return DL_EDEVICE;
        }
    }
    if ((rc = write_bits(s, mbits, wp, a.out_bits, n, a.mem))) return rc;
    tm.mark(3);
    if ((rc = check_status(ws, s))) return rc;
    if (st) {
        st->path_used = DL_PATH_BOOL_FP8;
        st->eps_used = eps;
        st->iters = t;
        gc.fill(st);
        st->final_resid = 0.0;
        st->recheck_sweeps = sweeps;
        st->model_ones = static_cast<int64_t>(host_scal(ws)[SC_ONES]);
        st->ms_factor = tm.ms(0, 1);
        st->ms_solve = tm.ms(1, 2);
        st->ms_epilogue = tm.ms(2, 3);
        st->ms_total = tm.ms(0, 3);
        st->gpu_launches = launches;
    }
    return DL_OK;
}

// DL_PATH_AUTO: tensor-core squarings and boolean sweeps, whichever is cheaper.
// A sweep (in place, M <- M | E | E M on bits) is one step of the paper's Iteration method
// (Sec. 7.1, eq. series:trcl) and adds at least one hop to every path; a squaring doubles
// the hop count but costs a dense 2 Np^3 product.  Sparse graphs are finished by sweeps
// alone; dense ones square first and let a few cheap sweeps (rows saturate quickly) finish.
// A sweep that changes nothing proves M = min1(I + E M), i.e. M is the reflexive closure;
// the model is then E M (the final sweep, which checks the same equation once more).
dl_status tc_auto(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a, dl_stats *st) {
    const int32_t n = a.n;
    const int64_t np = round_up(std::max<int64_t>(n, 1), 256);
    const int64_t wp = np / 64;
    Timer tm{ws.ev, s, "tc_auto"};
    int launches = 0;
    tm.mark(0);
    const uint8_t *E = nullptr;
    const uint64_t *Eb = nullptr;
    dl_status rc = a.E_bits ? stage_bits(ws, s, a.E_bits, n, a.mem, &Eb) : stage_input(ws, s, a.E, n, in_mem(a), "in0", &E);
    if (rc) return rc;
    uint8_t *C[2] = {static_cast<uint8_t *>(ws.get("c0", np * np)), static_cast<uint8_t *>(ws.get("c1", np * np))};
    auto *rbits = static_cast<uint64_t *>(ws.get("bits0", np * wp * 8));
    auto *mbits = static_cast<uint64_t *>(ws.get("bits1", np * wp * 8));
    auto *cnt = static_cast<int *>(ws.get("g_cnt", (np + 1) * 4));
    auto *ptr = static_cast<int *>(ws.get("g_ptr", (np + 1) * 4));
    auto *uoff = static_cast<int *>(ws.get("g_units", (np + 1) * 4));
    auto *colmask = static_cast<uint64_t *>(ws.get("g_colmask", wp * 8));
    NEED(C[0] && C[1] && rbits && mbits && cnt && ptr && uoff && colmask);
    CK(cudaMemsetAsync(ws.scal, 0, kScalars * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(ws.status, 0, sizeof(int), s));
    CK(cudaMemsetAsync(colmask, 0, wp * 8, s));
    // one pass over E: the bits of C_0 = I + E, 0/1 check, row counts, ||E||_inf, nnz,
    // self-loops (the e4m3 operand is only built if a squaring happens)
    if (Eb)
        CK(bits_ingest_checked(Eb, n, static_cast<int>(np), wp, cnt, ptr, rbits, ws.scal + SC_DMAX, ws.scal + SC_NNZ,
                               ws.scal + SC_COUNT0, ws.status, colmask, s));
    else
        CK(csr_pack_checked(E, n, static_cast<int>(np), wp, cnt, ptr, rbits, ws.scal + SC_DMAX, ws.scal + SC_NNZ,
                            ws.scal + SC_COUNT0, ws.status, colmask, s));
    launches += 2;

    SweepClock sc{ws, s};
    unsigned long long *vslot = ws.scal + 32;  // up to 16 violation counters, one per sweep
    constexpr int kFirstGroup = 8;
    // cost model (seconds): one squaring vs one sweep before rows saturate.  A sweep reads a
    // successor's row per fact; the bit matrix is L2-resident up to a few tens of MB.
    const double bit_bytes = static_cast<double>(np) * wp * 8;
    const TuneEntry tn = tuned(ctx, np);  // measured rates when the size bucket has been tuned
    const double sweep_rate = tn.sweep_rate > 0 ? tn.sweep_rate : bit_bytes <= 48e6 ? 6.0e12 : 3.0e12;
    const double t_sq = tn.t_sq > 0 ? tn.t_sq * static_cast<double>(np) * np * np /
                                          (static_cast<double>(tn.bucket) * tn.bucket * tn.bucket)
                                    : 2.0 * np * np * np / 3.4e15 + 15e-6;
    const double t_sw_min = 2.0 * bit_bytes / sweep_rate + 5e-6;  // a sweep with no facts
    // the speculative group never exceeds the sweeps a squaring is worth with no facts at all,
    // and is empty when the last closure here was settled by the single-row Iteration alone
    // (and no longer than the sweeps that settled the last closure here, when it settled in them)
    int spec_group =
        ws.last_rows_closed
            ? 0
            : static_cast<int>(std::max(4.0, std::min<double>(kFirstGroup, std::floor(t_sq / t_sw_min))));
    if (ws.last_spec_sweeps > 0) spec_group = std::min(spec_group, ws.last_spec_sweeps - 1);
    // the model E M, checking M = min1(I + E M) on the way (straight into a device output whose
    // rows have the same stride)
    const bool direct = a.mem == DL_MEM_DEVICE && (n + 63) / 64 == wp;
    uint64_t *model = direct ? a.out_bits : mbits;
    int *gate = reinterpret_cast<int *>(ws.scal + SC_GATE);
    int *col = nullptr;
    unsigned long long dmax = 0;
    auto emit = [&](const int *g) -> dl_status {
        CK(cudaMemsetAsync(ws.scal + SC_VIOL, 0, 2 * sizeof(unsigned long long), s));
        sc.start();
        CK(bits_sweep_csr(ptr, col, uoff, n, rbits, model, wp, 0, ws.scal + SC_VIOL, ws.scal + SC_ONES, &launches, s,
                          g ? 0 : static_cast<int>(dmax), nullptr, colmask, g));
        sc.stop();
        return DL_OK;
    };

    // Speculative start (rows of at most 256 words): the first steps run before the host knows
    // the CSR's size or ||E||_inf, so that a closure settled in them costs one host read.  The
    // CSR fill uses the column array as it is and, if the facts do not fit or a row has more
    // than 256 successors, writes nothing and sets the gate; every launch after it reads the
    // gate and does nothing then.  The single-row Iteration decides on the device whether the
    // graph is sparse enough; its open-row count lets the sweeps skip when it closed every row.
    // (not when the last closure on this workspace had heavy rows: they would stop it again)
    bool spec = row_direct(0, wp) && !ws.last_heavy, converged = false, emitted = false, iterated = false;
    int spec_sweeps = 0;
    if (spec) {
        const size_t want = std::max(ws.capacity("g_col"), static_cast<size_t>(np) * 8 * sizeof(int));
        col = static_cast<int *>(ws.get("g_col", want));
        NEED(col);
        const int64_t cap = static_cast<int64_t>(ws.capacity("g_col") / sizeof(int));
        CK(csr_fill_from_bits_guarded(rbits, n, wp, ptr, col, cap, ws.scal + SC_DMAX, 256, gate, s));
        ++launches;
        // the Iteration on single rows (it checks sparsity on the device; not launched when the
        // last closure here was too dense for it)
        iterated = row_iteration_fits(wp) && !ws.last_dense;
        if (iterated) {
            CK(row_iteration(ptr, col, n, wp, rbits, ws.scal + SC_OPEN, s, gate));
            ++launches;
        }
        sc.start();
        for (int k = 0; k < spec_group; ++k) {
            const unsigned long long *skip = k > 0 ? vslot + k - 1 : (iterated ? ws.scal + SC_OPEN : nullptr);
            CK(bits_sweep_csr(ptr, col, uoff, n, rbits, rbits, wp, 1, vslot + k, nullptr, &launches, s, 0, skip,
                              colmask, gate));
        }
        sc.stop();
        if ((rc = emit(gate))) return rc;
    }
    if ((rc = read_scalars(ws, s))) return rc;
    if ((rc = check_status(ws, s))) return rc;
    dmax = host_scal(ws)[SC_DMAX];
    ws.last_heavy = dmax > 256;
    double eps = 0;
    if ((rc = choose_eps(a.eps, 1.0 / (1.0 + static_cast<double>(dmax)), "Lemma 1 (1/(1+||E||))", &eps)))
        return rc;
    const int64_t nnz = static_cast<int64_t>(host_scal(ws)[SC_NNZ]);
    ws.last_dense = nnz > 2 * static_cast<int64_t>(n);
    // bytes a sweep reads at least: the CSR of E and every row of the bit matrix once
    const double sweep_min_bytes = 4.0 * (static_cast<double>(nnz) + n + 1) + static_cast<double>(n) * wp * 8.0;
    if (spec && *reinterpret_cast<const int *>(host_scal(ws) + SC_GATE) != 0) spec = false;  // nothing ran
    ws.last_rows_closed = false;
    ws.last_spec_sweeps = 0;
    if (spec) {
        if (iterated && host_scal(ws)[SC_OPEN] == 0) {
            converged = true;  // every row closed by the single-row Iteration (the sweeps skipped)
            ws.last_rows_closed = true;
        } else {
            // settled when a sweep changed nothing, or when the emitted certificate holds: the
            // sweeps only add facts of C*, and an M inside C* with M = min1(I + E M) is C*
            int working = -1;  // sweeps that were needed
            spec_sweeps = spec_group;
            for (int k = 0; k < spec_group; ++k)
                if (host_scal(ws)[32 + k] == 0) {
                    working = k;
                    spec_sweeps = k + 1;
                    break;
                }
            if (working < 0 && host_scal(ws)[SC_VIOL] == 0) working = spec_group;
            if (working >= 0) {
                converged = true;
                ws.last_spec_sweeps = working + 1;
            }
        }
        sc.account(spec_sweeps + 1, sweep_min_bytes);
        emitted = converged;
    } else {
        // planned on the host: the column array sized to the facts, work units for heavy rows
        col = static_cast<int *>(ws.get("g_col", static_cast<size_t>(std::max<int64_t>(nnz, 1)) * 4));
        NEED(col);
        CK(csr_fill_from_bits(rbits, n, wp, ptr, col, s));
        ++launches;
        if (!row_direct(static_cast<int>(dmax), wp)) {  // heavy rows: edge-parallel work units
            CK(sweep_units(ptr, n, cnt, uoff, s));
            launches += 2;
        }
    }
    tm.mark(1);
    // ones of C_0 = I + E over the padded size: the diagonal plus the facts off it
    unsigned long long prev = static_cast<unsigned long long>(np) + host_scal(ws)[SC_NNZ] - host_scal(ws)[SC_COUNT0];

    const double t_sw = (static_cast<double>(nnz) * wp * 8 + 2.0 * bit_bytes) / sweep_rate + 5e-6;
    // square first only when one unsaturated sweep costs more than a squaring (rows saturate
    // within a sweep or two on dense graphs, so later sweeps are cheap)
    const bool dense = t_sw > t_sq;
    // sweeps allowed between two squarings before a squaring is the cheaper way forward
    const int sweep_budget = static_cast<int>(std::max(4.0, std::floor(t_sq / t_sw)));

    GemmClock gc{ws, s};
    const int max_squarings = 2 + static_cast<int>(std::ceil(std::log2(static_cast<double>(np) + 1.0)));
    const int max_sweeps = static_cast<int>(std::min<int64_t>(2 * static_cast<int64_t>(n) + 16, 1 << 20));
    int cur = 0, squarings = 0, sweeps = spec_sweeps;
    bool c_valid = false;  // C[cur] holds the same matrix as rbits
    bool do_square = spec ? (!converged && sweeps >= sweep_budget) : dense;
    int since_square = sweeps;  // sweeps since the last squaring
    GemmProblem *dprobs = nullptr;
    int tiles = 0, grid = 0;
    const int bn = bool_bn(ctx, np);
    auto gemm_setup = [&]() -> dl_status {  // the two squaring problems, uploaded on first use
        if (dprobs) return DL_OK;
        GemmProblem probs[2];
        std::string err;
        for (int p = 0; p < 2; ++p) {
            if (!gemm_make_problem(&probs[p], KIND_F8, false, bn, static_cast<int>(np), static_cast<int>(np),
                                   static_cast<int>(np), square_op(C[p], np), square_op(C[p], np),
                                   bool_epi(C[1 - p], np, rbits, wp, ws.scal + SC_STEP0, nullptr), &err)) {
                set_error("%s", err.c_str());
                return DL_EDEVICE;
            }
        }
        dl_status r = upload_problems(ws, s, probs, 2, &dprobs);
        tiles = probs[0].tiles_m * probs[0].tiles_n;
        grid = std::min(tiles, ctx->sms);
        return r;
    };
    // sparse graphs planned on the host (at most two facts per row on average, no heavy rows):
    // the Iteration on single rows closes every row whose reachable set stays small in one
    // launch; the rows it leaves open keep what they reached and the sweeps below finish them
    if (!spec && !dense && nnz <= 2 * static_cast<int64_t>(n) && row_iteration_fits(wp) &&
        row_direct(static_cast<int>(dmax), wp)) {
        CK(cudaMemsetAsync(ws.scal + SC_OPEN, 0, sizeof(unsigned long long), s));
        sc.start();
        CK(row_iteration(ptr, col, n, wp, rbits, ws.scal + SC_OPEN, s));
        sc.stop();
        ++launches;
        if ((rc = emit(nullptr))) return rc;
        sc.account(1, sweep_min_bytes);
        if ((rc = read_scalars(ws, s))) return rc;
        if (host_scal(ws)[SC_OPEN] == 0) converged = emitted = ws.last_rows_closed = true;
    }
    while (!converged) {
        if (do_square) {
            if (squarings >= max_squarings) {
                set_error("closure did not converge in %d squarings", squarings);
                return DL_ENOTCONV;
            }
            if ((rc = gemm_setup())) return rc;
            if (!c_valid) {
                CK(bits_to_e4m3(rbits, wp, static_cast<int>(np), C[cur], s));
                ++launches;
            }
            CK(cudaMemsetAsync(ws.scal + SC_STEP0, 0, sizeof(unsigned long long), s));
            gc.start();
            CK(gemm_launch(KIND_F8, false, bn, EPI_BOOL, dprobs + cur, 1, tiles, grid, ws.status, ctx->budget_ns,
                           s));
            gc.stop(2.0 * np * np * np);
            ++launches;
            ++squarings;
            since_square = 0;
            cur ^= 1;
            c_valid = true;
            if ((rc = read_scalars(ws, s))) return rc;
            const unsigned long long c2 = host_scal(ws)[SC_STEP0];
            if (c2 == prev) {
                converged = true;
                break;
            }
            prev = c2;
        }
        // a group of in-place sweeps and, speculatively, the model (final if the group reached
        // the fixpoint), then one host read for all of it (after a squaring the rows are dense
        // and saturate within a few successors, so a short group is cheap)
        const int g = std::max(1, std::min(squarings == 0 ? kFirstGroup : 4, sweep_budget - since_square));
        CK(cudaMemsetAsync(vslot, 0, sizeof(unsigned long long) * g, s));
        sc.start();
        for (int k = 0; k < g; ++k)  // a sweep after one that changed nothing exits on the device
            CK(bits_sweep_csr(ptr, col, uoff, n, rbits, rbits, wp, 1, vslot + k, nullptr, &launches, s,
                              static_cast<int>(dmax), k > 0 ? vslot + k - 1 : nullptr, colmask));
        sc.stop();
        if ((rc = emit(nullptr))) return rc;
        if ((rc = read_scalars(ws, s))) return rc;
        int ran = g;
        for (int k = 0; k < g; ++k)
            if (host_scal(ws)[32 + k] == 0) {
                converged = true;
                ran = k + 1;
                break;
            }
        sc.account(ran + 1, sweep_min_bytes);
        sweeps += ran;
        since_square += g;
        emitted = converged;
        if (!converged) {
            c_valid = false;
            do_square = squarings > 0 || since_square >= sweep_budget;
            if (sweeps > max_sweeps) {
                set_error("closure did not converge in %d sweeps", sweeps);
                return DL_ENOTCONV;
            }
        }
    }
    tm.mark(2);
    if (!emitted) {  // converged by a squaring
        if ((rc = emit(nullptr))) return rc;
        sc.account(1, sweep_min_bytes);
        if ((rc = read_scalars(ws, s))) return rc;
    }
    if (host_scal(ws)[SC_VIOL] != 0) {
        set_error("internal: converged closure failed its certificate");
        return DL_EDEVICE;
    }
    if (!direct && (rc = write_bits(s, mbits, wp, a.out_bits, n, a.mem))) return rc;
    tm.mark(3);
    if ((rc = check_status(ws, s))) return rc;
    if (st) {
        st->path_used = DL_PATH_AUTO;
        st->eps_used = eps;
        st->iters = squarings;
        st->recheck_sweeps = sweeps + 1;
        gc.fill(st);
        sc.fill(st);
        st->model_ones = static_cast<int64_t>(host_scal(ws)[SC_ONES]);
        st->ms_factor = tm.ms(0, 1);
        st->ms_solve = tm.ms(1, 2);
        st->ms_epilogue = tm.ms(2, 3);
        st->ms_total = tm.ms(0, 3);
        st->gpu_launches = launches;
    }
    return DL_OK;
}

// After X > 0 went into mbits: the exact recheck (in-place sweeps until the bits satisfy
// M = min1(E + E M)), or with a.skip_recheck only the count of ones (SC_ONES).
dl_status recheck_bits(Workspace &ws, cudaStream_t s, const SolveArgs &a, const uint8_t *E, int32_t n, int64_t wp,
                       uint64_t *mbits, int *sweeps, unsigned long long *corrected, int *launches) {
    dl_status rc;
    *sweeps = 0;
    *corrected = 0;
    if (a.skip_recheck) {
        CK(cudaMemsetAsync(ws.scal + SC_ONES, 0, sizeof(unsigned long long), s));
        CK(bits_count(mbits, n, wp, ws.scal + SC_ONES, s));
        ++*launches;
        return read_scalars(ws, s);
    }
    for (;;) {
        CK(cudaMemsetAsync(ws.scal + SC_VIOL, 0, 2 * sizeof(unsigned long long), s));
        CK(bits_sweep(E, n, n, mbits, mbits, wp, 1, 0, ws.scal + SC_VIOL, ws.scal + SC_ONES, s));
        ++*launches;
        ++*sweeps;
        if ((rc = read_scalars(ws, s))) return rc;
        const unsigned long long v = host_scal(ws)[SC_VIOL];
        if (v == 0) return DL_OK;
        *corrected += v;
        if (*sweeps > n + 1) {
            set_error("recheck did not converge");
            return DL_ENOTCONV;
        }
    }
}

dl_status tc_fp64(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a, dl_stats *st) {
    const int32_t n = a.n;
    const int64_t np = round_up(std::max<int64_t>(n, 1), 64);
    const int64_t npb = round_up(std::max<int64_t>(n, 1), 256);
    const int64_t wp = npb / 64;
    Timer tm{ws.ev, s, "tc_fp64"};
    int launches = 0;
    tm.mark(0);
    const uint8_t *E = nullptr;
    dl_status rc = stage_input(ws, s, a.E, n, in_mem(a), "in0", &E);
    if (rc) return rc;
    auto *C0 = static_cast<uint8_t *>(ws.get("c0", npb * npb));
    auto *mbits = static_cast<uint64_t *>(ws.get("bits1", npb * wp * 8));
    const int64_t ldg = 2 * np;
    auto *G = static_cast<double *>(ws.get("fp64_G", np * ldg * 8));
    NEED(C0 && mbits && G);
    CK(cudaMemsetAsync(ws.scal, 0, kScalars * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(ws.status, 0, sizeof(int), s));
    // validation and row sums (the e4m3 copy is not used by this path)
    if ((rc = ingest(ctx, ws, s, E, n, npb, C0, 0, SC_DMAX, SC_NNZ, SC_COUNT0, &launches))) return rc;
    if ((rc = read_scalars(ws, s))) return rc;
    if ((rc = check_status(ws, s))) return rc;
    const unsigned long long dmax = host_scal(ws)[SC_DMAX];
    double eps = 0;
    if ((rc = choose_eps(a.eps, 1.0 / (1.0 + static_cast<double>(dmax)), "Lemma 1 (1/(1+||E||))", &eps)))
        return rc;
    if (a.rhs_real)
        CK(fp64_build_real(E, a.rhs_real, n, static_cast<int>(np), eps, G, ldg, s));
    else
        CK(fp64_build(E, a.rhs ? a.rhs : E, n, static_cast<int>(np), eps, G, ldg, s));
    ++launches;
    tm.mark(1);
    CK(fp64_solve(G, ldg, static_cast<int>(np), &launches, s));
    tm.mark(2);
    const double *X = G + np;
    const double tau = ctx->cfg.guard_tau > 0 ? ctx->cfg.guard_tau : 1e-30;
    CK(cudaMemsetAsync(mbits, 0, npb * wp * 8, s));  // the threshold writes rows < n, words < ceil(n/64)
    CK(thresh_pack_f64(X, ldg, n, static_cast<int>(np), tau, mbits, wp, ws.scal + SC_GUARD, s));
    ++launches;
    // recheck: in-place sweeps until the model satisfies R2 = min1(E + E R2)
    int sweeps = 0;
    unsigned long long corrected = 0;
    if ((rc = recheck_bits(ws, s, a, E, n, wp, mbits, &sweeps, &corrected, &launches))) return rc;
    if (a.out_bits && (rc = write_bits(s, mbits, wp, a.out_bits, n, a.mem))) return rc;
    if (a.out_rtilde) {
        CK(cudaMemcpy2DAsync(a.out_rtilde, static_cast<size_t>(n) * 8, X, ldg * 8,
                             static_cast<size_t>(n) * 8, n,
                             a.mem == DL_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    }
    tm.mark(3);
    if ((rc = check_status(ws, s))) return rc;
    if (st) {
        st->path_used = DL_PATH_FP64;
        st->eps_used = eps;
        st->iters = 0;
        st->final_resid = -1.0;
        st->guard_flagged = static_cast<int64_t>(host_scal(ws)[SC_GUARD]);
        st->rows_rechecked = static_cast<int64_t>(corrected);
        st->recheck_sweeps = sweeps;
        st->model_ones = static_cast<int64_t>(host_scal(ws)[SC_ONES]);
        st->ms_factor = tm.ms(0, 1);
        st->ms_solve = tm.ms(1, 2);
        st->ms_epilogue = tm.ms(2, 3);
        st->ms_total = tm.ms(0, 3);
        st->gpu_launches = launches;
    }
    return DL_OK;
}

dl_status tc_mixed_path(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a, dl_stats *st) {
    const int32_t n = a.n;
    const int64_t np = round_up(std::max<int64_t>(n, 1), 256);
    const int64_t wp = np / 64;
    Timer tm{ws.ev, s, "tc_mixed"};
    int launches = 0;
    tm.mark(0);
    const uint8_t *E = nullptr;
    dl_status rc = stage_input(ws, s, a.E, n, in_mem(a), "in0", &E);
    if (rc) return rc;
    auto *C0 = static_cast<uint8_t *>(ws.get("c0", np * np));
    auto *mbits = static_cast<uint64_t *>(ws.get("bits1", np * wp * 8));
    NEED(C0 && mbits);
    CK(cudaMemsetAsync(ws.scal, 0, kScalars * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(ws.status, 0, sizeof(int), s));
    // validation and row sums (the e4m3 copy is not used by this path)
    if ((rc = ingest(ctx, ws, s, E, n, np, C0, 0, SC_DMAX, SC_NNZ, SC_COUNT0, &launches))) return rc;
    if ((rc = read_scalars(ws, s))) return rc;
    if ((rc = check_status(ws, s))) return rc;
    const unsigned long long dmax = host_scal(ws)[SC_DMAX];
    double eps = 0;
    if ((rc = choose_eps(a.eps, 1.0 / (1.0 + static_cast<double>(dmax)), "Lemma 1 (1/(1+||E||))", &eps)))
        return rc;
    dl_stats local{};
    dl_stats *sx = st ? st : &local;
    if ((rc = tc_mixed(ctx, ws, s, a, sx, E, eps, dmax, &launches))) return rc;
    tm.mark(2);
    const auto *X = static_cast<const double *>(ws.get("mx_X64", np * np * 8));
    const double tau = ctx->cfg.guard_tau > 0 ? ctx->cfg.guard_tau : 1e-30;
    CK(cudaMemsetAsync(mbits, 0, np * wp * 8, s));  // the threshold writes rows < n, words < ceil(n/64)
    CK(thresh_pack_f64(X, np, n, static_cast<int>(np), tau, mbits, wp, ws.scal + SC_GUARD, s));
    ++launches;
    int sweeps = 0;
    unsigned long long corrected = 0;
    if ((rc = recheck_bits(ws, s, a, E, n, wp, mbits, &sweeps, &corrected, &launches))) return rc;
    if (a.out_bits && (rc = write_bits(s, mbits, wp, a.out_bits, n, a.mem))) return rc;
    if (a.out_rtilde) {
        CK(cudaMemcpy2DAsync(a.out_rtilde, static_cast<size_t>(n) * 8, X, np * 8, static_cast<size_t>(n) * 8, n,
                             a.mem == DL_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    }
    tm.mark(3);
    if ((rc = check_status(ws, s))) return rc;
    if (st) {
        st->path_used = DL_PATH_MIXED;
        st->eps_used = eps;
        st->guard_flagged = static_cast<int64_t>(host_scal(ws)[SC_GUARD]);
        st->rows_rechecked = static_cast<int64_t>(corrected);
        st->recheck_sweeps = sweeps;
        st->model_ones = static_cast<int64_t>(host_scal(ws)[SC_ONES]);
        st->ms_epilogue = tm.ms(2, 3);
        st->ms_total = tm.ms(0, 3);
        st->gpu_launches = launches;
    }
    return DL_OK;
}

}  // namespace

// The bytes of a bit-packed E on the device (the non-AUTO paths start from bytes); an input
// error is reported here, before the path runs.
dl_status unpack_input(Workspace &ws, cudaStream_t s, const SolveArgs &a, const uint8_t **out) {
    const uint64_t *Eb = nullptr;
    dl_status rc = stage_bits(ws, s, a.E_bits, a.n, a.mem, &Eb);
    if (rc) return rc;
    auto *E = static_cast<uint8_t *>(ws.get("in0u", std::max<size_t>(static_cast<size_t>(a.n) * a.n, 16)));
    NEED(E);
    CK(cudaMemsetAsync(ws.status, 0, sizeof(int), s));
    CK(unpack_bits_u8(Eb, a.n, E, ws.status, s));
    if ((rc = check_status(ws, s))) return rc;
    *out = E;
    return DL_OK;
}

dl_status solve_tc(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &in, dl_stats *st) {
    if (in.thr != 0.0) {
        set_error("thr must be 0: the model is R~ > 0 (Theorem 1)");
        return DL_EINVAL;
    }
    dl_status rc;
    SolveArgs a = in;
    if (a.E_bits && a.path != DL_PATH_AUTO) {  // AUTO ingests the bits as they are
        if (a.path != DL_PATH_BOOL_FP8 && a.path != DL_PATH_FP64 && a.path != DL_PATH_MIXED) {
            set_error("unknown path %d", static_cast<int>(a.path));
            return DL_EINVAL;
        }
        const uint8_t *E = nullptr;
        if ((rc = unpack_input(ws, s, a, &E))) return rc;
        a.E = E;
        a.E_bits = nullptr;
        a.e_device = true;
    }
    switch (a.path) {
        case DL_PATH_AUTO:
        case DL_PATH_BOOL_FP8:
            if (a.out_rtilde) {
                set_error("the boolean paths compute no real-valued R~; use DL_PATH_FP64 or DL_PATH_MIXED");
                return DL_EINVAL;
            }
            rc = a.path == DL_PATH_AUTO ? tc_auto(ctx, ws, s, a, st) : tc_bool(ctx, ws, s, a, st);
            break;
        case DL_PATH_FP64:
            rc = tc_fp64(ctx, ws, s, a, st);
            break;
        case DL_PATH_MIXED:
            rc = tc_mixed_path(ctx, ws, s, a, st);
            break;
        default:
            set_error("unknown path %d", static_cast<int>(a.path));
            return DL_EINVAL;
    }
    if (rc == DL_OK && st && st->ms_total > 0) {
        const double nn = static_cast<double>(a.n);
        st->tflops_equiv = (8.0 / 3.0) * nn * nn * nn / (st->ms_total * 1e-3) / 1e12;
    }
    return rc;
}

// Same generation by the Iteration method on bits: S_{t+1} = B | P S_t P^T, from S_0 = B
// (Kleene iteration from below, so an iteration that changes nothing has reached the least
// fixpoint).  One iteration: Y = P S_t^T (rows of P gather rows of S^T), X = Y^T = S_t P^T,
// S |= P X (rows of P gather rows of X); when B is symmetric so is every S_t and S^T = S.
// Returns with *done = false (and nothing written) if the rows are too wide or the
// iterations exceed the budget: the doubling below then solves the problem.
dl_status sg_iteration(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a, dl_stats *st, bool *done,
                       const uint64_t *seed = nullptr) {
    (void)ctx;
    *done = false;
    const int32_t n = a.n;
    const int64_t np = round_up(std::max<int64_t>(n, 1), 256);
    const int64_t wp = np / 64;
    if (wp > 256) return DL_OK;
    constexpr int kBudget = 64, kGroup = 8;
    Timer tm{ws.ev, s, "sg_iteration"};
    int launches = 0;
    tm.mark(0);
    const uint8_t *P = nullptr, *Bm = nullptr;
    dl_status rc = stage_input(ws, s, a.E, n, a.mem, "in0", &P);
    if (rc) return rc;
    if (a.E2 && (rc = stage_input(ws, s, a.E2, n, a.mem, "in1", &Bm))) return rc;
    auto *S = static_cast<uint64_t *>(ws.get("bits0", np * wp * 8));
    auto *Y = static_cast<uint64_t *>(ws.get("bits1", np * wp * 8));
    auto *X = static_cast<uint64_t *>(ws.get("bits2", np * wp * 8));
    auto *cnt = static_cast<int *>(ws.get("g_cnt", (np + 1) * 4));
    auto *ptr = static_cast<int *>(ws.get("g_ptr", (np + 1) * 4));
    auto *colmask = static_cast<uint64_t *>(ws.get("g_colmask", wp * 8));
    auto *uoff = static_cast<int *>(ws.get("g_units", (np + 1) * 4));
    NEED(S && Y && X && cnt && ptr && colmask && uoff);
    CK(cudaMemsetAsync(ws.scal, 0, kScalars * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(ws.status, 0, sizeof(int), s));
    CK(cudaMemsetAsync(colmask, 0, wp * 8, s));
    // the CSR of P (its bits of I + P go to X, a scratch here) and S_0 = B
    CK(csr_pack_checked(P, n, static_cast<int>(np), wp, cnt, ptr, X, ws.scal + SC_DMAX, ws.scal + SC_NNZ,
                        ws.scal + SC_COUNT0, ws.status, colmask, s));
    launches += 2;
    if (Bm) {  // is B symmetric?  (words of B and B^T that differ)
        CK(pack_bits(Bm, n, static_cast<int>(np), wp, S, ws.status, s));
        CK(bits_transpose(S, Y, static_cast<int>(np), wp, nullptr, s));
        CK(bits_diff(S, Y, np * wp, ws.scal + SC_CQ, s));
        launches += 3;
    } else {
        CK(bits_identity(S, n, static_cast<int>(np), wp, s));
        ++launches;
    }
    if (seed) {  // S_0 = B | seed (the seed lies inside the least model, so the limit is unchanged)
        CK(bits_or(S, seed, np * wp, s));
        ++launches;
    }
    if ((rc = read_scalars(ws, s))) return rc;
    if ((rc = check_status(ws, s))) return rc;
    const double dmax = static_cast<double>(host_scal(ws)[SC_DMAX]);
    double eps = 0;
    if ((rc = choose_eps(a.eps, 1.0 / (1.0 + dmax * dmax), "Sec. 7.2 (1/(1+||P||^2))", &eps))) return rc;
    const bool sym = seed == nullptr && (Bm == nullptr || host_scal(ws)[SC_CQ] == 0);
    const int64_t nnz = static_cast<int64_t>(host_scal(ws)[SC_NNZ]);
    auto *col = static_cast<int *>(ws.get("g_col", static_cast<size_t>(std::max<int64_t>(nnz, 1)) * 4));
    NEED(col);
    CK(csr_fill_from_bits(X, n, wp, ptr, col, s));
    ++launches;
    const int *units = nullptr;  // rows of more than 64 parents: edge-parallel gathers
    if (dmax > 64) {
        CK(sweep_units(ptr, n, cnt, uoff, s));
        launches += 2;
        units = uoff;
    }
    CK(cudaMemsetAsync(Y, 0, np * wp * 8, s));  // rows >= n stay zero (the gathers write rows < n)
    tm.mark(1);
    unsigned long long *vslot = ws.scal + 32;
    int iters = 0;
    bool converged = false;
    while (!converged) {
        if (iters >= kBudget) return DL_OK;  // deep derivations: doubling instead
        CK(cudaMemsetAsync(vslot, 0, sizeof(unsigned long long) * kGroup, s));
        for (int k = 0; k < kGroup; ++k) {  // an iteration after one that changed nothing exits at once
            const unsigned long long *skip = k > 0 ? vslot + k - 1 : nullptr;
            const uint64_t *src = S;
            if (!sym) {
                CK(bits_transpose(S, X, static_cast<int>(np), wp, skip, s));
                src = X;
                ++launches;
            }
            CK(bits_gather(ptr, col, units, n, src, Y, wp, 0, nullptr, skip, s));
            CK(bits_transpose(Y, X, static_cast<int>(np), wp, skip, s));
            CK(bits_gather(ptr, col, units, n, X, S, wp, 1, vslot + k, skip, s));
            launches += 3;
        }
        if ((rc = read_scalars(ws, s))) return rc;
        int ran = kGroup;
        for (int k = 0; k < kGroup; ++k)
            if (host_scal(ws)[32 + k] == 0) {
                converged = true;
                ran = k + 1;
                break;
            }
        iters += ran;
    }
    tm.mark(2);
    CK(bits_count(S, n, wp, ws.scal + SC_ONES, s));
    ++launches;
    if ((rc = write_bits(s, S, wp, a.out_bits, n, a.mem))) return rc;
    tm.mark(3);
    if ((rc = read_scalars(ws, s))) return rc;
    if ((rc = check_status(ws, s))) return rc;
    if (st) {
        st->path_used = DL_PATH_AUTO;
        st->eps_used = eps;
        st->iters = iters;
        st->recheck_sweeps = iters;
        st->model_ones = static_cast<int64_t>(host_scal(ws)[SC_ONES]);
        st->ms_factor = tm.ms(0, 1);
        st->ms_solve = tm.ms(1, 2);
        st->ms_epilogue = tm.ms(2, 3);
        st->ms_total = tm.ms(0, 3);
        st->gpu_launches = launches;
    }
    *done = true;
    return DL_OK;
}

dl_status sg_doubling(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a, dl_stats *st);

dl_status solve_sg(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a, dl_stats *st) {
    if (a.thr != 0.0) {
        set_error("thr must be 0: the model is S~ > 0 (Theorem 2)");
        return DL_EINVAL;
    }
    if (a.path != DL_PATH_AUTO && a.path != DL_PATH_BOOL_FP8) {
        set_error("same generation runs on DL_PATH_AUTO or DL_PATH_BOOL_FP8");
        return DL_ENOTIMPL;
    }
    // AUTO: the doubling costs about 30 Np^3 tensor flops (three products per step, about five
    // steps) and some 0.3 ms of fixed work; an iteration costs two row gathers, a transpose and
    // about 0.1 ms of launches, and about ten are needed.  The doubling is cheaper below
    // Np ~ 6000 (measured: 0.9 against 1.3 ms at N = 4096, 5.1 against 2.1 ms at N = 8192).
    const int64_t np = round_up(std::max<int64_t>(a.n, 1), 256);
    const int tuned_iteration = tuned(ctx, np).sg_iteration;  // measured crossover, when tuned
    if (a.path == DL_PATH_AUTO && (tuned_iteration >= 0 ? tuned_iteration == 1 : np >= 6144)) {
        bool done = false;
        const dl_status rc = sg_iteration(ctx, ws, s, a, st, &done);
        if (rc != DL_OK || done) return rc;
    }
    return sg_doubling(ctx, ws, s, a, st);
}

// Same generation by boolean doubling on the tensor cores: S_{2m} = min1(S_m + Q_m S_m Q_m^T),
// Q_{2m} = min1(Q_m^2), from S_1 = B, Q_1 = P.
dl_status sg_doubling(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a, dl_stats *st) {
    const int32_t n = a.n;
    const int64_t np = round_up(std::max<int64_t>(n, 1), 256);
    const int64_t wp = np / 64;
    Timer tm{ws.ev, s, "sg_doubling"};
    int launches = 0;
    tm.mark(0);
    const uint8_t *P = nullptr, *Bm = nullptr;
    dl_status rc = stage_input(ws, s, a.E, n, a.mem, "in0", &P);
    if (rc) return rc;
    if (a.E2 && (rc = stage_input(ws, s, a.E2, n, a.mem, "in1", &Bm))) return rc;
    uint8_t *Sa = static_cast<uint8_t *>(ws.get("c0", np * np));
    uint8_t *Sb = static_cast<uint8_t *>(ws.get("c1", np * np));
    uint8_t *Qa = static_cast<uint8_t *>(ws.get("c2", np * np));
    uint8_t *Qb = static_cast<uint8_t *>(ws.get("c3", np * np));
    uint8_t *T = static_cast<uint8_t *>(ws.get("c4", np * np));
    auto *sbits = static_cast<uint64_t *>(ws.get("bits0", np * wp * 8));
    NEED(Sa && Sb && Qa && Qb && T && sbits);
    CK(cudaMemsetAsync(ws.scal, 0, kScalars * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(ws.status, 0, sizeof(int), s));
    if ((rc = ingest(ctx, ws, s, P, n, np, Qa, 0, SC_DMAX, SC_NNZ, SC_COUNT0, &launches))) return rc;
    if (Bm) {
        if ((rc = ingest(ctx, ws, s, Bm, n, np, Sa, 0, SC_DMAX2, SC_NNZ2, SC_COUNT2, &launches))) return rc;
    } else {
        // identity: no source rows, diagonal added (rows past n are padding)
        if ((rc = ingest(ctx, ws, s, nullptr, 0, np, Sa, 1, SC_DMAX2, SC_NNZ2, SC_COUNT2, &launches)))
            return rc;
    }
    tm.mark(1);
    if ((rc = read_scalars(ws, s))) return rc;
    if ((rc = check_status(ws, s))) return rc;
    const double dmax = static_cast<double>(host_scal(ws)[SC_DMAX]);
    double eps = 0;
    if ((rc = choose_eps(a.eps, 1.0 / (1.0 + dmax * dmax), "Sec. 7.2 (1/(1+||P||^2))", &eps))) return rc;
    unsigned long long s_count = host_scal(ws)[SC_COUNT2];
    if (!Bm) s_count = static_cast<unsigned long long>(np);  // identity over padded size
    const unsigned long long q_count0 = host_scal(ws)[SC_COUNT0];

    // Tables per parity: [T = Q S, Q' = Q Q] (MN-major B) and [S' = T Q^T | S] (K-major B).
    const int bn = bool_bn(ctx, np);
    GemmProblem g1[4], g2[2];
    std::string err;
    for (int p = 0; p < 2; ++p) {
        uint8_t *Sc = p ? Sb : Sa, *Sn = p ? Sa : Sb, *Qc = p ? Qb : Qa, *Qn = p ? Qa : Qb;
        const int N = static_cast<int>(np);
        bool ok = gemm_make_problem(&g1[2 * p], KIND_F8, false, bn, N, N, N, square_op(Qc, np),
                                    square_op(Sc, np), bool_epi(T, np, nullptr, wp, nullptr, nullptr), &err) &&
                  gemm_make_problem(&g1[2 * p + 1], KIND_F8, false, bn, N, N, N, square_op(Qc, np),
                                    square_op(Qc, np), bool_epi(Qn, np, nullptr, wp, ws.scal + SC_CQ, nullptr),
                                    &err) &&
                  gemm_make_problem(&g2[p], KIND_F8, true, bn, N, N, N, square_op(T, np), square_op(Qc, np),
                                    bool_epi(Sn, np, sbits, wp, ws.scal + SC_CS, Sc), &err);
        if (!ok) {
            set_error("%s", err.c_str());
            return DL_EDEVICE;
        }
        g1[2 * p + 1].tile_start = g1[2 * p].tiles_m * g1[2 * p].tiles_n;
    }
    GemmProblem all[6] = {g1[0], g1[1], g1[2], g1[3], g2[0], g2[1]};
    GemmProblem *d = nullptr;
    if ((rc = upload_problems(ws, s, all, 6, &d))) return rc;
    const int tiles1 = g1[0].tiles_m * g1[0].tiles_n;
    const int grid1 = std::min(2 * tiles1, ctx->sms), grid2 = std::min(tiles1, ctx->sms);

    GemmClock gc{ws, s};
    int step = 0;
    (void)q_count0;  // P = 0 ends after one step (Q' = 0, S' = B)
    const int max_steps = 2 + static_cast<int>(std::ceil(std::log2(static_cast<double>(np) + 1.0)));
    for (;;) {
        if (step >= max_steps) {
            set_error("same-generation doubling did not converge in %d steps", step);
            return DL_ENOTCONV;
        }
        const int p = step & 1;
        CK(cudaMemsetAsync(ws.scal + SC_CQ, 0, 2 * sizeof(unsigned long long), s));
        gc.start();
        CK(gemm_launch(KIND_F8, false, bn, EPI_BOOL, d + 2 * p, 2, 2 * tiles1, grid1, ws.status,
                       ctx->budget_ns, s));
        gc.stop(4.0 * np * np * np);
        gc.start();
        CK(gemm_launch(KIND_F8, true, bn, EPI_BOOL, d + 4 + p, 1, tiles1, grid2, ws.status,
                       ctx->budget_ns, s));
        gc.stop(2.0 * np * np * np);
        launches += 2;
        ++step;
        if ((rc = read_scalars(ws, s))) return rc;
        const unsigned long long cs = host_scal(ws)[SC_CS], cq = host_scal(ws)[SC_CQ];
        const bool stop = cs == s_count || cq == 0;
        s_count = cs;
        if (stop) break;
    }
    tm.mark(2);
    if ((rc = write_bits(s, sbits, wp, a.out_bits, n, a.mem))) return rc;
    tm.mark(3);
    if ((rc = check_status(ws, s))) return rc;
    if (st) {
        st->path_used = DL_PATH_BOOL_FP8;
        st->eps_used = eps;
        st->iters = step;
        gc.fill(st);
        // ones of S over the padded size, less the padding's own diagonal when B = I
        st->model_ones = static_cast<int64_t>(s_count) - (Bm ? 0 : static_cast<int64_t>(np - n));
        st->ms_factor = tm.ms(0, 1);
        st->ms_solve = tm.ms(1, 2);
        st->ms_epilogue = tm.ms(2, 3);
        st->ms_total = tm.ms(0, 3);
        st->gpu_launches = launches;
    }
    return DL_OK;
}

dl_status solve_compose(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a,
                        dl_stats *st) {
    const int32_t n = a.n;
    const int64_t np = round_up(std::max<int64_t>(n, 1), 256);
    const int64_t wp = np / 64;
    Timer tm{ws.ev, s, "compose"};
    int launches = 0;
    tm.mark(0);
    const uint8_t *R1 = nullptr, *R2 = nullptr;
    dl_status rc = stage_input(ws, s, a.E, n, in_mem(a), "in0", &R1);
    if (rc) return rc;
    if ((rc = stage_input(ws, s, a.E2, n, in_mem(a), "in1", &R2))) return rc;
    auto *A8 = static_cast<uint8_t *>(ws.get("c0", np * np));
    auto *B8 = static_cast<uint8_t *>(ws.get("c1", np * np));
    auto *bits = static_cast<uint64_t *>(ws.get("bits0", np * wp * 8));
    NEED(A8 && B8 && bits);
    CK(cudaMemsetAsync(ws.scal, 0, kScalars * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(ws.status, 0, sizeof(int), s));
    if ((rc = ingest(ctx, ws, s, R1, n, np, A8, 0, SC_DMAX, SC_NNZ, SC_COUNT0, &launches))) return rc;
    if ((rc = ingest(ctx, ws, s, R2, n, np, B8, 0, SC_DMAX2, SC_NNZ2, SC_COUNT2, &launches))) return rc;
    tm.mark(1);
    GemmProblem pr;
    std::string err;
    const int bn = bool_bn(ctx, np);
    if (!gemm_make_problem(&pr, KIND_F8, false, bn, static_cast<int>(np), static_cast<int>(np),
                           static_cast<int>(np), square_op(A8, np), square_op(B8, np),
                           bool_epi(nullptr, np, bits, wp, ws.scal + SC_ONES, nullptr), &err)) {
        set_error("%s", err.c_str());
        return DL_EDEVICE;
    }
    GemmProblem *d = nullptr;
    if ((rc = upload_problems(ws, s, &pr, 1, &d))) return rc;
    const int tiles = pr.tiles_m * pr.tiles_n;
    GemmClock gc{ws, s};
    gc.start();
    CK(gemm_launch(KIND_F8, false, bn, EPI_BOOL, d, 1, tiles, std::min(tiles, ctx->sms), ws.status,
                   ctx->budget_ns, s));
    gc.stop(2.0 * np * np * np);
    ++launches;
    tm.mark(2);
    if ((rc = write_bits(s, bits, wp, a.out_bits, n, a.mem))) return rc;
    tm.mark(3);
    if ((rc = read_scalars(ws, s))) return rc;
    if ((rc = check_status(ws, s))) return rc;
    if (st) {
        st->path_used = DL_PATH_BOOL_FP8;
        gc.fill(st);
        st->model_ones = static_cast<int64_t>(host_scal(ws)[SC_ONES]);
        st->ms_factor = tm.ms(0, 1);
        st->ms_solve = tm.ms(1, 2);
        st->ms_epilogue = tm.ms(2, 3);
        st->ms_total = tm.ms(0, 3);
        st->gpu_launches = launches;
    }
    return DL_OK;
}

// The real least solution S~ = eps (B + P S~ P^T) of same generation (Sec. 7.2; its positive
// entries are the model, Theorem 2), in FP64, written to a.out_rtilde (n x n doubles).
//  * the series X_{t+1} = eps (B + P X_t P^T) from X_0 = 0 (FP64 gathers over the CSR of P;
//    X_{t+1} - X_t is X_t's residual, so a step whose change is at most tol eps ends it).  It
//    is exact after depth + 1 steps when P is nilpotent (a forest or a DAG);
//  * otherwise (DL_PATH_MIXED, or AUTO after 64 steps) refinement from the current X: the
//    residual in FP64, the correction D = sum_m (eps P)^m R (P^T)^m by Smith's doubling for
//    the Stein equation X = R + A X A^T with A = sqrt(eps) P on the TF32 tensor cores
//    (A_0 = A, A_{k+1} = A_k^2, X <- X + A_k X A_k^T; stopped when ||A_K||_inf^2 <= 1e-5, the
//    tail's relative size), X += D.
// The optional bits are S~ > 0 made exact by the boolean iteration S <- B | P S P^T started from
// B and those bits (an entry lost to underflow comes back; none can be spurious, since exact
// zeros stay exact through non-negative products and through the refinement).
dl_status solve_sg_real(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a, dl_stats *st) {
    if (a.thr != 0.0) {
        set_error("thr must be 0: the model is S~ > 0 (Theorem 2)");
        return DL_EINVAL;
    }
    if (a.path != DL_PATH_AUTO && a.path != DL_PATH_FP64 && a.path != DL_PATH_MIXED) {
        set_error("the real S~ runs on DL_PATH_AUTO, DL_PATH_FP64 or DL_PATH_MIXED");
        return DL_EINVAL;
    }
    const int32_t n = a.n;
    const int64_t np = round_up(std::max<int64_t>(n, 1), 256);
    const int64_t wp = np / 64;
    if (np * static_cast<int64_t>(sizeof(double)) > 227 * 1024) {
        set_error("n = %d: a row of S~ exceeds one block's shared memory", n);
        return DL_EINVAL;
    }
    Timer tm{ws.ev, s, "sg_real"};
    int launches = 0, gemm_launches = 0;
    tm.mark(0);
    const uint8_t *P = nullptr, *Bm = nullptr;
    dl_status rc = stage_input(ws, s, a.E, n, a.mem, "in0", &P);
    if (rc) return rc;
    if (a.E2 && (rc = stage_input(ws, s, a.E2, n, a.mem, "in1", &Bm))) return rc;
    const size_t nn = static_cast<size_t>(np) * np;
    auto *bits = static_cast<uint64_t *>(ws.get("bits0", np * wp * 8));
    auto *bitsB = static_cast<uint64_t *>(ws.get("bits1", np * wp * 8));
    auto *cnt = static_cast<int *>(ws.get("g_cnt", (np + 1) * 4));
    auto *ptr = static_cast<int *>(ws.get("g_ptr", (np + 1) * 4));
    auto *colmask = static_cast<uint64_t *>(ws.get("g_colmask", wp * 8));
    auto *Xd = static_cast<double *>(ws.get("sr_X", nn * 8));
    auto *Xn = static_cast<double *>(ws.get("sr_Xn", nn * 8));
    auto *U = static_cast<double *>(ws.get("sr_U", nn * 8));
    NEED(bits && bitsB && cnt && ptr && colmask && Xd && Xn && U);
    CK(cudaMemsetAsync(ws.scal, 0, kScalars * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(ws.status, 0, sizeof(int), s));
    CK(cudaMemsetAsync(colmask, 0, wp * 8, s));
    // P: 0/1 check, ||P||_inf, the CSR; B: 0/1 check
    CK(csr_pack_checked(P, n, static_cast<int>(np), wp, cnt, ptr, bits, ws.scal + SC_DMAX, ws.scal + SC_NNZ,
                        ws.scal + SC_COUNT0, ws.status, colmask, s));
    launches += 2;
    if (Bm) {
        CK(pack_bits(Bm, n, static_cast<int>(np), wp, bitsB, ws.status, s));
        ++launches;
    }
    if ((rc = read_scalars(ws, s))) return rc;
    if ((rc = check_status(ws, s))) return rc;
    const double dmax = static_cast<double>(host_scal(ws)[SC_DMAX]);
    double eps = 0;
    if ((rc = choose_eps(a.eps, 1.0 / (1.0 + dmax * dmax), "Sec. 7.2 (1/(1+||P||^2))", &eps))) return rc;
    const int64_t nnz = static_cast<int64_t>(host_scal(ws)[SC_NNZ]);
    auto *col = static_cast<int *>(ws.get("g_col", static_cast<size_t>(std::max<int64_t>(nnz, 1)) * 4));
    NEED(col);
    CK(csr_fill_from_bits(bits, n, wp, ptr, col, s));
    CK(cudaMemsetAsync(Xd, 0, nn * 8, s));
    ++launches;
    tm.mark(1);

    const double tol = ctx->cfg.refine_tol > 0 ? ctx->cfg.refine_tol : 1e-13;
    const bool fused = sg_real_fused(static_cast<int>(np), host_scal(ws)[SC_DMAX]);
    unsigned long long *slot = ws.scal + 32;  // per-step max |change|, bit patterns of doubles
    auto as_double = [](unsigned long long b) {
        double d;
        std::memcpy(&d, &b, sizeof d);
        return d;
    };
    bool done = false;
    int steps = 0, refine_steps = 0;
    double resid = 0.0;
    GemmClock gc{ws, s};
    if (a.path != DL_PATH_MIXED) {  // the series, four steps per host read
        constexpr int kGroup = 4;
        const int budget = a.path == DL_PATH_FP64 ? 100000 : 64;
        while (!done && steps < budget) {
            CK(cudaMemsetAsync(slot, 0, kGroup * sizeof(unsigned long long), s));
            for (int k = 0; k < kGroup; ++k) {
                CK(sg_real_step(ptr, col, n, static_cast<int>(np), eps, Bm, Xd, U, Xn, nullptr, slot + k, fused, s));
                std::swap(Xd, Xn);
                launches += 2;
            }
            if ((rc = read_scalars(ws, s))) return rc;
            for (int k = 0; k < kGroup; ++k) {
                ++steps;
                const unsigned long long code = host_scal(ws)[32 + k];  // max change < 2^(code - 4096)
                resid = code == 0 ? 0.0 : std::ldexp(1.0, static_cast<int>(code) - 4096) / eps;
                if (resid <= tol) {
                    done = true;  // the iterates after this step are at least as close
                    break;
                }
            }
        }
        if (!done && a.path == DL_PATH_FP64) {
            set_error("the series did not reach max|change|/eps <= %g in %d steps", tol, steps);
            return DL_ENOTCONV;
        }
    }
    tm.mark(2);
    if (!done) {  // refinement with Smith's doubling for the corrections
        constexpr int kMaxK = 40;
        constexpr int TB = 128;  // GEMM tile
        auto *Xs = static_cast<float *>(ws.get("sr_Xs", nn * 4));
        auto *W = static_cast<float *>(ws.get("sr_W", nn * 4));
        auto *WT = static_cast<float *>(ws.get("sr_WT", nn * 4));
        auto *AT = static_cast<float *>(ws.get("sr_AT", nn * 4));
        auto *dprob = static_cast<GemmProblem *>(ws.get("sr_probs", sizeof(GemmProblem) * (3 * kMaxK + 3)));
        NEED(Xs && W && WT && AT && dprob);
        std::vector<float *> A, NA;
        auto mat = [&](const char *base, int k) {
            return static_cast<float *>(ws.get(std::string(base) + std::to_string(k), nn * 4));
        };
        A.push_back(mat("sr_A", 0));
        NA.push_back(mat("sr_NA", 0));
        NEED(A[0] && NA[0]);
        CK(sg_scaled_p(P, n, static_cast<int>(np), static_cast<float>(std::sqrt(eps)), A[0], NA[0], s));
        ++launches;
        CK(gemm_prepare(KIND_TF32, true, TB, EPI_STORE_F32));
        CK(gemm_prepare(KIND_TF32, true, TB, EPI_SUB_F32));
        int nprob = 0;
        std::string err;
        auto op = [&](const float *m) { return Operand{m, np, np, np, 0, 0}; };
        // one problem C (=|-=) X Y^T of np x np operands, uploaded to slot nprob
        auto problem = [&](const float *X, const float *Y, float *C, GemmEpi /*the launch's epilogue*/,
                           int *slot_out) -> dl_status {
            GemmProblem p;
            GemmEpilogue e{};
            e.c32 = C;
            e.ld_c32 = np;
            if (!gemm_make_problem(&p, KIND_TF32, true, TB, static_cast<int>(np), static_cast<int>(np),
                                   static_cast<int>(np), op(X), op(Y), e, &err)) {
                set_error("same generation S~: %s", err.c_str());
                return DL_EDEVICE;
            }
            p.tile_start = 0;
            CK(cudaMemcpyAsync(dprob + nprob, &p, sizeof p, cudaMemcpyHostToDevice, s));
            *slot_out = nprob++;
            return DL_OK;
        };
        const int tiles = static_cast<int>((np / TB) * (np / TB));
        auto run = [&](int slot_i, GemmEpi epi) -> dl_status {
            gc.start();
            CK(gemm_launch(KIND_TF32, true, TB, epi, dprob + slot_i, 1, tiles, std::min(tiles, ctx->sms), ws.status,
                           ctx->budget_ns, s));
            gc.stop(2.0 * static_cast<double>(np) * np * np);
            ++launches;
            ++gemm_launches;
            return DL_OK;
        };
        // A_{k+1} = A_k^2 until ||A_K||_inf^2 <= 1e-5
        unsigned *nrm = reinterpret_cast<unsigned *>(ws.scal + 30);
        int K = 0;
        for (;;) {
            CK(cudaMemsetAsync(nrm, 0, sizeof(unsigned), s));
            CK(row_abs_sum_max(A[K], static_cast<int>(np), nrm, s));
            ++launches;
            if ((rc = read_scalars(ws, s))) return rc;
            unsigned nb_ = 0;
            std::memcpy(&nb_, host_scal(ws) + 30, sizeof nb_);
            float nk = 0.f;
            std::memcpy(&nk, &nb_, sizeof nk);
            if (nk == 0.0f || static_cast<double>(nk) * nk <= 1e-5) break;
            if (K + 1 > kMaxK) {
                set_error("same generation S~: ||(sqrt(eps) P)^(2^k)|| did not fall below 3e-3 in %d squarings", kMaxK);
                return DL_ENOTCONV;
            }
            A.push_back(mat("sr_A", K + 1));
            NA.push_back(mat("sr_NA", K + 1));
            NEED(A[K + 1] && NA[K + 1]);
            CK(transpose_f32(A[K], np, static_cast<int>(np), static_cast<int>(np), AT, np, s));
            int sq = 0;
            if ((rc = problem(A[K], AT, A[K + 1], EPI_STORE_F32, &sq))) return rc;
            if ((rc = run(sq, EPI_STORE_F32))) return rc;
            CK(negate_f32(A[K + 1], NA[K + 1], static_cast<int64_t>(nn), s));
            launches += 2;
            ++K;
        }
        // the doubling steps as problems: W = X_k A_k^T, then X_k -= (-A_k) (W^T)^T
        std::vector<int> p1(K), p2(K);
        for (int k = 0; k < K; ++k) {
            if ((rc = problem(Xs, A[k], W, EPI_STORE_F32, &p1[k]))) return rc;
            if ((rc = problem(NA[k], WT, Xs, EPI_SUB_F32, &p2[k]))) return rc;
        }
        double best = 0.0;
        int stall = 0;
        const int max_iters = ctx->cfg.refine_max_iters > 0 ? ctx->cfg.refine_max_iters : 30;
        for (;;) {
            CK(cudaMemsetAsync(slot, 0, sizeof(unsigned long long), s));
            CK(sg_real_step(ptr, col, n, static_cast<int>(np), eps, Bm, Xd, U, nullptr, Xs, slot, fused, s));  // Xs = R
            launches += 2;
            if ((rc = read_scalars(ws, s))) return rc;
            resid = as_double(host_scal(ws)[32]) / eps;
            if (resid <= tol) break;
            if (refine_steps == 0 || resid < 0.5 * best) {
                best = resid;
                stall = 0;
            } else if (++stall >= 2 && best <= 1e-8) {
                break;  // at the residual's rounding floor
            }
            if (refine_steps >= max_iters) {
                set_error("same generation S~: refinement stopped at max|R|/eps = %.3g after %d steps", resid,
                          refine_steps);
                return DL_ENOTCONV;
            }
            for (int k = 0; k < K; ++k) {  // Xs <- sum_m (A Xs A^T)-terms: the correction D
                if ((rc = run(p1[k], EPI_STORE_F32))) return rc;
                CK(transpose_f32(W, np, static_cast<int>(np), static_cast<int>(np), WT, np, s));
                ++launches;
                if ((rc = run(p2[k], EPI_SUB_F32))) return rc;
            }
            CK(add_f32_to_f64(Xd, Xs, static_cast<int64_t>(nn), s));
            ++launches;
            ++refine_steps;
        }
        steps += refine_steps;
    }
    tm.mark(3);
    CK(cudaMemcpy2DAsync(a.out_rtilde, static_cast<size_t>(n) * 8, Xd, static_cast<size_t>(np) * 8,
                         static_cast<size_t>(n) * 8, n,
                         a.mem == DL_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    tm.mark(4);
    CK(cudaEventSynchronize(ws.ev[4]));  // read before the boolean step reuses the events
    const double t_ingest = tm.ms(0, 1), t_series = tm.ms(1, 2), t_refine = tm.ms(2, 3), t_real = tm.ms(0, 4);
    const double t_gemm = gc.ms();  // before the boolean step reuses the GEMM events
    double t_bits = 0.0;
    int64_t model_ones = -1;
    unsigned long long guard = 0;
    if (a.out_bits) {
        auto *M = static_cast<uint64_t *>(ws.get("sr_bits", np * wp * 8));
        NEED(M);
        CK(cudaMemsetAsync(M, 0, np * wp * 8, s));  // the threshold writes rows < n, words < ceil(n/64)
        CK(cudaMemsetAsync(ws.scal + SC_GUARD, 0, sizeof(unsigned long long), s));
        const double tau = ctx->cfg.guard_tau > 0 ? ctx->cfg.guard_tau : 1e-30;
        CK(thresh_pack_f64(Xd, np, n, static_cast<int>(np), tau, M, wp, ws.scal + SC_GUARD, s));
        ++launches;
        if ((rc = read_scalars(ws, s))) return rc;
        guard = host_scal(ws)[SC_GUARD];
        dl_stats bs{};
        bool exact = false;
        SolveArgs b = a;
        b.path = DL_PATH_AUTO;
        b.eps = 0.0;
        if ((rc = sg_iteration(ctx, ws, s, b, &bs, &exact, M))) return rc;
        if (!exact && (rc = sg_doubling(ctx, ws, s, b, &bs))) return rc;
        launches += bs.gpu_launches;
        model_ones = bs.model_ones;
        t_bits = bs.ms_total;
        if (st) st->recheck_sweeps = bs.iters;
    }
    if (st) {
        st->path_used = done ? DL_PATH_FP64 : DL_PATH_MIXED;
        st->eps_used = eps;
        st->iters = steps;
        st->final_resid = resid;
        st->guard_flagged = static_cast<int64_t>(guard);
        st->model_ones = model_ones;
        st->ms_factor = t_ingest;
        st->ms_solve = t_series;
        st->ms_refine = t_refine;
        st->ms_epilogue = t_bits;
        st->ms_total = t_real + t_bits;
        st->gpu_launches = launches;
        st->gemm_launches = gemm_launches;
        st->ms_gemm = t_gemm;
        st->gemm_flops = gc.timed_flops;  // the flops of the timed launches, so the rate holds
    }
    return DL_OK;
}

// One equation of the tail recursive class (Sec. 6.1, eq. matrixeq:trec), its non-recursive
// part A already formed from the lower equations' solutions:
//     R~ = eps (A + B0 R~),  R~ = (I - eps B0)^-1 eps A,
// and its model, the least R with R = min1(A + B0 R) = min1((I + B0^+) A), B0^+ the transitive
// closure of B0 (a row of R is A's rows at every node reachable in zero or more B0 steps).
//  * the model: the closure of B0 (AUTO, or the squarings-only path), the identity added, one
//    boolean product with A on the FP8 tensor cores;
//  * R~ (DL_PATH_FP64 / DL_PATH_MIXED): the closure's real paths with the right-hand side eps A.
//    Exact zeros stay exact (an M-matrix and a non-negative right-hand side), so X > 0 lies
//    inside the model; the model's entries missing from it (underflow) are rows_rechecked.
dl_status solve_tail(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a, dl_stats *st) {
    if (a.thr != 0.0) {
        set_error("thr must be 0: the model is R~ > 0");
        return DL_EINVAL;
    }
    const bool real = a.path == DL_PATH_FP64 || a.path == DL_PATH_MIXED;
    if (!real && a.path != DL_PATH_AUTO && a.path != DL_PATH_BOOL_FP8) {
        set_error("unknown path %d", static_cast<int>(a.path));
        return DL_EINVAL;
    }
    if (a.out_rtilde && !real) {
        set_error("the boolean paths compute no real-valued R~; use DL_PATH_FP64 or DL_PATH_MIXED");
        return DL_EINVAL;
    }
    const int32_t n = a.n;
    const int64_t w = (n + 63) / 64;
    const uint8_t *B0 = nullptr, *A = nullptr;
    dl_status rc = stage_input(ws, s, a.E, n, a.mem, "tr_b0", &B0);
    if (rc) return rc;
    if ((rc = stage_input(ws, s, a.E2, n, a.mem, "tr_a", &A))) return rc;
    dl_stats sr{}, sc{}, sm{};
    int64_t thresh_ones = -1;
    if (real) {  // R~ with the right-hand side eps A; the model comes from the boolean route
        SolveArgs r = a;
        r.E = B0;
        r.E2 = nullptr;
        r.e_device = true;
        r.rhs = A;
        r.out_bits = nullptr;
        r.skip_recheck = true;
        if ((rc = solve_tc(ctx, ws, s, r, &sr))) return rc;
        thresh_ones = sr.model_ones;
    }
    auto *cl = static_cast<uint64_t *>(ws.get("tr_cl", static_cast<size_t>(n) * w * 8));
    auto *clb = static_cast<uint8_t *>(ws.get("tr_clb", std::max<size_t>(static_cast<size_t>(n) * n, 16)));
    NEED(cl && clb);
    SolveArgs c;
    c.n = n;
    c.E = B0;
    c.mem = DL_MEM_DEVICE;
    c.eps = a.eps;
    c.path = a.path == DL_PATH_BOOL_FP8 ? DL_PATH_BOOL_FP8 : DL_PATH_AUTO;
    c.out_bits = cl;
    if ((rc = solve_tc(ctx, ws, s, c, &sc))) return rc;  // B0^+ (and eps checked against ||B0||)
    CK(unpack_bits_u8(cl, n, clb, ws.status, s));
    CK(cudaMemset2DAsync(clb, static_cast<size_t>(n) + 1, 1, 1, n, s));  // + I: the diagonal bytes
    SolveArgs m;
    m.n = n;
    m.E = clb;
    m.E2 = A;
    m.e_device = true;
    m.mem = a.mem;
    m.out_bits = a.out_bits;
    if ((rc = solve_compose(ctx, ws, s, m, &sm))) return rc;  // min1((I + B0^+) A)
    if (st) {
        st->path_used = a.path;
        st->eps_used = real ? sr.eps_used : sc.eps_used;
        st->iters = real ? sr.iters : sc.iters;
        st->final_resid = real ? sr.final_resid : -1.0;
        st->guard_flagged = sr.guard_flagged;
        st->model_ones = sm.model_ones;
        st->rows_rechecked = thresh_ones >= 0 ? sm.model_ones - thresh_ones : 0;
        st->ms_factor = sr.ms_factor;
        st->ms_solve = sr.ms_solve;
        st->ms_refine = sr.ms_refine;
        st->ms_epilogue = sc.ms_total + sm.ms_total;
        st->ms_total = sr.ms_total + sc.ms_total + sm.ms_total;
        st->gpu_launches = sr.gpu_launches + sc.gpu_launches + sm.gpu_launches + 1;
        st->gemm_launches = sr.gemm_launches + sc.gemm_launches + sm.gemm_launches;
        st->gemm_flops = sr.gemm_flops + sc.gemm_flops + sm.gemm_flops;
        st->ms_gemm = sr.ms_gemm + sc.ms_gemm + sm.ms_gemm;
    }
    return DL_OK;
}

namespace {

// F = A1 (0/1 bytes) or 0, n x n FP64.
__global__ void rhs_init_kernel(const uint8_t *__restrict__ A1, int n, double *__restrict__ F) {
    const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (t < static_cast<int64_t>(n) * n) F[t] = A1 != nullptr && A1[t] ? 1.0 : 0.0;
}

// F += B R over the CSR of B:  F[i][j] += sum_{y in succ(i)} R[y][j]  (R n x n, row stride n).
__global__ void rhs_gather_kernel(const int *__restrict__ ptr, const int *__restrict__ col, int n,
                                  const double *__restrict__ R, double *__restrict__ F) {
    const int i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double acc = 0.0;
    const int q1 = ptr[i + 1];
    for (int q = ptr[i]; q < q1; ++q) acc += R[static_cast<int64_t>(col[q]) * n + j];
    F[static_cast<int64_t>(i) * n + j] += acc;
}

// out = [F > 0] (bytes) and *amax = max |F| (bits of a non-negative double).
__global__ void positive_bytes_kernel(const double *__restrict__ F, int64_t count, uint8_t *__restrict__ out,
                                      unsigned long long *amax) {
    unsigned long long m = 0;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < count;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double v = F[t];
        out[t] = v > 0.0 ? 1 : 0;
        const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v)) & 0x7FFFFFFFFFFFFFFFull;
        m = b > m ? b : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, m, o);
        m = other > m ? other : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(amax, m);
}

// dst |= src (bytes).
__global__ void or_bytes_kernel(uint8_t *__restrict__ dst, const uint8_t *__restrict__ src, int64_t count) {
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < count;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x)
        dst[t] |= src[t];
}

unsigned stream_grid(int64_t count) { return static_cast<unsigned>(std::min<int64_t>((count + 255) / 256, 16384)); }

}  // namespace

// One equation of the tail recursive class with the lower equations' real solutions
// (Sec. 6.1, eq. matrixeq:trec):
//     R~ = eps (A1 + B0 R~ + sum_q B_q R_q),   R~ = (I - eps B0)^-1 eps F,   F = A1 + sum_q B_q R_q,
// All pointers are device pointers (B0 / A1 may be null: zero); out_bits / out_rtilde in `mem`.
//  * F in FP64 by gathers over the CSR of each B_q;
//  * eps: default 1 / (1 + max_i (rowsum(B0)_i + sum_q rowsum(B_q)_i)), which makes
//    eps F[1, ..., 1] <= 1 when the R_q are at most 1 (Theorem 2) and keeps eps < 1 / ||B0||;
//  * the model: the least R with R = min1(A' + B0 R), A' = [F > 0] (the support of F is what the
//    lower models contribute, by the positivity of Lemma 5's kind), by solve_tail's boolean route;
//  * R~ (DL_PATH_FP64 / DL_PATH_MIXED, or AUTO with out_rtilde: mixed): the closure's real paths
//    with the real right-hand side F.
dl_status solve_tail_real(dl_ctx *ctx, Workspace &ws, cudaStream_t s, int32_t n, const uint8_t *B0,
                          const uint8_t *A1, int32_t nterms, const uint8_t *const *Bq, const double *const *Rq,
                          double eps_user, dl_path path, dl_mem mem, uint64_t *out_bits, double *out_rtilde,
                          dl_stats *st) {
    if (path != DL_PATH_AUTO && path != DL_PATH_BOOL_FP8 && path != DL_PATH_FP64 && path != DL_PATH_MIXED) {
        set_error("unknown path %d", static_cast<int>(path));
        return DL_EINVAL;
    }
    if (out_rtilde && path == DL_PATH_BOOL_FP8) {
        set_error("DL_PATH_BOOL_FP8 computes no real-valued R~; use DL_PATH_FP64 or DL_PATH_MIXED");
        return DL_EINVAL;
    }
    const int64_t nn = static_cast<int64_t>(n) * n, w = (n + 63) / 64;
    auto *F = static_cast<double *>(ws.get("tt_F", std::max<int64_t>(nn, 2) * 8));
    auto *Ab = static_cast<uint8_t *>(ws.get("tt_Ab", std::max<int64_t>(nn, 16)));
    auto *cnt = static_cast<int *>(ws.get("tt_cnt", (static_cast<size_t>(n) + 1) * 4));
    auto *ptr = static_cast<int *>(ws.get("tt_ptr", (static_cast<size_t>(n) + 1) * 4));
    auto *bits = static_cast<uint64_t *>(ws.get("tt_bits", std::max<int64_t>(n * w, 2) * 8));
    NEED(F && Ab && cnt && ptr && bits);
    const uint8_t *b0 = B0;
    if (!b0) {  // no recursive occurrence: B0 = 0
        auto *z = static_cast<uint8_t *>(ws.get("tt_zero", std::max<int64_t>(nn, 16)));
        NEED(z);
        CK(cudaMemsetAsync(z, 0, std::max<int64_t>(nn, 16), s));
        b0 = z;
    }
    CK(cudaMemsetAsync(ws.status, 0, sizeof(int), s));
    // row degrees of B0 and of every B_q (the default eps), and F
    std::vector<int> deg(static_cast<size_t>(n), 0), h(static_cast<size_t>(n) + 1);
    auto add_degrees = [&](const uint8_t *M) -> dl_status {
        CK(csr_build(M, n, cnt, ptr, s));
        CK(cudaMemcpyAsync(h.data(), cnt, static_cast<size_t>(n) * 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int32_t i = 0; i < n; ++i) deg[i] += h[i];
        return DL_OK;
    };
    dl_status rc;
    if ((rc = add_degrees(b0))) return rc;
    rhs_init_kernel<<<static_cast<unsigned>((nn + 255) / 256), 256, 0, s>>>(A1, n, F);
    CK(cudaGetLastError());
    int launches = 3;
    for (int32_t q = 0; q < nterms; ++q) {
        if ((rc = add_degrees(Bq[q]))) return rc;
        int nnz = 0;
        CK(cudaMemcpyAsync(&nnz, ptr + n, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        auto *col = static_cast<int *>(ws.get("tt_col", static_cast<size_t>(std::max(nnz, 1)) * 4));
        NEED(col);
        CK(csr_fill(Bq[q], n, ptr, col, s));
        dim3 grid(static_cast<unsigned>((n + 255) / 256), static_cast<unsigned>(n));
        rhs_gather_kernel<<<grid, 256, 0, s>>>(ptr, col, n, Rq[q], F);
        CK(cudaGetLastError());
        launches += 4;
    }
    const int dmax = *std::max_element(deg.begin(), deg.end());
    double eps = 0;
    if ((rc = choose_eps(eps_user, 1.0 / (1.0 + dmax), "Theorem 2 (eps F[1] <= 1)", &eps))) return rc;
    CK(cudaMemsetAsync(ws.scal + SC_GUARD, 0, sizeof(unsigned long long), s));
    positive_bytes_kernel<<<stream_grid(nn), 256, 0, s>>>(F, nn, Ab, ws.scal + SC_GUARD);
    CK(cudaGetLastError());
    ++launches;
    if ((rc = read_scalars(ws, s))) return rc;
    if ((rc = check_status(ws, s))) return rc;
    double fmax = 0.0;
    {
        const unsigned long long b = host_scal(ws)[SC_GUARD];
        std::memcpy(&fmax, &b, sizeof fmax);
    }
    // the model (unless the caller forms it from exact lower models: out_bits == nullptr)
    dl_stats sm{};
    if (out_bits) {
    SolveArgs m;
    m.n = n;
    m.E = b0;
    m.E2 = Ab;
    m.mem = DL_MEM_DEVICE;
    m.eps = eps;
    m.path = path == DL_PATH_BOOL_FP8 ? DL_PATH_BOOL_FP8 : DL_PATH_AUTO;
    m.out_bits = bits;
    if ((rc = solve_tail(ctx, ws, s, m, &sm))) return rc;
    CK(cudaMemcpyAsync(out_bits, bits, static_cast<size_t>(n) * w * 8,
                       mem == DL_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    }
    // R~
    dl_stats sr{};
    const bool real = path == DL_PATH_FP64 || path == DL_PATH_MIXED || out_rtilde != nullptr;
    if (real) {
        SolveArgs r;
        r.n = n;
        r.E = b0;
        r.e_device = true;
        r.rhs_real = F;
        r.rhs_bound = fmax;
        r.skip_recheck = true;
        r.mem = mem;
        r.eps = eps;
        r.path = path == DL_PATH_FP64 ? DL_PATH_FP64 : DL_PATH_MIXED;
        r.out_rtilde = out_rtilde;
        if ((rc = solve_tc(ctx, ws, s, r, &sr))) return rc;
    }
    CK(cudaStreamSynchronize(s));
    if (st) {
        st->path_used = real ? sr.path_used : sm.path_used;
        st->eps_used = eps;
        st->iters = real ? sr.iters : sm.iters;
        st->final_resid = real ? sr.final_resid : -1.0;
        st->model_ones = sm.model_ones;
        // model entries that X > 0 missed (underflow; X > 0 never holds outside the model)
        st->rows_rechecked = real && out_bits ? sm.model_ones - sr.model_ones : 0;
        st->ms_factor = sr.ms_factor;
        st->ms_solve = sr.ms_solve;
        st->ms_refine = sr.ms_refine;
        st->ms_epilogue = sm.ms_total;
        st->ms_total = sr.ms_total + sm.ms_total;
        st->gpu_launches = launches + sr.gpu_launches + sm.gpu_launches;
        st->gemm_launches = sr.gemm_launches + sm.gemm_launches;
        st->gemm_flops = sr.gemm_flops + sm.gemm_flops;
        st->ms_gemm = sr.ms_gemm + sm.ms_gemm;
    }
    return DL_OK;
}

// A layered system of tail recursive equations, solved in order (Sec. 6.1: each R~_h is solved with
// the lower ones substituted).  eqs[h].terms refer to equations j < h.  Real paths keep every R~_h
// on the device for the equations above it (FP64, n x n each); the boolean paths keep the models
// and form A'_h = min1(A1_h + sum_q B_q R_{j_q}) by FP8 products.
dl_status solve_tail_system(dl_ctx *ctx, Workspace &ws, cudaStream_t s, int32_t n, int32_t m, const dl_tail_eq *eqs,
                            dl_mem mem, dl_path path, uint64_t *const *out_bits, double *const *out_rtilde,
                            dl_stats *st) {
    const bool real = path == DL_PATH_FP64 || path == DL_PATH_MIXED;
    if (!real && path != DL_PATH_AUTO && path != DL_PATH_BOOL_FP8) {
        set_error("unknown path %d", static_cast<int>(path));
        return DL_EINVAL;
    }
    for (int32_t h = 0; h < m; ++h) {
        if (!out_bits[h]) {
            set_error("out_bits[%d] must not be NULL", h);
            return DL_EINVAL;
        }
        if (out_rtilde && out_rtilde[h] && !real) {
            set_error("out_rtilde needs DL_PATH_FP64 or DL_PATH_MIXED");
            return DL_EINVAL;
        }
        if (eqs[h].nterms < 0 || (eqs[h].nterms > 0 && (!eqs[h].B || !eqs[h].j))) {
            set_error("equation %d: bad terms", h);
            return DL_EINVAL;
        }
        for (int32_t q = 0; q < eqs[h].nterms; ++q)
            if (eqs[h].j[q] < 0 || eqs[h].j[q] >= h || !eqs[h].B[q]) {
                set_error("equation %d, term %d: j must name an equation below %d", h, q, h);
                return DL_EINVAL;
            }
    }
    const int64_t nn = static_cast<int64_t>(n) * n, w = (n + 63) / 64;
    auto key = [](const char *base, int a, int b = -1) {
        return std::string(base) + std::to_string(a) + (b >= 0 ? "_" + std::to_string(b) : std::string());
    };
    auto stage = [&](const uint8_t *src, const std::string &name, const uint8_t **out) -> dl_status {
        if (!src || mem == DL_MEM_DEVICE) {
            *out = src;
            return DL_OK;
        }
        auto *d = static_cast<uint8_t *>(ws.get(name, std::max<int64_t>(nn, 16)));
        NEED(d);
        CK(cudaMemcpyAsync(d, src, nn, cudaMemcpyHostToDevice, s));
        *out = d;
        return DL_OK;
    };
    dl_stats tot{};
    dl_status rc;
    for (int32_t h = 0; h < m; ++h) {
        const dl_tail_eq &eq = eqs[h];
        const uint8_t *A1 = nullptr, *B0 = nullptr;
        if ((rc = stage(eq.A1, key("ts_a", h), &A1)) || (rc = stage(eq.B0, key("ts_b", h), &B0))) return rc;
        std::vector<const uint8_t *> Bq(static_cast<size_t>(eq.nterms));
        for (int32_t q = 0; q < eq.nterms; ++q)
            if ((rc = stage(eq.B[q], key("ts_q", h, q), &Bq[q]))) return rc;
        auto *bits = static_cast<uint64_t *>(ws.get(key("ts_bits", h), std::max<int64_t>(n * w, 2) * 8));
        NEED(bits);
        dl_stats sh{};
        {   // the model from the lower models: A' = A1 | OR_q min1(B_q M_{j_q}) as bytes
            auto *Ap = static_cast<uint8_t *>(ws.get("ts_ap", std::max<int64_t>(nn, 16)));
            auto *cb = static_cast<uint64_t *>(ws.get("ts_cbits", std::max<int64_t>(n * w, 2) * 8));
            auto *cu = static_cast<uint8_t *>(ws.get("ts_cu8", std::max<int64_t>(nn, 16)));
            NEED(Ap && cb && cu);
            if (A1) CK(cudaMemcpyAsync(Ap, A1, nn, cudaMemcpyDeviceToDevice, s));
            else CK(cudaMemsetAsync(Ap, 0, nn, s));
            for (int32_t q = 0; q < eq.nterms; ++q) {
                const auto *Mj = static_cast<const uint8_t *>(ws.get(key("ts_m", eq.j[q]), static_cast<size_t>(nn)));
                SolveArgs c;
                c.n = n;
                c.E = Bq[q];
                c.E2 = Mj;
                c.mem = DL_MEM_DEVICE;
                c.out_bits = cb;
                dl_stats sc{};
                if ((rc = solve_compose(ctx, ws, s, c, &sc))) return rc;
                CK(unpack_bits_u8(cb, n, cu, ws.status, s));
                or_bytes_kernel<<<stream_grid(nn), 256, 0, s>>>(Ap, cu, nn);
                CK(cudaGetLastError());
                sh.gpu_launches += sc.gpu_launches + 2;
                sh.gemm_launches += sc.gemm_launches;
                sh.ms_total += sc.ms_total;
            }
            const uint8_t *b0 = B0;
            if (!b0) {
                auto *z = static_cast<uint8_t *>(ws.get("tt_zero", std::max<int64_t>(nn, 16)));
                NEED(z);
                CK(cudaMemsetAsync(z, 0, std::max<int64_t>(nn, 16), s));
                b0 = z;
            }
            SolveArgs t;
            t.n = n;
            t.E = b0;
            t.E2 = Ap;
            t.mem = DL_MEM_DEVICE;
            t.eps = eq.eps;
            t.path = path == DL_PATH_BOOL_FP8 ? DL_PATH_BOOL_FP8 : DL_PATH_AUTO;
            t.out_bits = bits;
            dl_stats stl{};
            if ((rc = solve_tail(ctx, ws, s, t, &stl))) return rc;
            sh.model_ones = stl.model_ones;
            sh.eps_used = stl.eps_used;
            sh.ms_total += stl.ms_total;
            sh.gpu_launches += stl.gpu_launches;
            sh.gemm_launches += stl.gemm_launches;
            auto *Mh = static_cast<uint8_t *>(ws.get(key("ts_m", h), std::max<int64_t>(nn, 16)));
            NEED(Mh);
            CK(unpack_bits_u8(bits, n, Mh, ws.status, s));
        }
        if (real) {  // R~_h from the lower R~ (kept on the device)
            std::vector<const double *> Rq(static_cast<size_t>(eq.nterms));
            for (int32_t q = 0; q < eq.nterms; ++q)
                Rq[q] = static_cast<const double *>(ws.get(key("ts_x", eq.j[q]), static_cast<size_t>(nn) * 8));
            auto *X = static_cast<double *>(ws.get(key("ts_x", h), std::max<int64_t>(nn, 2) * 8));
            NEED(X);
            dl_stats sr{};
            if ((rc = solve_tail_real(ctx, ws, s, n, B0, A1, eq.nterms, Bq.data(), Rq.data(), eq.eps, path,
                                      DL_MEM_DEVICE, nullptr, X, &sr)))
                return rc;
            if (out_rtilde && out_rtilde[h])
                CK(cudaMemcpyAsync(out_rtilde[h], X, static_cast<size_t>(nn) * 8,
                                   mem == DL_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
            sh.eps_used = sr.eps_used;
            sh.iters = sr.iters;
            sh.final_resid = sr.final_resid;
            sh.ms_total += sr.ms_total;
            sh.gpu_launches += sr.gpu_launches;
            sh.gemm_launches += sr.gemm_launches;
        }
        CK(cudaMemcpyAsync(out_bits[h], bits, static_cast<size_t>(n) * w * 8,
                           mem == DL_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        tot.ms_total += sh.ms_total;
        tot.gpu_launches += sh.gpu_launches;
        tot.gemm_launches += sh.gemm_launches;
        tot.model_ones += sh.model_ones;
        tot.iters += sh.iters;
        tot.final_resid = std::max(tot.final_resid, sh.final_resid);
        tot.rows_rechecked += sh.rows_rechecked;
        tot.eps_used = sh.eps_used;  // the last equation's
    }
    CK(cudaStreamSynchronize(s));
    if ((rc = check_status(ws, s))) return rc;
    if (st) {
        *st = tot;
        st->path_used = path;
    }
    return DL_OK;
}

size_t footprint_bytes(int kind, int32_t n) {
    const size_t np = static_cast<size_t>(round_up(std::max<int64_t>(n, 1), 256));
    const size_t mats = kind == 0 ? 3 : 7;  // staged inputs + operand buffers of the path
    return mats * np * np + 2 * np * (np / 8) + (1u << 20);
}

// ---- workspace ------------------------------------------------------------------------

namespace {

// The 0/1 bytes (n x n, row stride n) of an e4m3 0/1 matrix (row stride ldc).
__global__ void e4m3_to_u8_kernel(const uint8_t *__restrict__ C, int64_t ldc, int n, uint8_t *__restrict__ B) {
    const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (t >= static_cast<int64_t>(n) * n) return;
    const int64_t i = t / n, j = t - i * n;
    B[t] = C[i * ldc + j] != 0 ? 1 : 0;
}

}  // namespace

// The transposed class (Sec. 6.2), program prog:2:
//     r2(x,z) <- r1(x,z).      r2(x,z) <- r1(x,y), r2(z,y).
// Its completion R2 = min1(R1 + R1 R2^T) substituted into itself gives the two-sided equation
// R2 = min1(B + R1 R2 R1^T), B = min1(R1 + R1 R1^T) (eq. matrixeq:trans:2).  Both have the same
// least solution: the iterates of the two-step operator from 0 are every other iterate of the
// one-step operator, which increase to its least fixpoint.  So the model is one FP8 product
// (C = R1 R1^T with R1 added in the epilogue) and the same-generation solver with P = R1 and B.
// The real R~2 = eps (R1 + R1 R~2^T) (eq. matrixeq:trans:1; DL_PATH_FP64, or DL_PATH_AUTO when
// asked for): the increasing series X_{t+1} = eps (R1 + R1 X_t^T) from X_0 = 0 in FP64, four steps
// per host read, until a step changes no entry by more than tol eps; its positive entries are
// compared with the model (guard_flagged counts the bit words where they differ: only underflow
// can make them).
dl_status solve_transposed(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a, dl_stats *st) {
    if (a.thr != 0.0) {
        set_error("thr must be 0: the model is R~ > 0 (Theorem 2)");
        return DL_EINVAL;
    }
    if (a.path == DL_PATH_MIXED) {
        set_error("the transposed class has no mixed-precision path; use DL_PATH_FP64 or DL_PATH_AUTO");
        return DL_ENOTIMPL;
    }
    if (a.path != DL_PATH_AUTO && a.path != DL_PATH_BOOL_FP8 && a.path != DL_PATH_FP64) {
        set_error("unknown path %d", static_cast<int>(a.path));
        return DL_EINVAL;
    }
    if (a.path == DL_PATH_BOOL_FP8 && a.out_rtilde) {
        set_error("DL_PATH_BOOL_FP8 computes no real-valued R~; use DL_PATH_FP64 or DL_PATH_AUTO");
        return DL_EINVAL;
    }
    const int32_t n = a.n;
    const int64_t np = round_up(std::max<int64_t>(n, 1), 256);
    const int64_t wp = np / 64, w = (n + 63) / 64;
    Timer tm{ws.ev + 4, s, "transposed"};  // events 0-3 belong to the same-generation solver it calls
    int launches = 0;
    tm.mark(0);
    const uint8_t *R1 = nullptr;
    dl_status rc = stage_input(ws, s, a.E, n, a.mem, "tr_in0", &R1);
    if (rc) return rc;
    auto *R8 = static_cast<uint8_t *>(ws.get("tr_e8", np * np));
    auto *B8 = static_cast<uint8_t *>(ws.get("tr_b8", np * np));
    auto *Bu = static_cast<uint8_t *>(ws.get("tr_bu8", std::max<size_t>(static_cast<size_t>(n) * n, 16)));
    auto *Mw = static_cast<uint64_t *>(ws.get("tr_bits", std::max<size_t>(static_cast<size_t>(n) * w * 8, 16)));
    NEED(R8 && B8 && Bu && Mw);
    CK(cudaMemsetAsync(ws.scal, 0, kScalars * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(ws.status, 0, sizeof(int), s));
    if ((rc = ingest(ctx, ws, s, R1, n, np, R8, 0, SC_DMAX, SC_NNZ, SC_COUNT0, &launches))) return rc;
    if ((rc = read_scalars(ws, s))) return rc;
    if ((rc = check_status(ws, s))) return rc;
    const unsigned long long dmax = host_scal(ws)[SC_DMAX];
    double eps = 0;
    if ((rc = choose_eps(a.eps, 1.0 / (1.0 + static_cast<double>(dmax)), "Sec. 6.2 (1/(1+||R1||_inf))", &eps)))
        return rc;
    // B = min1(R1 + R1 R1^T): C[i][j] = sum_k R1[i][k] R1[j][k] (B operand K-major = R1 itself)
    GemmProblem pr;
    std::string err;
    const int bn = bool_bn(ctx, np);
    if (!gemm_make_problem(&pr, KIND_F8, true, bn, static_cast<int>(np), static_cast<int>(np), static_cast<int>(np),
                           square_op(R8, np), square_op(R8, np), bool_epi(B8, np, nullptr, wp, nullptr, R8), &err)) {
        set_error("%s", err.c_str());
        return DL_EDEVICE;
    }
    GemmProblem *d = nullptr;
    if ((rc = upload_problems(ws, s, &pr, 1, &d))) return rc;
    const int tiles = pr.tiles_m * pr.tiles_n;
    GemmClock gc{ws, s};
    gc.start();
    CK(gemm_launch(KIND_F8, true, bn, EPI_BOOL, d, 1, tiles, std::min(tiles, ctx->sms), ws.status, ctx->budget_ns, s));
    gc.stop(2.0 * np * np * np);
    const int64_t nn = static_cast<int64_t>(n) * n;
    e4m3_to_u8_kernel<<<static_cast<unsigned>((nn + 255) / 256), 256, 0, s>>>(B8, np, n, Bu);
    CK(cudaGetLastError());
    launches += 2;
    if ((rc = read_scalars(ws, s))) return rc;  // (the GEMM table's staging is free again)
    if ((rc = check_status(ws, s))) return rc;
    const double b_gemm_ms = gc.ms(), b_gemm_flops = gc.timed_flops;  // (its events are reused below)
    tm.mark(1);
    SolveArgs b = a;
    b.E = R1;
    b.E2 = Bu;
    b.mem = DL_MEM_DEVICE;
    b.e_device = false;
    b.eps = 0.0;
    b.path = a.path == DL_PATH_BOOL_FP8 ? DL_PATH_BOOL_FP8 : DL_PATH_AUTO;
    b.out_bits = Mw;
    b.out_rtilde = nullptr;
    dl_stats sgst{};
    if ((rc = solve_sg(ctx, ws, s, b, &sgst))) return rc;
    launches += sgst.gpu_launches;
    CK(cudaMemcpyAsync(a.out_bits, Mw, static_cast<size_t>(n) * w * 8,
                       a.mem == DL_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    tm.mark(2);
    int steps = 0;
    double resid = 0.0;
    unsigned long long differ = 0;
    const bool real = a.out_rtilde != nullptr || a.path == DL_PATH_FP64;
    if (real) {
        const size_t nq = static_cast<size_t>(np) * np;
        auto *cnt = static_cast<int *>(ws.get("tr_cnt", (np + 1) * 4));
        auto *ptr = static_cast<int *>(ws.get("tr_ptr", (np + 1) * 4));
        auto *X = static_cast<double *>(ws.get("tr_X", nq * 8));
        auto *Xn = static_cast<double *>(ws.get("tr_Xn", nq * 8));
        auto *U = static_cast<double *>(ws.get("tr_U", nq * 8));
        NEED(cnt && ptr && X && Xn && U);
        CK(csr_build(R1, n, cnt, ptr, s));
        int nnz = 0;
        CK(cudaMemcpyAsync(&nnz, ptr + n, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        auto *col = static_cast<int *>(ws.get("tr_col", static_cast<size_t>(std::max(nnz, 1)) * 4));
        NEED(col);
        CK(csr_fill(R1, n, ptr, col, s));
        CK(cudaMemsetAsync(X, 0, nq * 8, s));
        launches += 3;
        const double tol = ctx->cfg.refine_tol > 0 ? ctx->cfg.refine_tol : 1e-13;
        unsigned long long *slot = ws.scal + 32;
        constexpr int kGroup = 4, kBudget = 100000;
        bool done = false;
        while (!done && steps < kBudget) {
            CK(cudaMemsetAsync(slot, 0, kGroup * sizeof(unsigned long long), s));
            for (int k = 0; k < kGroup; ++k) {
                CK(trans_real_step(ptr, col, n, static_cast<int>(np), eps, R1, X, U, Xn, slot + k, s));
                std::swap(X, Xn);
                launches += 2;
            }
            if ((rc = read_scalars(ws, s))) return rc;
            for (int k = 0; k < kGroup; ++k) {
                ++steps;
                const unsigned long long code = host_scal(ws)[32 + k];  // max change < 2^(code - 4096)
                resid = code == 0 ? 0.0 : std::ldexp(1.0, static_cast<int>(code) - 4096) / eps;
                if (resid <= tol) {
                    done = true;  // the iterates after this step are at least as close
                    break;
                }
            }
        }
        if (!done) {
            set_error("transposed class: the series did not reach max|change|/eps <= %g in %d steps", tol, steps);
            return DL_ENOTCONV;
        }
        if (a.out_rtilde)
            CK(cudaMemcpy2DAsync(a.out_rtilde, static_cast<size_t>(n) * 8, X, static_cast<size_t>(np) * 8,
                                 static_cast<size_t>(n) * 8, n,
                                 a.mem == DL_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        // X > 0 against the model, word by word (np x wp layouts, rows < n)
        auto *T = static_cast<uint64_t *>(ws.get("tr_tbits", np * wp * 8));
        auto *Mp = static_cast<uint64_t *>(ws.get("tr_mbits", np * wp * 8));
        NEED(T && Mp);
        CK(cudaMemsetAsync(T, 0, np * wp * 8, s));
        CK(cudaMemsetAsync(Mp, 0, np * wp * 8, s));
        CK(cudaMemcpy2DAsync(Mp, wp * 8, Mw, w * 8, w * 8, n, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemsetAsync(ws.scal + SC_GUARD, 0, 2 * sizeof(unsigned long long), s));
        CK(thresh_pack_f64(X, np, n, static_cast<int>(np), 0.0, T, wp, ws.scal + SC_GUARD, s));
        CK(bits_diff(T, Mp, np * wp, ws.scal + SC_GUARD + 1, s));
        launches += 2;
        if ((rc = read_scalars(ws, s))) return rc;
        differ = host_scal(ws)[SC_GUARD + 1];
    }
    tm.mark(3);
    if ((rc = check_status(ws, s))) return rc;
    if (st) {
        st->path_used = real ? DL_PATH_FP64 : sgst.path_used;
        st->eps_used = eps;
        st->iters = real ? steps : sgst.iters;
        st->final_resid = resid;
        st->guard_flagged = static_cast<int64_t>(differ);
        st->model_ones = sgst.model_ones;
        st->ms_factor = tm.ms(0, 1);
        st->ms_solve = tm.ms(1, 2);
        st->ms_refine = tm.ms(2, 3);
        st->ms_total = tm.ms(0, 3);
        st->gpu_launches = launches;
        st->gemm_launches = 1 + sgst.gemm_launches;
        st->ms_gemm = b_gemm_ms + sgst.ms_gemm;
        st->gemm_flops = b_gemm_flops + sgst.gemm_flops;
    }
    return DL_OK;
}

cudaError_t Workspace::init() {
    if (ready) return cudaSuccess;
    // each piece only if it is missing, so a call after a failed one resumes without leaks
    cudaError_t e;
    if (!host_pinned) {
        if ((e = host_pinned_alloc(&host_pinned, kHostPinned)) != cudaSuccess) return e;
        host_bytes = kHostPinned;
    }
    if (!status && (e = device_alloc(reinterpret_cast<void **>(&status), 256)) != cudaSuccess) return e;
    if (!scal && (e = device_alloc(reinterpret_cast<void **>(&scal), kScalars * sizeof(unsigned long long))) !=
                     cudaSuccess)
        return e;
    for (auto &x : ev)
        if (!x && (e = cudaEventCreate(&x)) != cudaSuccess) return e;
    for (auto &x : gev)
        if (!x && (e = cudaEventCreate(&x)) != cudaSuccess) return e;
    for (auto &x : sev)
        if (!x && (e = cudaEventCreate(&x)) != cudaSuccess) return e;
    ready = true;
    return cudaSuccess;
}

void Workspace::release() {
    // the captured graph first: its nodes refer to the buffers, events and streams below
    if (mx_graph) cudaGraphExecDestroy(mx_graph);
    mx_graph = nullptr;
    mx_graph_key.clear();
    batch_plan_release(batch_plan);
    batch_plan = nullptr;
    for (auto &kv : bufs)
        if (kv.second.p) cudaFree(kv.second.p);
    bufs.clear();
    if (host_pinned) cudaFreeHost(host_pinned);
    if (status) cudaFree(status);
    if (scal) cudaFree(scal);
    for (auto &x : ev)
        if (x) cudaEventDestroy(x);
    for (auto &x : gev)
        if (x) cudaEventDestroy(x);
    for (auto &x : sev)
        if (x) cudaEventDestroy(x);
    for (auto &x : mx_ev)
        if (x) cudaEventDestroy(x);
    for (auto &x : mx_stream)
        if (x) cudaStreamDestroy(x);
    for (auto &x : mx_gev)
        if (x) cudaEventDestroy(x);
    for (auto &x : mx_gev) x = nullptr;
    for (auto &x : mx_ev) x = nullptr;
    for (auto &x : mx_stream) x = nullptr;
    for (auto &x : ev) x = nullptr;
    for (auto &x : gev) x = nullptr;
    for (auto &x : sev) x = nullptr;
    host_pinned = nullptr;
    status = nullptr;
    scal = nullptr;
    ready = false;
}

void *Workspace::get(const std::string &name, size_t bytes) {
    Buf &b = bufs[name];
    if (b.p && b.bytes >= bytes) return b.p;
    // grow by at least a quarter: buffers sized by data (facts, active rows) then rarely grow
    // again, and a regrowth's cudaFree waits for the whole device
    const size_t grown = b.p ? b.bytes + b.bytes / 4 : 0;
    if (b.p) {
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    size_t want = (std::max(bytes, grown) + 4095) & ~static_cast<size_t>(4095);
    if (device_alloc(&b.p, want) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return nullptr;
    }
    b.bytes = want;
    return b.p;
}

size_t Workspace::capacity(const std::string &name) const {
    const auto it = bufs.find(name);
    return it == bufs.end() ? 0 : it->second.bytes;
}

size_t Workspace::footprint() const {
    size_t t = 0;
    for (auto &kv : bufs) t += kv.second.bytes;
    return t;
}

}  // namespace dl
