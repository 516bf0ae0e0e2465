// dl_ctx.h -- the context behind the opaque dl_ctx handle and the per-call solve drivers.
#pragma once
#include <cuda_runtime.h>

#include <condition_variable>
#include <cstdarg>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/dl.h"
#include "dl_internal.h"

namespace dl {

void set_error(const char *fmt, ...);

struct BatchPlan;  // cached CUDA graph of the last dl_tc_batch call (dl_batch.cu)
void batch_plan_release(BatchPlan *p);

// Grow-only device buffers, one set per execution slot (a synchronous call or one serving
// slot), so concurrent slots never share scratch memory.
struct Workspace {
    struct Buf {
        void *p = nullptr;
        size_t bytes = 0;
    };
    std::map<std::string, Buf> bufs;
    void *host_pinned = nullptr;  // small pinned staging for scalars and GEMM tables
    size_t host_bytes = 0;
    int *status = nullptr;         // device status word
    unsigned long long *scal = nullptr;  // device scalars (counters)
    cudaEvent_t ev[8] = {};
    static constexpr int kGemmEvents = 128;  // start/stop pairs of timed GEMM launches
    cudaEvent_t gev[kGemmEvents] = {};
    cudaEvent_t sev[kGemmEvents] = {};       // start/stop pairs of timed sweep groups
    bool ready = false;
    // mixed path, created on first use: streams for the LU's critical chain (greatest priority),
    // its bulk updates (middle), the inverse (least), the row-panel transposes and each step's
    // off-chain row and column update (greatest), and events ordering them
    cudaStream_t mx_stream[5] = {};
    cudaEvent_t mx_ev[8] = {};
    cudaEvent_t mx_gev[32] = {};      // a group of the LU is final (the inverse may start on it)
    cudaGraphExec_t mx_graph = nullptr;  // the factorisation and inverse of the last size, captured
    std::string mx_graph_key;
    int mx_graph_launches = 0;
    BatchPlan *batch_plan = nullptr;
    bool last_heavy = false;  // the last closure on this workspace had rows of > 256 successors
    bool last_rows_closed = false;  // ... was closed by the Iteration on single rows alone
    bool last_dense = false;        // ... had more than two facts per row (no single-row Iteration)
    int last_spec_sweeps = 0;       // ... settled in its speculative phase after this many
                                    // working sweeps, plus one (0: it did not)

    cudaError_t init();
    void release();
    // device buffer of at least `bytes` (contents undefined); nullptr on failure
    void *get(const std::string &name, size_t bytes);
    // bytes held by buffer `name` (0 if it does not exist)
    size_t capacity(const std::string &name) const;
    size_t footprint() const;
};

struct Request;  // serving

// Tuned choices for one size bucket (dl_tune.cu); the defaults are the fixed rules.
struct TuneEntry {
    int bucket = 0;
    int sq_bn = 256;          // FP8 squaring tile width
    double t_sq = 0.0;        // seconds per squaring (0: the flop-rate model)
    double sweep_rate = 0.0;  // bytes per second of an unsaturated sweep (0: the size rule)
    int mx_reserve = 32;      // SMs the mixed LU's bulk update leaves to the chain
    int mx_pairs = -1;        // mixed LU steps taken in units sharing one bulk update (-1: half)
    int mx_group = 2;         // steps per such unit (2 or 4; K = that many blocks)
    int sg_iteration = -1;    // same generation on AUTO: 1 Iteration, 0 doubling, -1 by size
    bool measured = false;
};

struct Tuning {
    std::mutex mu;
    std::map<int, TuneEntry> by_bucket;
    std::string cache_path;
    std::string key_prefix;  // "<GPU name>|<driver version>|"
    bool autotune = false;
};

}  // namespace dl

struct dl_ctx {
    int device = 0;
    int sms = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    dl_config cfg{};
    uint64_t budget_ns = 2000000000ull;
    std::mutex mu;  // serialises synchronous calls
    dl::Workspace ws;

    dl::Tuning tune;  // tuned choices per size bucket (dl_tune.cu)

    // serving state (dl_serve.cpp)
    struct Serve;
    Serve *serve = nullptr;  // owned; freed by dl_serve_shutdown
};

namespace dl {

constexpr int kScalars = 64;  // device scalar slots per workspace
// scalar slot indices
enum : int {
    SC_DMAX = 0, SC_NNZ = 1, SC_COUNT0 = 2, SC_VIOL = 3, SC_ONES = 4, SC_GUARD = 5,
    SC_DMAX2 = 6, SC_NNZ2 = 7, SC_COUNT2 = 8, SC_CQ = 9, SC_CS = 10, SC_OPEN = 11, SC_GATE = 12, SC_STEP0 = 16
};

struct SolveArgs {
    int32_t n = 0;
    const uint8_t *E = nullptr;   // closure: E; same generation: P; compose: R1
    const uint64_t *E_bits = nullptr;  // closure: E bit-packed (n rows of ceil(n/64) words) instead
    bool e_device = false;        // E is on the device whatever mem says (unpacked from E_bits)
    const uint8_t *rhs = nullptr;  // tail recursive class: the right-hand side A of
                                   // X = eps (A + E X), a device pointer (NULL: A = E)
    const double *rhs_real = nullptr;  // a real right-hand side F of X = eps (F + E X) instead
                                       // (device, n x n FP64, row stride n; FP64 / mixed paths)
    double rhs_bound = 1.0;        // a bound on |F| (the mixed residual's fixed-point scale)
    bool skip_recheck = false;     // real paths: leave X > 0 in the bits unchecked, count its ones
    const uint8_t *E2 = nullptr;  // same generation: B (may be null); compose: R2
    dl_mem mem = DL_MEM_HOST;
    double eps = 0.0;
    double thr = 0.0;
    dl_path path = DL_PATH_AUTO;
    uint64_t *out_bits = nullptr;
    double *out_rtilde = nullptr;
};

// Drivers: run on (ws, stream); return a dl_status and fill stats.
dl_status solve_tc(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a, dl_stats *st);
dl_status solve_sg(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a, dl_stats *st);
// One equation of the tail recursive class: E = B0 (recursive coefficient), E2 = A (the
// non-recursive part); bits of the model, R~ into a.out_rtilde on the real paths.
dl_status solve_tail(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a, dl_stats *st);
// One tail recursive equation with real lower solutions, and a layered system of them.
dl_status solve_tail_real(dl_ctx *ctx, Workspace &ws, cudaStream_t s, int32_t n, const uint8_t *B0,
                          const uint8_t *A1, int32_t nterms, const uint8_t *const *Bq, const double *const *Rq,
                          double eps_user, dl_path path, dl_mem mem, uint64_t *out_bits, double *out_rtilde,
                          dl_stats *st);
dl_status solve_tail_system(dl_ctx *ctx, Workspace &ws, cudaStream_t s, int32_t n, int32_t m, const dl_tail_eq *eqs,
                            dl_mem mem, dl_path path, uint64_t *const *out_bits, double *const *out_rtilde,
                            dl_stats *st);
// The transposed class (program prog:2): E = R1; bits of the model, R~ into a.out_rtilde.
dl_status solve_transposed(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a, dl_stats *st);
// The real S~ of same generation into a.out_rtilde (n x n doubles); bits optional.
dl_status solve_sg_real(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a, dl_stats *st);
dl_status solve_compose(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a,
                        dl_stats *st);
dl_status solve_tc_batch(dl_ctx *ctx, Workspace &ws, cudaStream_t s, int32_t count,
                         const int32_t *ns, const uint8_t *const *Es, dl_mem mem,
                         uint64_t *const *out_bits, dl_stats *st);
// Mixed-precision solve (dl_mixed.cu): leaves X in the "mx_X64" buffer (np x np doubles).
// dmax = ||E||_inf (bounds the terms of the residual's sums).
dl_status tc_mixed(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a, dl_stats *st,
                   const uint8_t *E, double eps, unsigned long long dmax, int *launches_io);
// The program front-end (dl_program.cu).
dl_status program_create(dl_ctx *ctx, const char *text, dl_program **out);
void program_destroy(dl_program *p);
dl_status program_set(dl_program *p, cudaStream_t s, const char *pred, int32_t n, const uint8_t *R, dl_mem mem);
dl_status program_run(dl_ctx *ctx, Workspace &ws, cudaStream_t s, dl_program *p, dl_stats *st);
dl_status program_get(dl_program *p, Workspace &ws, cudaStream_t s, const char *pred, uint64_t *out_bits,
                      dl_mem mem);
std::string program_describe(const dl_program *p);
dl_ctx *program_ctx(const dl_program *p);
// The autotuner (dl_tune.cu).
int tune_bucket(int64_t np);
TuneEntry tuned(dl_ctx *ctx, int64_t np);  // the bucket's entry, or the defaults
void tune_init(dl_ctx *ctx);                 // key prefix, flags, cache read (dl_create)
dl_status autotune_bucket(dl_ctx *ctx, Workspace &ws, cudaStream_t s, int32_t n, bool force, TuneEntry *out,
                          std::string *source);
std::string tune_report(const dl_ctx *ctx, const TuneEntry &e, const std::string &source);
// Device bytes a request of this kind and size needs (serving admission).
size_t footprint_bytes(int kind, int32_t n);

}  // namespace dl

// Stop the serving threads of a context (no-op if serving never started).
void dl_serve_shutdown(dl_ctx *ctx);
