// dl_batch.cu -- many independent closure problems of uneven size in one call (dl_tc_batch).
//
// Every instance k runs the FP8 closure of dl_solve.cu (C_0 = I + E_k, C_{t+1} = min1(C_t^2),
// certificate C = min1(I + E C), model E C*), but all instances advance together in rounds:
//   round r:  one persistent grouped tcgen05 launch squares every still-active instance
//             (finished instances are gated off inside the kernel), a decide kernel marks
//             instances whose squaring added nothing, one batched sweep checks the
//             certificate of the others (and emits the model), a second decide kernel
//             retires instances whose certificate held.
// All decisions live on the device, so the rounds need no host round trip: the whole
// schedule (ingest + R rounds + copy-out) is captured once into a CUDA graph and launched
// as one unit; a repeated call on the same buffers relaunches the cached graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "dl_ctx.h"
#include "dl_internal.h"
#include "dl_ptx.cuh"
#include "dl_rows.cuh"

namespace dl {

namespace {

enum : int { B_ACTIVE = 0, B_EMIT = 1, B_DONE = 2 };

struct BatchInst {
    const uint8_t *E;  // n x n input on the device
    uint8_t *c0, *c1;  // ping-pong e4m3 operands, np x np
    uint64_t *rbits;   // bits of the latest C_t, np x wp
    uint64_t *mbits;   // model bits, np x wp
    uint64_t *out;     // user output (device memory) or null
    int32_t n, np;
    int64_t wp;
    int64_t prow0;  // first padded row of this instance in the global padded-row order
    int64_t row0;   // first real row in the global real-row order
};

// Per-instance device counters, laid out as arrays of `count` entries.
struct BatchCounters {
    int *state;
    unsigned long long *cnt_new, *cnt_old, *viol, *ones, *squarings;
};

__device__ __forceinline__ int find_by_prow(const BatchInst *inst, int count, int64_t g) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (inst[mid].prow0 <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_by_row(const BatchInst *inst, int count, int64_t g) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (inst[mid].row0 <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256)
    ingest_batch_kernel(const BatchInst *__restrict__ inst, int count, BatchCounters c, int *status) {
    const int64_t g = blockIdx.x;
    const int k = find_by_prow(inst, count, g);
    const BatchInst I = inst[k];
    const int r = static_cast<int>(g - I.prow0);
    uint32_t sum = 0, bad = 0, extra = 0;
    ingest_row(I.E, I.n, I.np, I.c0, 1, r, sum, bad, extra);
    block_reduce_sum_or(sum, bad);
    if (threadIdx.x == 0) {
        if (bad) atomicOr(status, ST_BAD_INPUT);
        if (sum + extra) atomicAdd(&c.cnt_old[k], static_cast<unsigned long long>(sum + extra));
    }
}

__global__ void __launch_bounds__(256)
    sweep_batch_kernel(const BatchInst *__restrict__ inst, int count, int64_t total_rows, BatchCounters c) {
    const int lane = threadIdx.x & 31;
    const int64_t g = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (g >= total_rows) return;
    const int k = find_by_row(inst, count, g);
    const int st = c.state[k];
    if (st == B_DONE) return;
    if (st == B_ACTIVE && warp_read_u64(&c.viol[k]) != 0ull) return;  // certificate already failed
    const BatchInst I = inst[k];
    const int r = static_cast<int>(g - I.row0);
    bool viol = false;
    uint32_t cnt = 0;
    sweep_row(I.E + static_cast<int64_t>(r) * I.n, I.n, I.rbits, I.mbits, I.wp, 0, r, lane, viol, cnt);
    if (lane == 0) {
        if (viol) atomicAdd(&c.viol[k], 1ull);
        if (cnt) atomicAdd(&c.ones[k], static_cast<unsigned long long>(cnt));
    }
}

// After a squaring: an active instance whose count of ones did not grow has reached its
// reflexive closure (it only needs the model emitted); the others record their new count.
__global__ void decide_after_square(int count, BatchCounters c) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count || c.state[k] != B_ACTIVE) return;
    c.squarings[k] += 1;
    if (c.cnt_new[k] == c.cnt_old[k]) c.state[k] = B_EMIT;
    else c.cnt_old[k] = c.cnt_new[k];
    c.cnt_new[k] = 0;
}

// After the sweep: a certificate that held, or an emission, retires the instance.
__global__ void decide_after_sweep(int count, BatchCounters c, int *status) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int st = c.state[k];
    if (st == B_ACTIVE) {
        if (c.viol[k] == 0) c.state[k] = B_DONE;
        else c.ones[k] = 0;
    } else if (st == B_EMIT) {
        c.state[k] = B_DONE;
        if (c.viol[k] != 0) atomicOr(status, ST_TIMEOUT_DEP);  // converged closure failed its check
    }
    c.viol[k] = 0;
}

// Copy each model (n rows of ceil(n/64) words) to its device output.
__global__ void copy_out_kernel(const BatchInst *__restrict__ inst, int count, int64_t total_rows) {
    const int lane = threadIdx.x & 31;
    const int64_t g = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (g >= total_rows) return;
    const int k = find_by_row(inst, count, g);
    const BatchInst I = inst[k];
    if (!I.out) return;
    const int r = static_cast<int>(g - I.row0);
    const int64_t w = (I.n + 63) / 64;
    for (int64_t q = lane; q < w; q += 32) I.out[r * w + q] = I.mbits[r * I.wp + q];
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

#define BCK(x)                                                                                  \
    do {                                                                                        \
        cudaError_t e_ = (x);                                                                   \
        if (e_ != cudaSuccess) {                                                                \
            set_error("batch: %s failed: %s (%s:%d)", #x, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return DL_EDEVICE;                                                                  \
        }                                                                                       \
    } while (0)

}  // namespace

// Cached schedule of the last batch (graph + the buffers it was built on).
struct BatchPlan {
    std::vector<int32_t> ns;
    std::vector<const void *> ins;
    std::vector<void *> outs;
    int mem = -1;
    int bn = 0;
    cudaGraphExec_t exec = nullptr;
    int rounds = 0;
    ~BatchPlan() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

dl_status solve_tc_batch(dl_ctx *ctx, Workspace &ws, cudaStream_t s, int32_t count, const int32_t *ns,
                         const uint8_t *const *Es, dl_mem mem, uint64_t *const *out_bits, dl_stats *st) {
    // instances with n > 0 take part; empty ones have nothing to write
    std::vector<int> live;
    for (int32_t k = 0; k < count; ++k)
        if (ns[k] > 0) live.push_back(k);
    if (live.empty()) return DL_OK;
    const int L = static_cast<int>(live.size());
    const int bn = 128;  // tile width for the batch (small instances waste less padding)
    std::vector<BatchInst> inst(L);
    int64_t in_bytes = 0, mat_bytes = 0, bit_words = 0, prow = 0, row = 0;
    int64_t max_np = 0;
    for (int i = 0; i < L; ++i) {
        const int32_t n = ns[live[i]];
        const int64_t np = round_up(n, 128);
        inst[i].n = n;
        inst[i].np = static_cast<int32_t>(np);
        inst[i].wp = np / 64;
        inst[i].prow0 = prow;
        inst[i].row0 = row;
        prow += np;
        row += n;
        in_bytes += round_up(static_cast<int64_t>(n) * n, 256);
        mat_bytes += np * np;
        bit_words += np * (np / 64);
        max_np = std::max(max_np, np);
    }
    const int64_t total_prows = prow, total_rows = row;
    auto *c0 = static_cast<uint8_t *>(ws.get("batch_c0", mat_bytes));
    auto *c1 = static_cast<uint8_t *>(ws.get("batch_c1", mat_bytes));
    auto *rb = static_cast<uint64_t *>(ws.get("batch_rbits", bit_words * 8));
    auto *mb = static_cast<uint64_t *>(ws.get("batch_mbits", bit_words * 8));
    auto *ctr = static_cast<unsigned long long *>(ws.get("batch_ctr", 5 * sizeof(unsigned long long) * L + 256));
    auto *state = static_cast<int *>(ws.get("batch_state", sizeof(int) * L + 256));
    auto *dinst = static_cast<BatchInst *>(ws.get("batch_inst", sizeof(BatchInst) * L));
    auto *dprob = static_cast<GemmProblem *>(ws.get("batch_probs", sizeof(GemmProblem) * 2 * L));
    uint8_t *staging = nullptr;
    if (mem == DL_MEM_HOST) staging = static_cast<uint8_t *>(ws.get("batch_in", std::max<int64_t>(in_bytes, 256)));
    if (!c0 || !c1 || !rb || !mb || !ctr || !state || !dinst || !dprob || (mem == DL_MEM_HOST && !staging)) {
        set_error("batch: device allocation failed (%.2f GB of operands)", 2.0 * mat_bytes / 1e9);
        return DL_ENOMEM;
    }
    BatchCounters bc{state, ctr, ctr + L, ctr + 2 * L, ctr + 3 * L, ctr + 4 * L};

    cudaEvent_t ev0 = ws.ev[0], ev1 = ws.ev[1];
    BCK(cudaEventRecord(ev0, s));
    // inputs on the device
    int64_t mo = 0, bo = 0, io = 0;
    for (int i = 0; i < L; ++i) {
        const int k = live[i];
        const int64_t np = inst[i].np, n = inst[i].n;
        if (mem == DL_MEM_HOST) {
            BCK(cudaMemcpyAsync(staging + io, Es[k], n * n, cudaMemcpyHostToDevice, s));
            inst[i].E = staging + io;
            io += round_up(n * n, 256);
        } else {
            inst[i].E = Es[k];
        }
        inst[i].c0 = c0 + mo;
        inst[i].c1 = c1 + mo;
        inst[i].rbits = rb + bo;
        inst[i].mbits = mb + bo;
        inst[i].out = mem == DL_MEM_DEVICE ? out_bits[k] : nullptr;
        mo += np * np;
        bo += np * (np / 64);
    }

    // reuse the captured schedule when the call repeats on the same buffers
    std::vector<int32_t> key_ns(L);
    std::vector<const void *> key_in(L);
    std::vector<void *> key_out(L);
    for (int i = 0; i < L; ++i) {
        key_ns[i] = inst[i].n;
        key_in[i] = inst[i].E;
        key_out[i] = out_bits[live[i]];
    }
    BatchPlan *&plan = ws.batch_plan;
    const bool reuse = plan && plan->mem == static_cast<int>(mem) && plan->bn == bn && plan->ns == key_ns &&
                       plan->ins == key_in && plan->outs == key_out;
    if (!reuse) {
        delete plan;
        plan = nullptr;
        BCK(cudaMemcpyAsync(dinst, inst.data(), sizeof(BatchInst) * L, cudaMemcpyHostToDevice, s));
        std::vector<GemmProblem> probs(2 * L);
        std::string err;
        int tiles = 0;
        for (int p = 0; p < 2; ++p) {
            int start = 0;
            for (int i = 0; i < L; ++i) {
                const int64_t np = inst[i].np;
                GemmEpilogue e{};
                e.out8 = p == 0 ? inst[i].c1 : inst[i].c0;
                e.ld_out8 = np;
                e.bits = reinterpret_cast<uint32_t *>(inst[i].rbits);
                e.ld_bits32 = 2 * inst[i].wp;
                e.count = bc.cnt_new + i;
                const Operand op{p == 0 ? inst[i].c0 : inst[i].c1, np, np, np, 0, 0};
                GemmProblem &pr = probs[p * L + i];
                if (!gemm_make_problem(&pr, KIND_F8, false, bn, static_cast<int>(np), static_cast<int>(np),
                                       static_cast<int>(np), op, op, e, &err)) {
                    set_error("batch: %s", err.c_str());
                    return DL_EDEVICE;
                }
                pr.gate = state + i;
                pr.tile_start = start;
                start += pr.tiles_m * pr.tiles_n;
            }
            tiles = start;
        }
        // pageable source: the copy has read `probs` when cudaMemcpyAsync returns
        BCK(cudaMemcpyAsync(dprob, probs.data(), sizeof(GemmProblem) * 2 * L, cudaMemcpyHostToDevice, s));
        BCK(gemm_prepare(KIND_F8, false, bn, EPI_BOOL));
        const int rounds = 2 + static_cast<int>(std::ceil(std::log2(static_cast<double>(max_np) + 1.0)));
        const int grid = std::min(tiles, ctx->sms);
        const int dgrid = (L + 255) / 256;
        const unsigned sweep_blocks = static_cast<unsigned>((total_rows + 7) / 8);
        // capture the schedule
        cudaGraph_t graph = nullptr;
        BCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        bool cap_ok = true;
        auto cap = [&](cudaError_t e) { cap_ok = cap_ok && e == cudaSuccess; };
        cap(cudaMemsetAsync(state, 0, sizeof(int) * L, s));
        cap(cudaMemsetAsync(ctr, 0, 5 * sizeof(unsigned long long) * L, s));
        ingest_batch_kernel<<<static_cast<unsigned>(total_prows), 256, 0, s>>>(dinst, L, bc, ws.status);
        cap(cudaGetLastError());
        for (int r = 0; r < rounds; ++r) {
            cap(gemm_launch(KIND_F8, false, bn, EPI_BOOL, dprob + (r & 1) * L, L, tiles, grid, ws.status,
                            ctx->budget_ns, s));
            decide_after_square<<<dgrid, 256, 0, s>>>(L, bc);
            cap(cudaGetLastError());
            sweep_batch_kernel<<<sweep_blocks, 256, 0, s>>>(dinst, L, total_rows, bc);
            cap(cudaGetLastError());
            decide_after_sweep<<<dgrid, 256, 0, s>>>(L, bc, ws.status);
            cap(cudaGetLastError());
        }
        if (mem == DL_MEM_DEVICE) {
            copy_out_kernel<<<sweep_blocks, 256, 0, s>>>(dinst, L, total_rows);
            cap(cudaGetLastError());
        }
        const cudaError_t ec = cudaStreamEndCapture(s, &graph);
        if (!cap_ok || ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            set_error("batch: stream capture failed (%s)", cudaGetErrorString(ec));
            return DL_EDEVICE;
        }
        plan = new BatchPlan();
        plan->ns = key_ns;
        plan->ins = key_in;
        plan->outs = key_out;
        plan->mem = static_cast<int>(mem);
        plan->bn = bn;
        plan->rounds = rounds;
        const cudaError_t ei = cudaGraphInstantiate(&plan->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            delete plan;
            plan = nullptr;
            set_error("batch: graph instantiation failed (%s)", cudaGetErrorString(ei));
            return DL_EDEVICE;
        }
    }
    BCK(cudaMemsetAsync(ws.status, 0, sizeof(int), s));
    BCK(cudaGraphLaunch(plan->exec, s));
    if (mem == DL_MEM_HOST) {
        for (int i = 0; i < L; ++i) {
            const int64_t n = inst[i].n, w = (n + 63) / 64;
            BCK(cudaMemcpy2DAsync(out_bits[live[i]], w * 8, inst[i].mbits, inst[i].wp * 8, w * 8, n,
                                  cudaMemcpyDeviceToHost, s));
        }
    }
    BCK(cudaEventRecord(ev1, s));
    std::vector<int> hstate(L);
    std::vector<unsigned long long> hctr(5 * static_cast<size_t>(L));
    BCK(cudaMemcpyAsync(hstate.data(), state, sizeof(int) * L, cudaMemcpyDeviceToHost, s));
    BCK(cudaMemcpyAsync(hctr.data(), ctr, sizeof(unsigned long long) * 5 * L, cudaMemcpyDeviceToHost, s));
    int hst = 0;
    BCK(cudaMemcpyAsync(&hst, ws.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    if (hst & ST_BAD_INPUT) {
        set_error("batch: an input matrix holds a byte that is neither 0 nor 1");
        return DL_EINVAL;
    }
    if (hst) {
        set_error("batch: device status 0x%x (a wait expired or a certificate failed)", hst);
        return DL_ETIMEOUT;
    }
    int max_sq = 0;
    int64_t ones = 0;
    double flops = 0.0;
    for (int i = 0; i < L; ++i) {
        if (hstate[i] != B_DONE) {
            set_error("batch: instance %d did not converge in %d rounds", live[i], plan->rounds);
            return DL_ENOTCONV;
        }
        const int sq = static_cast<int>(hctr[4 * L + i]);
        max_sq = std::max(max_sq, sq);
        ones += static_cast<int64_t>(hctr[3 * L + i]);
        const double np = inst[i].np;
        flops += 2.0 * np * np * np * sq;
    }
    if (st) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        double equiv = 0.0;
        for (int i = 0; i < L; ++i) {
            const double n = inst[i].n;
            equiv += (8.0 / 3.0) * n * n * n;
        }
        st->path_used = DL_PATH_BOOL_FP8;
        st->iters = max_sq;
        st->model_ones = ones;
        st->ms_total = ms;
        st->ms_solve = ms;
        st->tflops_equiv = ms > 0 ? equiv / (ms * 1e-3) / 1e12 : 0.0;
        st->gemm_launches = plan->rounds;
        st->gemm_flops = flops;
        st->gpu_launches = 1 + plan->rounds * 4 + (mem == DL_MEM_DEVICE ? 1 : 0);
    }
    return DL_OK;
}

void batch_plan_release(BatchPlan *p) { delete p; }

}  // namespace dl
