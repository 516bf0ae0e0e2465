// dl_bool.cu -- streaming kernels of the boolean path: ingest of the 0/1 base relation and
// the certificate / exact recheck sweep on packed bit matrices.
//
// Ingest (row sums give ||E||_inf, Sec. 2; eps = 1/(1 + ||E||_inf), Sec. 4) writes the FP8
// e4m3 operand of the tensor-core products: 1.0 (0x38) for a 1 and 0 elsewhere, padded with
// zero rows and columns to the GEMM tile size.  Padded constants have no facts, so they
// change nothing in the model of the real constants.
//
// The sweep checks a candidate closure M against the completed equation of the program,
// R2 = min1(E + E R2) (eq. matrixeq:trcl), row by row on bits:  row i of E R2 is the OR of
// the rows k of M with E[i][k] = 1.  A candidate that satisfies the equation and lies below
// the least model is the least model; a missing fact always shows up as a violated row
// (the fact with the shortest derivation that is missing has its successor's fact present).
#include <cuda_runtime.h>

#include <cstdint>

#include "dl_internal.h"
#include "dl_ptx.cuh"

namespace dl {

namespace {

constexpr int kIngestThreads = 256;

__global__ void __launch_bounds__(kIngestThreads)
    ingest_kernel(const uint8_t *__restrict__ src, int n, int np, uint8_t *__restrict__ dst,
                  int add_identity, unsigned long long *dmax, unsigned long long *nnz,
                  unsigned long long *count, int *status) {
    const int row = blockIdx.x;
    uint8_t *drow = dst + static_cast<int64_t>(row) * np;
    uint32_t sum = 0, bad = 0;
    if (row < n) {
        const uint8_t *srow = src + static_cast<int64_t>(row) * n;
        const bool vec = ((n & 15) == 0) && ((reinterpret_cast<uintptr_t>(src) & 15) == 0);
        if (vec) {
            const uint4 *s4 = reinterpret_cast<const uint4 *>(srow);
            uint4 *d4 = reinterpret_cast<uint4 *>(drow);
            for (int q = threadIdx.x; q < n / 16; q += blockDim.x) {
                const uint4 x = s4[q];
                const uint32_t w[4] = {x.x, x.y, x.z, x.w};
                uint32_t o[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    bad |= w[t] & 0xFEFEFEFEu;
                    sum += __popc(w[t] & 0x01010101u);
                    o[t] = (w[t] & 0x01010101u) * 0x38u;  // byte 1 -> 0x38 (e4m3 1.0)
                }
                d4[q] = make_uint4(o[0], o[1], o[2], o[3]);
            }
        } else {
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                const uint32_t b = srow[j];
                bad |= b & 0xFEu;
                sum += b & 1u;
                drow[j] = static_cast<uint8_t>((b & 1u) * 0x38u);
            }
        }
    }
    const int start = row < n ? n : 0;
    for (int j = start + threadIdx.x; j < np; j += blockDim.x) drow[j] = 0;
    __syncthreads();
    uint32_t extra = 0;
    if (add_identity && threadIdx.x == 0) {
        if (row >= n || drow[row] == 0) extra = 1;
        drow[row] = 0x38;
    }
    // block reduction of sum / bad
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    __shared__ uint32_t s_sum[kIngestThreads / 32], s_bad[kIngestThreads / 32];
    if ((threadIdx.x & 31) == 0) {
        s_sum[threadIdx.x >> 5] = sum;
        s_bad[threadIdx.x >> 5] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t ts = 0, tb = 0;
        for (int w = 0; w < kIngestThreads / 32; ++w) {
            ts += s_sum[w];
            tb |= s_bad[w];
        }
        if (tb) atomicOr(status, ST_BAD_INPUT);
        if (ts) {
            atomicMax(dmax, static_cast<unsigned long long>(ts));
            atomicAdd(nnz, static_cast<unsigned long long>(ts));
        }
        if (ts + extra) atomicAdd(count, static_cast<unsigned long long>(ts + extra));
    }
}

// One warp per row.  Lanes own words lane, lane+32, ... of the row (up to kWpl per lane per
// pass; wider rows take several passes over the E row).
constexpr int kWpl = 8;

__global__ void __launch_bounds__(256)
    sweep_kernel(const uint8_t *__restrict__ E, int64_t lde, int n, const uint64_t *M,
                 uint64_t *out, int64_t wp, int mode, int stop_early,
                 unsigned long long *violations, unsigned long long *ones) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= n) return;
    if (stop_early) {  // warp-uniform test: lane 0 reads, everyone follows
        unsigned long long seen =
            lane == 0 ? *reinterpret_cast<volatile unsigned long long *>(violations) : 0ull;
        seen = __shfl_sync(0xffffffffu, seen, 0);
        if (seen != 0ull) return;
    }
    const uint8_t *erow = E + static_cast<int64_t>(row) * lde;
    const uint64_t *mrow = M + static_cast<int64_t>(row) * wp;
    bool viol = false;
    uint32_t cnt = 0;
    // A row whose accumulator already holds all n columns cannot change any more: stop its
    // scan (single-pass rows only).  Most rows of a closure with a giant component are full.
    const bool single_pass = wp <= 32 * kWpl;
    uint64_t full[kWpl];
#pragma unroll
    for (int q = 0; q < kWpl; ++q) {
        const int64_t w = lane + 32 * q;
        const int64_t lo = w * 64;
        full[q] = (w >= wp || lo >= n) ? 0ull : (n - lo >= 64 ? ~0ull : ((1ull << (n - lo)) - 1ull));
    }
    for (int64_t w0 = 0; w0 < wp; w0 += 32 * kWpl) {
        uint64_t acc[kWpl];
#pragma unroll
        for (int t = 0; t < kWpl; ++t) acc[t] = 0;
        bool saturated = false;
        if (single_pass && mode == 1) {  // the row itself may already be full
            bool mine = true;
#pragma unroll
            for (int q = 0; q < kWpl; ++q) {
                const int64_t w = lane + 32 * q;
                if (w < wp) acc[q] = mrow[w];
                mine &= acc[q] == full[q];
            }
            saturated = __all_sync(0xffffffffu, mine);
        }
        for (int c0 = 0; c0 < n && !saturated; c0 += 512) {
            // lane looks at bytes c0 + 16*lane .. +15
            uint32_t mask = 0;
            const int base = c0 + 16 * lane;
#pragma unroll
            for (int t = 0; t < 16; ++t)
                if (base + t < n && erow[base + t]) mask |= 1u << t;
            uint32_t who = __ballot_sync(0xffffffffu, mask != 0);
            while (who) {
                const int src = __ffs(who) - 1;
                who &= who - 1;
                uint32_t m = __shfl_sync(0xffffffffu, mask, src);
                while (m) {
                    const int t = __ffs(m) - 1;
                    m &= m - 1;
                    const int k = c0 + 16 * src + t;
                    const uint64_t *mk = M + static_cast<int64_t>(k) * wp;
#pragma unroll
                    for (int q = 0; q < kWpl; ++q) {
                        const int64_t w = w0 + lane + 32 * q;
                        if (w < wp) acc[q] |= mk[w];
                    }
                    if (mode == 1) {  // the fact E[i][k] itself
                        const int64_t rel = (k >> 6) - w0;  // word index within this pass
                        if (rel >= 0 && rel < 32 * kWpl && (rel & 31) == lane) {
                            const int qk = static_cast<int>(rel >> 5);
#pragma unroll
                            for (int q = 0; q < kWpl; ++q)
                                if (q == qk) acc[q] |= 1ull << (k & 63);
                        }
                    }
                    if (single_pass) {
                        bool mine = true;
#pragma unroll
                        for (int q = 0; q < kWpl; ++q) mine &= acc[q] == full[q];
                        if (__all_sync(0xffffffffu, mine)) {
                            saturated = true;
                            m = 0;
                            who = 0;
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kWpl; ++q) {
            const int64_t w = w0 + lane + 32 * q;
            if (w >= wp) continue;
            const uint64_t old = mrow[w];
            uint64_t v = acc[q];
            if (mode == 0) {
                const uint64_t self = (w == (row >> 6)) ? (1ull << (row & 63)) : 0ull;
                if ((v | self) != old) viol = true;
                out[static_cast<int64_t>(row) * wp + w] = v;
            } else {
                v |= old;
                if (v != old) {
                    viol = true;
                    out[static_cast<int64_t>(row) * wp + w] = v;
                } else if (out != M) {
                    out[static_cast<int64_t>(row) * wp + w] = v;
                }
            }
            cnt += __popcll(v);
        }
    }
    const bool any = __any_sync(0xffffffffu, viol);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) {
        if (any) atomicAdd(violations, 1ull);
        if (ones && cnt) atomicAdd(ones, static_cast<unsigned long long>(cnt));
    }
}

}  // namespace

cudaError_t ingest_u8_to_e4m3(const uint8_t *src, int n, int np, uint8_t *dst, int add_identity,
                              unsigned long long *dmax, unsigned long long *nnz,
                              unsigned long long *count, int *status, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    ingest_kernel<<<np, kIngestThreads, 0, s>>>(src, n, np, dst, add_identity, dmax, nnz, count,
                                                 status);
    return cudaGetLastError();
}

cudaError_t bits_sweep(const uint8_t *E, int64_t lde, int n, const uint64_t *M, uint64_t *out,
                       int64_t wp, int mode, int stop_early, unsigned long long *violations,
                       unsigned long long *ones, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int rows_per_block = 8;
    sweep_kernel<<<(n + rows_per_block - 1) / rows_per_block, 32 * rows_per_block, 0, s>>>(
        E, lde, n, M, out, wp, mode, stop_early, violations, ones);
    return cudaGetLastError();
}

}  // namespace dl
