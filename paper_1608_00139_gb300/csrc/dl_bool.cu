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
#include "dl_rows.cuh"

namespace dl {

namespace {

constexpr int kIngestThreads = 256;

__global__ void __launch_bounds__(kIngestThreads)
    ingest_kernel(const uint8_t *__restrict__ src, int n, int np, uint8_t *__restrict__ dst,
                  int add_identity, unsigned long long *dmax, unsigned long long *nnz,
                  unsigned long long *count, int *status) {
    uint32_t sum = 0, bad = 0, extra = 0;
    ingest_row(src, n, np, dst, add_identity, static_cast<int>(blockIdx.x), sum, bad, extra);
    block_reduce_sum_or(sum, bad);
    if (threadIdx.x == 0) {
        if (bad) atomicOr(status, ST_BAD_INPUT);
        if (sum) {
            atomicMax(dmax, static_cast<unsigned long long>(sum));
            atomicAdd(nnz, static_cast<unsigned long long>(sum));
        }
        if (sum + extra) atomicAdd(count, static_cast<unsigned long long>(sum + extra));
    }
}

__global__ void __launch_bounds__(256)
    sweep_kernel(const uint8_t *__restrict__ E, int64_t lde, int n, const uint64_t *M,
                 uint64_t *out, int64_t wp, int mode, int stop_early,
                 unsigned long long *violations, unsigned long long *ones) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= n) return;
    if (stop_early && warp_read_u64(violations) != 0ull) return;
    bool viol = false;
    uint32_t cnt = 0;
    sweep_row(E + static_cast<int64_t>(row) * lde, n, M, out, wp, mode, row, lane, viol, cnt);
    if (lane == 0) {
        if (viol) atomicAdd(violations, 1ull);
        if (ones && cnt) atomicAdd(ones, static_cast<unsigned long long>(cnt));
    }
}

// ---- edge-parallel sweeps on the CSR of E -------------------------------------------------
// Work unit = (row i, up to kUnit consecutive successors of i); unit_off[i] = first unit of row i.
// The OR over a row's successors is split across units and combined with 64-bit atomicOr,
// so rows with thousands of successors (heavy-tailed degrees) do not serialise a sweep.
constexpr int kUnit = 64;

__global__ void unit_count_kernel(const int *__restrict__ ptr, int n, int *cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cnt[i] = (ptr[i + 1] - ptr[i] + kUnit - 1) / kUnit;
}

__device__ __forceinline__ int unit_row(const int *unit_off, int n, int u) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (unit_off[mid] <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// OR of the successors' rows of one unit into dst row i (atomically).  with_self: also set
// the successors' own bits (the facts E[i][k]).  skip_full: skip the unit if dst row i is
// already full (nothing can change).  Returns (warp-uniform) whether any word of dst changed.
__device__ __forceinline__ bool or_unit(const int *__restrict__ col, int q0, int q1, int n, int i,
                                        const uint64_t *M, uint64_t *dst, int64_t wp, bool with_self,
                                        bool skip_full, int lane) {
    const bool single = wp <= 32 * kSweepWpl;
    uint64_t *drow = dst + static_cast<int64_t>(i) * wp;
    bool changed = false;
    for (int64_t w0 = 0; w0 < wp; w0 += 32 * kSweepWpl) {
        uint64_t acc[kSweepWpl], full[kSweepWpl], have[kSweepWpl];
        bool mine_full = true;
#pragma unroll
        for (int q = 0; q < kSweepWpl; ++q) {
            acc[q] = 0;
            const int64_t w = w0 + lane + 32 * q;
            const int64_t lo = w * 64;
            full[q] = (w >= wp || lo >= n) ? 0ull : (n - lo >= 64 ? ~0ull : ((1ull << (n - lo)) - 1ull));
            have[q] = (skip_full && single && w < wp) ? drow[w] : 0ull;  // snapshot of dst row i
            mine_full &= have[q] == full[q];
        }
        if (skip_full && single && __all_sync(0xffffffffu, mine_full)) return false;
        for (int qq = q0; qq < q1; ++qq) {
            const int k = col[qq];
            const uint64_t *mk = M + static_cast<int64_t>(k) * wp;
#pragma unroll
            for (int q = 0; q < kSweepWpl; ++q) {
                const int64_t w = w0 + lane + 32 * q;
                if (w < wp) acc[q] |= mk[w];
            }
            if (with_self) {
                const int64_t rel = (k >> 6) - w0;
                if (rel >= 0 && rel < 32 * kSweepWpl && (rel & 31) == lane) {
                    const int qk = static_cast<int>(rel >> 5);
#pragma unroll
                    for (int q = 0; q < kSweepWpl; ++q)
                        if (q == qk) acc[q] |= 1ull << (k & 63);
                }
            }
            if (skip_full && single) {  // the row is covered: later successors add nothing
                bool mine = true;
#pragma unroll
                for (int q = 0; q < kSweepWpl; ++q) mine &= (have[q] | acc[q]) == full[q];
                if (__all_sync(0xffffffffu, mine)) break;
            }
        }
#pragma unroll
        for (int q = 0; q < kSweepWpl; ++q) {
            const int64_t w = w0 + lane + 32 * q;
            if (w >= wp || acc[q] == 0ull) continue;
            if ((drow[w] | acc[q]) == drow[w]) continue;  // nothing new for this word
            const unsigned long long old =
                atomicOr(reinterpret_cast<unsigned long long *>(drow + w), static_cast<unsigned long long>(acc[q]));
            if ((old | acc[q]) != old) changed = true;
        }
    }
    return __any_sync(0xffffffffu, changed);
}

// Row-direct variants (used when every row has at most kRowDirect successors): one warp per
// row, lanes own WPL words each (the whole row in one pass, wp <= 32 * WPL), successor rows
// loaded two at a time, stop as soon as the row is full, plain stores (the warp is the row's
// only writer).
constexpr int kRowDirect = 256;

// The most a row can hold: the columns with an incoming edge (colmask), plus bit self if
// self >= 0; all n columns without a mask.
template <int WPL>
__device__ __forceinline__ void full_mask(int n, int64_t wp, int lane, const uint64_t *colmask, int self,
                                          uint64_t (&full)[WPL]) {
#pragma unroll
    for (int q = 0; q < WPL; ++q) {
        const int64_t w = lane + 32 * q;
        const int64_t lo = w * 64;
        if (w >= wp || lo >= n) {
            full[q] = 0ull;
        } else if (colmask != nullptr) {
            full[q] = colmask[w] | ((self >= 0 && w == (self >> 6)) ? 1ull << (self & 63) : 0ull);
        } else {
            full[q] = n - lo >= 64 ? ~0ull : ((1ull << (n - lo)) - 1ull);
        }
        asm volatile("" : "+l"(full[q]));  // keep the bound in a register (no reloads in the loops)
    }
}

// acc |= rows k (and, if with_self, bit k) for the successors [q0, q1), stopping when full.
template <int WPL>
__device__ __forceinline__ void or_successors(const int *__restrict__ col, int q0, int q1, const uint64_t *M,
                                              int64_t wp, int lane, bool with_self, const uint64_t (&full)[WPL],
                                              uint64_t (&acc)[WPL]) {
    int qq = q0;
    for (; qq + 1 < q1; qq += 2) {
        const int k1 = col[qq], k2 = col[qq + 1];
        const uint64_t *m1 = M + static_cast<int64_t>(k1) * wp;
        const uint64_t *m2 = M + static_cast<int64_t>(k2) * wp;
        uint64_t a[WPL], b[WPL];
#pragma unroll
        for (int q = 0; q < WPL; ++q) {
            const int64_t w = lane + 32 * q;
            a[q] = w < wp ? m1[w] : 0ull;
            b[q] = w < wp ? m2[w] : 0ull;
        }
        bool mine = true;
#pragma unroll
        for (int q = 0; q < WPL; ++q) {
            const int64_t w = lane + 32 * q;
            acc[q] |= a[q] | b[q];
            if (with_self) {
                if (w == (k1 >> 6)) acc[q] |= 1ull << (k1 & 63);
                if (w == (k2 >> 6)) acc[q] |= 1ull << (k2 & 63);
            }
            mine &= acc[q] == full[q];
        }
        if (__all_sync(0xffffffffu, mine)) return;
    }
    if (qq < q1) {
        const int k = col[qq];
        const uint64_t *m = M + static_cast<int64_t>(k) * wp;
#pragma unroll
        for (int q = 0; q < WPL; ++q) {
            const int64_t w = lane + 32 * q;
            if (w < wp) acc[q] |= m[w];
            if (with_self && w == (k >> 6)) acc[q] |= 1ull << (k & 63);
        }
    }
}

// mode 1 (in place): M_i |= E_i | OR_{k in succ(i)} M_k; counts changed rows.  A sweep that
// follows one which changed nothing has nothing to do: with skip_if_zero pointing at the
// previous sweep's counter, the grid leaves at once.
template <int WPL>
__global__ void __launch_bounds__(256)
    sweep_rows_step_kernel(const int *__restrict__ ptr, const int *__restrict__ col, int n, uint64_t *M, int64_t wp,
                           unsigned long long *changed_rows, const unsigned long long *skip_if_zero,
                           const uint64_t *__restrict__ colmask, const int *gate) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    if (skip_if_zero != nullptr && *skip_if_zero == 0) return;  // the previous sweep changed nothing
    if (gate != nullptr && *gate != 0) return;
    const int q0 = ptr[i], q1 = ptr[i + 1];
    if (q0 == q1) return;
    uint64_t *mrow = M + static_cast<int64_t>(i) * wp;
    uint64_t full[WPL], acc[WPL];
    full_mask<WPL>(n, wp, lane, colmask, i, full);
    bool mine = true;
#pragma unroll
    for (int q = 0; q < WPL; ++q) {
        const int64_t w = lane + 32 * q;
        acc[q] = w < wp ? mrow[w] : 0ull;
        mine &= acc[q] == full[q];
    }
    if (__all_sync(0xffffffffu, mine)) return;  // already full
    uint64_t before[WPL];
#pragma unroll
    for (int q = 0; q < WPL; ++q) before[q] = acc[q];
    or_successors<WPL>(col, q0, q1, M, wp, lane, true, full, acc);
    bool changed = false;
#pragma unroll
    for (int q = 0; q < WPL; ++q) {
        const int64_t w = lane + 32 * q;
        if (w < wp && acc[q] != before[q]) {
            mrow[w] = acc[q];
            changed = true;
        }
    }
    if (__any_sync(0xffffffffu, changed) && lane == 0) atomicAdd(changed_rows, 1ull);
}

// mode 0: out_i = OR_{k in succ(i)} M_k; violation iff (out_i | e_i) != M_i; ones of out.
template <int WPL>
__global__ void __launch_bounds__(256)
    sweep_rows_emit_kernel(const int *__restrict__ ptr, const int *__restrict__ col, int n, const uint64_t *M,
                           uint64_t *out, int64_t wp, unsigned long long *violations, unsigned long long *ones,
                           const uint64_t *__restrict__ colmask, const int *gate) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    if (gate != nullptr && *gate != 0) return;
    uint64_t full[WPL], acc[WPL];
    full_mask<WPL>(n, wp, lane, colmask, -1, full);
#pragma unroll
    for (int q = 0; q < WPL; ++q) acc[q] = 0ull;
    or_successors<WPL>(col, ptr[i], ptr[i + 1], M, wp, lane, false, full, acc);
    const uint64_t *mrow = M + static_cast<int64_t>(i) * wp;
    bool viol = false;
    uint32_t cnt = 0;
#pragma unroll
    for (int q = 0; q < WPL; ++q) {
        const int64_t w = lane + 32 * q;
        if (w >= wp) continue;
        const uint64_t self = (w == (i >> 6)) ? (1ull << (i & 63)) : 0ull;
        if ((acc[q] | self) != mrow[w]) viol = true;
        out[static_cast<int64_t>(i) * wp + w] = acc[q];
        cnt += __popcll(acc[q]);
    }
    const bool any = __any_sync(0xffffffffu, viol);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) {
        if (any) atomicAdd(violations, 1ull);
        if (ones && cnt) atomicAdd(ones, static_cast<unsigned long long>(cnt));
    }
}

template <int WPL>
cudaError_t launch_rows(const int *ptr, const int *col, int n, const uint64_t *M, uint64_t *out, int64_t wp,
                        int mode, unsigned long long *violations, unsigned long long *ones,
                        const unsigned long long *skip, const uint64_t *colmask, const int *gate, cudaStream_t s) {
    if (mode == 1)
        sweep_rows_step_kernel<WPL><<<(n + 7) / 8, 256, 0, s>>>(ptr, col, n, const_cast<uint64_t *>(M), wp,
                                                                 violations, skip, colmask, gate);
    else
        sweep_rows_emit_kernel<WPL><<<(n + 7) / 8, 256, 0, s>>>(ptr, col, n, M, out, wp, violations, ones,
                                                                 colmask, gate);
    return cudaGetLastError();
}

// mode 1 (closure step, in place): M_i |= E_i | OR_{k in succ(i)} M_k; counts changed units.
__global__ void __launch_bounds__(256)
    sweep_units_step_kernel(const int *__restrict__ ptr, const int *__restrict__ col, const int *__restrict__ unit_off,
                            int n, uint64_t *M, int64_t wp, unsigned long long *changed_units,
                            const unsigned long long *skip_if_zero) {
    const int lane = threadIdx.x & 31;
    if (skip_if_zero != nullptr && *skip_if_zero == 0) return;  // the previous sweep changed nothing
    const int total = unit_off[n];
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < total; u += warps) {
        const int i = unit_row(unit_off, n, u);
        const int q0 = ptr[i] + (u - unit_off[i]) * kUnit;
        const int q1 = min(q0 + kUnit, ptr[i + 1]);
        if (or_unit(col, q0, q1, n, i, M, M, wp, true, true, lane) && lane == 0) atomicAdd(changed_units, 1ull);
    }
}

// mode 0, pass 1 (out cleared beforehand): out_i = OR_{k in succ(i)} M_k.
__global__ void __launch_bounds__(256)
    sweep_units_or_kernel(const int *__restrict__ ptr, const int *__restrict__ col, const int *__restrict__ unit_off,
                          int n, const uint64_t *M, uint64_t *out, int64_t wp) {
    const int lane = threadIdx.x & 31;
    const int total = unit_off[n];
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < total; u += warps) {
        const int i = unit_row(unit_off, n, u);
        const int q0 = ptr[i] + (u - unit_off[i]) * kUnit;
        const int q1 = min(q0 + kUnit, ptr[i + 1]);
        or_unit(col, q0, q1, n, i, M, out, wp, false, true, lane);
    }
}

// mode 0, pass 2: violation iff (out_i | e_i) != M_i; ones of out.
__global__ void __launch_bounds__(256)
    sweep_check_kernel(int n, const uint64_t *__restrict__ M, const uint64_t *__restrict__ out, int64_t wp,
                       unsigned long long *violations, unsigned long long *ones) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    bool viol = false;
    uint32_t cnt = 0;
    for (int64_t w = lane; w < wp; w += 32) {
        const uint64_t v = out[static_cast<int64_t>(i) * wp + w];
        const uint64_t self = (w == (i >> 6)) ? (1ull << (i & 63)) : 0ull;
        if ((v | self) != M[static_cast<int64_t>(i) * wp + w]) viol = true;
        cnt += __popcll(v);
    }
    const bool any = __any_sync(0xffffffffu, viol);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) {
        if (any) atomicAdd(violations, 1ull);
        if (ones && cnt) atomicAdd(ones, static_cast<unsigned long long>(cnt));
    }
}

// e4m3 0/1 matrix (np x np, 0x38 = 1) from bits; one thread per 64-column word.
__global__ void bits_to_e4m3_kernel(const uint64_t *__restrict__ bits, int64_t wp, int np, uint8_t *__restrict__ C) {
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= static_cast<int64_t>(np) * wp) return;
    const int64_t r = t / wp, w = t % wp;
    const uint64_t x = bits[t];
    uint4 *dst = reinterpret_cast<uint4 *>(C + r * np + w * 64);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t o[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const uint32_t nib = static_cast<uint32_t>(x >> (16 * q + 4 * b)) & 0xFu;
            o[b] = ((nib & 1u) * 0x38u) | (((nib >> 1) & 1u) * 0x3800u) | (((nib >> 2) & 1u) * 0x380000u) |
                   (((nib >> 3) & 1u) * 0x38000000u);
        }
        dst[q] = make_uint4(o[0], o[1], o[2], o[3]);
    }
}

// Rows of the reflexive closure by the Iteration on single rows (see iterate_row).  With a
// gate the launch decides on the device: if *gate is set or the graph has more than two facts
// per row it does nothing but count every row as open.
__global__ void __launch_bounds__(256)
    row_iteration_kernel(const int *__restrict__ ptr, const int *__restrict__ col, int n, int wp, uint64_t *M,
                         unsigned long long *open_rows, const int *gate) {
    if (gate != nullptr && (*gate != 0 || ptr[n] > 2 * n)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(open_rows, static_cast<unsigned long long>(n));
        return;
    }
    extern __shared__ uint64_t row_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t *bits = row_smem + static_cast<size_t>(wid) * (wp + kRowFront + 1);
    const int i = blockIdx.x * (blockDim.x >> 5) + wid;
    if (i >= n) return;
    if (!iterate_row(ptr, col, i, wp, bits, M + static_cast<int64_t>(i) * wp, lane) && lane == 0)
        atomicAdd(open_rows, 1ull);
}

// ---- same generation on bits --------------------------------------------------------------
// 64 x 64 bit-block transpose, one warp per block (lane l holds rows l and l + 32 of the
// block; bit c of a word is column c): the off-diagonal j x j sub-blocks of every 2j x 2j
// block are exchanged for j = 32, 16, ..., 1 (the first step inside a lane, the others between
// lanes l and l ^ j).
__global__ void __launch_bounds__(256)
    bits_transpose_kernel(const uint64_t *__restrict__ src, uint64_t *__restrict__ dst, int nb, int64_t wp,
                          const unsigned long long *skip_if_zero) {
    if (skip_if_zero != nullptr && *skip_if_zero == 0) return;
    const int lane = threadIdx.x & 31;
    const int64_t b = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= static_cast<int64_t>(nb) * nb) return;
    const int64_t R = b / nb, C = b % nb;
    uint64_t x0 = src[(64 * R + lane) * wp + C], x1 = src[(64 * R + 32 + lane) * wp + C];
    {
        const uint64_t t = ((x0 >> 32) ^ x1) & 0x00000000FFFFFFFFull;
        x1 ^= t;
        x0 ^= t << 32;
    }
    const uint64_t masks[5] = {0x0000FFFF0000FFFFull, 0x00FF00FF00FF00FFull, 0x0F0F0F0F0F0F0F0Full,
                               0x3333333333333333ull, 0x5555555555555555ull};
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int j = 16 >> s;
        const uint64_t m = masks[s];
        const uint64_t y0 = __shfl_xor_sync(0xffffffffu, x0, j), y1 = __shfl_xor_sync(0xffffffffu, x1, j);
        if ((lane & j) == 0) {  // upper row of the pair: takes the partner's low part
            x0 ^= (((x0 >> j) ^ y0) & m) << j;
            x1 ^= (((x1 >> j) ^ y1) & m) << j;
        } else {
            x0 ^= ((y0 >> j) ^ x0) & m;
            x1 ^= ((y1 >> j) ^ x1) & m;
        }
    }
    dst[(64 * C + lane) * wp + R] = x0;
    dst[(64 * C + 32 + lane) * wp + R] = x1;
}

// dst_i = [dst_i if accumulate] | OR_{k in succ(i)} src_k, one warp per row i < n (lanes own
// WPL words, successor rows loaded in pairs, stop once the row holds every column).  With
// accumulate, *changed counts the rows whose words changed; without, every word is written.
template <int WPL>
__global__ void __launch_bounds__(256)
    gather_rows_kernel(const int *__restrict__ ptr, const int *__restrict__ col, int n, const uint64_t *src,
                       uint64_t *dst, int64_t wp, int accumulate, unsigned long long *changed,
                       const unsigned long long *skip_if_zero) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    if (skip_if_zero != nullptr && *skip_if_zero == 0) return;
    uint64_t *drow = dst + static_cast<int64_t>(i) * wp;
    uint64_t acc[WPL], full[WPL];
    full_mask<WPL>(n, wp, lane, nullptr, -1, full);
#pragma unroll
    for (int q = 0; q < WPL; ++q) {
        const int64_t w = lane + 32 * q;
        acc[q] = (accumulate && w < wp) ? drow[w] : 0ull;
    }
    or_successors<WPL>(col, ptr[i], ptr[i + 1], src, wp, lane, false, full, acc);
    bool ch = false;
#pragma unroll
    for (int q = 0; q < WPL; ++q) {
        const int64_t w = lane + 32 * q;
        if (w >= wp) continue;
        if (!accumulate) {
            drow[w] = acc[q];
        } else if (acc[q] != drow[w]) {  // only this warp writes row i
            drow[w] = acc[q];
            ch = true;
        }
    }
    if (accumulate && __any_sync(0xffffffffu, ch) && lane == 0) atomicAdd(changed, 1ull);
}

// The same gather split into work units of at most kUnit successors (rows with hundreds of
// successors would serialise a warp), combined with atomicOr; dst rows < n must start zero
// unless accumulate.  With accumulate, *changed counts units that changed a word.
__global__ void __launch_bounds__(256)
    gather_units_kernel(const int *__restrict__ ptr, const int *__restrict__ col, const int *__restrict__ unit_off,
                        int n, const uint64_t *src, uint64_t *dst, int64_t wp, int accumulate,
                        unsigned long long *changed, const unsigned long long *skip_if_zero) {
    if (skip_if_zero != nullptr && *skip_if_zero == 0) return;
    const int lane = threadIdx.x & 31;
    const int total = unit_off[n];
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < total; u += warps) {
        const int i = unit_row(unit_off, n, u);
        const int q0 = ptr[i] + (u - unit_off[i]) * kUnit;
        const int q1 = min(q0 + kUnit, ptr[i + 1]);
        if (or_unit(col, q0, q1, n, i, src, dst, wp, false, true, lane) && accumulate && lane == 0)
            atomicAdd(changed, 1ull);
    }
}

// Ones in rows < n of a bit matrix.
__global__ void bits_count_kernel(const uint64_t *__restrict__ M, int n, int64_t wp, unsigned long long *ones) {
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    uint32_t c = t < static_cast<int64_t>(n) * wp ? __popcll(M[t]) : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(ones, static_cast<unsigned long long>(c));
}

// Rows < n get the identity, every other word is zero (np rows).
__global__ void bits_identity_kernel(uint64_t *M, int n, int np, int64_t wp) {
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= static_cast<int64_t>(np) * wp) return;
    const int64_t r = t / wp, w = t % wp;
    M[t] = (r < n && w == (r >> 6)) ? 1ull << (r & 63) : 0ull;
}

// Words where A and B differ (counted).
__global__ void bits_diff_kernel(const uint64_t *__restrict__ A, const uint64_t *__restrict__ B, int64_t words,
                                 unsigned long long *diff) {
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const bool d = t < words && A[t] != B[t];
    const unsigned bal = __ballot_sync(0xffffffffu, d);
    if ((threadIdx.x & 31) == 0 && bal) atomicAdd(diff, static_cast<unsigned long long>(__popc(bal)));
}

}  // namespace

bool row_direct(int max_deg, int64_t wp) { return max_deg >= 0 && max_deg <= kRowDirect && wp <= 256; }

cudaError_t sweep_units(const int *ptr, int n, int *cnt, int *unit_off, cudaStream_t s) {
    unit_count_kernel<<<(n + 255) / 256, 256, 0, s>>>(ptr, n, cnt);
    return exclusive_scan(cnt, n, unit_off, s);
}

cudaError_t bits_sweep_csr(const int *ptr, const int *col, const int *unit_off, int n, const uint64_t *M,
                           uint64_t *out, int64_t wp, int mode, unsigned long long *violations,
                           unsigned long long *ones, int *launches, cudaStream_t s, int max_deg,
                           const unsigned long long *skip_if_zero, const uint64_t *colmask, const int *gate) {
    if (n <= 0) return cudaSuccess;
    if (row_direct(max_deg, wp)) {  // no heavy rows: row-direct kernels
        if (launches) *launches += 1;
        if (wp <= 64)
            return launch_rows<2>(ptr, col, n, M, out, wp, mode, violations, ones, skip_if_zero, colmask, gate, s);
        if (wp <= 128)
            return launch_rows<4>(ptr, col, n, M, out, wp, mode, violations, ones, skip_if_zero, colmask, gate, s);
        return launch_rows<8>(ptr, col, n, M, out, wp, mode, violations, ones, skip_if_zero, colmask, gate, s);
    }
    if (gate != nullptr) return cudaErrorInvalidValue;  // gated launches are row-direct only
    const unsigned grid = static_cast<unsigned>(num_sms() * 8);
    if (mode == 1) {
        sweep_units_step_kernel<<<grid, 256, 0, s>>>(ptr, col, unit_off, n, const_cast<uint64_t *>(M), wp,
                                                      violations, skip_if_zero);
        if (launches) *launches += 1;
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(out, 0, static_cast<size_t>(n) * wp * 8, s);
    if (e != cudaSuccess) return e;
    sweep_units_or_kernel<<<grid, 256, 0, s>>>(ptr, col, unit_off, n, M, out, wp);
    sweep_check_kernel<<<(n + 7) / 8, 256, 0, s>>>(n, M, out, wp, violations, ones);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

cudaError_t bits_to_e4m3(const uint64_t *bits, int64_t wp, int np, uint8_t *C, cudaStream_t s) {
    const int64_t words = static_cast<int64_t>(np) * wp;
    bits_to_e4m3_kernel<<<static_cast<unsigned>((words + 255) / 256), 256, 0, s>>>(bits, wp, np, C);
    return cudaGetLastError();
}

cudaError_t ingest_u8_to_e4m3(const uint8_t *src, int n, int np, uint8_t *dst, int add_identity,
                              unsigned long long *dmax, unsigned long long *nnz,
                              unsigned long long *count, int *status, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    ingest_kernel<<<np, kIngestThreads, 0, s>>>(src, n, np, dst, add_identity, dmax, nnz, count,
                                                 status);
    return cudaGetLastError();
}

cudaError_t load_ingest_and_sweep() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, ingest_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, sweep_kernel);
    return e;
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

bool row_iteration_fits(int64_t wp) { return wp <= 256; }

cudaError_t row_iteration(const int *ptr, const int *col, int n, int64_t wp, uint64_t *M,
                          unsigned long long *open_rows, cudaStream_t s, const int *gate) {
    if (n <= 0) return cudaSuccess;
    if (!row_iteration_fits(wp)) return cudaErrorInvalidValue;
    const size_t smem = 8 * (static_cast<size_t>(wp) + kRowFront + 1) * sizeof(uint64_t);
    row_iteration_kernel<<<(n + 7) / 8, 256, smem, s>>>(ptr, col, n, static_cast<int>(wp), M, open_rows, gate);
    return cudaGetLastError();
}

cudaError_t bits_transpose(const uint64_t *src, uint64_t *dst, int np, int64_t wp, const unsigned long long *skip,
                           cudaStream_t s) {
    if (np % 64 != 0 || wp * 64 != np) return cudaErrorInvalidValue;
    const int nb = np / 64;
    const int64_t blocks = (static_cast<int64_t>(nb) * nb + 7) / 8;
    bits_transpose_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(src, dst, nb, wp, skip);
    return cudaGetLastError();
}

cudaError_t bits_gather(const int *ptr, const int *col, const int *unit_off, int n, const uint64_t *src, uint64_t *dst,
                        int64_t wp, int accumulate, unsigned long long *changed, const unsigned long long *skip,
                        cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (unit_off != nullptr) {
        if (!accumulate) {
            const cudaError_t e = cudaMemsetAsync(dst, 0, static_cast<size_t>(n) * wp * 8, s);
            if (e != cudaSuccess) return e;
        }
        gather_units_kernel<<<static_cast<unsigned>(num_sms() * 8), 256, 0, s>>>(ptr, col, unit_off, n, src, dst, wp,
                                                                                accumulate, changed, skip);
        return cudaGetLastError();
    }
    const unsigned grid = static_cast<unsigned>((n + 7) / 8);
    if (wp <= 64) gather_rows_kernel<2><<<grid, 256, 0, s>>>(ptr, col, n, src, dst, wp, accumulate, changed, skip);
    else if (wp <= 128) gather_rows_kernel<4><<<grid, 256, 0, s>>>(ptr, col, n, src, dst, wp, accumulate, changed, skip);
    else if (wp <= 256) gather_rows_kernel<8><<<grid, 256, 0, s>>>(ptr, col, n, src, dst, wp, accumulate, changed, skip);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t bits_count(const uint64_t *M, int n, int64_t wp, unsigned long long *ones, cudaStream_t s) {
    const int64_t words = static_cast<int64_t>(n) * wp;
    if (words <= 0) return cudaSuccess;
    bits_count_kernel<<<static_cast<unsigned>((words + 255) / 256), 256, 0, s>>>(M, n, wp, ones);
    return cudaGetLastError();
}

cudaError_t bits_identity(uint64_t *M, int n, int np, int64_t wp, cudaStream_t s) {
    const int64_t words = static_cast<int64_t>(np) * wp;
    bits_identity_kernel<<<static_cast<unsigned>((words + 255) / 256), 256, 0, s>>>(M, n, np, wp);
    return cudaGetLastError();
}

cudaError_t bits_diff(const uint64_t *A, const uint64_t *B, int64_t words, unsigned long long *diff, cudaStream_t s) {
    if (words <= 0) return cudaSuccess;
    bits_diff_kernel<<<static_cast<unsigned>((words + 255) / 256), 256, 0, s>>>(A, B, words, diff);
    return cudaGetLastError();
}

}  // namespace dl
