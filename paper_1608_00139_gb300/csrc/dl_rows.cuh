// dl_rows.cuh -- per-row device routines shared by the single-problem and batched kernels:
// ingest of one row of a 0/1 base relation, and one row of the certificate / recheck sweep.
#pragma once
#include <cstdint>

#include "dl_internal.h"

namespace dl {

// One CTA writes padded row `row` of the e4m3 operand (np bytes): 0x38 where the source byte
// is 1, zero elsewhere and in the padding, and 1.0 on the diagonal if add_identity.  The
// calling thread's partial row sum and "bad byte" bits are returned in sum / bad; thread 0
// sets extra = 1 if it added a diagonal one that the source lacked.
__device__ __forceinline__ void ingest_row(const uint8_t *__restrict__ src, int n, int np,
                                           uint8_t *__restrict__ dst, int add_identity, int row,
                                           uint32_t &sum, uint32_t &bad, uint32_t &extra) {
    uint8_t *drow = dst + static_cast<int64_t>(row) * np;
    if (row < n) {
        const uint8_t *srow = src + static_cast<int64_t>(row) * n;
        const bool vec = ((n & 15) == 0) && ((reinterpret_cast<uintptr_t>(src) & 15) == 0) &&
                         ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) && ((np & 15) == 0);
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
    if (add_identity && threadIdx.x == 0) {
        if (row >= n || drow[row] == 0) extra = 1;
        drow[row] = 0x38;
    }
}

// Block-wide sum (of a) and OR (of b); the result is valid in thread 0.
__device__ __forceinline__ void block_reduce_sum_or(uint32_t &a, uint32_t &b) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b |= __shfl_xor_sync(0xffffffffu, b, o);
    }
    __shared__ uint32_t s_a[32], s_b[32];
    const int warps = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_a[threadIdx.x >> 5] = a;
        s_b[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t ta = 0, tb = 0;
        for (int w = 0; w < warps; ++w) {
            ta += s_a[w];
            tb |= s_b[w];
        }
        a = ta;
        b = tb;
    }
}

// Warp-uniform read of a counter another warp may be incrementing.
__device__ __forceinline__ unsigned long long warp_read_u64(const unsigned long long *p) {
    unsigned long long v = (threadIdx.x & 31) == 0 ? *reinterpret_cast<const volatile unsigned long long *>(p) : 0ull;
    return __shfl_sync(0xffffffffu, v, 0);
}

// Lanes own words lane, lane+32, ... of a row (up to kSweepWpl per lane per pass; wider
// rows take several passes over the E row).
constexpr int kSweepWpl = 8;

// One warp processes row `row` of the sweep over bit matrix M (wp 64-bit words per row):
//   mode 0: out_row = OR_{k : E[row][k]} M_k;  violation iff (out_row | e_row) != M_row
//   mode 1: out_row = M_row | E_row | OR_{k : E[row][k]} M_k;  violation iff it changed
// (out may equal M in mode 1).  viol and cnt (ones in out_row) are warp-uniform on return.
__device__ __forceinline__ void sweep_row(const uint8_t *__restrict__ erow, int n, const uint64_t *M,
                                          uint64_t *out, int64_t wp, int mode, int row, int lane,
                                          bool &viol_out, uint32_t &cnt_out) {
    const uint64_t *mrow = M + static_cast<int64_t>(row) * wp;
    bool viol = false;
    uint32_t cnt = 0;
    // A row whose accumulator already holds all n columns cannot change any more: stop its
    // scan (single-pass rows only).  Most rows of a closure with a giant component are full.
    const bool single_pass = wp <= 32 * kSweepWpl;
    uint64_t full[kSweepWpl];
#pragma unroll
    for (int q = 0; q < kSweepWpl; ++q) {
        const int64_t w = lane + 32 * q;
        const int64_t lo = w * 64;
        full[q] = (w >= wp || lo >= n) ? 0ull : (n - lo >= 64 ? ~0ull : ((1ull << (n - lo)) - 1ull));
    }
    for (int64_t w0 = 0; w0 < wp; w0 += 32 * kSweepWpl) {
        uint64_t acc[kSweepWpl];
#pragma unroll
        for (int t = 0; t < kSweepWpl; ++t) acc[t] = 0;
        bool saturated = false;
        if (single_pass && mode == 1) {  // the row itself may already be full
            bool mine = true;
#pragma unroll
            for (int q = 0; q < kSweepWpl; ++q) {
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
                    for (int q = 0; q < kSweepWpl; ++q) {
                        const int64_t w = w0 + lane + 32 * q;
                        if (w < wp) acc[q] |= mk[w];
                    }
                    if (mode == 1) {  // the fact E[i][k] itself
                        const int64_t rel = (k >> 6) - w0;  // word index within this pass
                        if (rel >= 0 && rel < 32 * kSweepWpl && (rel & 31) == lane) {
                            const int qk = static_cast<int>(rel >> 5);
#pragma unroll
                            for (int q = 0; q < kSweepWpl; ++q)
                                if (q == qk) acc[q] |= 1ull << (k & 63);
                        }
                    }
                    if (single_pass) {
                        bool mine = true;
#pragma unroll
                        for (int q = 0; q < kSweepWpl; ++q) mine &= acc[q] == full[q];
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
        for (int q = 0; q < kSweepWpl; ++q) {
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
    viol_out = __any_sync(0xffffffffu, viol);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    cnt_out = cnt;
}

}  // namespace dl
