// dl_rows.cuh -- per-row device routines shared by the single-problem and batched kernels:
// ingest of one row of a 0/1 base relation (as e4m3 or as bits), successor lists from bits,
// and one row of the certificate / recheck sweep.
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

// Low bits of the four bytes of x as a 4-bit mask (byte b -> bit b).
__device__ __forceinline__ uint32_t byte_lsbs(uint32_t x) { return ((x & 0x01010101u) * 0x01020408u) >> 24; }
// Bytes of x with any of bits 1..7 set, as a 4-bit mask.
__device__ __forceinline__ uint32_t byte_bad(uint32_t x) {
    const uint32_t t = (x >> 1) & 0x7F7F7F7Fu;
    return byte_lsbs(((t + 0x7F7F7F7Fu) | t) >> 7);
}

// One warp packs row r of a 0/1 byte matrix (the n bytes at a, any alignment) into wp 64-bit
// words at `row`, plus the identity bit r.  The row is read as aligned 16-byte chunks: lane
// L of segment s holds the 64 bytes that start 64 (32 s + L) bytes after the aligned address
// below a, and each model word is two of those 64-bit groups shifted by the misalignment.
// Bytes outside the row are masked off (they are never counted or checked).  Every lane
// returns the row's count of ones (without the identity) and whether a byte was not 0/1.
// With colmask (shared memory, wp words) the row's facts are also ORed into it; without
// identity the bit r is not added.
__device__ __forceinline__ void pack_row_bits(const uint8_t *a, int n, int r, int wp, uint64_t *row, int lane,
                                              int &count, bool &bad_byte, uint64_t *colmask = nullptr,
                                              bool identity = true) {
    const int idw = identity ? r >> 6 : -1;
    const uint64_t idb = 1ull << (r & 63);
    const int off = static_cast<int>(reinterpret_cast<uintptr_t>(a) & 15);
    const uint8_t *base = a - off;
    const int lim = off + n;  // the row occupies bytes [off, lim) from base
    const int nseg = wp / 32 + 1;
    uint32_t bad = 0;
    int c = 0;
    uint64_t carry = 0;
    auto shifted = [off](uint64_t lo, uint64_t hi) { return off ? (lo >> off) | (hi << (64 - off)) : lo; };
    // the next segment's chunks are loaded before this one is processed (two in flight)
    uint4 cur[4];
    auto load = [&](int sg, uint4 (&x)[4]) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int v0 = 64 * (32 * sg + lane) + 16 * j;
            x[j] = v0 < lim ? *reinterpret_cast<const uint4 *>(base + v0) : make_uint4(0u, 0u, 0u, 0u);
        }
    };
    load(0, cur);
    for (int sg = 0; sg < nseg; ++sg) {
        const int u = 32 * sg + lane;
        uint4 nx[4] = {};
        if (sg + 1 < nseg) load(sg + 1, nx);
        uint64_t vw = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int v0 = 64 * u + 16 * j;
            if (v0 < lim) {
                const uint4 x = cur[j];
                const int lo = max(0, off - v0), hi = min(16, lim - v0);
                const uint32_t valid = ((1u << hi) - 1u) & ~((1u << lo) - 1u);
                const uint32_t m = byte_lsbs(x.x) | (byte_lsbs(x.y) << 4) | (byte_lsbs(x.z) << 8) |
                                   (byte_lsbs(x.w) << 12);
                const uint32_t b = byte_bad(x.x) | (byte_bad(x.y) << 4) | (byte_bad(x.z) << 8) |
                                   (byte_bad(x.w) << 12);
                vw |= static_cast<uint64_t>(m & valid) << (16 * j);
                bad |= b & valid;
            }
        }
        c += __popcll(vw);
        const uint64_t nxt = __shfl_down_sync(0xffffffffu, vw, 1);
        const uint64_t first = __shfl_sync(0xffffffffu, vw, 0);
        auto put = [&](int w, uint64_t e) {  // e: the facts of word w
            row[w] = e | (w == idw ? idb : 0ull);
            if (colmask != nullptr && e != 0ull) atomicOr(reinterpret_cast<unsigned long long *>(colmask + w), e);
        };
        if (sg > 0 && lane == 31) {
            const int w = 32 * (sg - 1) + 31;
            if (w < wp) put(w, shifted(carry, first));
        }
        if (lane < 31) {
            const int w = 32 * sg + lane;
            if (w < wp) put(w, shifted(vw, nxt));
        }
        carry = vw;
#pragma unroll
        for (int j = 0; j < 4; ++j) cur[j] = nx[j];
    }
    if (lane == 31) {
        const int w = 32 * (nseg - 1) + 31;
        if (w < wp) {
            const uint64_t e = shifted(carry, 0ull);
            row[w] = e | (w == idw ? idb : 0ull);
            if (colmask != nullptr && e != 0ull) atomicOr(reinterpret_cast<unsigned long long *>(colmask + w), e);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(0xffffffffu, c, o);
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    count = c;
    bad_byte = bad != 0;
}

// One warp writes the successor list of row r into col[pos0 .. pos1) from its packed bits
// (I + E: the identity bit belongs to E only when the row holds pos1 - pos0 ones).
__device__ __forceinline__ void fill_row_from_bits(const uint64_t *row, int wp, int r, int pos0, int pos1, int *col,
                                                   int lane) {
    int ones = 0;
    for (int w = lane; w < wp; w += 32) ones += __popcll(row[w]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ones += __shfl_xor_sync(0xffffffffu, ones, o);
    const bool self = ones == pos1 - pos0;
    int pos = pos0;
    for (int w0 = 0; w0 < wp; w0 += 32) {
        const int w = w0 + lane;
        uint64_t x = w < wp ? row[w] : 0ull;
        if (!self && w == (r >> 6)) x &= ~(1ull << (r & 63));
        const int c = __popcll(x);
        int inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        int p = pos + inc - c;
        while (x) {
            const int b = __ffsll(static_cast<long long>(x)) - 1;
            x &= x - 1;
            col[p++] = 64 * w + b;
        }
        pos += __shfl_sync(0xffffffffu, inc, 31);
    }
}

// Single-row Iteration (eq. series:trcl on one row vector x_i, x <- min1(e_i + x E) for the
// successor relation), semi-naive: one warp keeps the row's bits in shared memory (`bits`:
// wp words, then two frontiers of kRowFront ints and a counter) and expands only the nodes
// that entered x in the last step, lanes taking frontier nodes and setting their successors'
// bits with shared-memory atomicOr.  ptr/col: the CSR with column indices local to the
// problem (ptr may be offset so that ptr[k] is local row k).  When the frontier empties, x
// is the exact row i of the reflexive closure; a frontier larger than kRowFront or more than
// kRowSteps steps (long paths are left to squarings) ends the row early.  Either way the bits
// reached (all reachable from i) go to mrow; returns whether the row is exact.
constexpr int kRowFront = 256;
constexpr int kRowSteps = 64;

__device__ __forceinline__ bool iterate_row(const int *__restrict__ ptr, const int *__restrict__ col, int i, int wp,
                                            uint64_t *bits, uint64_t *mrow, int lane) {
    int *front = reinterpret_cast<int *>(bits + wp);  // two frontiers of kRowFront
    int *next_cnt = front + 2 * kRowFront;
    for (int w = lane; w < wp; w += 32) bits[w] = w == (i >> 6) ? 1ull << (i & 63) : 0ull;
    if (lane == 0) front[0] = i;
    int cur = 0, cnt = 1, steps = 0;
    bool ok = true;
    __syncwarp();
    while (cnt > 0) {
        if (++steps > kRowSteps) {
            ok = false;
            break;
        }
        if (lane == 0) *next_cnt = 0;
        __syncwarp();
        const int *fc = front + cur * kRowFront;
        int *fn = front + (cur ^ 1) * kRowFront;
        for (int f = lane; f < cnt; f += 32) {
            const int k = fc[f];
            const int q1 = ptr[k + 1];
            for (int q = ptr[k]; q < q1; ++q) {
                const int j = col[q];
                const unsigned long long b = 1ull << (j & 63);
                const unsigned long long old = atomicOr(reinterpret_cast<unsigned long long *>(bits + (j >> 6)), b);
                if (!(old & b)) {
                    const int pos = atomicAdd(next_cnt, 1);
                    if (pos < kRowFront) fn[pos] = j;
                }
            }
        }
        __syncwarp();
        cnt = *next_cnt;
        __syncwarp();  // every lane has read the count before lane 0 clears it
        if (cnt > kRowFront) {
            ok = false;
            break;
        }
        cur ^= 1;
    }
    __syncwarp();
    for (int w = lane; w < wp; w += 32) mrow[w] = bits[w];
    return ok;
}

}  // namespace dl
