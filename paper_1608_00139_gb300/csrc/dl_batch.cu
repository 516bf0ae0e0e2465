// dl_batch.cu -- many independent closure problems of uneven size in one call (dl_tc_batch).
//
// Every instance k gets the AUTO closure of dl_solve.cu (Iteration steps on bits, with
// repeated squaring of the reflexive closure for the instances that keep changing), but all
// instances advance together and every decision is taken on the device:
//   1. (every call) one pass over all inputs packs the bits of I + E_k, checks that every
//      byte is 0/1 and counts successors; a scan gives one CSR over all instances' rows.
//   2. (captured CUDA graph) fill the CSR column indices from the packed bits; 24 batched
//      in-place sweeps M <- M | E | E M; an instance whose sweep changes nothing holds its
//      reflexive closure and leaves the active list.  Then rounds for the instances still
//      active: their bits become e4m3 operands, one persistent grouped tcgen05 launch squares
//      exactly those instances (a tile schedule written on the device), 4 more sweeps.
//      Finally the model E_k C_k* of every instance with its certificate C = min1(I + E C).
// After every sweep a single-CTA kernel rebuilds the list of active instances (their rows,
// padded rows and GEMM tiles as prefix sums), so that later kernels touch only live rows and
// a round with nothing left active costs a few empty launches.  The graph is cached and
// relaunched while the inputs and outputs stay the same buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "dl_ctx.h"
#include "dl_internal.h"
#include "dl_rows.cuh"

namespace dl {

namespace {

constexpr unsigned kFull = 0xffffffffu;
enum : int { B_ACTIVE = 0, B_EMIT = 1, B_DONE = 2 };
constexpr int kFirstSweeps = 24;  // sweeps before any squaring
constexpr int kRoundSweeps = 4;   // sweeps after each squaring round
constexpr int kMainRounds = 2;    // squaring rounds in the main graph (the rest only if needed)
constexpr int kChunk = 32;        // rows a warp claims at a time in the row kernels
constexpr int kListThreads = 1024;

struct BatchInst {
    const uint8_t *E;  // n x n input bytes on the device (row stride n)
    uint8_t *c0;       // e4m3 operand, np x np
    uint64_t *rbits;   // reflexive-closure candidate M, np x wp
    uint64_t *mbits;   // model bits, np x wp (host outputs are copied from here)
    uint64_t *out;     // user output (device memory, n rows of ceil(n/64) words) or null
    uint64_t *colmask; // the columns with an incoming edge, wp words
    int32_t n, np;
    int32_t wp;
    int32_t tiles;  // GEMM tiles of the squaring
    int32_t prow0;  // first padded row in the order of all instances
    int32_t row0;   // first real row in the order of all instances
};

// Per-instance counters (arrays of `count` entries) and the active-instance counter.
struct BatchCounters {
    int *state;
    unsigned long long *chg, *viol, *ones, *squarings, *sweeps;
};
constexpr int kCounterArrays = 5;

// The instances in one state, as prefix sums over the selected instances.
//   hdr[0] entries A, hdr[1] rows, hdr[2] padded rows, hdr[3] tiles, hdr[4] chunk counter
//   k[j] instance of entry j; row[j], prow[j] exclusive prefixes (A + 1 entries)
//   sched: the GEMM schedule (see gemm_launch) over the same entries
struct BatchList {
    int *hdr;
    int *k, *row, *prow;
    int *sched;
};

__device__ __forceinline__ int last_le(const int *pre, int count, int x) {  // largest j: pre[j] <= x
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Padded row -> instance, rebuilt every call (one CTA per instance).
__global__ void batch_map_kernel(const BatchInst *__restrict__ inst, int *pinst) {
    const BatchInst I = inst[blockIdx.x];
    for (int r = threadIdx.x; r < I.np; r += blockDim.x) pinst[I.prow0 + r] = blockIdx.x;
}

// Bits of row r of I + E_k into M, the row's successor count and the 0/1 check.  A warp takes
// kPackRows consecutive padded rows and looks the instance up again only where the rows cross
// into the next one (rows are short: per-row lookups would put two dependent loads before
// every row's own).
constexpr int kPackRows = 4;

__global__ void __launch_bounds__(256, 4)
    batch_pack_kernel(const BatchInst *__restrict__ inst, const int *__restrict__ pinst, int total_prows,
                      int *cnt, int *status) {
    const int lane = threadIdx.x & 31;
    const int g0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kPackRows;
    if (g0 >= total_prows) return;
    const int g1 = min(g0 + kPackRows, total_prows);
    int k = pinst[g0];
    const uint8_t *E = inst[k].E;
    uint64_t *rbits = inst[k].rbits;
    int n = inst[k].n, np = inst[k].np, wp = inst[k].wp, prow0 = inst[k].prow0, row0 = inst[k].row0;
    for (int g = g0; g < g1; ++g) {
        if (g - prow0 >= np) {  // the next instance
            k = pinst[g];
            E = inst[k].E;
            rbits = inst[k].rbits;
            n = inst[k].n;
            np = inst[k].np;
            wp = inst[k].wp;
            prow0 = inst[k].prow0;
            row0 = inst[k].row0;
        }
        const int r = g - prow0;
        uint64_t *row = rbits + static_cast<int64_t>(r) * wp;
        if (r >= n) {  // padding: identity only
            for (int w = lane; w < wp; w += 32) row[w] = w == (r >> 6) ? 1ull << (r & 63) : 0ull;
            continue;
        }
        int c = 0;
        bool bad = false;
        pack_row_bits(E + static_cast<int64_t>(r) * n, n, r, wp, row, lane, c, bad);
        if (lane == 0) {
            cnt[row0 + r] = c;
            if (bad) atomicOr(status, ST_BAD_INPUT);
        }
    }
}

// Successor lists from the packed bits (one warp per padded row, real rows only).
__global__ void __launch_bounds__(256)
    batch_fill_kernel(const BatchInst *__restrict__ inst, const int *__restrict__ pinst, int total_prows,
                      const int *__restrict__ ptr, int *col) {
    const int lane = threadIdx.x & 31;
    const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (g >= total_prows) return;
    const BatchInst I = inst[pinst[g]];
    const int r = g - I.prow0;
    if (r >= I.n) return;
    const int gr = I.row0 + r;
    fill_row_from_bits(I.rbits + static_cast<int64_t>(r) * I.wp, I.wp, r, ptr[gr], ptr[gr + 1], col, lane);
}

// Column mask of every instance (CTA per instance): the columns its CSR names.  No row of
// the reflexive closure leaves the mask plus its own bit, no row of E M leaves the mask.
__global__ void __launch_bounds__(256)
    batch_colmask_kernel(const BatchInst *__restrict__ inst, const int *__restrict__ ptr, const int *__restrict__ col) {
    extern __shared__ unsigned long long cm_s[];
    const BatchInst I = inst[blockIdx.x];
    for (int w = threadIdx.x; w < I.wp; w += blockDim.x) cm_s[w] = 0ull;
    __syncthreads();
    for (int q = ptr[I.row0] + threadIdx.x; q < ptr[I.row0 + I.n]; q += blockDim.x)
        atomicOr(&cm_s[col[q] >> 6], 1ull << (col[q] & 63));
    __syncthreads();
    for (int w = threadIdx.x; w < I.wp; w += blockDim.x) I.colmask[w] = cm_s[w];
}

// Instances whose whole bit matrix fits in shared memory (at most kSmallNp padded rows of at
// most 16 words: 128 KB) are closed by one CTA each, before the batched machinery: in-place
// sweeps M_i |= E_i | OR_{s in succ(i)} M_s on the shared copy (rows of an instance share a
// warp in lane groups sized to the row) until one changes nothing (__syncthreads_or over the
// CTA), then the model E M with its certificate straight to the output.  An instance still
// changing after kSmallSweeps sweeps writes its bits back and stays active for the batched
// sweeps and squarings.
constexpr int kSmallNp = 1024;
constexpr int kSmallThreads = 1024;
constexpr int kSmallSweeps = 64;

__global__ void __launch_bounds__(kSmallThreads)
    batch_small_kernel(const BatchInst *__restrict__ inst, const int *__restrict__ small_ids,
                       const int *__restrict__ ptr, const int *__restrict__ col, BatchCounters c, int *status) {
    extern __shared__ uint64_t small_s[];
    __shared__ unsigned int ones_s;
    const int k = small_ids[blockIdx.x];
    const BatchInst I = inst[k];
    const int wp = I.wp, n = I.n;
    uint64_t *Ms = small_s;  // np x wp
    for (int t = threadIdx.x; t < I.np * wp; t += blockDim.x) Ms[t] = I.rbits[t];
    if (threadIdx.x == 0) ones_s = 0u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int G = 32;
    while (G > 1 && (G >> 1) >= wp) G >>= 1;
    const int R = 32 / G, grp = lane / G, w = lane % G;
    const bool wv = w < wp;
    const uint64_t cm = wv ? I.colmask[w] : 0ull;
    const int *iptr = ptr + I.row0;  // iptr[r]: local row r
    __syncthreads();
    int it = 0;
    bool conv = false;
    while (it < kSmallSweeps) {
        bool ch = false;
        for (int r = warp * R + grp; r < n; r += nwarps * R) {
            if (!wv) continue;
            uint64_t acc = Ms[r * wp + w];
            const uint64_t before = acc;
            const uint64_t full = cm | (w == (r >> 6) ? 1ull << (r & 63) : 0ull);
            for (int q = iptr[r]; q < iptr[r + 1] && acc != full; ++q) {
                const int sidx = col[q];
                acc |= Ms[sidx * wp + w] | (w == (sidx >> 6) ? 1ull << (sidx & 63) : 0ull);
            }
            if (acc != before) {
                Ms[r * wp + w] = acc;
                ch = true;
            }
        }
        ++it;
        if (!__syncthreads_or(ch)) {
            conv = true;
            break;
        }
    }
    if (!conv) {  // hand over: the batched machinery continues from these bits
        for (int t = threadIdx.x; t < I.np * wp; t += blockDim.x) I.rbits[t] = Ms[t];
        if (threadIdx.x == 0) c.sweeps[k] = it;
        return;
    }
    // the model E M and the certificate (out_r | e_r) = M_r
    const int wout = (n + 63) >> 6;
    bool viol = false;
    unsigned int ones = 0;
    for (int r = warp * R + grp; r < n; r += nwarps * R) {
        if (!wv) continue;
        uint64_t out = 0ull;
        for (int q = iptr[r]; q < iptr[r + 1] && out != cm; ++q) out |= Ms[col[q] * wp + w];
        const uint64_t self = w == (r >> 6) ? 1ull << (r & 63) : 0ull;
        viol |= (out | self) != Ms[r * wp + w];
        ones += __popcll(out);
        if (I.out) {
            if (w < wout) I.out[static_cast<int64_t>(r) * wout + w] = out;
        } else {
            I.mbits[static_cast<int64_t>(r) * wp + w] = out;
        }
    }
    if (ones) atomicAdd(&ones_s, ones);
    const int any_viol = __syncthreads_or(viol);
    if (threadIdx.x == 0) {
        c.sweeps[k] = it;
        c.ones[k] = ones_s;
        c.state[k] = B_DONE;
        if (any_viol) {  // a converged closure that fails its certificate: an internal error
            c.viol[k] = 1;
            atomicOr(status, ST_TIMEOUT_DEP);
        }
    }
}

// Block-wide exclusive scan of four counters at once (kListThreads threads).
__device__ __forceinline__ int4 block_scan4(int4 v, int4 *total) {
    __shared__ int4 part[kListThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int4 inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(kFull, inc.x, o), b = __shfl_up_sync(kFull, inc.y, o);
        const int c = __shfl_up_sync(kFull, inc.z, o), d = __shfl_up_sync(kFull, inc.w, o);
        if (lane >= o) inc = make_int4(inc.x + a, inc.y + b, inc.z + c, inc.w + d);
    }
    if (lane == 31) part[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int4 p = part[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int a = __shfl_up_sync(kFull, p.x, o), b = __shfl_up_sync(kFull, p.y, o);
            const int c = __shfl_up_sync(kFull, p.z, o), d = __shfl_up_sync(kFull, p.w, o);
            if (lane >= o) p = make_int4(p.x + a, p.y + b, p.z + c, p.w + d);
        }
        part[lane] = p;
    }
    __syncthreads();
    const int4 before = warp > 0 ? part[warp - 1] : make_int4(0, 0, 0, 0);
    *total = part[kListThreads / 32 - 1];
    return make_int4(before.x + inc.x - v.x, before.y + inc.y - v.y, before.z + inc.z - v.z,
                     before.w + inc.w - v.w);
}

// The list of instances in state `target` (single CTA).  With decide set, first the verdict of
// the sweep that just ran: an active instance whose sweep changed no row is converged.
__global__ void __launch_bounds__(kListThreads)
    batch_list_kernel(const BatchInst *__restrict__ inst, int L, BatchCounters c, BatchList list, int target,
                      int decide) {
    const int per = (L + kListThreads - 1) / kListThreads;
    const int k0 = min(L, static_cast<int>(threadIdx.x) * per), k1 = min(L, k0 + per);
    int4 mine = make_int4(0, 0, 0, 0);
    for (int k = k0; k < k1; ++k) {
        if (decide && c.state[k] == B_ACTIVE) {
            c.sweeps[k] += 1;
            if (c.chg[k] == 0) c.state[k] = B_EMIT;
            c.chg[k] = 0;
        }
        if (c.state[k] == target) {
            const BatchInst &I = inst[k];
            mine = make_int4(mine.x + 1, mine.y + I.n, mine.z + I.np, mine.w + I.tiles);
        }
    }
    int4 tot;
    int4 at = block_scan4(mine, &tot);
    int *tile_start = list.sched + 2 + L;
    for (int k = k0; k < k1; ++k) {
        if (c.state[k] != target) continue;
        const BatchInst &I = inst[k];
        list.k[at.x] = k;
        list.row[at.x] = at.y;
        list.prow[at.x] = at.z;
        list.sched[2 + at.x] = k;
        tile_start[at.x] = at.w;
        at = make_int4(at.x + 1, at.y + I.n, at.z + I.np, at.w + I.tiles);
    }
    if (threadIdx.x == 0) {
        list.hdr[0] = tot.x;
        list.hdr[1] = tot.y;
        list.hdr[2] = tot.z;
        list.hdr[3] = tot.w;
        list.hdr[4] = 0;
        list.row[tot.x] = tot.y;
        list.prow[tot.x] = tot.z;
        list.sched[0] = tot.x;
        list.sched[1] = tot.w;
        tile_start[tot.x] = tot.w;
    }
}

// Rows of the listed instances, claimed kChunk at a time.  With WPL == 1 a row takes G lanes
// (G = wp rounded up to a power of two) and a warp works on 32 / G rows of one instance at
// once; with WPL > 1 a row takes the warp and each lane WPL words.  Successors are taken U at
// a time, their rows loaded before any is combined.
//   EMIT == false (sweep):  M_i <- M_i | E_i | OR_{s in succ(i)} M_s in place; a group stops
//                           once its row is full; instance k's change counter counts steps
//                           that changed a row.
//   EMIT == true:           out_i = OR_{s in succ(i)} M_s; violation iff (out_i | e_i) != M_i.
template <int WPL, bool EMIT>
__global__ void __launch_bounds__(256)
    batch_rows_kernel(const BatchInst *__restrict__ inst, BatchList list, const int *__restrict__ ptr,
                      const int *__restrict__ col, BatchCounters c) {
    constexpr int U = WPL <= 2 ? 4 : 2;
    const int lane = threadIdx.x & 31;
    const int nrows = list.hdr[1];
    const int entries = list.hdr[0];
    if (nrows == 0) return;
    // rows per claim: kChunk while there are plenty, fewer as the active rows thin out (every
    // warp of the grid should have rows to work on)
    const int warps = gridDim.x * (blockDim.x >> 5);
    const int per = max(1, min(kChunk, nrows / warps));
    for (;;) {
        int chunk = 0;
        if (lane == 0) chunk = atomicAdd(list.hdr + 4, 1);
        chunk = __shfl_sync(kFull, chunk, 0);
        int r = chunk * per;
        if (r >= nrows) return;
        const int rend = min(nrows, r + per);
        int j = last_le(list.row, entries, r);
        while (r < rend) {
            const int k = list.k[j];
            const int ib = list.row[j];
            const int lim = min(rend, list.row[j + 1]);
            const BatchInst I = inst[k];
            const uint64_t *M = I.rbits;
            int G = 32;
            if (WPL == 1)
                while (G > 1 && (G >> 1) >= I.wp) G >>= 1;
            const int grp = lane / G, w0 = lane % G;
            const unsigned gmask = G == 32 ? kFull : (((1u << G) - 1u) << (grp * G));
            const int wout = (I.n + 63) >> 6;
            for (; r < lim; r += 32 / G) {
                const int i = r + grp - ib;
                const bool act = r + grp < lim;
                int q0 = 0, q1 = 0;
                if (act) {
                    q0 = ptr[I.row0 + i];
                    q1 = ptr[I.row0 + i + 1];
                }
                uint64_t acc[WPL], mi[WPL], fullw[WPL];
                bool sat = true;
#pragma unroll
                for (int q = 0; q < WPL; ++q) {
                    const int w = w0 + G * q;
                    const bool v = act && w < I.wp;
                    // the most the row can hold (kept in a register across the successor loop)
                    fullw[q] = v ? I.colmask[w] | ((!EMIT && w == (i >> 6)) ? 1ull << (i & 63) : 0ull) : 0ull;
                    asm volatile("" : "+l"(fullw[q]));
                    mi[q] = v ? M[static_cast<int64_t>(i) * I.wp + w] : 0ull;
                    acc[q] = EMIT ? 0ull : mi[q];
                    sat &= acc[q] == fullw[q];
                }
                unsigned bal = __ballot_sync(kFull, sat);
                int deg = act ? q1 - q0 : 0;
                if (!EMIT && (bal & gmask) == gmask) deg = 0;
                for (int t = 0; __any_sync(kFull, t < deg); t += U) {
                    int s[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) s[u] = t + u < deg ? col[q0 + t + u] : -1;
                    uint64_t v[U][WPL];
#pragma unroll
                    for (int u = 0; u < U; ++u)
#pragma unroll
                        for (int q = 0; q < WPL; ++q) {
                            const int w = w0 + G * q;
                            v[u][q] = (s[u] >= 0 && w < I.wp) ? M[static_cast<int64_t>(s[u]) * I.wp + w] : 0ull;
                        }
                    sat = true;
#pragma unroll
                    for (int q = 0; q < WPL; ++q) {
                        const int w = w0 + G * q;
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            acc[q] |= v[u][q];
                            if (!EMIT && s[u] >= 0 && w == (s[u] >> 6)) acc[q] |= 1ull << (s[u] & 63);
                        }
                        sat &= acc[q] == fullw[q];
                    }
                    bal = __ballot_sync(kFull, sat);
                    if ((bal & gmask) == gmask) deg = 0;  // the row is full: nothing more can be added
                }
                if (!EMIT) {
                    bool changed = false;
#pragma unroll
                    for (int q = 0; q < WPL; ++q) {
                        const int w = w0 + G * q;
                        if (act && w < I.wp && acc[q] != mi[q]) {
                            I.rbits[static_cast<int64_t>(i) * I.wp + w] = acc[q];
                            changed = true;
                        }
                    }
                    if (__any_sync(kFull, changed) && lane == 0) atomicAdd(&c.chg[k], 1ull);
                } else {
                    bool viol = false;
                    uint32_t ones = 0;
#pragma unroll
                    for (int q = 0; q < WPL; ++q) {
                        const int w = w0 + G * q;
                        if (!act || w >= I.wp) continue;
                        const uint64_t self = w == (i >> 6) ? 1ull << (i & 63) : 0ull;
                        viol |= (acc[q] | self) != mi[q];
                        ones += __popcll(acc[q]);
                        if (I.out) {
                            if (w < wout) I.out[static_cast<int64_t>(i) * wout + w] = acc[q];
                        } else {
                            I.mbits[static_cast<int64_t>(i) * I.wp + w] = acc[q];
                        }
                    }
                    const bool any = __any_sync(kFull, viol);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) ones += __shfl_xor_sync(kFull, ones, o);
                    if (lane == 0) {
                        if (any) atomicAdd(&c.viol[k], 1ull);
                        if (ones) atomicAdd(&c.ones[k], static_cast<unsigned long long>(ones));
                    }
                }
            }
            r = lim;
            ++j;
        }
    }
}

// e4m3 operands of the listed instances from their bits (warp per padded row, 16 rows per
// claim); an instance's first row counts its squaring.
__global__ void __launch_bounds__(256)
    batch_to_e4m3_kernel(const BatchInst *__restrict__ inst, BatchList list, BatchCounters c) {
    const int lane = threadIdx.x & 31;
    const int nprows = list.hdr[2];
    if (nprows == 0) return;
    const int entries = list.hdr[0];
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int p0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 16; p0 < nprows; p0 += warps * 16) {
        int j = last_le(list.prow, entries, p0);
        for (int p = p0; p < min(nprows, p0 + 16); ++p) {
            while (list.prow[j + 1] <= p) ++j;
            const int k = list.k[j];
            const BatchInst &I = inst[k];
            const int r = p - list.prow[j];
            if (r == 0 && lane == 0) c.squarings[k] += 1;
            const uint64_t *src = I.rbits + static_cast<int64_t>(r) * I.wp;
            uint4 *dst = reinterpret_cast<uint4 *>(I.c0 + static_cast<int64_t>(r) * I.np);
            for (int w = lane; w < I.wp; w += 32) {
                const uint64_t x = src[w];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t o[4];
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const uint32_t nib = static_cast<uint32_t>(x >> (16 * q + 4 * b)) & 0xFu;
                        o[b] = ((nib & 1u) * 0x38u) | (((nib >> 1) & 1u) * 0x3800u) |
                               (((nib >> 2) & 1u) * 0x380000u) | (((nib >> 3) & 1u) * 0x38000000u);
                    }
                    dst[4 * w + q] = make_uint4(o[0], o[1], o[2], o[3]);
                }
            }
        }
    }
}

// After the emission: a certificate that failed is an internal error; all instances retire.
__global__ void decide_final(int count, BatchCounters c, int *status) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    if (c.state[k] == B_EMIT) {
        c.state[k] = B_DONE;
        if (c.viol[k] != 0) atomicOr(status, ST_TIMEOUT_DEP);
    }
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

template <bool EMIT>
void launch_rows(int wpl, int grid, const BatchInst *d, const BatchList &l, const int *ptr, const int *col,
                 const BatchCounters &bc, cudaStream_t s) {
    if (wpl == 1) batch_rows_kernel<1, EMIT><<<grid, 256, 0, s>>>(d, l, ptr, col, bc);
    else if (wpl == 2) batch_rows_kernel<2, EMIT><<<grid, 256, 0, s>>>(d, l, ptr, col, bc);
    else if (wpl == 4) batch_rows_kernel<4, EMIT><<<grid, 256, 0, s>>>(d, l, ptr, col, bc);
    else batch_rows_kernel<8, EMIT><<<grid, 256, 0, s>>>(d, l, ptr, col, bc);
}

}  // namespace

// Cached schedule of the last batch (graph + the buffers it was built on).
struct BatchPlan {
    std::vector<int32_t> ns;
    std::vector<const void *> ins;
    std::vector<void *> outs;
    const void *col = nullptr;
    int mem = -1;
    // main: CSR fill, first sweeps, the first squaring rounds, emission of the converged
    // instances; more: the remaining rounds and their emission (launched only if an instance
    // is still active after main)
    cudaGraphExec_t exec = nullptr, exec_more = nullptr;
    int rounds = 0, rounds_more = 0;
    int launches = 0, launches_more = 0;  // kernels in each graph
    ~BatchPlan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (exec_more) cudaGraphExecDestroy(exec_more);
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
    const int bn = 128;  // GEMM tile width for the batch (small instances waste less padding)
    const int tm = gemm_tile_m();
    std::vector<BatchInst> inst(L);
    int64_t in_bytes = 0, mat_bytes = 0, bit_words = 0, prow = 0, row = 0, max_np = 0, max_wp = 0, tiles = 0,
            wp_words = 0;
    for (int i = 0; i < L; ++i) {
        const int32_t n = ns[live[i]];
        const int64_t np = round_up(n, 128);
        inst[i].n = n;
        inst[i].np = static_cast<int32_t>(np);
        inst[i].wp = static_cast<int32_t>(np / 64);
        inst[i].tiles = static_cast<int32_t>(((np + tm - 1) / tm) * ((np + bn - 1) / bn));
        inst[i].prow0 = static_cast<int32_t>(std::min<int64_t>(prow, INT32_MAX));
        inst[i].row0 = static_cast<int32_t>(std::min<int64_t>(row, INT32_MAX));
        prow += np;
        row += n;
        tiles += inst[i].tiles;
        in_bytes += round_up(static_cast<int64_t>(n) * n, 256);
        mat_bytes += np * np;
        bit_words += np * (np / 64);
        wp_words += np / 64;
        max_np = std::max(max_np, np);
        max_wp = std::max(max_wp, np / 64);
    }
    const int64_t total_prows = prow, total_rows = row;
    if (max_wp > 256) {
        set_error("batch: instances are limited to n <= 16384");
        return DL_EINVAL;
    }
    if (total_prows > (1ll << 31) - 2 || tiles > (1ll << 31) - 1) {
        set_error("batch: too many rows (%lld padded rows)", static_cast<long long>(total_prows));
        return DL_EINVAL;
    }
    const int wpl = max_wp <= 32 ? 1 : max_wp <= 64 ? 2 : max_wp <= 128 ? 4 : 8;
    const int scan_blocks = static_cast<int>((total_rows + 1023) / 1024);
    auto *c0 = static_cast<uint8_t *>(ws.get("batch_c0", mat_bytes));
    auto *rb = static_cast<uint64_t *>(ws.get("batch_rbits", bit_words * 8));
    auto *mb = static_cast<uint64_t *>(ws.get("batch_mbits", bit_words * 8));
    auto *cmask = static_cast<uint64_t *>(ws.get("batch_colmask", std::max<int64_t>(wp_words, 1) * 8));
    auto *ctr = static_cast<unsigned long long *>(ws.get("batch_ctr", kCounterArrays * sizeof(unsigned long long) * L));
    auto *state = static_cast<int *>(ws.get("batch_state", sizeof(int) * L));
    auto *lists = static_cast<int *>(ws.get("batch_list", sizeof(int) * (8 + 3 * (L + 1) + 2 + 2 * L + 1)));
    auto *dinst = static_cast<BatchInst *>(ws.get("batch_inst", sizeof(BatchInst) * L));
    auto *dprob = static_cast<GemmProblem *>(ws.get("batch_probs", sizeof(GemmProblem) * L));
    auto *pinst = static_cast<int *>(ws.get("batch_pinst", sizeof(int) * total_prows));
    auto *gcnt = static_cast<int *>(ws.get("batch_cnt", sizeof(int) * (total_rows + 1)));
    auto *gptr = static_cast<int *>(ws.get("batch_ptr", sizeof(int) * (total_rows + 1)));
    auto *scratch = static_cast<int *>(ws.get("batch_scan", sizeof(int) * 2 * (scan_blocks + 1)));
    uint8_t *staging = nullptr;
    if (mem == DL_MEM_HOST) staging = static_cast<uint8_t *>(ws.get("batch_in", std::max<int64_t>(in_bytes, 256)));
    if (!c0 || !rb || !mb || !cmask || !ctr || !state || !lists || !dinst || !dprob || !pinst || !gcnt || !gptr ||
        !scratch || (mem == DL_MEM_HOST && !staging)) {
        set_error("batch: device allocation failed (%.2f GB of operands)", 1.0 * mat_bytes / 1e9);
        return DL_ENOMEM;
    }
    const BatchCounters bc{state, ctr, ctr + L, ctr + 2 * L, ctr + 3 * L, ctr + 4 * L};
    const BatchList bl{lists, lists + 8, lists + 8 + (L + 1), lists + 8 + 2 * (L + 1), lists + 8 + 3 * (L + 1)};

    cudaEvent_t ev0 = ws.ev[0], ev1 = ws.ev[1];
    BCK(cudaEventRecord(ev0, s));
    int64_t mo = 0, bo = 0, io = 0, co = 0;
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
        inst[i].rbits = rb + bo;
        inst[i].mbits = mb + bo;
        inst[i].out = mem == DL_MEM_DEVICE ? out_bits[k] : nullptr;
        inst[i].colmask = cmask + co;
        co += np / 64;
        mo += np * np;
        bo += np * (np / 64);
    }
    BCK(cudaMemcpyAsync(dinst, inst.data(), sizeof(BatchInst) * L, cudaMemcpyHostToDevice, s));

    // 1. bits of I + E, counts and checks over all inputs, then the CSR row pointers (every
    //    call: the contents, hence the number of facts, may differ between calls)
    BCK(cudaMemsetAsync(ws.status, 0, sizeof(int), s));
    batch_map_kernel<<<L, 256, 0, s>>>(dinst, pinst);
    const unsigned pack_blocks = static_cast<unsigned>((total_prows + 8 * kPackRows - 1) / (8 * kPackRows));
    batch_pack_kernel<<<pack_blocks, 256, 0, s>>>(dinst, pinst, static_cast<int>(total_prows), gcnt, ws.status);
    BCK(cudaGetLastError());
    BCK(exclusive_scan_large(gcnt, static_cast<int>(total_rows), gptr, scratch, s));
    const int pre_launches = 2 + (total_rows > 64 * 1024 ? 3 : 1);
    int nnz_total = 0, hst = 0;
    BCK(cudaMemcpyAsync(&nnz_total, gptr + total_rows, sizeof(int), cudaMemcpyDeviceToHost, s));
    BCK(cudaMemcpyAsync(&hst, ws.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    if (hst & ST_BAD_INPUT) {
        set_error("batch: an input matrix holds a byte that is neither 0 nor 1");
        return DL_EINVAL;
    }
    auto *gcol = static_cast<int *>(ws.get("batch_col", sizeof(int) * static_cast<size_t>(std::max(nnz_total, 1))));
    if (!gcol) {
        set_error("batch: device allocation failed (CSR of %d facts)", nnz_total);
        return DL_ENOMEM;
    }

    // 2. the captured schedule (rebuilt when the buffers change)
    std::vector<int32_t> key_ns(L);
    std::vector<const void *> key_in(L);
    std::vector<void *> key_out(L);
    for (int i = 0; i < L; ++i) {
        key_ns[i] = inst[i].n;
        key_in[i] = inst[i].E;
        key_out[i] = out_bits[live[i]];
    }
    BatchPlan *&plan = ws.batch_plan;
    const bool reuse = plan && plan->mem == static_cast<int>(mem) && plan->ns == key_ns && plan->ins == key_in &&
                       plan->outs == key_out && plan->col == gcol;
    if (!reuse) {
        delete plan;
        plan = nullptr;
        std::vector<GemmProblem> probs(L);
        std::string err;
        int64_t tile0 = 0;
        for (int i = 0; i < L; ++i) {
            const int64_t np = inst[i].np;
            GemmEpilogue e{};
            e.bits = reinterpret_cast<uint32_t *>(inst[i].rbits);  // M <- min1(M^2), bits only
            e.ld_bits32 = 2 * inst[i].wp;
            const Operand op{inst[i].c0, np, np, np, 0, 0};
            GemmProblem &pr = probs[i];
            if (!gemm_make_problem(&pr, KIND_F8, false, bn, static_cast<int>(np), static_cast<int>(np),
                                   static_cast<int>(np), op, op, e, &err)) {
                set_error("batch: %s", err.c_str());
                return DL_EDEVICE;
            }
            pr.tile_start = static_cast<int>(tile0);
            tile0 += pr.tiles_m * pr.tiles_n;
        }
        // pageable source: the copy has read `probs` when cudaMemcpyAsync returns
        BCK(cudaMemcpyAsync(dprob, probs.data(), sizeof(GemmProblem) * L, cudaMemcpyHostToDevice, s));
        BCK(gemm_prepare(KIND_F8, false, bn, EPI_BOOL));
        // instances closed in shared memory by one CTA each
        std::vector<int> small;
        size_t small_smem = 0;
        for (int i = 0; i < L; ++i)
            if (inst[i].np <= kSmallNp) {
                small.push_back(i);
                small_smem = std::max(small_smem, static_cast<size_t>(inst[i].np) * inst[i].wp * 8);
            }
        int *dsmall = nullptr;
        if (!small.empty()) {
            dsmall = static_cast<int *>(ws.get("batch_small", sizeof(int) * small.size()));
            if (!dsmall) {
                set_error("batch: device allocation failed (small-instance list)");
                return DL_ENOMEM;
            }
            BCK(cudaMemcpyAsync(dsmall, small.data(), sizeof(int) * small.size(), cudaMemcpyHostToDevice, s));
            BCK(cudaFuncSetAttribute(batch_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(small_smem)));
        }
        const int rounds = 1 + static_cast<int>(std::ceil(std::log2(static_cast<double>(max_np) + 1.0)));
        const int ggrid = static_cast<int>(std::min<int64_t>(tiles, ctx->sms));
        const int rgrid = ctx->sms * 8;  // row kernels: 8 CTAs of 8 warps per SM, rows claimed in chunks
        const unsigned prow_grid = static_cast<unsigned>((total_prows + 7) / 8);
        int launches = 0;
        auto sweep = [&]() {
            launch_rows<false>(wpl, rgrid, dinst, bl, gptr, gcol, bc, s);
            batch_list_kernel<<<1, kListThreads, 0, s>>>(dinst, L, bc, bl, B_ACTIVE, 1);
            launches += 2;
        };
        const int rounds_main = std::min(rounds, kMainRounds);
        auto round = [&]() {
            batch_to_e4m3_kernel<<<rgrid, 256, 0, s>>>(dinst, bl, bc);
            const cudaError_t e = gemm_launch(KIND_F8, false, bn, EPI_BOOL, dprob, L, static_cast<int>(tiles), ggrid,
                                              ws.status, ctx->budget_ns, s, bl.sched);
            launches += 2;
            for (int k = 0; k < kRoundSweeps; ++k) sweep();
            return e;
        };
        auto emit = [&]() {
            batch_list_kernel<<<1, kListThreads, 0, s>>>(dinst, L, bc, bl, B_EMIT, 0);
            launch_rows<true>(wpl, rgrid, dinst, bl, gptr, gcol, bc, s);
            decide_final<<<(L + 255) / 256, 256, 0, s>>>(L, bc, ws.status);
            launches += 3;
        };
        // capture one schedule; body() issues its launches and returns the first error
        auto capture = [&](auto body, cudaGraphExec_t *out) -> dl_status {
            cudaGraph_t graph = nullptr;
            BCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = body();
            if (e == cudaSuccess) e = cudaGetLastError();
            const cudaError_t ec = cudaStreamEndCapture(s, &graph);
            if (e != cudaSuccess || ec != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
                set_error("batch: stream capture failed (%s)", cudaGetErrorString(e != cudaSuccess ? e : ec));
                return DL_EDEVICE;
            }
            const cudaError_t ei = cudaGraphInstantiate(out, graph, 0);
            cudaGraphDestroy(graph);
            if (ei != cudaSuccess) {
                set_error("batch: graph instantiation failed (%s)", cudaGetErrorString(ei));
                return DL_EDEVICE;
            }
            return DL_OK;
        };
        plan = new BatchPlan();
        plan->ns = key_ns;
        plan->ins = key_in;
        plan->outs = key_out;
        plan->col = gcol;
        plan->mem = static_cast<int>(mem);
        dl_status rc = capture(
            [&]() -> cudaError_t {
                cudaError_t e = cudaMemsetAsync(state, 0, sizeof(int) * L, s);
                if (e == cudaSuccess) e = cudaMemsetAsync(ctr, 0, kCounterArrays * sizeof(unsigned long long) * L, s);
                batch_fill_kernel<<<prow_grid, 256, 0, s>>>(dinst, pinst, static_cast<int>(total_prows), gptr, gcol);
                batch_colmask_kernel<<<L, 256, static_cast<size_t>(max_wp) * 8, s>>>(dinst, gptr, gcol);
                if (!small.empty()) {
                    batch_small_kernel<<<static_cast<unsigned>(small.size()), kSmallThreads, small_smem, s>>>(
                        dinst, dsmall, gptr, gcol, bc, ws.status);
                    ++launches;
                }
                batch_list_kernel<<<1, kListThreads, 0, s>>>(dinst, L, bc, bl, B_ACTIVE, 0);
                launches += 3;
                for (int k = 0; k < kFirstSweeps; ++k) sweep();
                for (int r = 0; r < rounds_main && e == cudaSuccess; ++r) e = round();
                emit();
                return e;
            },
            &plan->exec);
        plan->rounds = rounds_main;
        plan->launches = launches;
        launches = 0;
        if (rc == DL_OK && rounds > rounds_main)
            rc = capture(
                [&]() -> cudaError_t {
                    batch_list_kernel<<<1, kListThreads, 0, s>>>(dinst, L, bc, bl, B_ACTIVE, 0);
                    ++launches;
                    cudaError_t e = cudaSuccess;
                    for (int r = rounds_main; r < rounds && e == cudaSuccess; ++r) e = round();
                    emit();
                    return e;
                },
                &plan->exec_more);
        plan->rounds_more = rounds - rounds_main;
        plan->launches_more = launches;
        if (rc != DL_OK) {
            delete plan;
            plan = nullptr;
            return rc;
        }
    }
    BCK(cudaGraphLaunch(plan->exec, s));
    std::vector<int> hstate(L);
    BCK(cudaMemcpyAsync(hstate.data(), state, sizeof(int) * L, cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    const bool more = std::any_of(hstate.begin(), hstate.end(), [](int x) { return x == B_ACTIVE; });
    if (more && plan->exec_more) BCK(cudaGraphLaunch(plan->exec_more, s));
    if (mem == DL_MEM_HOST) {
        for (int i = 0; i < L; ++i) {
            const int64_t n = inst[i].n, w = (n + 63) / 64;
            BCK(cudaMemcpy2DAsync(out_bits[live[i]], w * 8, inst[i].mbits, inst[i].wp * 8, w * 8, n,
                                  cudaMemcpyDeviceToHost, s));
        }
    }
    BCK(cudaEventRecord(ev1, s));
    std::vector<unsigned long long> hctr(kCounterArrays * static_cast<size_t>(L));
    BCK(cudaMemcpyAsync(hstate.data(), state, sizeof(int) * L, cudaMemcpyDeviceToHost, s));
    BCK(cudaMemcpyAsync(hctr.data(), ctr, sizeof(unsigned long long) * kCounterArrays * L, cudaMemcpyDeviceToHost,
                        s));
    BCK(cudaMemcpyAsync(&hst, ws.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    if (hst) {
        set_error("batch: device status 0x%x (a wait expired or a certificate failed)", hst);
        return DL_ETIMEOUT;
    }
    int max_sq = 0, max_sw = 0;
    int64_t ones = 0;
    double flops = 0.0;
    for (int i = 0; i < L; ++i) {
        if (hstate[i] != B_DONE) {
            set_error("batch: instance %d did not converge", live[i]);
            return DL_ENOTCONV;
        }
        const int sq = static_cast<int>(hctr[3 * L + i]);
        max_sq = std::max(max_sq, sq);
        max_sw = std::max(max_sw, static_cast<int>(hctr[4 * L + i]));
        ones += static_cast<int64_t>(hctr[2 * L + i]);
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
        st->path_used = DL_PATH_AUTO;
        st->iters = max_sq;
        st->recheck_sweeps = max_sw;
        st->model_ones = ones;
        st->ms_total = ms;
        st->ms_solve = ms;
        st->tflops_equiv = ms > 0 ? equiv / (ms * 1e-3) / 1e12 : 0.0;
        st->gemm_launches = plan->rounds + (more ? plan->rounds_more : 0);
        st->gemm_flops = flops;
        st->gpu_launches = pre_launches + plan->launches + (more ? plan->launches_more : 0);
    }
    return DL_OK;
}

void batch_plan_release(BatchPlan *p) { delete p; }

}  // namespace dl
