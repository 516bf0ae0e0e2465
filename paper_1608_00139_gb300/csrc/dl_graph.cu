// dl_graph.cu -- graph utilities on the device: the CSR (successor lists) of a dense 0/1
// matrix, used by the FP64 residual of the mixed path and by the boolean sweeps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "dl_internal.h"
#include "dl_rows.cuh"

namespace dl {

namespace {

// Successor counts, one warp per row (16-byte loads when rows are 16-byte aligned).  Bytes are
// 0/1 (validated by the ingest); the low bit is the fact.
__global__ void csr_count_kernel(const uint8_t *__restrict__ E, int n, int *cnt) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    const uint8_t *row = E + static_cast<int64_t>(i) * n;
    int c = 0;
    if ((n & 15) == 0 && (reinterpret_cast<uintptr_t>(E) & 15) == 0) {
        const uint4 *r4 = reinterpret_cast<const uint4 *>(row);
        for (int q = lane; q < n / 16; q += 32) {
            const uint4 x = r4[q];
            c += __popc(x.x & 0x01010101u) + __popc(x.y & 0x01010101u) + __popc(x.z & 0x01010101u) +
                 __popc(x.w & 0x01010101u);
        }
    } else {
        for (int j = lane; j < n; j += 32) c += row[j] & 1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[i] = c;
}

// One pass over E (warp per padded row): bits of I + E into M, successor counts, the 0/1
// check, ||E||_inf (max row count), nnz and the number of self-loops.
__global__ void __launch_bounds__(256, 4)
    csr_pack_check_kernel(const uint8_t *__restrict__ E, int n, int np, int wp, int *cnt, uint64_t *M,
                          unsigned long long *dmax, unsigned long long *nnz, unsigned long long *diag,
                          int *status, uint64_t *colmask) {
    extern __shared__ uint64_t colmask_s[];  // the CTA's rows' facts, merged into colmask at the end
    for (int w = threadIdx.x; w < wp; w += blockDim.x) colmask_s[w] = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    uint64_t *row = M + static_cast<int64_t>(r) * wp;
    if (r >= n && r < np) {  // padding: identity only
        for (int w = lane; w < wp; w += 32) row[w] = w == (r >> 6) ? 1ull << (r & 63) : 0ull;
    } else if (r < n) {
        const uint8_t *a = E + static_cast<int64_t>(r) * n;
        int c = 0;
        bool bad = false;
        pack_row_bits(a, n, r, wp, row, lane, c, bad, colmask_s);
        if (lane == 0) {
            cnt[r] = c;
            if (bad) atomicOr(status, ST_BAD_INPUT);
            if (c) {
                atomicMax(dmax, static_cast<unsigned long long>(c));
                atomicAdd(nnz, static_cast<unsigned long long>(c));
            }
            if (a[r] & 1) atomicAdd(diag, 1ull);
        }
    }
    __syncthreads();
    for (int w = threadIdx.x; w < wp; w += blockDim.x)
        if (colmask_s[w] != 0ull) atomicOr(reinterpret_cast<unsigned long long *>(colmask + w), colmask_s[w]);
}

// The same outputs from a bit-packed E: row r is ceil(n/64) words at Eb + r ceil(n/64), bit
// (j mod 64) of word j/64 holding E[r][j].  A set bit at a column >= n is an input error
// (ST_BAD_PAD) and is dropped.  Warp per padded row, a word per lane and step (coalesced).
__global__ void __launch_bounds__(256, 4)
    bits_ingest_check_kernel(const uint64_t *__restrict__ Eb, int n, int np, int wp, int *cnt, uint64_t *M,
                             unsigned long long *dmax, unsigned long long *nnz, unsigned long long *diag,
                             int *status, uint64_t *colmask) {
    extern __shared__ uint64_t colmask_s[];
    for (int w = threadIdx.x; w < wp; w += blockDim.x) colmask_s[w] = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    uint64_t *row = M + static_cast<int64_t>(r) * wp;
    const int idw = r >> 6;
    const uint64_t idb = 1ull << (r & 63);
    if (r >= n && r < np) {
        for (int w = lane; w < wp; w += 32) row[w] = w == idw ? idb : 0ull;
    } else if (r < n) {
        const int w_in = (n + 63) >> 6;
        const uint64_t *a = Eb + static_cast<int64_t>(r) * w_in;
        const uint64_t last = (n & 63) ? (1ull << (n & 63)) - 1ull : ~0ull;  // columns < n of the last word
        int c = 0;
        bool bad = false, self = false;
        for (int w = lane; w < wp; w += 32) {
            uint64_t e = w < w_in ? a[w] : 0ull;
            if (w == w_in - 1) {
                bad = (e & ~last) != 0ull;
                e &= last;
            }
            if (w == idw) self = (e & idb) != 0ull;
            c += __popcll(e);
            if (e != 0ull) atomicOr(reinterpret_cast<unsigned long long *>(colmask_s + w), e);
            row[w] = e | (w == idw ? idb : 0ull);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        bad = __any_sync(0xffffffffu, bad);
        self = __any_sync(0xffffffffu, self);
        if (lane == 0) {
            cnt[r] = c;
            if (bad) atomicOr(status, ST_BAD_PAD);
            if (c) {
                atomicMax(dmax, static_cast<unsigned long long>(c));
                atomicAdd(nnz, static_cast<unsigned long long>(c));
            }
            if (self) atomicAdd(diag, 1ull);
        }
    }
    __syncthreads();
    for (int w = threadIdx.x; w < wp; w += blockDim.x)
        if (colmask_s[w] != 0ull) atomicOr(reinterpret_cast<unsigned long long *>(colmask + w), colmask_s[w]);
}

// Byte (b) of a bit-packed row spread over 8 bytes, bit k to the low bit of byte k: the four
// high bits move up 28 places, then pairs 14, then single bits 7.
__device__ __forceinline__ uint64_t spread_byte(uint64_t b) {
    b = (b | (b << 28)) & 0x0000000F0000000Full;
    b = (b | (b << 14)) & 0x0003000300030003ull;
    return (b | (b << 7)) & 0x0101010101010101ull;
}

// Bytes of a bit-packed E (n x n, row-major): thread per 8 columns of a row; 8-byte stores
// when rows are 8-byte aligned, else byte stores.  The first thread of a row checks the bits
// at columns >= n (ST_BAD_PAD).
__global__ void __launch_bounds__(256) unpack_bits_u8_kernel(const uint64_t *__restrict__ Eb, int n, uint8_t *E,
                                                             int *status) {
    const int w_in = (n + 63) >> 6;
    const int64_t groups = (static_cast<int64_t>(n) + 7) >> 3;
    const int64_t total = groups * n;
    const bool aligned = (n & 7) == 0 && (reinterpret_cast<uintptr_t>(E) & 7) == 0;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = t / groups;
        const int g = static_cast<int>(t - r * groups);
        const uint64_t word = Eb[r * w_in + (g >> 3)];
        if (g == 0 && (n & 63) != 0) {
            const uint64_t tail = Eb[r * w_in + w_in - 1] >> (n & 63);
            if (tail != 0ull) atomicOr(status, ST_BAD_PAD);
        }
        const uint64_t v = spread_byte((word >> (8 * (g & 7))) & 0xFFull);
        uint8_t *dst = E + r * n + 8 * static_cast<int64_t>(g);
        if (aligned) {
            *reinterpret_cast<uint64_t *>(dst) = v;
        } else {
            const int m = min(8, n - 8 * g);
            for (int k = 0; k < m; ++k) dst[k] = static_cast<uint8_t>((v >> (8 * k)) & 1ull);
        }
    }
}

// Column indices from the packed bits.  Guarded form (cap >= 0): every thread first reads the
// number of facts and ||E||_inf; if the facts do not fit cap entries or a row has more than
// max_deg successors nothing is written and *gate = 1 (a later step re-plans on the host).
__global__ void __launch_bounds__(256)
    csr_fill_bits_kernel(const uint64_t *__restrict__ M, int n, int wp, const int *__restrict__ ptr, int *col,
                         int64_t cap, const unsigned long long *dmax, int max_deg, int *gate) {
    if (cap >= 0) {
        const bool stop = ptr[n] > cap || *dmax > static_cast<unsigned long long>(max_deg);
        if (blockIdx.x == 0 && threadIdx.x == 0) *gate = stop ? 1 : 0;
        if (stop) return;
    }
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= n) return;
    fill_row_from_bits(M + static_cast<int64_t>(r) * wp, wp, r, ptr[r], ptr[r + 1], col, lane);
}

// Bits of E alone (no identity; rows >= n zero), the 0/1 check; warp per padded row.
__global__ void __launch_bounds__(256, 4)
    pack_bits_kernel(const uint8_t *__restrict__ E, int n, int np, int wp, uint64_t *M, int *status) {
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= np) return;
    uint64_t *row = M + static_cast<int64_t>(r) * wp;
    if (r >= n) {
        for (int w = lane; w < wp; w += 32) row[w] = 0ull;
        return;
    }
    int c = 0;
    bool bad = false;
    pack_row_bits(E + static_cast<int64_t>(r) * n, n, r, wp, row, lane, c, bad, nullptr, false);
    if (lane == 0 && bad) atomicOr(status, ST_BAD_INPUT);
}

// Exclusive scan in one CTA: each thread holds 16 consecutive counts in registers, a warp
// scan and a scan of the warp totals place them; long inputs go round in tiles of 16384.
__global__ void __launch_bounds__(1024) exclusive_scan_kernel(const int *cnt, int n, int *ptr) {
    __shared__ int warp_tot[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool vec = (reinterpret_cast<uintptr_t>(cnt) & 15) == 0;
    int carry = 0;
    for (int base = 0; base < n; base += 1024 * 16) {
        const int b = base + static_cast<int>(threadIdx.x) * 16;
        int v[16];
        if (vec && b + 16 <= n) {
            const int4 *c4 = reinterpret_cast<const int4 *>(cnt + b);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int4 x = c4[q];
                v[4 * q] = x.x;
                v[4 * q + 1] = x.y;
                v[4 * q + 2] = x.z;
                v[4 * q + 3] = x.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = b + j < n ? cnt[b + j] : 0;
        }
        int sum = 0;
#pragma unroll
        for (int j = 0; j < 16; ++j) sum += v[j];
        int inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) warp_tot[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            int w = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            warp_tot[lane] = w;
        }
        __syncthreads();
        int run = carry + (warp > 0 ? warp_tot[warp - 1] : 0) + inc - sum;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (b + j < n) ptr[b + j] = run;
            run += v[j];
        }
        carry += warp_tot[31];
        __syncthreads();  // warp_tot is rewritten by the next tile
    }
    if (threadIdx.x == 0) ptr[n] = carry;
}

// Column indices in increasing order, one warp per row: each lane takes 16 bytes of a
// 512-byte chunk, a warp prefix sum of the lanes' counts places its indices.
__global__ void csr_fill_kernel(const uint8_t *__restrict__ E, int n, const int *__restrict__ ptr, int *col) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    const uint8_t *row = E + static_cast<int64_t>(i) * n;
    const bool vec = (n & 15) == 0 && (reinterpret_cast<uintptr_t>(E) & 15) == 0;
    int base = ptr[i];
    for (int c0 = 0; c0 < n; c0 += 512) {
        const int j0 = c0 + 16 * lane;
        uint32_t m = 0;
        if (vec) {
            if (j0 < n) {
                const uint4 x = *reinterpret_cast<const uint4 *>(row + j0);
                const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int b = 0; b < 4; ++b) m |= ((w[q] >> (8 * b)) & 1u) << (4 * q + b);
            }
        } else {
#pragma unroll
            for (int t = 0; t < 16; ++t)
                if (j0 + t < n && (row[j0 + t] & 1)) m |= 1u << t;
        }
        const int cnt = __popc(m);
        int pre = cnt;  // inclusive warp scan
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= o) pre += v;
        }
        int pos = base + pre - cnt;
        while (m) {
            const int t = __ffs(m) - 1;
            m &= m - 1;
            col[pos++] = j0 + t;
        }
        base += __shfl_sync(0xffffffffu, pre, 31);
    }
}

}  // namespace

cudaError_t csr_build(const uint8_t *E, int n, int *cnt, int *ptr, cudaStream_t s) {
    csr_count_kernel<<<static_cast<unsigned>((n + 7) / 8), 256, 0, s>>>(E, n, cnt);
    exclusive_scan_kernel<<<1, 1024, 0, s>>>(cnt, n, ptr);
    return cudaGetLastError();
}

cudaError_t csr_pack_checked(const uint8_t *E, int n, int np, int64_t wp, int *cnt, int *ptr, uint64_t *M,
                             unsigned long long *dmax, unsigned long long *nnz, unsigned long long *diag, int *status,
                             uint64_t *colmask, cudaStream_t s) {
    if (wp > 6144) return cudaErrorInvalidValue;  // the CTA's column mask lives in shared memory
    const size_t smem = static_cast<size_t>(wp) * sizeof(uint64_t);
    csr_pack_check_kernel<<<static_cast<unsigned>((np + 7) / 8), 256, smem, s>>>(
        E, n, np, static_cast<int>(wp), cnt, M, dmax, nnz, diag, status, colmask);
    exclusive_scan_kernel<<<1, 1024, 0, s>>>(cnt, n, ptr);
    return cudaGetLastError();
}

cudaError_t bits_ingest_checked(const uint64_t *Eb, int n, int np, int64_t wp, int *cnt, int *ptr, uint64_t *M,
                                unsigned long long *dmax, unsigned long long *nnz, unsigned long long *diag,
                                int *status, uint64_t *colmask, cudaStream_t s) {
    if (wp > 6144) return cudaErrorInvalidValue;  // the CTA's column mask lives in shared memory
    const size_t smem = static_cast<size_t>(wp) * sizeof(uint64_t);
    bits_ingest_check_kernel<<<static_cast<unsigned>((np + 7) / 8), 256, smem, s>>>(
        Eb, n, np, static_cast<int>(wp), cnt, M, dmax, nnz, diag, status, colmask);
    exclusive_scan_kernel<<<1, 1024, 0, s>>>(cnt, n, ptr);
    return cudaGetLastError();
}

cudaError_t unpack_bits_u8(const uint64_t *Eb, int n, uint8_t *E, int *status, cudaStream_t s) {
    const int64_t total = ((static_cast<int64_t>(n) + 7) >> 3) * n;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 16);
    unpack_bits_u8_kernel<<<static_cast<unsigned>(std::max<int64_t>(blocks, 1)), 256, 0, s>>>(Eb, n, E, status);
    return cudaGetLastError();
}

cudaError_t pack_bits(const uint8_t *E, int n, int np, int64_t wp, uint64_t *M, int *status, cudaStream_t s) {
    pack_bits_kernel<<<static_cast<unsigned>((np + 7) / 8), 256, 0, s>>>(E, n, np, static_cast<int>(wp), M, status);
    return cudaGetLastError();
}

cudaError_t csr_fill_from_bits(const uint64_t *M, int n, int64_t wp, const int *ptr, int *col, cudaStream_t s) {
    csr_fill_bits_kernel<<<static_cast<unsigned>((n + 7) / 8), 256, 0, s>>>(M, n, static_cast<int>(wp), ptr, col, -1,
                                                                           nullptr, 0, nullptr);
    return cudaGetLastError();
}

cudaError_t csr_fill_from_bits_guarded(const uint64_t *M, int n, int64_t wp, const int *ptr, int *col, int64_t cap,
                                       const unsigned long long *dmax, int max_deg, int *gate, cudaStream_t s) {
    csr_fill_bits_kernel<<<static_cast<unsigned>((n + 7) / 8), 256, 0, s>>>(M, n, static_cast<int>(wp), ptr, col, cap,
                                                                           dmax, max_deg, gate);
    return cudaGetLastError();
}

// Two-level scan for long arrays: block sums of 1024 elements, a scan of those sums (the
// single-CTA kernel), then every block rescans its elements from its offset.
__global__ void __launch_bounds__(1024) block_sums_kernel(const int *cnt, int n, int *sums) {
    __shared__ int part[32];
    const int i = blockIdx.x * 1024 + threadIdx.x;
    int v = i < n ? cnt[i] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        int w = part[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (threadIdx.x == 0) sums[blockIdx.x] = w;
    }
}

__global__ void __launch_bounds__(1024) block_scan_kernel(const int *cnt, int n, const int *offs, int *out) {
    __shared__ int part[32];
    const int i = blockIdx.x * 1024 + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int v = i < n ? cnt[i] : 0;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) part[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = part[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        part[lane] = w;  // inclusive prefix of warp totals
    }
    __syncthreads();
    const int before = offs[blockIdx.x] + (warp > 0 ? part[warp - 1] : 0) + inc - v;
    if (i < n) out[i] = before;
    if (i == n - 1) out[n] = before + v;
}

cudaError_t exclusive_scan(const int *cnt, int n, int *out, cudaStream_t s) {
    exclusive_scan_kernel<<<1, 1024, 0, s>>>(cnt, n, out);
    return cudaGetLastError();
}

cudaError_t exclusive_scan_large(const int *cnt, int n, int *out, int *scratch, cudaStream_t s) {
    if (n <= 64 * 1024) return exclusive_scan(cnt, n, out, s);
    const int blocks = (n + 1023) / 1024;  // scratch: 2 * (blocks + 1) ints
    block_sums_kernel<<<blocks, 1024, 0, s>>>(cnt, n, scratch);
    exclusive_scan_kernel<<<1, 1024, 0, s>>>(scratch, blocks, scratch + blocks + 1);
    block_scan_kernel<<<blocks, 1024, 0, s>>>(cnt, n, scratch + blocks + 1, out);
    return cudaGetLastError();
}

cudaError_t csr_fill(const uint8_t *E, int n, const int *ptr, int *col, cudaStream_t s) {
    csr_fill_kernel<<<static_cast<unsigned>((n + 7) / 8), 256, 0, s>>>(E, n, ptr, col);
    return cudaGetLastError();
}

}  // namespace dl
