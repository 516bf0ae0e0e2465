// dl_graph.cu -- graph utilities on the device: the CSR (successor lists) of a dense 0/1
// matrix, used by the FP64 residual of the mixed path and by the boolean sweeps.
#include <cuda_runtime.h>

#include <cstdint>

#include "dl_internal.h"

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

__global__ void __launch_bounds__(1024) exclusive_scan_kernel(const int *cnt, int n, int *ptr) {
    __shared__ int part[1024];
    const int t = threadIdx.x;
    const int chunk = (n + 1023) / 1024;
    const int b = t * chunk, e = min(n, b + chunk);
    int s = 0;
    for (int i = b; i < e; ++i) s += cnt[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive Hillis-Steele scan of the partial sums
        const int v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = t > 0 ? part[t - 1] : 0;
    for (int i = b; i < e; ++i) {
        ptr[i] = run;
        run += cnt[i];
    }
    if (t == 1023) ptr[n] = part[1023];
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

cudaError_t exclusive_scan(const int *cnt, int n, int *out, cudaStream_t s) {
    exclusive_scan_kernel<<<1, 1024, 0, s>>>(cnt, n, out);
    return cudaGetLastError();
}

cudaError_t csr_fill(const uint8_t *E, int n, const int *ptr, int *col, cudaStream_t s) {
    csr_fill_kernel<<<static_cast<unsigned>((n + 7) / 8), 256, 0, s>>>(E, n, ptr, col);
    return cudaGetLastError();
}

}  // namespace dl
