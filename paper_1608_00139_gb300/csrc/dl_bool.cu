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
