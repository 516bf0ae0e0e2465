// dl_sgreal.cu -- kernels of the real least solution S~ of the same-generation equation
// (Sec. 7.2; the two-sided class of Sec. 6.3):
//     S~ = eps (B + P S~ P^T),   eps = 1 / (1 + ||P||_inf^2).
// One step of the fixpoint series X <- eps (B + P X P^T) is two gather passes over the CSR of P
// in FP64 (U = X P^T, then eps (B + P U)); the same passes give the residual
// eps (B + P X P^T) - X of the refinement.  The FP32 helpers serve Smith's doubling for the
// Stein equation on the TF32 tensor cores (the GEMMs themselves are dl_umma.cu's).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "dl_internal.h"

namespace dl {

namespace {

// Bound on the change of a series step without FP64 arithmetic.  The series is monotone in
// floating point too (every operation is monotone on non-negative values), so v >= x and
// k = bits(v) - bits(x) >= 0 counts the doubles between them; then v - x < 2^(bitlength(k) +
// exponent(v) - 1075).  Returned as that power plus 4096 (0: no change), for an integer max.
__device__ __forceinline__ unsigned long long change_code(double v, double x) {
    const long long bv = __double_as_longlong(v), bx = __double_as_longlong(x);
    long long k = bv - bx;
    if (k == 0) return 0ull;
    if (k < 0) k = -k;  // not reached by the series; kept as a bound
    const int ev = static_cast<int>((bv >> 52) & 0x7FF);
    return static_cast<unsigned long long>((64 - __clzll(k)) + max(ev, 1) - 1075 + 4096);
}

// U = X P^T:  U[i][j] = sum_{w : P[j][w] = 1} X[i][w].  One block per row i, the row staged in
// shared memory; rows and columns >= n are zero.
__global__ void __launch_bounds__(256) sg_xpt_kernel(const int *__restrict__ ptr, const int *__restrict__ col, int n,
                                                     int np, const double *__restrict__ X, double *__restrict__ U) {
    extern __shared__ double xs[];
    const int i = blockIdx.x;
    const double *xr = X + static_cast<int64_t>(i) * np;
    for (int t = threadIdx.x; t < np; t += blockDim.x) xs[t] = xr[t];
    __syncthreads();
    double *ur = U + static_cast<int64_t>(i) * np;
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
        double s = 0.0;
        if (i < n && j < n) {
            const int q1 = ptr[j + 1];
            for (int q = ptr[j]; q < q1; ++q) s += xs[col[q]];
        }
        ur[j] = s;
    }
}

// V[i][j] = eps (B[i][j] + sum_{y : P[i][y] = 1} U[y][j])  (B = NULL: the identity), and
// D = V - X.  Xn (optional) <- V (a series step); R (optional, FP32) <- D (the residual).
// With R: *dmax = max |D| as the bit pattern of a non-negative double; without: *dmax = the
// max of change_code(V, X).
// Grid: x over columns (256 per block), y over rows.
__global__ void __launch_bounds__(256) sg_pu_kernel(const int *__restrict__ ptr, const int *__restrict__ col, int n,
                                                    int np, double eps, const uint8_t *__restrict__ B,
                                                    const double *__restrict__ U, const double *__restrict__ X,
                                                    double *__restrict__ Xn, float *__restrict__ R,
                                                    unsigned long long *dmax) {
    const int i = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long m = 0;
    if (j < np) {
        double v = 0.0;
        if (i < n && j < n) {
            double s = B != nullptr ? static_cast<double>(B[static_cast<int64_t>(i) * n + j] & 1) : (i == j ? 1.0 : 0.0);
            const int q1 = ptr[i + 1];
            for (int q = ptr[i]; q < q1; ++q) s += U[static_cast<int64_t>(col[q]) * np + j];
            v = eps * s;
        }
        const int64_t at = static_cast<int64_t>(i) * np + j;
        if (R != nullptr) {  // the residual: the real difference
            const double d = v - X[at];
            R[at] = static_cast<float>(d);
            m = static_cast<unsigned long long>(__double_as_longlong(d)) & 0x7FFFFFFFFFFFFFFFull;  // |d|
        } else {
            m = change_code(v, X[at]);
        }
        if (Xn != nullptr) Xn[at] = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, m, o);
        m = other > m ? other : m;
    }
    if ((threadIdx.x & 31) == 0 && m != 0) atomicMax(dmax, m);
}

constexpr int kFusedMaxNp = 16384;  // 1024 threads x 16 columns

// The same step in one pass when every node has few parents:
//   V[i][j] = eps ([B_ij] + sum_{y in P_i} sum_{w in P_j} X[y][w]).
// One block per row i; the rows y of X (the parents of i) go through shared memory one at a
// time and each thread keeps the sums of its columns j = t + THREADS c in registers (512 x 8
// up to np = 4096, two blocks per SM; else 1024 x 16).  A sum starts
// from its first term (no 0 + x) and B's term is added only where it is 1, so a column with one
// parent pair costs one FP64 multiply.
template <int THREADS, int COLS>
__global__ void __launch_bounds__(THREADS)
    sg_fused_kernel(const int *__restrict__ ptr, const int *__restrict__ col, int n, int np, double eps,
                    const uint8_t *__restrict__ B, const double *__restrict__ X, double *__restrict__ Xn,
                    float *__restrict__ R, unsigned long long *dmax) {
    extern __shared__ double xs[];
    const int i = blockIdx.x;
    double acc[COLS];
    unsigned started = 0;  // bit c: column c's sum has a term
#pragma unroll
    for (int c = 0; c < COLS; ++c) acc[c] = 0.0;
    const int q0 = i < n ? ptr[i] : 0, q1 = i < n ? ptr[i + 1] : 0;
    for (int q = q0; q < q1; ++q) {  // parents y of i (block-uniform)
        const double *xr = X + static_cast<int64_t>(col[q]) * np;
        __syncthreads();
        for (int t = threadIdx.x; t < np; t += THREADS) xs[t] = xr[t];
        __syncthreads();
#pragma unroll
        for (int c = 0; c < COLS; ++c) {
            const int j = threadIdx.x + c * THREADS;
            if (j >= n) break;
            int w = ptr[j];
            const int w1 = ptr[j + 1];
            if (w < w1 && !((started >> c) & 1)) {  // a first term is assigned, not added to 0
                acc[c] = xs[col[w]];
                started |= 1u << c;
                ++w;
            }
            for (; w < w1; ++w) acc[c] += xs[col[w]];
        }
    }
    unsigned long long m = 0;
#pragma unroll
    for (int c = 0; c < COLS; ++c) {
        const int j = threadIdx.x + c * THREADS;
        if (j >= np) break;
        double v = 0.0;
        if (i < n && j < n) {
            const bool b = B != nullptr ? (B[static_cast<int64_t>(i) * n + j] & 1) != 0 : i == j;
            double s = acc[c];
            if (b) s = (started >> c) & 1 ? s + 1.0 : 1.0;
            v = eps * s;
        }
        const int64_t at = static_cast<int64_t>(i) * np + j;
        if (Xn != nullptr) Xn[at] = v;
        if (R != nullptr) {  // the residual: the real difference
            const double d = v - X[at];
            R[at] = static_cast<float>(d);
            const unsigned long long ad = static_cast<unsigned long long>(__double_as_longlong(d)) & 0x7FFFFFFFFFFFFFFFull;
            m = ad > m ? ad : m;
        } else if (dmax != nullptr) {  // a series step: the integer bound
            const unsigned long long cc = change_code(v, X[at]);
            m = cc > m ? cc : m;
        }
    }
    if (dmax != nullptr) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, m, o);
            m = other > m ? other : m;
        }
        if ((threadIdx.x & 31) == 0 && m != 0) atomicMax(dmax, m);
    }
}

// A = s P (FP32, np x np, zero padding) and NA = -A.
__global__ void sg_scaled_p_kernel(const uint8_t *__restrict__ P, int n, int np, float s, float *__restrict__ A,
                                   float *__restrict__ NA) {
    const int64_t total = static_cast<int64_t>(np) * np;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = t / np, j = t - i * np;
        const float v = (i < n && j < n && (P[i * n + j] & 1)) ? s : 0.0f;
        A[t] = v;
        NA[t] = -v;
    }
}

// *out = max over rows of sum_j |A[i][j]| (FP32 bit patterns of non-negative sums, atomicMax).
__global__ void __launch_bounds__(256) row_abs_sum_max_kernel(const float *__restrict__ A, int np, unsigned *out) {
    __shared__ float part[8];
    const int i = blockIdx.x;
    float s = 0.0f;
    for (int j = threadIdx.x; j < np; j += blockDim.x) s += fabsf(A[static_cast<int64_t>(i) * np + j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += part[w];
        atomicMax(out, __float_as_uint(t));
    }
}

__global__ void negate_f32_kernel(const float *__restrict__ a, float *__restrict__ b, int64_t count) {
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < count;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x)
        b[t] = -a[t];
}

__global__ void add_f32_to_f64_kernel(double *__restrict__ x, const float *__restrict__ d, int64_t count) {
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < count;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x)
        x[t] += static_cast<double>(d[t]);
}

__global__ void bits_or_kernel(uint64_t *__restrict__ dst, const uint64_t *__restrict__ src, int64_t words) {
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < words;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x)
        dst[t] |= src[t];
}

constexpr int kTT = 32;

// dst[c][r] = src[r][c] for an rows x cols block (32 x 32 tiles through shared memory).
template <class T>
__global__ void transpose_tile_kernel(const T *__restrict__ src, int64_t lds, int rows, int cols, T *__restrict__ dst,
                                      int64_t ldd) {
    __shared__ T tile[kTT][kTT + 1];
    const int c0 = blockIdx.x * kTT, r0 = blockIdx.y * kTT;
    for (int y = threadIdx.y; y < kTT; y += blockDim.y) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[y][threadIdx.x] = src[static_cast<int64_t>(r) * lds + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < kTT; y += blockDim.y) {
        const int c = c0 + y, r = r0 + threadIdx.x;
        if (r < rows && c < cols) dst[static_cast<int64_t>(c) * ldd + r] = tile[threadIdx.x][y];
    }
}

unsigned stream_blocks(int64_t count) {
    return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, 152 * 32)));
}

}  // namespace

bool sg_real_fused(int np, unsigned long long max_parents) {
    return np <= kFusedMaxNp && max_parents <= 4;
}

cudaError_t sg_real_step(const int *ptr, const int *col, int n, int np, double eps, const uint8_t *B, const double *X,
                         double *U, double *Xn, float *R, unsigned long long *dmax, bool fused, cudaStream_t s) {
    const size_t smem = sizeof(double) * static_cast<size_t>(np);
    if (fused && np <= 4096) {
        cudaError_t e = cudaFuncSetAttribute(sg_fused_kernel<512, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        sg_fused_kernel<512, 8><<<static_cast<unsigned>(np), 512, smem, s>>>(ptr, col, n, np, eps, B, X, Xn, R, dmax);
        return cudaGetLastError();
    }
    if (fused) {
        cudaError_t e = cudaFuncSetAttribute(sg_fused_kernel<1024, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        sg_fused_kernel<1024, 16><<<static_cast<unsigned>(np), 1024, smem, s>>>(ptr, col, n, np, eps, B, X, Xn, R,
                                                                               dmax);
        return cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(sg_xpt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    sg_xpt_kernel<<<static_cast<unsigned>(np), 256, smem, s>>>(ptr, col, n, np, X, U);
    dim3 grid(static_cast<unsigned>((np + 255) / 256), static_cast<unsigned>(np));
    sg_pu_kernel<<<grid, 256, 0, s>>>(ptr, col, n, np, eps, B, U, X, Xn, R, dmax);
    return cudaGetLastError();
}

cudaError_t sg_scaled_p(const uint8_t *P, int n, int np, float scale, float *A, float *NA, cudaStream_t s) {
    sg_scaled_p_kernel<<<stream_blocks(static_cast<int64_t>(np) * np), 256, 0, s>>>(P, n, np, scale, A, NA);
    return cudaGetLastError();
}

cudaError_t row_abs_sum_max(const float *A, int np, unsigned *out, cudaStream_t s) {
    row_abs_sum_max_kernel<<<static_cast<unsigned>(np), 256, 0, s>>>(A, np, out);
    return cudaGetLastError();
}

cudaError_t negate_f32(const float *a, float *b, int64_t count, cudaStream_t s) {
    negate_f32_kernel<<<stream_blocks(count), 256, 0, s>>>(a, b, count);
    return cudaGetLastError();
}

cudaError_t add_f32_to_f64(double *x, const float *d, int64_t count, cudaStream_t s) {
    add_f32_to_f64_kernel<<<stream_blocks(count), 256, 0, s>>>(x, d, count);
    return cudaGetLastError();
}

cudaError_t bits_or(uint64_t *dst, const uint64_t *src, int64_t words, cudaStream_t s) {
    bits_or_kernel<<<stream_blocks(words), 256, 0, s>>>(dst, src, words);
    return cudaGetLastError();
}

cudaError_t transpose_f32(const float *src, int64_t lds, int rows, int cols, float *dst, int64_t ldd, cudaStream_t s) {
    dim3 grid(static_cast<unsigned>((cols + kTT - 1) / kTT), static_cast<unsigned>((rows + kTT - 1) / kTT));
    transpose_tile_kernel<float><<<grid, dim3(kTT, 8), 0, s>>>(src, lds, rows, cols, dst, ldd);
    return cudaGetLastError();
}

cudaError_t trans_real_step(const int *ptr, const int *col, int n, int np, double eps, const uint8_t *R1,
                            const double *X, double *U, double *Xn, unsigned long long *dmax, cudaStream_t s) {
    dim3 tgrid(static_cast<unsigned>((np + kTT - 1) / kTT), static_cast<unsigned>((np + kTT - 1) / kTT));
    transpose_tile_kernel<double><<<tgrid, dim3(kTT, 8), 0, s>>>(X, np, np, np, U, np);  // U = X^T
    dim3 grid(static_cast<unsigned>((np + 255) / 256), static_cast<unsigned>(np));
    sg_pu_kernel<<<grid, 256, 0, s>>>(ptr, col, n, np, eps, R1, U, X, Xn, nullptr, dmax);
    return cudaGetLastError();
}

}  // namespace dl
