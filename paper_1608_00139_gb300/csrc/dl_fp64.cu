// dl_fp64.cu -- the plain FP64 route: R~ = (I - eps E)^-1 eps E (Proposition 1) by blocked
// Gaussian elimination without pivoting, all in FP64 on the CUDA cores, then threshold > 0
// (Theorem 1).
//
// A = I - eps E is strictly diagonally dominant by rows for 0 < eps <= 1/(1 + ||E||_inf)
// (proof of Proposition 1: eps ||E||_inf <= 1 - eps < 1 = a_ii - |eps e_ii| margin), so the
// unpivoted LU exists.  The elimination runs on the augmented matrix G = [A | eps E]
// (np x 2np, padded rows/columns: identity in A, zero in eps E), so the forward substitution
// L Y = eps E happens inside the factorisation; afterwards G = [U | Y] and a blocked
// backward substitution leaves X = U^-1 Y in the right half.
//
// Per block column k (width b = 64):
//   1. diag_lu:   L11 U11 = G11 (one CTA, the b x b block in shared memory)
//   2. trsm_row:  [U12 | Y1] = L11^-1 [G12 | B1]      (one thread per column)
//   3. trsm_col:  L21 = G21 U11^-1                   (one thread per row)
//   4. dgemm:     [G22 | B2] -= L21 [U12 | Y1]       (64 x 64 tiles, FP64 FMA)
// Backward, block k from the last: Y_k = U_kk^-1 Y_k, then Y_{<k} -= U_{<k,k} Y_k.
#include <cuda_runtime.h>

#include <cstdint>

#include "dl_internal.h"
#include "dl_ptx.cuh"

namespace dl {

namespace {

constexpr int B = 64;  // block size of the blocked elimination

__global__ void build_kernel(const uint8_t *__restrict__ E, const uint8_t *__restrict__ A, int n, int np, double eps,
                             double *__restrict__ G, int64_t ldg) {
    const int64_t row = blockIdx.y;
    for (int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; c < 2 * np;
         c += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        double v;
        if (c < np) {
            const double e = (row < n && c < n && E[row * n + c]) ? eps : 0.0;
            v = (c == row ? 1.0 : 0.0) - e;
        } else {
            const int64_t cc = c - np;
            v = (row < n && cc < n && A[row * n + cc]) ? eps : 0.0;
        }
        G[row * ldg + c] = v;
    }
}

// G = [I - eps E | eps F] with a real right-hand side F (n x n FP64, row stride n).
__global__ void build_real_kernel(const uint8_t *__restrict__ E, const double *__restrict__ F, int n, int np,
                                  double eps, double *__restrict__ G, int64_t ldg) {
    const int64_t row = blockIdx.y;
    for (int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; c < 2 * np;
         c += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        double v;
        if (c < np) {
            const double e = (row < n && c < n && E[row * n + c]) ? eps : 0.0;
            v = (c == row ? 1.0 : 0.0) - e;
        } else {
            const int64_t cc = c - np;
            v = (row < n && cc < n) ? eps * F[row * n + cc] : 0.0;
        }
        G[row * ldg + c] = v;
    }
}

// Unpivoted LU of the b x b block at g (row stride ldg), in place: unit L below, U on/above.
__global__ void __launch_bounds__(256) diag_lu_kernel(double *g, int64_t ldg) {
    __shared__ double s[B][B + 1];
    for (int t = threadIdx.x; t < B * B; t += blockDim.x) s[t / B][t % B] = g[(t / B) * ldg + t % B];
    __syncthreads();
    for (int k = 0; k < B; ++k) {
        const double piv = s[k][k];
        for (int i = k + 1 + threadIdx.x; i < B; i += blockDim.x) s[i][k] /= piv;
        __syncthreads();
        for (int t = threadIdx.x; t < (B - k - 1) * (B - k - 1); t += blockDim.x) {
            const int i = k + 1 + t / (B - k - 1), j = k + 1 + t % (B - k - 1);
            s[i][j] -= s[i][k] * s[k][j];
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < B * B; t += blockDim.x) g[(t / B) * ldg + t % B] = s[t / B][t % B];
}

// X = L11^-1 X for the b rows starting at g (columns [c0, c1)), L11 unit lower in diag.
__global__ void __launch_bounds__(128) trsm_row_kernel(const double *diag, int64_t ldg, double *g,
                                                       int64_t ncols) {
    __shared__ double L[B][B];
    for (int t = threadIdx.x; t < B * B; t += blockDim.x) L[t / B][t % B] = diag[(t / B) * ldg + t % B];
    __syncthreads();
    const int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (c >= ncols) return;
    double x[B];
#pragma unroll
    for (int r = 0; r < B; ++r) x[r] = g[r * ldg + c];
#pragma unroll
    for (int r = 1; r < B; ++r) {
        double acc = x[r];
#pragma unroll
        for (int q = 0; q < r; ++q) acc -= L[r][q] * x[q];
        x[r] = acc;
    }
#pragma unroll
    for (int r = 0; r < B; ++r) g[r * ldg + c] = x[r];
}

// X = X U11^-1 for nrows rows starting at g (b columns), U11 upper in diag.
__global__ void __launch_bounds__(128) trsm_col_kernel(const double *diag, int64_t ldg, double *g,
                                                       int64_t nrows) {
    __shared__ double U[B][B];
    for (int t = threadIdx.x; t < B * B; t += blockDim.x) U[t / B][t % B] = diag[(t / B) * ldg + t % B];
    __syncthreads();
    const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (r >= nrows) return;
    double x[B];
#pragma unroll
    for (int c = 0; c < B; ++c) x[c] = g[r * ldg + c];
#pragma unroll
    for (int c = 0; c < B; ++c) {
        double acc = x[c];
#pragma unroll
        for (int q = 0; q < c; ++q) acc -= x[q] * U[q][c];
        x[c] = acc / U[c][c];
    }
#pragma unroll
    for (int c = 0; c < B; ++c) g[r * ldg + c] = x[c];
}

// X = U11^-1 X for the b rows starting at g (ncols columns), U11 upper (non-unit) in diag.
__global__ void __launch_bounds__(128) trsm_upper_kernel(const double *diag, int64_t ldg, double *g,
                                                         int64_t ncols) {
    __shared__ double U[B][B];
    for (int t = threadIdx.x; t < B * B; t += blockDim.x) U[t / B][t % B] = diag[(t / B) * ldg + t % B];
    __syncthreads();
    const int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (c >= ncols) return;
    double x[B];
#pragma unroll
    for (int r = 0; r < B; ++r) x[r] = g[r * ldg + c];
#pragma unroll
    for (int r = B - 1; r >= 0; --r) {
        double acc = x[r];
#pragma unroll
        for (int q = r + 1; q < B; ++q) acc -= U[r][q] * x[q];
        x[r] = acc / U[r][r];
    }
#pragma unroll
    for (int r = 0; r < B; ++r) g[r * ldg + c] = x[r];
}

// C(M x N) -= A(M x 64) * Bm(64 x N); all row-major with stride ldg; M, N multiples of 64.
constexpr int TM = 64, TN = 64, TK = 16;
__global__ void __launch_bounds__(256) dgemm_sub_kernel(const double *__restrict__ A,
                                                        const double *__restrict__ Bm,
                                                        double *__restrict__ C, int64_t ldg) {
    __shared__ double sA[TK][TM + 1];
    __shared__ double sB[TK][TN];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t r0 = static_cast<int64_t>(blockIdx.y) * TM, c0 = static_cast<int64_t>(blockIdx.x) * TN;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < B; k0 += TK) {
        for (int t = threadIdx.x; t < TM * TK; t += 256) {
            const int i = t / TK, k = t % TK;
            sA[k][i] = A[(r0 + i) * ldg + k0 + k];
        }
        for (int t = threadIdx.x; t < TK * TN; t += 256) {
            const int k = t / TN, j = t % TN;
            sB[k][j] = Bm[(k0 + k) * ldg + c0 + j];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TK; ++k) {
            double a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = sA[k][ty + 16 * q];
                b[q] = sB[k][tx + 16 * q];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) C[(r0 + ty + 16 * i) * ldg + c0 + tx + 16 * j] -= acc[i][j];
}

cudaError_t dgemm_sub(const double *A, const double *Bm, double *C, int64_t ldg, int64_t M, int64_t N,
                      cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid(static_cast<unsigned>(N / TN), static_cast<unsigned>(M / TM));
    dgemm_sub_kernel<<<grid, 256, 0, s>>>(A, Bm, C, ldg);
    return cudaGetLastError();
}

// Threshold X > 0 into bits (and count the guard band).
// Spread the 32 bits of x to the even bit positions of a 64-bit word (bit l -> bit 2l).
__device__ __forceinline__ uint64_t spread_even(uint32_t x) {
    uint64_t v = x;
    v = (v | (v << 16)) & 0x0000FFFF0000FFFFull;
    v = (v | (v << 8)) & 0x00FF00FF00FF00FFull;
    v = (v | (v << 4)) & 0x0F0F0F0F0F0F0F0Full;
    v = (v | (v << 2)) & 0x3333333333333333ull;
    v = (v | (v << 1)) & 0x5555555555555555ull;
    return v;
}

constexpr int kThreshWords = 8;  // 64-bit words (512 columns) per warp

// A warp takes kThreshWords consecutive words of one row: every lane issues its 16-byte loads
// (columns 2 lane, 2 lane + 1 of each word) before it tests any, and the even and odd columns'
// ballots are interleaved into the word.  Rows are 16-byte aligned (ldx even).
__global__ void __launch_bounds__(256) thresh_pack_kernel(const double *__restrict__ X, int64_t ldx, int n,
                                                          double tau, uint64_t *__restrict__ bits, int64_t wp,
                                                          unsigned long long *guard) {
    const int lane = threadIdx.x & 31;
    const int64_t words = (n + 63) / 64, groups = (words + kThreshWords - 1) / kThreshWords;
    const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (gw >= static_cast<int64_t>(n) * groups) return;
    const int64_t row = gw / groups, w0 = (gw % groups) * kThreshWords;
    const double *xr = X + row * ldx;
    double2 v[kThreshWords];
#pragma unroll
    for (int q = 0; q < kThreshWords; ++q) {
        const int64_t c = (w0 + q) * 64 + 2 * lane;
        v[q] = c + 1 < n ? __ldcs(reinterpret_cast<const double2 *>(xr + c))
                         : make_double2(c < n ? xr[c] : 0.0, 0.0);
    }
    uint32_t gcount = 0;
#pragma unroll
    for (int q = 0; q < kThreshWords; ++q) {
        if (w0 + q >= words) break;
        const uint32_t ev = __ballot_sync(0xffffffffu, v[q].x > 0.0);
        const uint32_t od = __ballot_sync(0xffffffffu, v[q].y > 0.0);
        const bool gx = v[q].x < 0.0 || (v[q].x > 0.0 && v[q].x <= tau);  // guard band: |X| <= tau or X < 0
        const bool gy = v[q].y < 0.0 || (v[q].y > 0.0 && v[q].y <= tau);
        gcount += __popc(__ballot_sync(0xffffffffu, gx)) + __popc(__ballot_sync(0xffffffffu, gy));
        if (lane == q) bits[row * wp + w0 + q] = spread_even(ev) | (spread_even(od) << 1);
    }
    if (lane == 0 && gcount) atomicAdd(guard, static_cast<unsigned long long>(gcount));
}

}  // namespace

cudaError_t fp64_build(const uint8_t *E, const uint8_t *A, int n, int np, double eps, double *G, int64_t ldg,
                       cudaStream_t s) {
    dim3 grid(static_cast<unsigned>((2 * np + 255) / 256 < 64 ? (2 * np + 255) / 256 : 64),
              static_cast<unsigned>(np));
    build_kernel<<<grid, 256, 0, s>>>(E, A, n, np, eps, G, ldg);
    return cudaGetLastError();
}

cudaError_t fp64_build_real(const uint8_t *E, const double *F, int n, int np, double eps, double *G, int64_t ldg,
                            cudaStream_t s) {
    dim3 grid(static_cast<unsigned>((2 * np + 255) / 256 < 64 ? (2 * np + 255) / 256 : 64),
              static_cast<unsigned>(np));
    build_real_kernel<<<grid, 256, 0, s>>>(E, F, n, np, eps, G, ldg);
    return cudaGetLastError();
}

cudaError_t fp64_solve(double *G, int64_t ldg, int np, int *launches, cudaStream_t s) {
    cudaError_t e;
    int L = 0;
    const int nb = np / B;
    for (int k = 0; k < nb; ++k) {
        const int64_t kb = static_cast<int64_t>(k) * B;
        double *g11 = G + kb * ldg + kb;
        diag_lu_kernel<<<1, 256, 0, s>>>(g11, ldg);
        ++L;
        const int64_t ncols = 2 * static_cast<int64_t>(np) - kb - B;  // U12 and the RHS
        trsm_row_kernel<<<static_cast<unsigned>((ncols + 127) / 128), 128, 0, s>>>(g11, ldg, g11 + B, ncols);
        ++L;
        const int64_t nrows = np - kb - B;
        if (nrows > 0) {
            trsm_col_kernel<<<static_cast<unsigned>((nrows + 127) / 128), 128, 0, s>>>(g11, ldg, g11 + B * ldg, nrows);
            ++L;
            if ((e = dgemm_sub(g11 + B * ldg, g11 + B, g11 + B * ldg + B, ldg, nrows, ncols, s)) != cudaSuccess)
                return e;
            ++L;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    double *Y = G + np;  // right half
    for (int k = nb - 1; k >= 0; --k) {
        const int64_t kb = static_cast<int64_t>(k) * B;
        trsm_upper_kernel<<<static_cast<unsigned>((np + 127) / 128), 128, 0, s>>>(G + kb * ldg + kb, ldg,
                                                                                Y + kb * ldg, np);
        ++L;
        if (kb > 0) {
            if ((e = dgemm_sub(G + kb, Y + kb * ldg, Y, ldg, kb, np, s)) != cudaSuccess) return e;
            ++L;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (launches) *launches += L;
    return cudaSuccess;
}

cudaError_t thresh_pack_f64(const double *X, int64_t ldx, int n, int np, double tau, uint64_t *bits,
                            int64_t wp, unsigned long long *guard, cudaStream_t s) {
    (void)np;
    if (n <= 0) return cudaSuccess;
    if (ldx % 2 != 0 || (reinterpret_cast<uintptr_t>(X) & 15) != 0) return cudaErrorInvalidValue;
    const int64_t groups = ((n + 63) / 64 + kThreshWords - 1) / kThreshWords;
    const int64_t threads = static_cast<int64_t>(n) * groups * 32;
    thresh_pack_kernel<<<static_cast<unsigned>((threads + 255) / 256), 256, 0, s>>>(X, ldx, n, tau, bits, wp,
                                                                                   guard);
    return cudaGetLastError();
}

}  // namespace dl
