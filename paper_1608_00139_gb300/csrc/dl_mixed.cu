// dl_mixed.cu -- R~ = (I - eps E)^-1 eps E (Proposition 1) on the TF32 tensor cores, with FP64
// iterative refinement (DL_PATH_MIXED).
//
//   1. A = I - eps E in FP32 (padded with the identity).  The right-hand side is kept
//      transposed: Z = X^T, starting from Z = (eps E)^T, so that every product below is a
//      "TN" GEMM whose operands are both stored with K contiguous (the form the TF32 tensor
//      cores run here).
//   2. Blocked right-looking LU of A without pivoting (A is strictly diagonally dominant by
//      rows, proof of Proposition 1), block b = 128.  Per block k:
//        diag_lu_inv:  L11 U11 = A11 on the CUDA cores (FP32) and the explicit inverses
//                      L11^-1, U11^-1 (and U11^-T);
//        T = A12^T (transpose of the 128-wide row panel);
//        one grouped tcgen05 launch:  T = T L11^-T (= U12^T)  and  L21 = A21 U11^-1;
//        A12 = T^T (U12 kept row-major for the backward substitution);
//        one tcgen05 launch:  A22 -= L21 U12  (B operand U12^T = T).
//   3. Z = (eps E)^T U^-T L^-T, i.e. X = U^-1 L^-1 eps E, by block forward and backward
//      substitution on the columns of Z:  Z_k = Z_k L_kk^-T,  Z_{>k} -= Z_k L_{>k,k}^T,
//      then Z_k = Z_k U_kk^-T,  Z_{<k} -= Z_k U_{<k,k}^T  (L and U blocks read as stored).
//   4. Refinement in FP64 on Z: R^T = (eps E - A X)^T, i.e.
//      R^T[j][i] = eps * sum_{k : E[i][k]} (Z[j][k] + [k = j]) - Z[j][i]
//      (E is 0/1, so E X is a sum of rows of X: FP64 additions only); D^T = R^T U^-T L^-T on
//      the tensor cores; Z += D^T; until max|R| <= tol * eps.  Each step contracts the error
//      by about kappa(A) u_tf32, kappa_inf(A) <= (1 + eps ||E||) / eps <= 2 (1 + ||E||).
//   5. X = Z^T; model X > 0 (Theorem 1); entries in the guard band are counted and the exact
//      boolean recheck of R2 = min1(E + E R2) confirms the model or adds lost facts.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "dl_ctx.h"
#include "dl_internal.h"

namespace dl {

namespace {

constexpr int BL = 128;  // LU block size = GEMM tile
constexpr int TT = 32;   // transpose tile

__global__ void build_a_kernel(const uint8_t *__restrict__ E, int n, int np, float eps, float *__restrict__ A) {
    const int64_t row = blockIdx.y;
    for (int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; c < np;
         c += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float e = (row < n && c < n && E[row * n + c]) ? eps : 0.0f;
        A[row * np + c] = (c == row ? 1.0f : 0.0f) - e;
    }
}

// Z = (eps E)^T, np x np (zero padding); 32 x 32 tiles through shared memory.
__global__ void build_zt_kernel(const uint8_t *__restrict__ E, int n, int np, float eps, float *__restrict__ Z) {
    __shared__ float tile[TT][TT + 1];
    const int c0 = blockIdx.x * TT, r0 = blockIdx.y * TT;
    for (int y = threadIdx.y; y < TT; y += blockDim.y) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        tile[y][threadIdx.x] = (r < n && c < n && E[static_cast<int64_t>(r) * n + c]) ? eps : 0.0f;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < TT; y += blockDim.y) {
        const int r = c0 + y, c = r0 + threadIdx.x;  // Z[r][c] = eps E[c][r]
        if (r < np && c < np) Z[static_cast<int64_t>(r) * np + c] = tile[threadIdx.x][y];
    }
}

// dst (cols x rows) = src (rows x cols)^T
template <class T>
__global__ void transpose_kernel(const T *__restrict__ src, int64_t lds, int rows, int cols, T *__restrict__ dst,
                                 int64_t ldd) {
    __shared__ T tile[TT][TT + 1];
    const int c0 = blockIdx.x * TT, r0 = blockIdx.y * TT;
    for (int y = threadIdx.y; y < TT; y += blockDim.y) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[y][threadIdx.x] = src[static_cast<int64_t>(r) * lds + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < TT; y += blockDim.y) {
        const int r = c0 + y, c = r0 + threadIdx.x;
        if (r < cols && c < rows) dst[static_cast<int64_t>(r) * ldd + c] = tile[threadIdx.x][y];
    }
}

template <class T>
cudaError_t transpose(const T *src, int64_t lds, int rows, int cols, T *dst, int64_t ldd, cudaStream_t s) {
    dim3 grid(static_cast<unsigned>((cols + TT - 1) / TT), static_cast<unsigned>((rows + TT - 1) / TT));
    transpose_kernel<T><<<grid, dim3(TT, 8), 0, s>>>(src, lds, rows, cols, dst, ldd);
    return cudaGetLastError();
}

// Unpivoted LU of the BL x BL block at A (row stride lda) with the inverses of its factors,
// FP32, blocked by 32 in shared memory: one CTA of 1024 threads holds the block, L^-1 and
// U^-1 (three BL x (BL + 4) float arrays).
//  1. right-looking LU by 32-column panels: warp 0 factors the panel's 32 x 32 diagonal block
//     (lane = row; the pivot row, final once the earlier steps are done, is read back from
//     shared memory), warps 1-3 form L21 = A21 U11^-1 (lane = row) and warps 4-6 form
//     U12 = L11^-1 A12 (lane = column) by substitution, then all warps update A22 -= L21 U12
//     in strips of 8 rows x 32 columns;
//  2. the inverses of the 32 x 32 diagonal blocks of L and U by substitution (a warp each),
//     then the blocks off the diagonal at distance d = 1, 2, 3 from it, each from blocks
//     nearer the diagonal:  X_ij = -X_ii sum_{k=j..i-1} L_ik X_kj  (X = L^-1, i > j) and
//     Y_ij = -Y_ii sum_{k=i+1..j} U_ik Y_kj  (Y = U^-1, i < j).
// Writes L^-1 (unit lower), U^-1 and U^-T, BL x BL each; a zero pivot sets ST_BAD_INPUT.
constexpr int kDiagThreads = 1024;
constexpr int kDiagLd = BL + 4;  // padded shared-memory row (keeps float4 alignment)
constexpr size_t kDiagSmem = 3ull * BL * kDiagLd * sizeof(float) + 16;
constexpr int kSolveGroup = 8;  // panels per group of the N-RHS solves
constexpr size_t kResidualSmem = 227 * 1024;  // dynamic shared memory of one residual block

// acc[r] += sum_{k < 32} A[r][k] B[k][lane] for an 8 x 32 strip A and a 32 x 32 block B, both in
// shared memory with row stride kDiagLd (A's rows read as broadcast float4s).
__device__ __forceinline__ void strip_product(const float *A, const float *B, int lane, float (&acc)[8]) {
#pragma unroll
    for (int k = 0; k < 32; k += 4) {
        const float b0 = B[(k + 0) * kDiagLd + lane], b1 = B[(k + 1) * kDiagLd + lane];
        const float b2 = B[(k + 2) * kDiagLd + lane], b3 = B[(k + 3) * kDiagLd + lane];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const float4 a = *reinterpret_cast<const float4 *>(A + r * kDiagLd + k);
            acc[r] = fmaf(a.x, b0, acc[r]);
            acc[r] = fmaf(a.y, b1, acc[r]);
            acc[r] = fmaf(a.z, b2, acc[r]);
            acc[r] = fmaf(a.w, b3, acc[r]);
        }
    }
}

__device__ __forceinline__ void load_row32(const float *p, float (&r)[32]) {
#pragma unroll
    for (int c = 0; c < 32; c += 4) {
        const float4 v = *reinterpret_cast<const float4 *>(p + c);
        r[c] = v.x;
        r[c + 1] = v.y;
        r[c + 2] = v.z;
        r[c + 3] = v.w;
    }
}

__device__ __forceinline__ void store_row32(float *p, const float (&r)[32]) {
#pragma unroll
    for (int c = 0; c < 32; c += 4) *reinterpret_cast<float4 *>(p + c) = make_float4(r[c], r[c + 1], r[c + 2], r[c + 3]);
}

__global__ void __launch_bounds__(kDiagThreads) diag_lu_inv_kernel(const float *A, int64_t lda, float *Linv,
                                                                   float *Uinv, float *UinvT, int *status) {
    static_assert(BL == 128, "four 32-column panels");
    extern __shared__ float4 diag_smem[];
    float *S = reinterpret_cast<float *>(diag_smem);  // the block; then L (strictly lower) and U in place
    float *XL = S + BL * kDiagLd;                      // L^-1
    float *XU = XL + BL * kDiagLd;                     // U^-1
    int *bad = reinterpret_cast<int *>(XU + BL * kDiagLd);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) *bad = 0;
    for (int e = t; e < BL * BL / 4; e += kDiagThreads) {
        const int r = e >> 5, c = (e & 31) * 4;
        *reinterpret_cast<float4 *>(S + r * kDiagLd + c) = *reinterpret_cast<const float4 *>(A + r * lda + c);
    }
    __syncthreads();

    // ---- 1. LU by 32-column panels ----
    for (int o = 0; o < BL; o += 32) {
        const int rem = BL - o - 32;  // rows (and columns) after the panel
        if (warp == 0) {
            float *rowp = S + (o + lane) * kDiagLd + o;
            float r[32];
            load_row32(rowp, r);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (lane == j) store_row32(rowp, r);  // row j is final after steps 0 .. j-1
                __syncwarp();
                const float *pj = S + (o + j) * kDiagLd + o;
                if (lane > j) {
                    const float l = r[j] / pj[j];
                    r[j] = l;
#pragma unroll
                    for (int c = j + 1; c < 32; ++c) r[c] = fmaf(-l, pj[c], r[c]);
                }
            }
            store_row32(rowp, r);
            const float d = S[(o + lane) * kDiagLd + o + lane];  // U_ii (this lane's row, stored above)
            if (!(fabsf(d) > 0.0f) || !isfinite(d)) atomicOr(bad, 1);
        }
        __syncthreads();
        if (*bad) {  // uniform: every thread reads the flag after the barrier
            if (t == 0) atomicOr(status, ST_BAD_INPUT);
            return;
        }
        if (rem == 0) break;
        if (warp >= 1 && warp <= 3 && 32 * (warp - 1) < rem) {  // L21 = A21 U11^-1, lane = row
            float *rowp = S + (o + 32 + 32 * (warp - 1) + lane) * kDiagLd + o;
            float r[32];
            load_row32(rowp, r);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float *uj = S + (o + j) * kDiagLd + o;
                r[j] = r[j] / uj[j];
#pragma unroll
                for (int c = j + 1; c < 32; ++c) r[c] = fmaf(-r[j], uj[c], r[c]);
            }
            store_row32(rowp, r);
        } else if (warp >= 4 && warp <= 6 && 32 * (warp - 4) < rem) {  // U12 = L11^-1 A12, lane = column
            const int c = o + 32 + 32 * (warp - 4) + lane;
            float x[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) x[i] = S[(o + i) * kDiagLd + c];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
#pragma unroll
                for (int i = j + 1; i < 32; ++i) x[i] = fmaf(-S[(o + i) * kDiagLd + o + j], x[j], x[i]);
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) S[(o + i) * kDiagLd + c] = x[i];
        }
        __syncthreads();
        const int nbk = rem / 32, tasks = nbk * nbk * 4;  // A22 -= L21 U12: 4 strips per 32 x 32 block
        for (int task = warp; task < tasks; task += 32) {
            const int blk = task >> 2, strip = task & 3;
            const int row0 = o + 32 + 32 * (blk / nbk) + 8 * strip, col0 = o + 32 + 32 * (blk % nbk);
            float acc[8] = {};
            strip_product(S + row0 * kDiagLd + o, S + o * kDiagLd + col0, lane, acc);
#pragma unroll
            for (int r = 0; r < 8; ++r) S[(row0 + r) * kDiagLd + col0 + lane] -= acc[r];
        }
        __syncthreads();
    }

    // ---- 2a. inverses of the diagonal blocks (lane = column) ----
    if (warp < 4) {  // L_pp^-1, unit lower: forward substitution on e_lane
        const int o = 32 * warp;
        float x[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) x[i] = i == lane ? 1.0f : 0.0f;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
#pragma unroll
            for (int i = k + 1; i < 32; ++i) x[i] = fmaf(-S[(o + i) * kDiagLd + o + k], x[k], x[i]);
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) XL[(o + i) * kDiagLd + o + lane] = x[i];
    } else if (warp < 8) {  // U_pp^-1 by rows: row lane of U^-1 solves U^T z = e_lane (forward)
        const int o = 32 * (warp - 4);
        float z[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) z[i] = i == lane ? 1.0f : 0.0f;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const float *uk = S + (o + k) * kDiagLd + o;  // row k of U
            z[k] = z[k] / uk[k];
#pragma unroll
            for (int i = k + 1; i < 32; ++i) z[i] = fmaf(-uk[i], z[k], z[i]);
        }
        store_row32(XU + (o + lane) * kDiagLd + o, z);
    }
    __syncthreads();

    // ---- 2b. blocks off the diagonal, by distance d: warp -> (side, j, strip) ----
    for (int d = 1; d < 4; ++d) {
        const int nblk = 4 - d, tasks = 2 * nblk * 4;  // at most 24 <= 32 warps
        const bool has = warp < tasks;
        const int task = has ? warp : 0;  // idle warps take task 0's indices and access nothing
        const int side = task / (nblk * 4), j = (task % (nblk * 4)) >> 2, strip = task & 3;
        // L side: block (j + d, j) of X;  U side: block (j, j + d) of Y
        const int bi = side == 0 ? j + d : j, bj = side == 0 ? j : j + d;
        float *X = side == 0 ? XL : XU;
        float *dst = X + (32 * bi + 8 * strip) * kDiagLd + 32 * bj;
        if (has) {  // T = sum_k L_{bi,k} X_{k,bj} (k = bj .. bi-1), or U_{bi,k} Y_{k,bj} (k = bi+1 .. bj)
            float acc[8] = {};
            const int k0 = side == 0 ? bj : bi + 1, k1 = side == 0 ? bi - 1 : bj;
            for (int k = k0; k <= k1; ++k)
                strip_product(S + (32 * bi + 8 * strip) * kDiagLd + 32 * k, X + 32 * k * kDiagLd + 32 * bj, lane, acc);
#pragma unroll
            for (int r = 0; r < 8; ++r) dst[r * kDiagLd + lane] = acc[r];
        }
        __syncthreads();
        float acc[8] = {};
        if (has)  // -X_{bi,bi} T (the whole T block is read: products first, stores after a barrier)
            strip_product(X + (32 * bi + 8 * strip) * kDiagLd + 32 * bi, X + 32 * bi * kDiagLd + 32 * bj, lane, acc);
        __syncthreads();
        if (has) {
#pragma unroll
            for (int r = 0; r < 8; ++r) dst[r * kDiagLd + lane] = -acc[r];
        }
        __syncthreads();
    }

    for (int e = t; e < BL * BL; e += kDiagThreads) {
        const int r = e >> 7, c = e & (BL - 1);
        Linv[e] = c < r ? XL[r * kDiagLd + c] : (c == r ? 1.0f : 0.0f);
        Uinv[e] = c >= r ? XU[r * kDiagLd + c] : 0.0f;
        UinvT[e] = r >= c ? XU[c * kDiagLd + r] : 0.0f;  // U^-T[r][c] = U^-1[c][r]
    }
}

// round(z 2^e) from the bits of z with integer operations only (GB300's FP64 units are the scarce
// resource of the residual); the caller keeps |z| 2^e below 2^62.  Zero and subnormal z give 0.
__device__ __forceinline__ long long fixed_of(long long bits, int e) {
    const int ex = static_cast<int>((bits >> 52) & 0x7FF);
    if (ex == 0) return 0;
    const long long m = (bits & 0xFFFFFFFFFFFFFll) | 0x10000000000000ll;  // |z| = m 2^(ex - 1075)
    const int sh = ex - 1075 + e;
    long long v = 0;
    if (sh >= 0) v = m << sh;
    else if (sh > -64) v = (m + (1ll << (-sh - 1))) >> (-sh);  // nearest, ties away from zero
    return bits < 0 ? -v : v;
}

// Residual of the transposed system for G rows j of Z per block (the rows share each read of
// the CSR):  R^T[j][i] = eps * sum_{k in succ(i)} (Z[j][k] + [k = j]) - Z[j][i]  (right-hand side
// eps E; with At, the bytes of A^T, the term [k = j] becomes A[i][j]: right-hand side eps A),  stored as FP32
// (right-hand side of the correction solve); max |R| -> *rmax.  The sums are exact in 64-bit
// fixed point: row j sits in shared memory as round((Z[j][k] + [k = j]) 2^e_j), e_j chosen from
// the row's largest exponent and 2^deg_bits >= ||E||_inf so that no sum reaches 2^62.  Each
// term is rounded once (at most 2^-(e_j + 1), below one FP64 ulp of the row's largest entry);
// the scaling by eps 2^-e_j and the subtraction are one FP64 fma.
template <int G>
__global__ void __launch_bounds__(1024, 1)
    residual_fixed_kernel(const int *__restrict__ ptr, const int *__restrict__ col, int n, int np, int deg_bits,
                          double eps, const double *__restrict__ Z, float *__restrict__ R, unsigned long long *rmax,
                          const uint8_t *__restrict__ At) {
    extern __shared__ long long zi[];  // G rows of np entries
    __shared__ int ex_max[G];
    const int j0 = blockIdx.x * G;
    if (threadIdx.x < G) ex_max[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int g = 0; g < G; ++g) {  // stage the raw bits and find the largest exponent
        const int j = j0 + g;
        int ex = 0;
        if (j < np) {
            const long long *zb = reinterpret_cast<const long long *>(Z + static_cast<int64_t>(j) * np);
            for (int k = threadIdx.x; k < np; k += blockDim.x) {
                const long long b = zb[k];
                zi[g * np + k] = b;
                ex = max(ex, static_cast<int>((b >> 52) & 0x7FF));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, o));
        if ((threadIdx.x & 31) == 0) atomicMax(&ex_max[g], ex);
    }
    __syncthreads();
    int e[G];
    double scale[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        // every term, the +1 included, is below 2^hb; a sum of at most 2^deg_bits terms below 2^62
        const int hb = max(ex_max[g] - 1022, 0) + 1;
        e[g] = max(0, 62 - deg_bits - hb);
        scale[g] = ldexp(eps, -e[g]);
    }
#pragma unroll
    for (int g = 0; g < G; ++g)
        for (int k = threadIdx.x; k < np; k += blockDim.x) zi[g * np + k] = fixed_of(zi[g * np + k], e[g]);
    __syncthreads();
    if (threadIdx.x < G && At == nullptr) {  // the eps E[i][j] term, as k = j
        const int g = threadIdx.x, j = j0 + g;
        if (j < n) zi[g * np + j] += 1ll << e[g];
    }
    __syncthreads();
    float m = 0.0f;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        long long sum[G] = {};
        if (i < n) {
            const int q1 = ptr[i + 1];
            int q = ptr[i];
            for (; q + 4 <= q1; q += 4) {  // four successor indices in flight
                const int c0 = col[q], c1 = col[q + 1], c2 = col[q + 2], c3 = col[q + 3];
#pragma unroll
                for (int g = 0; g < G; ++g)
                    sum[g] += (zi[g * np + c0] + zi[g * np + c1]) + (zi[g * np + c2] + zi[g * np + c3]);
            }
            for (; q < q1; ++q) {
                const int c = col[q];
#pragma unroll
                for (int g = 0; g < G; ++g) sum[g] += zi[g * np + c];
            }
            if (At != nullptr) {  // a general right-hand side: the eps A[i][j] term from A^T's row j
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int j = j0 + g;
                    if (j < n && At[static_cast<int64_t>(j) * n + i]) sum[g] += 1ll << e[g];
                }
            }
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int j = j0 + g;
            if (j >= np) break;
            float r = 0.0f;
            if (i < n && j < n)
                r = static_cast<float>(fma(scale[g], static_cast<double>(sum[g]), -Z[static_cast<int64_t>(j) * np + i]));
            R[static_cast<int64_t>(j) * np + i] = r;
            m = fmaxf(m, fabsf(r));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0f)
        atomicMax(rmax, static_cast<unsigned long long>(__double_as_longlong(static_cast<double>(m))));
}

// Y = I on every group's rows (groups of gw rows starting at multiples of gw; row r of a group
// holds its identity entry at column r mod gw), for both group-inverse buffers (zeroed before).
__global__ void group_identity_kernel(float *YL, float *YU, int np, int gw) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= np) return;
    const int64_t at = static_cast<int64_t>(r) * gw + r % gw;
    YL[at] = 1.0f;
    YU[at] = 1.0f;
}

__global__ void f32_to_f64_kernel(const float *__restrict__ a, double *__restrict__ b, int64_t count) {
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < count;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x)
        b[t] = static_cast<double>(a[t]);
}

__global__ void add_f32_kernel(double *__restrict__ x, const float *__restrict__ d, int64_t count) {
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < count;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x)
        x[t] += static_cast<double>(d[t]);
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

#define MCK(x)                                                                                   \
    do {                                                                                         \
        cudaError_t e_ = (x);                                                                    \
        if (e_ != cudaSuccess) {                                                                 \
            set_error("mixed path: %s failed: %s (%s:%d)", #x, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return DL_EDEVICE;                                                                   \
        }                                                                                        \
    } while (0)

struct Launch {
    int first, count, tiles;  // problems [first, first + count) of the table
    GemmEpi epi;
};

}  // namespace

dl_status tc_mixed(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a, dl_stats *st,
                   const uint8_t *E, double eps, unsigned long long dmax, int *launches_io) {
    const int32_t n = a.n;
    const int64_t np = round_up(std::max<int64_t>(n, 1), 256);
    const int nb = static_cast<int>(np / BL);
    const int N = static_cast<int>(np);
    int launches = 0;
    auto *A32 = static_cast<float *>(ws.get("mx_A", np * np * 4));
    auto *Z32 = static_cast<float *>(ws.get("mx_Z", np * np * 4));
    auto *Z64 = static_cast<double *>(ws.get("mx_Z64", np * np * 8));
    auto *X64 = static_cast<double *>(ws.get("mx_X64", np * np * 8));
    auto *T = static_cast<float *>(ws.get("mx_T", np * BL * 4));
    auto *Linv = static_cast<float *>(ws.get("mx_Linv", np * BL * 4));
    auto *Uinv = static_cast<float *>(ws.get("mx_Uinv", np * BL * 4));
    auto *UinvT = static_cast<float *>(ws.get("mx_UinvT", np * BL * 4));
    // group inverses of the solves: a group is kSolveGroup panels (GW columns)
    const int64_t GW = std::min<int64_t>(np, static_cast<int64_t>(kSolveGroup) * BL);
    auto *YL = static_cast<float *>(ws.get("mx_YL", np * GW * 4));
    auto *YU = static_cast<float *>(ws.get("mx_YU", np * GW * 4));
    auto *GL = static_cast<float *>(ws.get("mx_GL", np * GW * 4));
    auto *GU = static_cast<float *>(ws.get("mx_GU", np * GW * 4));
    auto *Tg = static_cast<float *>(ws.get("mx_Tg", np * GW * 4));
    if (!YL || !YU || !GL || !GU || !Tg) {
        set_error("mixed path: device allocation failed (group inverses)");
        return DL_ENOMEM;
    }
    auto *csr_cnt = static_cast<int *>(ws.get("mx_cnt", (np + 1) * 4));
    auto *csr_ptr = static_cast<int *>(ws.get("mx_ptr", (np + 1) * 4));
    if (!A32 || !Z32 || !Z64 || !X64 || !T || !Linv || !Uinv || !UinvT || !csr_cnt || !csr_ptr) {
        set_error("mixed path: device allocation failed");
        return DL_ENOMEM;
    }
    cudaEvent_t *ev = ws.ev;
    MCK(cudaEventRecord(ev[4], s));
    {
        dim3 grid(static_cast<unsigned>(std::min<int64_t>((np + 255) / 256, 64)), static_cast<unsigned>(np));
        build_a_kernel<<<grid, 256, 0, s>>>(E, n, N, static_cast<float>(eps), A32);
        MCK(cudaGetLastError());
        dim3 tgrid(static_cast<unsigned>(np / TT), static_cast<unsigned>(np / TT));
        build_zt_kernel<<<tgrid, dim3(TT, 8), 0, s>>>(a.rhs ? a.rhs : E, n, N, static_cast<float>(eps), Z32);
        MCK(cudaGetLastError());
        launches += 2;
    }
    // a general right-hand side A: its transpose (bytes) for the residual's A[i][j] terms
    uint8_t *At = nullptr;
    if (a.rhs) {
        At = static_cast<uint8_t *>(ws.get("mx_At", std::max<size_t>(static_cast<size_t>(n) * n, 16)));
        if (!At) {
            set_error("mixed path: device allocation failed (A^T)");
            return DL_ENOMEM;
        }
        MCK(transpose(a.rhs, n, n, n, At, n, s));
        ++launches;
    }
    // CSR of E for the residual
    MCK(csr_build(E, n, csr_cnt, csr_ptr, s));
    int nnz = 0;
    MCK(cudaMemcpyAsync(&nnz, csr_ptr + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
    auto *csr_col = static_cast<int *>(ws.get("mx_col", static_cast<size_t>(std::max(nnz, 1)) * 4));
    if (!csr_col) {
        set_error("mixed path: device allocation failed (CSR)");
        return DL_ENOMEM;
    }
    MCK(csr_fill(E, n, csr_ptr, csr_col, s));
    launches += 3;

    // ---- GEMM table (every product is C (=|-=) A B'^T, both operands K-major) --------------
    std::vector<GemmProblem> probs;
    std::vector<Launch> lu, ginv, fwd, bwd;
    // a solve step: a GEMM launch of fwd/bwd, or (launch < 0) the copy of the group panel Tg
    // back into Z's columns [gs, gs + w)
    struct Step {
        int launch, gs, w;
    };
    std::vector<Step> fwd_steps, bwd_steps;
    std::string err;
    double flops_lu = 0, flops_solve = 0;
    auto add = [&](std::vector<Launch> &list, GemmEpi epi, int M, int Nn, int K, const Operand &Aop,
                   const Operand &Bop, float *C, int64_t ldc, int r0, int c0, bool group_with_prev,
                   double *fl) -> bool {
        GemmProblem p;
        GemmEpilogue e{};
        e.c32 = C;
        e.ld_c32 = ldc;
        e.out_row0 = r0;
        e.out_col0 = c0;
        if (!gemm_make_problem(&p, KIND_TF32, true, BL, M, Nn, K, Aop, Bop, e, &err)) return false;
        const int t = p.tiles_m * p.tiles_n;
        if (group_with_prev && !list.empty() && list.back().epi == epi &&
            list.back().first + list.back().count == static_cast<int>(probs.size())) {
            p.tile_start = list.back().tiles;
            list.back().count += 1;
            list.back().tiles += t;
        } else {
            p.tile_start = 0;
            list.push_back(Launch{static_cast<int>(probs.size()), 1, t, epi});
        }
        probs.push_back(p);
        *fl += 2.0 * M * Nn * K;
        return true;
    };
    auto at = [](Operand o, int r, int c) {
        o.row0 = r;
        o.col0 = c;
        return o;
    };
    const Operand opA{A32, np, np, np, 0, 0};
    const Operand opZ{Z32, np, np, np, 0, 0};
    const Operand opT{T, np, BL, BL, 0, 0};
    const Operand opL{Linv, np, BL, BL, 0, 0};
    const Operand opU{Uinv, np, BL, BL, 0, 0};
    const Operand opUT{UinvT, np, BL, BL, 0, 0};
    bool ok = true;
    std::vector<int> lu_panel(nb, -1), lu_trail(nb, -1);
    for (int k = 0; k < nb && ok; ++k) {
        const int kb = k * BL, rem = N - kb - BL;
        if (rem <= 0) break;
        lu_panel[k] = static_cast<int>(lu.size());
        // U12^T = A12^T L11^-T (in T), L21 = A21 U11^-1 (in place)
        ok = add(lu, EPI_STORE_F32, rem, BL, BL, opT, at(opL, kb, 0), T, BL, 0, 0, false, &flops_lu) &&
             add(lu, EPI_STORE_F32, rem, BL, BL, at(opA, kb + BL, kb), at(opUT, kb, 0), A32, np, kb + BL, kb, true,
                 &flops_lu);
        lu_trail[k] = static_cast<int>(lu.size());
        // A22 -= L21 U12
        ok = ok && add(lu, EPI_SUB_F32, rem, rem, BL, at(opA, kb + BL, kb), opT, A32, np, kb + BL, kb + BL, false,
                       &flops_lu);
    }
    // Inverses of the diagonal groups (kSolveGroup panels each), once per factorisation: the
    // forward machinery on rows Y = I of a group gives Y L_gg^T = I, i.e. Y = L_gg^-T, and the
    // backward one Y = U_gg^-T; every step is one launch over all groups.  (Transposed after.)
    const Operand opYL{YL, np, GW, GW, 0, 0}, opYU{YU, np, GW, GW, 0, 0};
    const Operand opGL{GL, np, GW, GW, 0, 0}, opGU{GU, np, GW, GW, 0, 0};
    const Operand opTg{Tg, np, GW, GW, 0, 0};
    const int ng = (nb + kSolveGroup - 1) / kSolveGroup;
    for (int kl = 0; kl < kSolveGroup && ok; ++kl) {
        for (int g = 0; g < ng && ok; ++g) {  // Y_k = Y_k L_kk^-T
            const int g0 = g * kSolveGroup, g1 = std::min(nb, g0 + kSolveGroup), gs = g0 * BL, w = (g1 - g0) * BL;
            if (g0 + kl < g1)
                ok = add(ginv, EPI_STORE_F32, w, BL, BL, at(opYL, gs, kl * BL), at(opL, gs + kl * BL, 0), YL, GW, gs,
                         kl * BL, true, &flops_lu);
        }
        for (int g = 0; g < ng && ok; ++g) {  // Y_{>k} -= Y_k L_{>k,k}^T
            const int g0 = g * kSolveGroup, g1 = std::min(nb, g0 + kSolveGroup), gs = g0 * BL, ge = g1 * BL,
                      w = ge - gs, kb = gs + kl * BL;
            if (g0 + kl < g1 && kb + BL < ge)
                ok = add(ginv, EPI_SUB_F32, w, ge - kb - BL, BL, at(opYL, gs, kl * BL), at(opA, kb + BL, kb), YL, GW,
                         gs, (kl + 1) * BL, true, &flops_lu);
        }
    }
    for (int kl = kSolveGroup - 1; kl >= 0 && ok; --kl) {
        for (int g = 0; g < ng && ok; ++g) {  // Y_k = Y_k U_kk^-T
            const int g0 = g * kSolveGroup, g1 = std::min(nb, g0 + kSolveGroup), gs = g0 * BL, w = (g1 - g0) * BL;
            if (g0 + kl < g1)
                ok = add(ginv, EPI_STORE_F32, w, BL, BL, at(opYU, gs, kl * BL), at(opU, gs + kl * BL, 0), YU, GW, gs,
                         kl * BL, true, &flops_lu);
        }
        for (int g = 0; g < ng && ok; ++g) {  // Y_{<k} -= Y_k U_{<k,k}^T
            const int g0 = g * kSolveGroup, g1 = std::min(nb, g0 + kSolveGroup), gs = g0 * BL, w = (g1 - g0) * BL,
                      kb = gs + kl * BL;
            if (g0 + kl < g1 && kb > gs)
                ok = add(ginv, EPI_SUB_F32, w, kb - gs, BL, at(opYU, gs, kl * BL), at(opA, gs, kb), YU, GW, gs, 0,
                         true, &flops_lu);
        }
    }
    // The N-RHS solves by groups: Z_g = Z_g G_g^T (G_g = L_gg^-1 or U_gg^-1, one GEMM with
    // K = the group's width, into Tg and copied back), then one update with the same K carries
    // the group to the columns beyond it (forward) or before it (backward).
    for (int g = 0; g < ng && ok; ++g) {
        const int g0 = g * kSolveGroup, g1 = std::min(nb, g0 + kSolveGroup), gs = g0 * BL, ge = g1 * BL, w = ge - gs;
        fwd_steps.push_back(Step{static_cast<int>(fwd.size()), gs, w});
        ok = add(fwd, EPI_STORE_F32, N, w, w, at(opZ, 0, gs), at(opGL, gs, 0), Tg, GW, 0, 0, false, &flops_solve);
        fwd_steps.push_back(Step{-1, gs, w});
        if (ok && ge < N) {
            fwd_steps.push_back(Step{static_cast<int>(fwd.size()), gs, w});
            ok = add(fwd, EPI_SUB_F32, N, N - ge, w, at(opTg, 0, 0), at(opA, ge, gs), Z32, np, 0, ge, false,
                     &flops_solve);
        }
    }
    for (int g = ng - 1; g >= 0 && ok; --g) {
        const int g0 = g * kSolveGroup, g1 = std::min(nb, g0 + kSolveGroup), gs = g0 * BL, ge = g1 * BL, w = ge - gs;
        bwd_steps.push_back(Step{static_cast<int>(bwd.size()), gs, w});
        ok = add(bwd, EPI_STORE_F32, N, w, w, at(opZ, 0, gs), at(opGU, gs, 0), Tg, GW, 0, 0, false, &flops_solve);
        bwd_steps.push_back(Step{-1, gs, w});
        if (ok && gs > 0) {
            bwd_steps.push_back(Step{static_cast<int>(bwd.size()), gs, w});
            ok = add(bwd, EPI_SUB_F32, N, gs, w, at(opTg, 0, 0), at(opA, 0, gs), Z32, np, 0, 0, false, &flops_solve);
        }
    }
    if (!ok) {
        set_error("mixed path: %s", err.c_str());
        return DL_EDEVICE;
    }
    auto *dprob = static_cast<GemmProblem *>(ws.get("mx_probs", sizeof(GemmProblem) * probs.size()));
    if (!dprob) {
        set_error("mixed path: device allocation failed (table)");
        return DL_ENOMEM;
    }
    MCK(cudaMemcpyAsync(dprob, probs.data(), sizeof(GemmProblem) * probs.size(), cudaMemcpyHostToDevice, s));
    MCK(gemm_prepare(KIND_TF32, true, BL, EPI_STORE_F32));
    MCK(gemm_prepare(KIND_TF32, true, BL, EPI_SUB_F32));

    auto run = [&](const Launch &L) -> cudaError_t {
        ++launches;
        return gemm_launch(KIND_TF32, true, BL, L.epi, dprob + L.first, L.count, L.tiles,
                           std::min(L.tiles, ctx->sms), ws.status, ctx->budget_ns, s);
    };

    // ---- LU ----------------------------------------------------------------------------
    MCK(cudaFuncSetAttribute(diag_lu_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kDiagSmem)));
    for (int k = 0; k < nb; ++k) {
        const int64_t kb = static_cast<int64_t>(k) * BL;
        diag_lu_inv_kernel<<<1, kDiagThreads, kDiagSmem, s>>>(A32 + kb * np + kb, np, Linv + kb * BL, Uinv + kb * BL,
                                                      UinvT + kb * BL, ws.status);
        MCK(cudaGetLastError());
        ++launches;
        if (lu_panel[k] >= 0) {
            const int rem = N - static_cast<int>(kb) - BL;
            MCK(transpose(A32 + kb * np + kb + BL, np, BL, rem, T, BL, s));  // T = A12^T
            MCK(run(lu[lu_panel[k]]));                                        // T = U12^T, L21
            MCK(transpose(T, BL, rem, BL, A32 + kb * np + kb + BL, np, s));  // A12 = U12
            MCK(run(lu[lu_trail[k]]));                                        // A22 -= L21 U12
            launches += 2;
        }
    }
    // group inverses: Y = I on each group's rows, the grouped steps, then G = Y^T per group
    MCK(cudaMemsetAsync(YL, 0, np * GW * 4, s));
    MCK(cudaMemsetAsync(YU, 0, np * GW * 4, s));
    group_identity_kernel<<<static_cast<unsigned>((np + 255) / 256), 256, 0, s>>>(YL, YU, N, static_cast<int>(GW));
    MCK(cudaGetLastError());
    ++launches;
    for (const Launch &L : ginv) MCK(run(L));
    for (int64_t gs = 0; gs < np; gs += GW) {
        const int w = static_cast<int>(std::min<int64_t>(GW, np - gs));
        MCK(transpose(YL + gs * GW, GW, w, w, GL + gs * GW, GW, s));
        MCK(transpose(YU + gs * GW, GW, w, w, GU + gs * GW, GW, s));
        launches += 2;
    }
    MCK(cudaEventRecord(ev[5], s));
    auto solve = [&]() -> cudaError_t {
        cudaError_t e;
        for (int pass = 0; pass < 2; ++pass) {
            const std::vector<Step> &steps = pass == 0 ? fwd_steps : bwd_steps;
            const std::vector<Launch> &list = pass == 0 ? fwd : bwd;
            for (const Step &st_ : steps) {
                if (st_.launch >= 0) {
                    if ((e = run(list[st_.launch])) != cudaSuccess) return e;
                } else if ((e = cudaMemcpy2DAsync(Z32 + st_.gs, np * 4, Tg, GW * 4, static_cast<size_t>(st_.w) * 4, np,
                                                  cudaMemcpyDeviceToDevice, s)) != cudaSuccess) {
                    return e;
                }
            }
        }
        return cudaSuccess;
    };
    MCK(solve());
    const int64_t cnt = np * np;
    const unsigned eblocks = static_cast<unsigned>(std::min<int64_t>((cnt + 255) / 256, 8 * 1024));
    f32_to_f64_kernel<<<eblocks, 256, 0, s>>>(Z32, Z64, cnt);
    MCK(cudaGetLastError());
    ++launches;
    MCK(cudaEventRecord(ev[6], s));

    // ---- refinement ----------------------------------------------------------------------
    const double tol = ctx->cfg.refine_tol > 0 ? ctx->cfg.refine_tol : 1e-13;
    const int max_iters = ctx->cfg.refine_max_iters > 0 ? ctx->cfg.refine_max_iters : 30;
    // rows of Z per residual block: as many (up to 3) as shared memory holds
    const size_t row_bytes = sizeof(long long) * static_cast<size_t>(np);
    const int rows_per_block = static_cast<int>(std::min<size_t>(3, kResidualSmem / row_bytes));
    if (rows_per_block < 1) {
        set_error("mixed path: n = %d exceeds the residual's shared-memory row (%zu bytes)", n, kResidualSmem);
        return DL_EINVAL;
    }
    const size_t res_smem = row_bytes * rows_per_block;
    int deg_bits = 0;  // 2^deg_bits >= ||E||_inf (the terms of one sum)
    while ((1ull << deg_bits) < std::max<unsigned long long>(dmax, 1)) ++deg_bits;
    auto residual = [&](unsigned long long *rmax_p) -> cudaError_t {
        const unsigned grid = static_cast<unsigned>((np + rows_per_block - 1) / rows_per_block);
        cudaError_t e;
        switch (rows_per_block) {
            case 3:
                if ((e = cudaFuncSetAttribute(residual_fixed_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              static_cast<int>(res_smem))) != cudaSuccess)
                    return e;
                residual_fixed_kernel<3><<<grid, 1024, res_smem, s>>>(csr_ptr, csr_col, n, N, deg_bits, eps, Z64, Z32,
                                                                     rmax_p, At);
                break;
            case 2:
                if ((e = cudaFuncSetAttribute(residual_fixed_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              static_cast<int>(res_smem))) != cudaSuccess)
                    return e;
                residual_fixed_kernel<2><<<grid, 1024, res_smem, s>>>(csr_ptr, csr_col, n, N, deg_bits, eps, Z64, Z32,
                                                                     rmax_p, At);
                break;
            default:
                if ((e = cudaFuncSetAttribute(residual_fixed_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              static_cast<int>(res_smem))) != cudaSuccess)
                    return e;
                residual_fixed_kernel<1><<<grid, 1024, res_smem, s>>>(csr_ptr, csr_col, n, N, deg_bits, eps, Z64, Z32,
                                                                     rmax_p, At);
        }
        return cudaGetLastError();
    };
    unsigned long long *rmax_d = ws.scal + 20;
    double rmax = 0.0, best = 0.0;
    int it = 0, stall = 0;
    // The FP64 residual has a rounding floor of about (row length) * u * max|X|; refinement
    // stops at tol, or when it no longer halves the residual once that is below 1e-8 * eps.
    const double floor_ok = 1e-8 * eps;
    for (;;) {
        MCK(cudaMemsetAsync(rmax_d, 0, sizeof(unsigned long long), s));
        MCK(residual(rmax_d));
        ++launches;
        unsigned long long h = 0;
        MCK(cudaMemcpyAsync(&h, rmax_d, sizeof(h), cudaMemcpyDeviceToHost, s));
        MCK(cudaStreamSynchronize(s));
        std::memcpy(&rmax, &h, sizeof(rmax));
        if (rmax <= tol * eps) break;
        if (it == 0 || rmax < 0.5 * best) {
            best = rmax;
            stall = 0;
        } else if (++stall >= 2 && best <= floor_ok) {
            break;
        }
        if (it >= max_iters) {
            set_error("mixed path: refinement stopped at max|R|/eps = %.3g after %d steps", rmax / eps, it);
            return DL_ENOTCONV;
        }
        MCK(solve());
        add_f32_kernel<<<eblocks, 256, 0, s>>>(Z64, Z32, cnt);
        MCK(cudaGetLastError());
        ++launches;
        ++it;
    }
    MCK(transpose(Z64, np, N, N, X64, np, s));  // X = Z^T
    ++launches;
    MCK(cudaEventRecord(ev[7], s));
    MCK(cudaEventSynchronize(ev[7]));
    if (st) {
        st->iters = it;
        st->final_resid = rmax / eps;
        st->gemm_flops = flops_lu + flops_solve * (1 + it);
        st->gemm_launches = static_cast<int>(lu.size() + ginv.size() + (fwd.size() + bwd.size()) * (1 + it));
        float t1 = 0, t2 = 0, t3 = 0;
        cudaEventElapsedTime(&t1, ev[4], ev[5]);
        cudaEventElapsedTime(&t2, ev[5], ev[6]);
        cudaEventElapsedTime(&t3, ev[6], ev[7]);
        st->ms_factor = t1;
        st->ms_solve = t2;
        st->ms_refine = t3;
    }
    *launches_io += launches;
    return DL_OK;
}

}  // namespace dl
