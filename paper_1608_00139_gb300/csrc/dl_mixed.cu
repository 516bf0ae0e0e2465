// dl_mixed.cu -- R~ = (I - eps E)^-1 eps E (Proposition 1) on the TF32 tensor cores, with FP64
// iterative refinement (DL_PATH_MIXED).
//
//   1. A = I - eps E in FP32 (padded with the identity).
//   2. Block LU of A without pivoting, blocks of b = 128 (A is strictly diagonally dominant by
//      rows, proof of Proposition 1, so every Schur complement is too and block elimination is
//      stable):  A = L U with L unit block lower (L_ik = A_ik S_kk^-1) and U block upper
//      (U_kj = A_kj after the eliminations before k, diagonal blocks S_kk).  Per block k:
//        update: block row and column k receive the updates of the steps since the last bulk
//               update (left-looking, one GEMM, K up to 4 b);
//        diag:  S_kk^-1 (one CTA: Gauss-Jordan on the CUDA cores, products on mma.sync TF32);
//        L21 = A21 S_kk^-1 (in place), T = A12^T;
//        bulk:  after every unit of G = 2 or 4 steps (single steps at the end), the rest of the
//               trailing matrix, A22 -= L21 U12 with K = G b for the whole unit.
//      The chain (the diagonal block's update, diag, L21) runs on a stream of the greatest
//      priority as programmatic launches, the rest of each step's update and the transposes on
//      two more, the bulk update on a middle priority and on all SMs but a reserve (tuned per
//      size), so the chain of 128 x 128 steps proceeds while the bulk update streams through HBM.
//   3. W = A^-1 in FP32: the block solves applied to the identity (kept transposed, Z = I A^-T,
//      by groups of 8 blocks with precomputed inverses of the groups' diagonal parts, so that
//      every product is a tensor-core GEMM with K = 1024), then W = Z^T.
//   4. Refinement in FP64 on Z = X^T, from Z = 0:  R^T = (eps E - A X)^T, i.e.
//        R^T[j][i] = eps * sum_{k : E[i][k]} (Z[j][k] + [k = j]) - Z[j][i]
//      (E is 0/1: E X is a sum of rows of X, summed exactly in 64-bit fixed point);
//      D^T = R^T W^T, one TF32 GEMM of n x n x n; Z += D^T; until max|R| <= tol * eps.  The first
//      step (Z = 0, R^T = (eps E)^T) is the solve itself; each later one contracts the error by
//      about ||I - W A||, a few TF32 units times kappa(A), kappa_inf(A) <= 2 (1 + ||E||_inf).
//   5. X = Z^T; model X > 0 (Theorem 1); entries in the guard band are counted and the exact
//      boolean recheck of R2 = min1(E + E R2) confirms the model or adds lost facts.
// Every product is a "TN" GEMM (both operands stored with K contiguous), the form the TF32
// tensor cores run here; that is why the right-hand side is kept transposed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "dl_ctx.h"
#include "dl_internal.h"
#include "dl_ptx.cuh"

namespace dl {

namespace {

constexpr int BL = 128;        // LU block size = GEMM tile
constexpr int TT = 32;         // transpose tile
constexpr int kSolveGroup = 8;  // blocks per group of the solves (1024 columns)
constexpr int kMaxGroup = 4;    // LU steps per unit sharing one bulk update, at most

__global__ void build_a_kernel(const uint8_t *__restrict__ E, int n, int np, float eps, float *__restrict__ A) {
    const int64_t row = blockIdx.y;
    for (int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; c < np;
         c += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float e = (row < n && c < n && E[row * n + c]) ? eps : 0.0f;
        A[row * np + c] = (c == row ? 1.0f : 0.0f) - e;
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

// S^-1 of the BL x BL block at A (row stride lda), one CTA of 256 threads, by block inversion of
// its 64 x 64 quarters  S = [[P, B], [C, D]]:
//     P^-1;  Y = P^-1 B;  X = C P^-1;  Sd = (D - C Y)^-1;
//     S^-1 = [[P^-1 - (-Y Sd) X, -Y Sd], [-Sd X, Sd]]
// (Schur complement; A is strictly diagonally dominant by rows and so are P and D - C Y, so no
// pivoting is needed).  The two 64 x 64 inverses by Gauss-Jordan on the CUDA cores (4 x 4 register
// tiles, two pivots per barrier: every thread applies step k and forms row and column k + 1 as
// step k leaves them from the same published values); the six 64 x 64 products on the tensor
// cores (mma.sync m16n8k8, TF32 operands rounded to nearest, FP32 accumulate).  S^-1 comes out
// within TF32 accuracy, below what the LU's TF32 products use it at: it only preconditions the
// refinement.  A pivot that is not positive sets ST_BAD_INPUT.  Writes S^-1 and S^-T (BL x BL,
// row-major).  Dynamic shared memory: kDiagSmem bytes.
constexpr int kDiagThreads = 256;
constexpr int kHB = BL / 2;                 // quarter size
constexpr int kLdS = BL + 4, kLdH = kHB + 8;  // shared-memory row strides
constexpr size_t kDiagSmem = (static_cast<size_t>(BL) * kLdS + 2 * kHB * kLdH + 8 * kHB) * sizeof(float);

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// out (64 x 64, ldo) = alpha P Q + beta out (P, Q 64 x 64 in shared memory, not aliasing out);
// warp w computes rows 16 (w mod 4) .. + 16 and columns 32 (w / 4) .. + 32 as four 16 x 8 tiles.
__device__ void quarter_product(const float *P, int ldp, const float *Q, int ldq, float *out, int ldo, float alpha,
                                float beta) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = 16 * (warp & 3);
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[j][r] = 0.f;
#pragma unroll
    for (int k0 = 0; k0 < kHB; k0 += 8) {
        const uint32_t a0 = to_tf32(P[(m0 + g) * ldp + k0 + t]);
        const uint32_t a1 = to_tf32(P[(m0 + g + 8) * ldp + k0 + t]);
        const uint32_t a2 = to_tf32(P[(m0 + g) * ldp + k0 + t + 4]);
        const uint32_t a3 = to_tf32(P[(m0 + g + 8) * ldp + k0 + t + 4]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n0 = 8 * ((warp >> 2) * 4 + j);
            const uint32_t b0 = to_tf32(Q[(k0 + t) * ldq + n0 + g]);
            const uint32_t b1 = to_tf32(Q[(k0 + t + 4) * ldq + n0 + g]);
            asm volatile(
                "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+f"(acc[j][0]), "+f"(acc[j][1]), "+f"(acc[j][2]), "+f"(acc[j][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int n0 = 8 * ((warp >> 2) * 4 + j);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            float *o = out + (m0 + g + 8 * (r >> 1)) * ldo + n0 + 2 * t + (r & 1);
            *o = beta != 0.f ? fmaf(alpha, acc[j][r], beta * *o) : alpha * acc[j][r];
        }
    }
}

// One elimination step on a thread's 4 x 4 tile, pivot kk of the tile (ro / co: the tile holds the
// pivot row / column; c = the pivot column at the tile's rows, rp = the pivot row at the tile's
// columns times p = 1 / pivot).  Written as one update a <- a - c' rp' for every element, with
// c'[kk] = c[kk] - 1 on the pivot row, rp'[kk] = p on the pivot column and the pivot column of a
// replaced by the unit vector e_k: that gives the pivot row times p, the pivot column times -p, p
// at the pivot and a - c rp elsewhere, one FMA per element instead of a select per element.
template <int kk>
__device__ __forceinline__ void gj_step(float (&a)[4][4], bool ro, bool co, const float (&c)[4], const float (&rp)[4],
                                        float p) {
    float cc[4], rr[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) cc[i] = c[i], rr[i] = rp[i];
    if (ro) cc[kk] -= 1.f;
    if (co) {
        rr[kk] = p;
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i][kk] = (ro && i == kk) ? 1.f : 0.f;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) a[i][j] = fmaf(-cc[i], rr[j], a[i][j]);
}

// Steps k = kb + kk and k + 1 from one publication of rows and columns k, k + 1 (buffer buf).
template <int kk>
__device__ __forceinline__ void gj_pair(float (&a)[4][4], int r0, int c0, int k, bool ro, bool co,
                                        float (*rowbuf)[kHB], float (*colbuf)[kHB], bool *bad) {
    const float2 s0 = *reinterpret_cast<const float2 *>(&rowbuf[0][k]);
    const float2 s1 = *reinterpret_cast<const float2 *>(&rowbuf[1][k]);
    const float s00 = s0.x, s01 = s0.y, s10 = s1.x, s11 = s1.y;
    const float4 cv = *reinterpret_cast<const float4 *>(&colbuf[0][r0]);
    const float4 c1v = *reinterpret_cast<const float4 *>(&colbuf[1][r0]);
    const float4 rv = *reinterpret_cast<const float4 *>(&rowbuf[0][c0]);
    const float4 r1v = *reinterpret_cast<const float4 *>(&rowbuf[1][c0]);
    const float p = __fdividef(1.0f, s00);
    const float c[4] = {cv.x, cv.y, cv.z, cv.w}, c1[4] = {c1v.x, c1v.y, c1v.z, c1v.w};
    const float rp[4] = {rv.x * p, rv.y * p, rv.z * p, rv.w * p}, r1[4] = {r1v.x, r1v.y, r1v.z, r1v.w};
    gj_step<kk>(a, ro, co, c, rp, p);  // step k
    // row and column k + 1 as step k leaves them (the same uniform update), and the next pivot
    const float s01p = s01 * p;
    const float piv2 = fmaf(-s10, s01p, s11);
    const float p2 = __fdividef(1.0f, piv2);
    *bad |= !(s00 > 0.0f) || !isfinite(p) || !(piv2 > 0.0f) || !isfinite(p2);
    float c2[4], rp2[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) c2[i] = fmaf(-(ro && i == kk ? c[i] - 1.f : c[i]), s01p, c1[i]);
#pragma unroll
    for (int j = 0; j < 4; ++j) rp2[j] = (co && j == kk ? -s10 * p : fmaf(-s10, rp[j], r1[j])) * p2;
    gj_step<kk + 1>(a, ro, co, c2, rp2, p2);  // step k + 1
}

// In-place Gauss-Jordan inverse of the 64 x 64 quarter at R (row stride ld); two pivots per
// barrier.  rowbuf / colbuf: [buffer][pivot row or column k, k + 1][64].
__device__ void quarter_inverse(float *R, int ld, float (*rowbuf)[2][kHB], float (*colbuf)[2][kHB], bool *bad) {
    const int r0 = 4 * (threadIdx.x >> 4), c0 = 4 * (threadIdx.x & 15);
    float a[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) a[i][j] = R[(r0 + i) * ld + c0 + j];
#pragma unroll 1
    for (int kb = 0; kb < kHB; kb += 4) {
        const bool ro = r0 == kb, co = c0 == kb;
#pragma unroll
        for (int kk = 0; kk < 4; kk += 2) {
            const int k = kb + kk, buf = (k >> 1) & 1;
            if (ro)
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    *reinterpret_cast<float4 *>(&rowbuf[buf][h][c0]) =
                        make_float4(a[kk + h][0], a[kk + h][1], a[kk + h][2], a[kk + h][3]);
            if (co)
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    *reinterpret_cast<float4 *>(&colbuf[buf][h][r0]) =
                        make_float4(a[0][kk + h], a[1][kk + h], a[2][kk + h], a[3][kk + h]);
            __syncthreads();
            if (kk == 0) gj_pair<0>(a, r0, c0, k, ro, co, rowbuf[buf], colbuf[buf], bad);
            else gj_pair<2>(a, r0, c0, k, ro, co, rowbuf[buf], colbuf[buf], bad);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) R[(r0 + i) * ld + c0 + j] = a[i][j];
}

__global__ void __launch_bounds__(kDiagThreads) diag_inv_kernel(const float *__restrict__ A, int64_t lda,
                                                                float *__restrict__ Sinv, float *__restrict__ SinvT,
                                                                int *status) {
    static_assert(BL == 128 && kDiagThreads == 256, "64 x 64 quarters, 4 x 4 tiles");
    grid_dep_launch();  // the successor (L21) may launch now: it waits for this kernel's end
    grid_dep_wait();    // the diagonal block as its update before leaves it
    extern __shared__ __align__(16) float dsm[];
    float *S = dsm;                 // BL x kLdS
    float *Yq = S + BL * kLdS;      // kHB x kLdH
    float *Xq = Yq + kHB * kLdH;    // kHB x kLdH
    auto *rowbuf = reinterpret_cast<float(*)[2][kHB]>(Xq + kHB * kLdH);
    auto *colbuf = rowbuf + 2;
    for (int e = threadIdx.x; e < BL * BL / 4; e += kDiagThreads) {
        const int r = e / (BL / 4), c = 4 * (e % (BL / 4));
        *reinterpret_cast<float4 *>(S + r * kLdS + c) = *reinterpret_cast<const float4 *>(A + r * lda + c);
    }
    __syncthreads();
    float *Pq = S, *Bq = S + kHB, *Cq = S + kHB * kLdS, *Dq = S + kHB * kLdS + kHB;
    bool bad = false;
    quarter_inverse(Pq, kLdS, rowbuf, colbuf, &bad);           // P^-1
    __syncthreads();
    quarter_product(Pq, kLdS, Bq, kLdS, Yq, kLdH, 1.f, 0.f);   // Y = P^-1 B
    quarter_product(Cq, kLdS, Pq, kLdS, Xq, kLdH, 1.f, 0.f);   // X = C P^-1
    __syncthreads();
    quarter_product(Cq, kLdS, Yq, kLdH, Dq, kLdS, -1.f, 1.f);  // D - C Y
    __syncthreads();
    quarter_inverse(Dq, kLdS, rowbuf, colbuf, &bad);           // Sd
    __syncthreads();
    quarter_product(Dq, kLdS, Xq, kLdH, Cq, kLdS, -1.f, 0.f);  // lower left: -Sd X
    quarter_product(Yq, kLdH, Dq, kLdS, Bq, kLdS, -1.f, 0.f);  // upper right: -Y Sd
    __syncthreads();
    quarter_product(Bq, kLdS, Xq, kLdH, Pq, kLdS, -1.f, 1.f);  // upper left: P^-1 - (-Y Sd) X
    __syncthreads();
    if (bad) atomicOr(status, ST_BAD_INPUT);
    for (int e = threadIdx.x; e < BL * BL / 4; e += kDiagThreads) {  // S^-1, row-major
        const int r = e / (BL / 4), c = 4 * (e % (BL / 4));
        *reinterpret_cast<float4 *>(Sinv + r * BL + c) = *reinterpret_cast<const float4 *>(S + r * kLdS + c);
    }
    // S^-T through a 32 x 33 tile per warp (in the quarter buffers, free now): conflict-free
    // shared-memory reads and whole 128-byte rows written
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *tw = Yq + warp * 32 * 33;
    for (int t = warp; t < (BL / 32) * (BL / 32); t += kDiagThreads / 32) {
        const int tr = 32 * (t / (BL / 32)), tc = 32 * (t % (BL / 32));
        for (int i = 0; i < 32; ++i) tw[lane * 33 + i] = S[(tr + i) * kLdS + tc + lane];
        __syncwarp();
        for (int j = 0; j < 32; ++j) SinvT[(tc + j) * BL + tr + lane] = tw[j * 33 + lane];
        __syncwarp();
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

// Scale of row j of Z in the residual: every term of a sum (the +1 or A[i][j] included) stays
// below 2^hb, hb from the row's largest exponent field, and a sum of at most 2^deg_bits terms
// below 2^62.
__device__ __forceinline__ int row_scale(int ex_max, int deg_bits, int min_hb = 1) {
    const int hb = max(max(ex_max - 1022, 0) + 1, min_hb);
    return max(0, 62 - deg_bits - hb);
}

// floor(s * eps_q / 2^62) for |s| < 2^62, 0 <= eps_q <= 2^62: eps s in fixed point, with
// eps_q = round(eps 2^62) (a 128-bit product, integer units only).
__device__ __forceinline__ long long mul_eps(long long s, long long eps_q) {
    const unsigned long long lo = static_cast<unsigned long long>(s) * static_cast<unsigned long long>(eps_q);
    const long long hi = __mul64hi(s, eps_q);
    return static_cast<long long>((static_cast<unsigned long long>(hi) << 2) | (lo >> 62));
}

// r (|r| < 2^62) as a float, within one rounding of the nearest: two exact 32-bit conversions
// of its halves combined by one fma.
__device__ __forceinline__ float float_of(long long r) {
    const float hi = static_cast<float>(static_cast<int>(r >> 31));
    const float lo = static_cast<float>(static_cast<unsigned>(r & 0x7FFFFFFFll));
    return fmaf(hi, 2147483648.0f, lo);
}

// Residual of the transposed system:
//     R^T[j][i] = eps * sum_{k in succ(i)} (Z[j][k] + [k = j]) - Z[j][i]
// (right-hand side eps E; with rhs, a general right-hand side eps A, the [k = j] term becomes
// A[i][j]), as FP32 (right-hand side of the next correction), and max |R| into *rmax (bits of a
// non-negative float).  The sums are exact in 64-bit fixed point: Zf[j][k] = round(Z[j][k] 2^e_j)
// (plus 2^e_j at k = j for the closure's right-hand side), written by add_fix_kernel with e_j
// chosen so that no sum reaches 2^62; eps times a sum is an exact 128-bit product with
// eps_q = round(eps 2^62), floored; the result is rounded once to FP32.  Every error is below
// 2^-(62 - deg_bits) of the row's largest entry, under one FP64 ulp of it, and no FP64 unit is
// used.  Two kernels compute it, by the density of E:

// R^T[j][i] from the fixed-point sum and Zf[j][i] (the result's last step).
__device__ __forceinline__ float residual_entry(long long sum, long long z, int i, int j, int n, int e,
                                                long long eps_q, float inv, const uint8_t *rhs, const double *rhsr) {
    if (rhsr != nullptr) {
        sum += fixed_of(__double_as_longlong(rhsr[static_cast<int64_t>(i) * n + j]), e);
    } else if (rhs != nullptr) {
        if (rhs[static_cast<int64_t>(i) * n + j]) sum += 1ll << e;
    } else if (i == j) {
        z -= 1ll << e;  // Zf carries the [k = j] term
    }
    return float_of(mul_eps(sum, eps_q) - z) * inv;
}

// (1) Sparse E: G rows j of Zf per block in shared memory, a thread per row i walking its
// successors (few gathers per row; Zf is read once).
template <int G>
__global__ void __launch_bounds__(1024, 1)
    residual_rows_kernel(const int *__restrict__ ptr, const int *__restrict__ col, int n, int np, long long eps_q,
                         const int *__restrict__ escale, const long long *__restrict__ Zf, float *__restrict__ R,
                         unsigned *rmax, const uint8_t *__restrict__ rhs, const double *__restrict__ rhsr) {
    extern __shared__ long long zi[];  // G rows of np
    const int j0 = blockIdx.x * G;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const longlong2 *src = reinterpret_cast<const longlong2 *>(Zf + static_cast<int64_t>(j0 + g) * np);
        longlong2 *dst = reinterpret_cast<longlong2 *>(zi + g * np);
        const bool live = j0 + g < np;
#pragma unroll 4
        for (int t = threadIdx.x; t < np / 2; t += blockDim.x) dst[t] = live ? src[t] : make_longlong2(0, 0);
    }
    __syncthreads();
    int e[G];
    float inv[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        e[g] = j0 + g < np ? escale[j0 + g] : 0;
        inv[g] = __int_as_float((127 - e[g]) << 23);  // 2^-e (0 <= e <= 62)
    }
    float m = 0.0f;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        long long sum[G];
#pragma unroll
        for (int g = 0; g < G; ++g) sum[g] = 0;
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
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int j = j0 + g;
            if (j >= np) break;
            float r = 0.0f;
            if (i < n && j < n) r = residual_entry(sum[g], zi[g * np + i], i, j, n, e[g], eps_q, inv[g], rhs, rhsr);
            R[static_cast<int64_t>(j) * np + i] = r;
            m = fmaxf(m, fabsf(r));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(rmax, __float_as_uint(m));
}

// (2) Denser E: a block is kRJ = 32 rows j (one per lane) by kRI = 512 rows i (kIW = 32 per warp
// of kRWarps = 16).  It reads the fixed-point Z transposed, ZfT[k][j] = Zf[j][k], so that the
// band of kBand columns k of its 32 rows j is a kBand x 32 tile of 256-byte rows: TMA copies it
// into shared memory (two buffers, the next band's copy in flight during this band's gathers), and
// the 32 lanes reading one k read 256 contiguous bytes (no bank conflict).  The edges come
// bucketed by (i-tile, band) with band-local columns (bucket_*_kernel): a warp copies its rows'
// edges of the band into a shared buffer with coalesced loads, then row by row every lane adds
// its row's entry at each edge's column.  Bands without edges in the i-tile are skipped.  Every
// index read serves 32 rows of Z.  The copies complete on mbarriers whose waits are bounded: on
// expiry the kernel records ST_TIMEOUT_FULL, waits (bounded) for its copies still in flight and
// returns.
constexpr int kRJ = 32, kIW = 32, kRWarps = 16, kRI = kRWarps * kIW, kBand = 384, kBox = 128;
constexpr int kEdgeBuf = 256;  // band-local columns per warp buffered at once
constexpr size_t kBandBytes = sizeof(long long) * kBand * kRJ;
constexpr size_t kResidualSmem = 2 * kBandBytes + sizeof(uint16_t) * kRWarps * kEdgeBuf + 64;

// Bucketed edges: segment (t, b) holds the edges (i, k) with i in i-tile t (kRI rows) and k in
// band b (kBand columns), ordered by (i, k); off[(t * nbd + b) * kRI + il] is the first edge of
// row t kRI + il in it (flat exclusive scan of the counts, so the next entry is the row's end).
// cnt: one count per (segment, row), zeroed by the caller; a warp per row.
__global__ void bucket_count_kernel(const int *__restrict__ ptr, const int *__restrict__ col, int n, int nbd,
                                    int *__restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    const int t = i / kRI, il = i - t * kRI;
    for (int q = ptr[i] + lane; q < ptr[i + 1]; q += 32)
        atomicAdd(&cnt[(t * nbd + col[q] / kBand) * kRI + il], 1);
}

__global__ void bucket_fill_kernel(const int *__restrict__ ptr, const int *__restrict__ col, int n, int nbd,
                                   const int *__restrict__ off, uint16_t *__restrict__ edges) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    const int t = i / kRI, il = i - t * kRI;
    const int q0 = ptr[i], q1 = ptr[i + 1];
    for (int q = q0 + lane; q < q1; q += 32) {
        const int k = col[q], b = k / kBand;
        int lo = q0, hi = q;  // first successor of row i in band b (columns sorted)
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (col[mid] < b * kBand) lo = mid + 1;
            else hi = mid;
        }
        edges[off[(t * nbd + b) * kRI + il] + (q - lo)] = static_cast<uint16_t>(k - b * kBand);
    }
}

// ZfT[k][j] = round(Z[j][k] 2^e_j), plus 2^e_j at k = j < n when add_identity; 32 x 32 tiles.
__global__ void fix_transpose_kernel(const double *__restrict__ Z, const int *__restrict__ escale, int n, int np,
                                     int add_identity, long long *__restrict__ ZfT) {
    __shared__ long long tile[TT][TT + 1];
    const int k0 = blockIdx.x * TT, j0 = blockIdx.y * TT;
    for (int y = threadIdx.y; y < TT; y += blockDim.y) {
        const int j = j0 + y, k = k0 + threadIdx.x;
        const int e = escale[j];
        long long v = fixed_of(__double_as_longlong(Z[static_cast<int64_t>(j) * np + k]), e);
        if (add_identity && k == j && j < n) v += 1ll << e;
        tile[y][threadIdx.x] = v;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < TT; y += blockDim.y)
        ZfT[static_cast<int64_t>(k0 + y) * np + j0 + threadIdx.x] = tile[threadIdx.x][y];
}

__global__ void __launch_bounds__(32 * kRWarps, 1)
    residual_band_kernel(const __grid_constant__ CUtensorMap zmap, int n, int np, int nbd, const int *__restrict__ off,
                         const uint16_t *__restrict__ edges, long long eps_q, const int *__restrict__ escale,
                         const long long *__restrict__ ZfT, float *__restrict__ R, unsigned *rmax,
                         const uint8_t *__restrict__ rhs, const double *__restrict__ rhsr, int *status,
                         uint64_t budget_ns) {
    extern __shared__ __align__(1024) uint8_t rsmem[];
    uint16_t *ebuf = reinterpret_cast<uint16_t *>(rsmem + 2 * kBandBytes) + (threadIdx.x >> 5) * kEdgeBuf;
    uint64_t *full = reinterpret_cast<uint64_t *>(rsmem + 2 * kBandBytes + sizeof(uint16_t) * kRWarps * kEdgeBuf);
    __shared__ int abort_s;
    const unsigned fullmask = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ni = (np + kRI - 1) / kRI;
    const int it = blockIdx.x % ni, jt = blockIdx.x / ni;  // the i-tiles of one j-tile are adjacent
    const int j0 = jt * kRJ, i0 = it * kRI + warp * kIW;   // i0 < np or the warp only helps
    const int j = j0 + lane;
    const int e = escale[j];
    const int *seg = off + it * nbd * kRI;  // segment b's row starts at seg + b kRI
    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        fence_barrier_init();
        abort_s = 0;
    }
    __syncthreads();
    // the bands with edges in this i-tile, in order: b is live iff seg[b kRI] != seg[(b + 1) kRI]
    auto next_live = [&](int b) {
        while (b < nbd && seg[b * kRI] == seg[(b + 1) * kRI]) ++b;
        return b;
    };
    auto slab = [&](int buf) { return reinterpret_cast<long long *>(rsmem + buf * kBandBytes); };
    auto issue = [&](int b, int buf) {  // one thread: the band's kBand x 32 tile of ZfT
        mbar_arrive_expect_tx(&full[buf], static_cast<uint32_t>(kBandBytes));
        for (int c = 0; c < kBand / kBox; ++c)
            tma_load_2d(&zmap, slab(buf) + c * kBox * kRJ, &full[buf], j0, b * kBand + c * kBox);
    };
    long long acc[kIW];
#pragma unroll
    for (int q = 0; q < kIW; ++q) acc[q] = 0;
    int b = next_live(0), use = 0;
    uint32_t phases = 0u;    // bit u: parity of buffer u's next completion
    uint32_t inflight = 0u;  // bit u: thread 0 issued a copy into buffer u that nobody has waited on
    if (b < nbd && threadIdx.x == 0) {
        issue(b, 0);
        inflight = 1u;
    }
    while (b < nbd) {
        const int bn = next_live(b + 1);
        if (bn < nbd && threadIdx.x == 0) {  // the other buffer was freed by the previous barrier
            issue(bn, use ^ 1);
            inflight |= 1u << (use ^ 1);
        }
        const bool ok = mbar_wait_bounded(&full[use], (phases >> use) & 1u, budget_ns, status, ST_TIMEOUT_FULL);
        if (ok) {
            phases ^= 1u << use;
            inflight &= ~(1u << use);
        } else {
            atomicOr(&abort_s, 1);
        }
        if (__syncthreads_or(abort_s)) {  // every thread leaves together; thread 0 drains its copies
            if (threadIdx.x == 0)
                for (int u = 0; u < 2; ++u)
                    if ((inflight >> u) & 1u)
                        mbar_wait_bounded(&full[u], (phases >> u) & 1u, budget_ns, status, ST_TIMEOUT_DRAIN);
            return;
        }
        const long long *sl = slab(use);
        const int *so = seg + b * kRI;
        const int rs = so[min(warp * kIW + lane, kRI)];      // lane l: start of row il = l
        const int re = so[min(warp * kIW + lane + 1, kRI)];  // ... and its end
        const int ws = __shfl_sync(fullmask, rs, 0), we = __shfl_sync(fullmask, re, kIW - 1);
        for (int w0 = ws; w0 < we; w0 += kEdgeBuf) {
            const int wl = min(kEdgeBuf, we - w0);
            __syncwarp();
            for (int p = lane; p < wl; p += 32) ebuf[p] = edges[w0 + p];
            __syncwarp();
#pragma unroll
            for (int il = 0; il < kIW; ++il) {
                const int lo = max(__shfl_sync(fullmask, rs, il), w0) - w0;
                const int hi = min(__shfl_sync(fullmask, re, il), w0 + wl) - w0;
                long long a = acc[il];
                for (int p = lo; p < hi; ++p) a += sl[ebuf[p] * kRJ + lane];
                acc[il] = a;
            }
        }
        __syncthreads();  // this buffer's gathers are done: it may be refilled
        b = bn;
        use ^= 1;
    }
    if (i0 >= np) return;
    // R^T[j][i0 .. i0 + kIW - 1]: lane j writes kIW consecutive entries of its row
    float m = 0.0f;
    const float inv = __int_as_float((127 - e) << 23);  // 2^-e (0 <= e <= 62)
    float *rrow = R + static_cast<int64_t>(j) * np + i0;
#pragma unroll
    for (int il = 0; il < kIW; il += 4) {
        float v4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + il + u;
            const long long z = ZfT[static_cast<int64_t>(i) * np + j];
            v4[u] = i < n && j < n ? residual_entry(acc[il + u], z, i, j, n, e, eps_q, inv, rhs, rhsr) : 0.0f;
            m = fmaxf(m, fabsf(v4[u]));
        }
        *reinterpret_cast<float4 *>(rrow + il) = make_float4(v4[0], v4[1], v4[2], v4[3]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(fullmask, m, o));
    if (lane == 0 && m > 0.0f) atomicMax(rmax, __float_as_uint(m));
}

// Z += D for row j (one block per row, the new row kept in shared memory), then the row's scale
// e_j = row_scale(largest exponent field, deg_bits, min_hb) into escale[j] (min_hb: a real right-
// hand side's terms are below 2^min_hb too) and the fixed-point row
// Zf[j][k] = round(Z[j][k] 2^e_j), plus 2^e_j at k = j < n when add_identity (the closure's
// [k = j] term of the residual).
__global__ void __launch_bounds__(256) add_fix_kernel(double *__restrict__ Z, const float *__restrict__ D, int n,
                                                      int np, int deg_bits, int min_hb, int add_identity,
                                                      int *__restrict__ escale, long long *__restrict__ Zf) {
    // (Zf == nullptr: only Z and escale; fix_transpose_kernel then writes the transposed copy)
    extern __shared__ double zrow_s[];
    __shared__ int wmax[8];
    const int j = blockIdx.x;
    const int64_t base = static_cast<int64_t>(j) * np;
    int ex = 0;
    for (int k = threadIdx.x * 4; k < np; k += blockDim.x * 4) {
        const float4 d = *reinterpret_cast<const float4 *>(D + base + k);
        double2 z0 = *reinterpret_cast<const double2 *>(Z + base + k);
        double2 z1 = *reinterpret_cast<const double2 *>(Z + base + k + 2);
        z0.x += static_cast<double>(d.x);
        z0.y += static_cast<double>(d.y);
        z1.x += static_cast<double>(d.z);
        z1.y += static_cast<double>(d.w);
        *reinterpret_cast<double2 *>(Z + base + k) = z0;
        *reinterpret_cast<double2 *>(Z + base + k + 2) = z1;
        *reinterpret_cast<double2 *>(zrow_s + k) = z0;
        *reinterpret_cast<double2 *>(zrow_s + k + 2) = z1;
        ex = max(ex, max(max(static_cast<int>((__double_as_longlong(z0.x) >> 52) & 0x7FF),
                             static_cast<int>((__double_as_longlong(z0.y) >> 52) & 0x7FF)),
                         max(static_cast<int>((__double_as_longlong(z1.x) >> 52) & 0x7FF),
                             static_cast<int>((__double_as_longlong(z1.y) >> 52) & 0x7FF))));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = ex;
    __syncthreads();
    int m = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) m = max(m, wmax[w]);
    const int e = row_scale(m, deg_bits, min_hb);
    if (threadIdx.x == 0) escale[j] = e;
    if (Zf == nullptr) return;
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        long long v = fixed_of(__double_as_longlong(zrow_s[k]), e);
        if (add_identity && k == j && j < n) v += 1ll << e;
        Zf[base + k] = v;
    }
}

// R^T = (eps F)^T for a real F (n x n FP64), FP32, zero padding.
__global__ void build_rt_real_kernel(const double *__restrict__ F, int n, int np, double eps, float *__restrict__ R) {
    __shared__ float tile[TT][TT + 1];
    const int c0 = blockIdx.x * TT, r0 = blockIdx.y * TT;
    for (int y = threadIdx.y; y < TT; y += blockDim.y) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        tile[y][threadIdx.x] = (r < n && c < n) ? static_cast<float>(eps * F[static_cast<int64_t>(r) * n + c]) : 0.0f;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < TT; y += blockDim.y) {
        const int r = c0 + y, c = r0 + threadIdx.x;
        if (r < np && c < np) R[static_cast<int64_t>(r) * np + c] = tile[threadIdx.x][y];
    }
}

// R^T = (eps A)^T (np x np, zero padding): the residual of Z = 0, the first right-hand side.
__global__ void build_rt_kernel(const uint8_t *__restrict__ A, int n, int np, float eps, float *__restrict__ R) {
    __shared__ float tile[TT][TT + 1];
    const int c0 = blockIdx.x * TT, r0 = blockIdx.y * TT;
    for (int y = threadIdx.y; y < TT; y += blockDim.y) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        tile[y][threadIdx.x] = (r < n && c < n && A[static_cast<int64_t>(r) * n + c]) ? eps : 0.0f;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < TT; y += blockDim.y) {
        const int r = c0 + y, c = r0 + threadIdx.x;  // R[r][c] = eps A[c][r]
        if (r < np && c < np) R[static_cast<int64_t>(r) * np + c] = tile[threadIdx.x][y];
    }
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

// Z = I (np x np, zeroed before).
__global__ void identity_kernel(float *Z, int np) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < np) Z[static_cast<int64_t>(r) * np + r] = 1.0f;
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
    int bn;
};

// The GEMM table of one mixed solve (every product is C (=|-=) A B'^T, both operands K-major).
struct Table {
    std::vector<GemmProblem> probs;
    std::string err;
    // Append one problem to `list`: grouped into the list's last launch when asked and the
    // kinds match, else as a launch of its own.
    bool add(std::vector<Launch> &list, GemmEpi epi, int bn, int M, int N, int K, const Operand &A,
             const Operand &B, float *C, int64_t ldc, int r0, int c0, bool group_with_prev, double *fl) {
        GemmProblem p;
        GemmEpilogue e{};
        e.c32 = C;
        e.ld_c32 = ldc;
        e.out_row0 = r0;
        e.out_col0 = c0;
        if (!gemm_make_problem(&p, KIND_TF32, true, bn, M, N, K, A, B, e, &err)) return false;
        const int t = p.tiles_m * p.tiles_n;
        if (group_with_prev && !list.empty() && list.back().epi == epi && list.back().bn == bn &&
            list.back().first + list.back().count == static_cast<int>(probs.size())) {
            p.tile_start = list.back().tiles;
            list.back().count += 1;
            list.back().tiles += t;
        } else {
            p.tile_start = 0;
            list.push_back(Launch{static_cast<int>(probs.size()), 1, t, epi, bn});
        }
        probs.push_back(p);
        *fl += 2.0 * M * N * K;
        return true;
    }
};

Operand at(Operand o, int r, int c) {
    o.row0 = r;
    o.col0 = c;
    return o;
}

dl_status mixed_streams(Workspace &ws) {
    if (ws.mx_stream[0]) return DL_OK;
    int least = 0, greatest = 0;
    MCK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    // the chain (and beside it the transposes and each step's off-chain update) first, then the
    // bulk update, then the inverse's early groups (which fill the SMs the chain-bound end of the
    // factorisation leaves idle)
    MCK(cudaStreamCreateWithPriority(&ws.mx_stream[0], cudaStreamNonBlocking, greatest));
    MCK(cudaStreamCreateWithPriority(&ws.mx_stream[1], cudaStreamNonBlocking, std::max(greatest, least - 1)));
    MCK(cudaStreamCreateWithPriority(&ws.mx_stream[2], cudaStreamNonBlocking, least));
    MCK(cudaStreamCreateWithPriority(&ws.mx_stream[3], cudaStreamNonBlocking, greatest));
    MCK(cudaStreamCreateWithPriority(&ws.mx_stream[4], cudaStreamNonBlocking, greatest));
    for (auto &e : ws.mx_ev) MCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    for (auto &e : ws.mx_gev) MCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return DL_OK;
}

}  // namespace

// The first product of the refinement when E is sparse: with Z = 0 the residual is R = eps E, and
// D^T = R^T W^T has rows  D^T[j][:] = eps * sum_{k : E[k][j] = 1} W^T[k][:]  (rows of W^T, row-major
// in WT, gathered over the predecessors of j from the CSR of E^T): nnz(E) rows read instead of an
// n^3 product.  Rows j >= n are zero; columns i >= n come out zero (W's padded rows are identity
// rows).
constexpr int kFirstThreads = 256;

__global__ void __launch_bounds__(kFirstThreads) first_product_kernel(const int *__restrict__ pptr,
                                                                      const int *__restrict__ pcol, int n, int np,
                                                                      float eps, const float *__restrict__ WT,
                                                                      float *__restrict__ D) {
    const int j = blockIdx.x;
    float *dj = D + static_cast<int64_t>(j) * np;
    const int q0 = j < n ? pptr[j] : 0, q1 = j < n ? pptr[j + 1] : 0;
    for (int c = 4 * threadIdx.x; c < np; c += 4 * kFirstThreads) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        int q = q0;
        for (; q + 4 <= q1; q += 4) {  // four rows in flight
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                v[u] = *reinterpret_cast<const float4 *>(WT + static_cast<int64_t>(pcol[q + u]) * np + c);
#pragma unroll
            for (int u = 0; u < 4; ++u) acc.x += v[u].x, acc.y += v[u].y, acc.z += v[u].z, acc.w += v[u].w;
        }
        for (; q < q1; ++q) {
            const float4 v = *reinterpret_cast<const float4 *>(WT + static_cast<int64_t>(pcol[q]) * np + c);
            acc.x += v.x, acc.y += v.y, acc.z += v.z, acc.w += v.w;
        }
        *reinterpret_cast<float4 *>(dj + c) = make_float4(eps * acc.x, eps * acc.y, eps * acc.z, eps * acc.w);
    }
}

// Graphs with at most this many facts per constant take the gathered first product.
constexpr int64_t kSparseFirstDegree = 12;

// Consecutive NVTX ranges, one open at a time.
struct Phases {
    bool open = false;
    void to(const char *name) {
        if (open) nvtxRangePop();
        nvtxRangePushA(name);
        open = true;
    }
    ~Phases() {
        if (open) nvtxRangePop();
    }
};

dl_status tc_mixed(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a, dl_stats *st,
                   const uint8_t *E, double eps, unsigned long long dmax, int *launches_io) {
    const int32_t n = a.n;
    const int64_t np = round_up(std::max<int64_t>(n, 1), 256);
    const int nb = static_cast<int>(np / BL);
    const int N = static_cast<int>(np);
    int launches = 0;
    dl_status rc = mixed_streams(ws);
    if (rc) return rc;
    cudaStream_t P = ws.mx_stream[0], U = ws.mx_stream[1], V = ws.mx_stream[2], Q = ws.mx_stream[3];
    cudaStream_t Rs = ws.mx_stream[4];
    auto *A32 = static_cast<float *>(ws.get("mx_A", np * np * 4));
    auto *W32 = static_cast<float *>(ws.get("mx_W", np * np * 4));   // Z = A^-T, then R
    auto *Wt = static_cast<float *>(ws.get("mx_Wt", np * np * 4));   // W = A^-1
    auto *D32 = static_cast<float *>(ws.get("mx_D", np * np * 4));
    auto *Z64 = static_cast<double *>(ws.get("mx_Z64", np * np * 8));
    auto *X64 = static_cast<double *>(ws.get("mx_X64", np * np * 8));
    // transposed row panels: two slots of np rows (indexed by the absolute column) x kMaxGroup BL
    // (the panels of a unit of steps side by side)
    auto *T2 = static_cast<float *>(ws.get("mx_T", 2 * np * kMaxGroup * BL * 4));
    auto *Sinv = static_cast<float *>(ws.get("mx_Sinv", np * BL * 4));
    auto *SinvT = static_cast<float *>(ws.get("mx_SinvT", np * BL * 4));
    const int64_t GW = std::min<int64_t>(np, static_cast<int64_t>(kSolveGroup) * BL);
    auto *YL = static_cast<float *>(ws.get("mx_YL", np * GW * 4));
    auto *YU = static_cast<float *>(ws.get("mx_YU", np * GW * 4));
    auto *GL = static_cast<float *>(ws.get("mx_GL", np * GW * 4));
    auto *GU = static_cast<float *>(ws.get("mx_GU", np * GW * 4));
    auto *Tg = static_cast<float *>(ws.get("mx_Tg", np * GW * 4));
    auto *csr_cnt = static_cast<int *>(ws.get("mx_cnt", (np + 1) * 4));
    auto *csr_ptr = static_cast<int *>(ws.get("mx_ptr", (np + 1) * 4));
    if (!A32 || !W32 || !Wt || !D32 || !Z64 || !X64 || !T2 || !Sinv || !SinvT || !YL || !YU || !GL || !GU || !Tg ||
        !csr_cnt || !csr_ptr) {
        set_error("mixed path: device allocation failed");
        return DL_ENOMEM;
    }
    float *R32 = W32;  // the residual reuses Z's buffer once W = Z^T is formed
    cudaEvent_t *ev = ws.ev;
    Phases ph;  // NVTX ranges of the host-side phases
    ph.to("mixed:set-up");
    MCK(cudaEventRecord(ev[4], s));
    {
        dim3 grid(static_cast<unsigned>(std::min<int64_t>((np + 255) / 256, 64)), static_cast<unsigned>(np));
        build_a_kernel<<<grid, 256, 0, s>>>(E, n, N, static_cast<float>(eps), A32);
        MCK(cudaGetLastError());
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

    // ---- GEMM table ---------------------------------------------------------------------
    Table tb;
    std::vector<Launch> l21, udiag, urest, bulk, wfwd, wbwd, refine;
    double flops_lu = 0, flops_w = 0, flops_ref = 0;
    const Operand opA{A32, np, np, np, 0, 0};
    const Operand opS{Sinv, np, BL, BL, 0, 0}, opST{SinvT, np, BL, BL, 0, 0};
    bool ok = true;
    std::vector<int> has_bulk(nb, -1), has_udiag(nb, -1), has_urest(nb, -1), has_l21(nb, -1);
    // Steps k < grouped go in units of G consecutive steps (G = 2 or 4), later steps are single.
    // Within a unit the updates are left-looking: before step j's pivot, block row and column j
    // receive, in one GEMM with K = (j - s) BL, the updates of every step s .. j - 1 since the
    // unit's start (of the whole previous unit when j starts a unit) -- its diagonal block as one
    // launch on the chain, the rest beside the diagonal inverse.  The unit's last step then issues
    // one bulk update, K = G BL, of the rows and columns from the second block after it.  So the
    // chain carries one small GEMM per step, each block row and column is read and written once
    // per unit, and the trailing matrix G times less often.  G and the grouped steps: tuned per size.
    const TuneEntry tn = tuned(ctx, np);
    const int G = tn.mx_group == 4 ? 4 : 2;
    int grouped = tn.mx_pairs >= 0 ? tn.mx_pairs : nb / 2;
    grouped = std::max(0, std::min(grouped, nb - 6)) / G * G;
    auto unit_of = [&](int k) { return k < grouped ? k / G : grouped / G + (k - grouped); };
    auto pos_of = [&](int k) { return k < grouped ? k % G : 0; };          // q, the step's place in its unit
    auto size_of = [&](int k) { return k < grouped ? G : 1; };             // the unit's number of steps
    auto start_of = [&](int k) { return k - pos_of(k); };
    const int64_t ldT = static_cast<int64_t>(kMaxGroup) * BL;
    // T(k) = A_{k, >k}^T of every step of a unit, side by side (row = absolute column), two units' worth
    auto opT_of = [&](int k) {
        return Operand{T2 + static_cast<int64_t>(unit_of(k) & 1) * np * ldT, np, ldT, ldT, 0, 0};
    };
    for (int j = 0; j < nb && ok; ++j) {
        const int jb = j * BL, rem = N - jb - BL;
        const int q = pos_of(j), gu = size_of(j), k0 = start_of(j);
        if (j > 0) {  // the left-looking update of block row and column j
            const int s = q >= 1 ? k0 : start_of(j - 1), K = (j - s) * BL;
            const Operand opTs = opT_of(s);
            has_udiag[j] = static_cast<int>(udiag.size());
            ok = tb.add(udiag, EPI_SUB_F32, BL, BL, BL, K, at(opA, jb, s * BL), at(opTs, jb, 0), A32, np, jb, jb,
                        false, &flops_lu);
            if (ok && rem > 0) {
                has_urest[j] = static_cast<int>(urest.size());
                ok = tb.add(urest, EPI_SUB_F32, BL, rem, BL, K, at(opA, jb + BL, s * BL), at(opTs, jb, 0), A32, np,
                            jb + BL, jb, false, &flops_lu);
                ok = ok && tb.add(urest, EPI_SUB_F32, BL, BL, rem, K, at(opA, jb, s * BL), at(opTs, jb + BL, 0), A32,
                                  np, jb, jb + BL, true, &flops_lu);
            }
        }
        if (!ok || rem <= 0) break;
        // L21 = A21 S^-1 (in place: each output tile reads only its own rows of A21)
        has_l21[j] = static_cast<int>(l21.size());
        ok = tb.add(l21, EPI_STORE_F32, BL, rem, BL, BL, at(opA, jb + BL, jb), at(opST, jb, 0), A32, np, jb + BL, jb,
                    false, &flops_lu);
        if (ok && q == gu - 1 && rem > BL) {  // the unit's bulk update (K = gu BL)
            has_bulk[j] = static_cast<int>(bulk.size());
            ok = tb.add(bulk, EPI_SUB_F32, 256, rem - BL, rem - BL, gu * BL, at(opA, jb + 2 * BL, k0 * BL),
                        at(opT_of(j), jb + 2 * BL, 0), A32, np, jb + 2 * BL, jb + 2 * BL, false, &flops_lu);
        }
    }
    // Inverses of the diagonal groups (kSolveGroup blocks each), once per factorisation.
    // L_gg is unit block lower: Y = I, Y_{>k} -= Y_k L_{>k,k}^T for k in order gives Y = L_gg^-T.
    // U_gg is block upper with diagonal blocks S_kk: Y = I, then for k descending
    // Y_k = Y_k S_kk^-T, Y_{<k} -= Y_k U_{<k,k}^T gives Y = U_gg^-T.  Every step is one launch over
    // all groups; transposed afterwards (GL = L_gg^-1, GU = U_gg^-1).
    const Operand opYL{YL, np, GW, GW, 0, 0}, opYU{YU, np, GW, GW, 0, 0};
    const Operand opGL{GL, np, GW, GW, 0, 0}, opGU{GU, np, GW, GW, 0, 0};
    const Operand opTg{Tg, np, GW, GW, 0, 0};
    const int ng = (nb + kSolveGroup - 1) / kSolveGroup;
    if (ng > static_cast<int>(sizeof(ws.mx_gev) / sizeof(ws.mx_gev[0]))) {
        set_error("mixed path: n = %d has more solve groups than supported", n);
        return DL_EINVAL;
    }
    std::vector<std::vector<Launch>> ginv(ng);  // one list per group (a group's inverse runs once its LU is final)
    for (int g = 0; g < ng && ok; ++g) {
        const int g0 = g * kSolveGroup, g1 = std::min(nb, g0 + kSolveGroup), gs = g0 * BL, ge = g1 * BL, w = ge - gs;
        for (int kl = 0; g0 + kl < g1 && ok; ++kl) {
            const int kb = gs + kl * BL;
            if (kb + BL < ge)
                ok = tb.add(ginv[g], EPI_SUB_F32, BL, w, ge - kb - BL, BL, at(opYL, gs, kl * BL), at(opA, kb + BL, kb),
                            YL, GW, gs, (kl + 1) * BL, false, &flops_lu);
        }
        for (int kl = g1 - g0 - 1; kl >= 0 && ok; --kl) {
            const int kb = gs + kl * BL;
            // Y_k = Y_k S_kk^-T (in place: N = BL), then Y_{<k} -= Y_k U_{<k,k}^T
            ok = tb.add(ginv[g], EPI_STORE_F32, BL, w, BL, BL, at(opYU, gs, kl * BL), at(opS, kb, 0), YU, GW, gs,
                        kl * BL, false, &flops_lu);
            if (ok && kb > gs)
                ok = tb.add(ginv[g], EPI_SUB_F32, BL, w, kb - gs, BL, at(opYU, gs, kl * BL), at(opA, gs, kb), YU, GW, gs,
                            0, false, &flops_lu);
        }
    }
    // W: the solves on Z = I.  Forward by groups, Z_g = Z_g L_gg^-T (into Tg, copied back) and
    // Z_{>g} -= Z_g L_{>g,g}^T; Z = L^-T is block upper triangular, so the forward steps of group g
    // touch rows [0, ge) only.  Backward by groups, Z_g = Z_g U_gg^-T, Z_{<g} -= Z_g U_{<g,g}^T.
    struct Step {
        int launch, gs, w, rows;  // launch < 0: copy Tg back into Z's columns [gs, gs + w), rows rows
    };
    std::vector<Step> fwd_steps, bwd_steps;
    const Operand opZ{W32, np, np, np, 0, 0};
    for (int g = 0; g < ng && ok; ++g) {
        const int g0 = g * kSolveGroup, g1 = std::min(nb, g0 + kSolveGroup), gs = g0 * BL, ge = g1 * BL, w = ge - gs;
        fwd_steps.push_back(Step{static_cast<int>(wfwd.size()), gs, w, ge});
        ok = tb.add(wfwd, EPI_STORE_F32, 256, ge, w, w, at(opZ, 0, gs), at(opGL, gs, 0), Tg, GW, 0, 0, false, &flops_w);
        fwd_steps.push_back(Step{-1, gs, w, ge});
        if (ok && ge < N) {
            fwd_steps.push_back(Step{static_cast<int>(wfwd.size()), gs, w, ge});
            ok = tb.add(wfwd, EPI_SUB_F32, 256, ge, N - ge, w, at(opTg, 0, 0), at(opA, ge, gs), W32, np, 0, ge, false,
                        &flops_w);
        }
    }
    for (int g = ng - 1; g >= 0 && ok; --g) {
        const int g0 = g * kSolveGroup, g1 = std::min(nb, g0 + kSolveGroup), gs = g0 * BL, ge = g1 * BL, w = ge - gs;
        bwd_steps.push_back(Step{static_cast<int>(wbwd.size()), gs, w, N});
        ok = tb.add(wbwd, EPI_STORE_F32, 256, N, w, w, at(opZ, 0, gs), at(opGU, gs, 0), Tg, GW, 0, 0, false, &flops_w);
        bwd_steps.push_back(Step{-1, gs, w, N});
        if (ok && gs > 0) {
            bwd_steps.push_back(Step{static_cast<int>(wbwd.size()), gs, w, N});
            ok = tb.add(wbwd, EPI_SUB_F32, 256, N, gs, w, at(opTg, 0, 0), at(opA, 0, gs), W32, np, 0, 0, false,
                        &flops_w);
        }
    }
    // refinement product D^T = R^T W^T (B operand W = A^-1, row-major)
    ok = ok && tb.add(refine, EPI_STORE_F32, 256, N, N, N, Operand{R32, np, np, np, 0, 0},
                      Operand{Wt, np, np, np, 0, 0}, D32, np, 0, 0, false, &flops_ref);
    if (!ok) {
        set_error("mixed path: %s", tb.err.c_str());
        return DL_EDEVICE;
    }
    auto *dprob = static_cast<GemmProblem *>(ws.get("mx_probs", sizeof(GemmProblem) * tb.probs.size()));
    if (!dprob) {
        set_error("mixed path: device allocation failed (table)");
        return DL_ENOMEM;
    }
    MCK(cudaMemcpyAsync(dprob, tb.probs.data(), sizeof(GemmProblem) * tb.probs.size(), cudaMemcpyHostToDevice, s));
    for (int bn : {128, 256}) {
        MCK(gemm_prepare(KIND_TF32, true, bn, EPI_STORE_F32));
        MCK(gemm_prepare(KIND_TF32, true, bn, EPI_SUB_F32));
    }
    MCK(cudaFuncSetAttribute(diag_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kDiagSmem)));
    auto run = [&](const Launch &L, int max_grid, cudaStream_t on, bool pdl = false) -> cudaError_t {
        ++launches;
        return gemm_launch(KIND_TF32, true, L.bn, L.epi, dprob + L.first, L.count, L.tiles,
                           std::min(L.tiles, max_grid), ws.status, ctx->budget_ns, on, nullptr, pdl);
    };
    const int sms = ctx->sms;
    // SMs the bulk update leaves to the chain (tuned per size bucket, else 32)
    const int reserve = std::min(std::max(1, tuned(ctx, np).mx_reserve), std::max(1, sms - 1));

    // ---- LU, then W = A^-1 (enqueued on s, P, Rs, Q, U, V; all join s) ----------------------
    auto enqueue = [&]() -> dl_status {
    ph.to("mixed:lu");
    MCK(cudaEventRecord(ws.mx_ev[0], s));  // the table and A are ready on s
    MCK(cudaStreamWaitEvent(P, ws.mx_ev[0], 0));
    MCK(cudaStreamWaitEvent(U, ws.mx_ev[0], 0));
    MCK(cudaStreamWaitEvent(V, ws.mx_ev[0], 0));
    MCK(cudaStreamWaitEvent(Q, ws.mx_ev[0], 0));
    // The inverse (on V, least priority): the group inverses and the forward solve of group g
    // start as soon as the LU's steps of group g are done (its L and U blocks, and L below it, are
    // final then: later steps write only block rows and columns beyond the group), so they fill
    // SMs the chain-bound end of the factorisation leaves idle; the backward solve needs all of U.
    MCK(cudaMemsetAsync(YL, 0, np * GW * 4, V));
    MCK(cudaMemsetAsync(YU, 0, np * GW * 4, V));
    group_identity_kernel<<<static_cast<unsigned>((np + 255) / 256), 256, 0, V>>>(YL, YU, N, static_cast<int>(GW));
    MCK(cudaGetLastError());
    MCK(cudaMemsetAsync(W32, 0, np * np * 4, V));
    identity_kernel<<<static_cast<unsigned>((np + 255) / 256), 256, 0, V>>>(W32, N);
    MCK(cudaGetLastError());
    launches += 2;
    // After the LU, V's GEMMs are programmatic launches as well (during it they are not: their
    // early CTAs would hold SMs the chain needs).
    bool lu_done = false;
    auto run_steps = [&](const std::vector<Step> &steps, const std::vector<Launch> &list, int gs_only) -> cudaError_t {
        for (const Step &sp : steps) {
            if (gs_only >= 0 && sp.gs != gs_only) continue;
            cudaError_t e;
            if (sp.launch >= 0) {
                if ((e = run(list[sp.launch], sms, V, lu_done)) != cudaSuccess) return e;
            } else if ((e = cudaMemcpy2DAsync(W32 + sp.gs, np * 4, Tg, GW * 4, static_cast<size_t>(sp.w) * 4, sp.rows,
                                              cudaMemcpyDeviceToDevice, V)) != cudaSuccess) {
                return e;
            }
        }
        return cudaSuccess;
    };
    int groups_started = 0;
    auto inverse_group = [&](int g) -> cudaError_t {  // on V, after the group's LU steps
        cudaError_t e;
        for (const Launch &L : ginv[g])
            if ((e = run(L, sms, V, lu_done)) != cudaSuccess) return e;
        const int64_t gs = static_cast<int64_t>(g) * GW;
        const int w = static_cast<int>(std::min<int64_t>(GW, np - gs));
        if ((e = transpose(YL + gs * GW, GW, w, w, GL + gs * GW, GW, V)) != cudaSuccess) return e;
        if ((e = transpose(YU + gs * GW, GW, w, w, GU + gs * GW, GW, V)) != cudaSuccess) return e;
        launches += 2;
        groups_started = g + 1;
        return run_steps(fwd_steps, wfwd, static_cast<int>(gs));
    };
    cudaEvent_t evT[2] = {ws.mx_ev[0], ws.mx_ev[1]}, evB[2] = {ws.mx_ev[2], ws.mx_ev[3]};
    cudaEvent_t evR = ws.mx_ev[4], evQ = ws.mx_ev[5], evL = ws.mx_ev[6];
    // Bulk updates issued and not yet waited for by the chain: (the issuing step, its event).  The
    // bulk issued at step j covers the rows and columns from block j + 2.
    std::vector<std::pair<int, int>> bulks;
    // Per step j, on P (the chain): the update of diagonal block j, diag(j), L21(j); on Rs beside
    // diag(j): the rest of block row and column j's update, which L21(j) and T(j) wait for; on Q:
    // T(j).  The chain's kernels are programmatic launches: each one's launch and set-up overlap
    // the end of the one before it on P (diag lets L21 launch at once: L21's CTAs wait on SMs it
    // does not use).
    auto diag = [&](int64_t kb) -> cudaError_t {
        ++launches;
        return launch_programmatic(diag_inv_kernel, dim3(1), dim3(kDiagThreads), kDiagSmem, P,
                                   static_cast<const float *>(A32 + kb * np + kb), static_cast<int64_t>(np),
                                   Sinv + kb * BL, SinvT + kb * BL, ws.status);
    };
    for (int j = 0; j < nb; ++j) {
        const int64_t jb = static_cast<int64_t>(j) * BL;
        const int rem = N - static_cast<int>(jb) - BL;
        if (j > 0) {
            MCK(cudaStreamWaitEvent(P, evQ, 0));  // T(j - 1)
            const int jp = j - 1;
            if (has_bulk[jp] >= 0) {  // the bulk update of the unit that step j - 1 ends
                const int par = unit_of(jp) & 1;
                for (const auto &b : bulks)  // (an event is re-recorded only after its last wait)
                    if (b.second == par) MCK(cudaStreamWaitEvent(P, evB[par], 0));
                MCK(cudaEventRecord(evT[par], P));
                MCK(cudaStreamWaitEvent(U, evT[par], 0));
                MCK(run(bulk[has_bulk[jp]], std::max(1, sms - reserve), U));
                MCK(cudaEventRecord(evB[par], U));
                bulks.emplace_back(jp, par);
            }
            // the bulk updates whose region holds block row and column j
            while (!bulks.empty() && bulks.front().first + 2 <= j) {
                MCK(cudaStreamWaitEvent(P, evB[bulks.front().second], 0));
                bulks.erase(bulks.begin());
            }
            MCK(cudaEventRecord(evL, P));
            MCK(run(udiag[has_udiag[j]], sms, P, true));
            if (has_urest[j] >= 0) {
                MCK(cudaStreamWaitEvent(Rs, evL, 0));
                MCK(run(urest[has_urest[j]], sms, Rs));
                MCK(cudaEventRecord(evR, Rs));
            }
        }
        MCK(diag(jb));
        if (rem <= 0) break;
        if (j > 0) MCK(cudaStreamWaitEvent(P, evR, 0));  // column j below the diagonal block
        // L21 runs beside a bulk update, which leaves it `reserve` SMs
        MCK(run(l21[has_l21[j]], bulks.empty() ? sms : reserve, P, true));
        if ((j + 1) % kSolveGroup == 0) {  // group (j + 1) / kSolveGroup - 1 is final
            const int g = (j + 1) / kSolveGroup - 1;
            MCK(cudaEventRecord(ws.mx_gev[g], P));
            MCK(cudaStreamWaitEvent(V, ws.mx_gev[g], 0));
            MCK(inverse_group(g));
        }
        if (j > 0) MCK(cudaStreamWaitEvent(Q, evR, 0));  // row j
        float *Tj = T2 + static_cast<int64_t>(unit_of(j) & 1) * np * ldT + (jb + BL) * ldT + pos_of(j) * BL;
        MCK(transpose(A32 + jb * np + jb + BL, np, BL, rem, Tj, ldT, Q));
        ++launches;
        MCK(cudaEventRecord(evQ, Q));
    }
    MCK(cudaEventRecord(ws.mx_ev[0], U));  // (evT[0] is no longer needed)
    MCK(cudaStreamWaitEvent(P, ws.mx_ev[0], 0));
    MCK(cudaEventRecord(ws.mx_ev[1], P));
    MCK(cudaStreamWaitEvent(s, ws.mx_ev[1], 0));

    MCK(cudaEventRecordWithFlags(ev[5], s, cudaEventRecordExternal));  // the LU's end (a node in a graph)

    // ---- W = A^-1: the remaining groups' inverses and forward solves, then the backward solve --
    ph.to("mixed:inverse");
    MCK(cudaStreamWaitEvent(V, ws.mx_ev[1], 0));  // the whole LU
    lu_done = true;
    for (int g = groups_started; g < ng; ++g) MCK(inverse_group(g));
    MCK(run_steps(bwd_steps, wbwd, -1));
    MCK(transpose(W32, np, N, N, Wt, np, V));  // W = (A^-T)^T
    ++launches;
    MCK(cudaEventRecord(ws.mx_ev[2], V));
    MCK(cudaStreamWaitEvent(s, ws.mx_ev[2], 0));
    return DL_OK;
    };
    // The work above is a fixed sequence of about six hundred small launches for a given size:
    // it is captured once as a CUDA graph (per workspace, size, tuned shape and buffers) and
    // replayed, which removes most of the host launch cost and the gaps between dependent
    // launches on the chain.
    char gkey[512];
    std::snprintf(gkey, sizeof gkey, "%d %lld %d %d %d %d %llu %p %p %p %p %p %p %p %p %p %p %p %p %p %p", N,
                  static_cast<long long>(np), nb, G, grouped, reserve, static_cast<unsigned long long>(ctx->budget_ns),
                  static_cast<void *>(A32), static_cast<void *>(T2), static_cast<void *>(Sinv),
                  static_cast<void *>(SinvT), static_cast<void *>(YL), static_cast<void *>(YU), static_cast<void *>(GL),
                  static_cast<void *>(GU), static_cast<void *>(Tg), static_cast<void *>(W32), static_cast<void *>(Wt),
                  static_cast<void *>(dprob), static_cast<void *>(ws.status), static_cast<void *>(s));
    if (!ws.mx_graph || ws.mx_graph_key != gkey) {
        if (ws.mx_graph) {
            cudaGraphExecDestroy(ws.mx_graph);
            ws.mx_graph = nullptr;
        }
        const int before = launches;
        MCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        const dl_status rcap = enqueue();
        cudaGraph_t graph = nullptr;
        const cudaError_t ecap = cudaStreamEndCapture(s, &graph);
        if (rcap != DL_OK || ecap != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            if (rcap != DL_OK) return rcap;
            set_error("mixed path: capture of the factorisation failed: %s", cudaGetErrorString(ecap));
            return DL_EDEVICE;
        }
        const cudaError_t einst = cudaGraphInstantiate(&ws.mx_graph, graph, 0);
        cudaGraphDestroy(graph);
        if (einst != cudaSuccess) {
            ws.mx_graph = nullptr;
            set_error("mixed path: graph instantiation failed: %s", cudaGetErrorString(einst));
            return DL_EDEVICE;
        }
        ws.mx_graph_key = gkey;
        ws.mx_graph_launches = launches - before;
        launches = before;
    }
    MCK(cudaGraphLaunch(ws.mx_graph, s));
    launches += ws.mx_graph_launches;
    MCK(cudaEventRecord(ev[6], s));

    // ---- refinement from Z = 0 -------------------------------------------------------------
    ph.to("mixed:refine");
    const double tol = ctx->cfg.refine_tol > 0 ? ctx->cfg.refine_tol : 1e-13;
    const int max_iters = ctx->cfg.refine_max_iters > 0 ? ctx->cfg.refine_max_iters : 30;
    int deg_bits = 0;  // 2^deg_bits >= ||E||_inf + 1 (the terms of one sum, the +1 or A[i][j] included)
    while ((1ull << deg_bits) < std::max<unsigned long long>(dmax, 1) + 1) ++deg_bits;
    const bool general_rhs = a.rhs != nullptr || a.rhs_real != nullptr;
    int min_hb = 1;  // a real right-hand side's terms are below 2^min_hb as well
    if (a.rhs_real) {
        int ex = 0;
        std::frexp(std::max(a.rhs_bound, 1.0), &ex);  // rhs_bound < 2^ex
        min_hb = std::max(1, ex);
    }
    const long long eps_q = std::llround(std::ldexp(eps, 62));
    auto *escale = static_cast<int *>(ws.get("mx_escale", np * 4));
    auto *Zf = static_cast<long long *>(ws.get("mx_Zf", np * np * 8));
    if (!escale || !Zf) {
        set_error("mixed path: device allocation failed (row scales)");
        return DL_ENOMEM;
    }
    const size_t row_smem = static_cast<size_t>(np) * sizeof(double);
    if (row_smem > 227 * 1024) {
        set_error("mixed path: n = %d exceeds the refinement's shared-memory row (%zu bytes)", n, row_smem);
        return DL_EINVAL;
    }
    MCK(cudaFuncSetAttribute(add_fix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(row_smem)));
    // the residual kernel by density: rows of Zf per block for sparse E, bucketed bands otherwise
    const bool banded = static_cast<int64_t>(nnz) >= 32ll * n;
    const int rows_per_block = static_cast<int>(std::min<size_t>(3, (227 * 1024) / row_smem));
    const int nbd = (n + kBand - 1) / kBand, ni = static_cast<int>((np + kRI - 1) / kRI);
    int *boff = nullptr;
    uint16_t *bedges = nullptr;
    CUtensorMap zmap{};  // ZfT (banded residual)
    const bool need_x = a.out_rtilde != nullptr;  // (see the refinement loop below)
    if (banded && need_x) {
        const int64_t cells = static_cast<int64_t>(ni) * nbd * kRI;
        auto *bcnt = static_cast<int *>(ws.get("mx_bcnt", (cells + 1) * 4));
        boff = static_cast<int *>(ws.get("mx_boff", (cells + 1) * 4));
        auto *bscr = static_cast<int *>(ws.get("mx_bscr", (2 * (cells / 1024 + 2)) * 4));
        bedges = static_cast<uint16_t *>(ws.get("mx_bedges", std::max<size_t>(static_cast<size_t>(nnz), 8) * 2));
        if (!bcnt || !boff || !bscr || !bedges) {
            set_error("mixed path: device allocation failed (residual buckets)");
            return DL_ENOMEM;
        }
        MCK(cudaMemsetAsync(bcnt, 0, (cells + 1) * 4, s));
        bucket_count_kernel<<<static_cast<unsigned>((n + 7) / 8), 256, 0, s>>>(csr_ptr, csr_col, n, nbd, bcnt);
        MCK(cudaGetLastError());
        MCK(exclusive_scan_large(bcnt, static_cast<int>(cells), boff, bscr, s));
        bucket_fill_kernel<<<static_cast<unsigned>((n + 7) / 8), 256, 0, s>>>(csr_ptr, csr_col, n, nbd, boff, bedges);
        MCK(cudaGetLastError());
        launches += 3;
        MCK(cudaFuncSetAttribute(residual_band_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(kResidualSmem)));
        std::string err;
        if (!tensor_map_2d(&zmap, CU_TENSOR_MAP_DATA_TYPE_INT64, 8, Zf, np, np, np, kRJ, kBox, &err)) {
            set_error("mixed path: %s (residual)", err.c_str());
            return DL_EDEVICE;
        }
    } else {
        const int smem = static_cast<int>(row_smem * rows_per_block);
        MCK(cudaFuncSetAttribute(residual_rows_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        MCK(cudaFuncSetAttribute(residual_rows_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        MCK(cudaFuncSetAttribute(residual_rows_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    }
    auto residual = [&](unsigned *rmax_p) -> cudaError_t {
        if (banded) {
            dim3 tgrid(static_cast<unsigned>(np / TT), static_cast<unsigned>(np / TT));
            fix_transpose_kernel<<<tgrid, dim3(TT, 8), 0, s>>>(Z64, escale, n, N, general_rhs ? 0 : 1, Zf);
            residual_band_kernel<<<static_cast<unsigned>((np / kRJ) * ni), 32 * kRWarps, kResidualSmem, s>>>(
                zmap, n, N, nbd, boff, bedges, eps_q, escale, Zf, R32, rmax_p, a.rhs, a.rhs_real, ws.status,
                ctx->budget_ns);
            return cudaGetLastError();
        }
        const unsigned grid = static_cast<unsigned>((np + rows_per_block - 1) / rows_per_block);
        const size_t smem = row_smem * rows_per_block;
        if (rows_per_block == 3)
            residual_rows_kernel<3><<<grid, 1024, smem, s>>>(csr_ptr, csr_col, n, N, eps_q, escale, Zf, R32, rmax_p, a.rhs,
                                                             a.rhs_real);
        else if (rows_per_block == 2)
            residual_rows_kernel<2><<<grid, 1024, smem, s>>>(csr_ptr, csr_col, n, N, eps_q, escale, Zf, R32, rmax_p, a.rhs,
                                                             a.rhs_real);
        else
            residual_rows_kernel<1><<<grid, 1024, smem, s>>>(csr_ptr, csr_col, n, N, eps_q, escale, Zf, R32, rmax_p, a.rhs,
                                                             a.rhs_real);
        return cudaGetLastError();
    };
    // The first product as a gather for sparse E (the closure's own right-hand side eps E): the
    // CSR of E^T from a transposed byte copy of E.
    const bool sparse_first = !general_rhs && static_cast<int64_t>(nnz) <= kSparseFirstDegree * n;
    int *pptr = nullptr, *pcol = nullptr;
    if (sparse_first) {
        auto *Et = static_cast<uint8_t *>(ws.get("mx_Et", static_cast<size_t>(n) * n));
        auto *pcnt = static_cast<int *>(ws.get("mx_pcnt", (np + 1) * 4));
        pptr = static_cast<int *>(ws.get("mx_pptr", (np + 1) * 4));
        pcol = static_cast<int *>(ws.get("mx_pcol", static_cast<size_t>(std::max(nnz, 1)) * 4));
        if (!Et || !pcnt || !pptr || !pcol) {
            set_error("mixed path: device allocation failed (CSR of E^T)");
            return DL_ENOMEM;
        }
        MCK(transpose(E, n, n, n, Et, n, s));
        MCK(csr_build(Et, n, pcnt, pptr, s));
        MCK(csr_fill(Et, n, pptr, pcol, s));
        launches += 3;
    }
    // Without an R~ output only the model is wanted: X > 0 after the solve is already exact where
    // it is positive (A is an M-matrix and every quantity of the factorisation keeps its sign, so
    // no entry cancels to a spurious value), entries lost to underflow land in the guard band, and
    // the caller's certificate and recheck settle them; the refinement is then skipped.
    unsigned *rmax_d = reinterpret_cast<unsigned *>(ws.scal + 20);
    double rmax = 0.0, best = 0.0;
    int products = 0, stall = 0, gemm_products = 0;
    // The residual has a rounding floor of about (row length) * 2^-53 * max|X|; refinement stops
    // at tol, or when it no longer halves the residual once that is below 1e-8 * eps.
    const double floor_ok = 1e-8 * eps;
    MCK(cudaMemsetAsync(Z64, 0, np * np * 8, s));
    if (!sparse_first) {
        dim3 tgrid(static_cast<unsigned>(np / TT), static_cast<unsigned>(np / TT));
        if (a.rhs_real)
            build_rt_real_kernel<<<tgrid, dim3(TT, 8), 0, s>>>(a.rhs_real, n, N, eps, R32);
        else
            build_rt_kernel<<<tgrid, dim3(TT, 8), 0, s>>>(a.rhs ? a.rhs : E, n, N, static_cast<float>(eps), R32);
        MCK(cudaGetLastError());
        ++launches;
    }
    for (;;) {
        if (products == 0 && sparse_first) {
            // W^T row-major is still in W32 (the residual overwrites it from the first residual on)
            first_product_kernel<<<static_cast<unsigned>(np), kFirstThreads, 0, s>>>(pptr, pcol, n, N,
                                                                                   static_cast<float>(eps), W32, D32);
            MCK(cudaGetLastError());
            ++launches;
        } else {
            MCK(run(refine[0], sms, s));  // D^T = R^T W^T
            ++gemm_products;
        }
        add_fix_kernel<<<static_cast<unsigned>(np), 256, row_smem, s>>>(Z64, D32, n, N, deg_bits, min_hb,
                                                                      general_rhs ? 0 : 1, escale,
                                                                      banded || !need_x ? nullptr : Zf);
        MCK(cudaGetLastError());
        ++launches;
        ++products;
        if (!need_x) break;  // the model only: no refinement
        MCK(cudaMemsetAsync(rmax_d, 0, sizeof(unsigned), s));
        MCK(residual(rmax_d));
        ++launches;
        unsigned h = 0;
        MCK(cudaMemcpyAsync(&h, rmax_d, sizeof(h), cudaMemcpyDeviceToHost, s));
        MCK(cudaStreamSynchronize(s));
        float hf = 0.0f;
        std::memcpy(&hf, &h, sizeof(hf));
        rmax = hf;
        if (rmax <= tol * eps) break;
        if (products == 1 || rmax < 0.5 * best) {  // refinement steps must keep halving the residual
            best = rmax;
            stall = 0;
        } else if (++stall >= 2 && best <= floor_ok) {
            break;
        }
        if (products > max_iters) {
            set_error("mixed path: refinement stopped at max|R|/eps = %.3g after %d steps", rmax / eps, products - 1);
            return DL_ENOTCONV;
        }
    }
    MCK(transpose(Z64, np, N, N, X64, np, s));  // X = Z^T
    ++launches;
    MCK(cudaEventRecord(ev[7], s));
    MCK(cudaEventSynchronize(ev[7]));
    if (st) {
        st->iters = std::max(products - 1, 0);  // refinement steps after the first product (the solve)
        st->final_resid = need_x ? rmax / eps : -1.0;  // -1: no residual was formed (model only)
        st->gemm_flops = flops_lu + flops_w + flops_ref * gemm_products;
        size_t ginv_n = 0;
        for (const auto &gl : ginv) ginv_n += gl.size();
        st->gemm_launches = static_cast<int>(l21.size() + udiag.size() + urest.size() + bulk.size() + ginv_n + wfwd.size() +
                                             wbwd.size()) + gemm_products;
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
