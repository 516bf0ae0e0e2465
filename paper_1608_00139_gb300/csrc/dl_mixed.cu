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
// FP32, by Gauss-Jordan elimination held in registers: 1024 threads, thread t owns columns
// (t & 7) + 8 q, q = 0 .. 31, of row t >> 3 of the augmented BL x 2BL matrix (interleaved, so
// that the 8 threads of a row read 8 different shared-memory banks of the pivot row).
//  1. forward elimination of [A | I] (row_r -= (a_rk / a_kk) row_k for r > k) leaves [U | L^-1];
//  2. backward elimination of [U | I] (row_k /= u_kk, then row_i -= u_ik row_k for i < k; the
//     multipliers are U's entries, unchanged by the later steps) leaves U^-1 on the right.
// One barrier per step: the pivot row goes through a double-buffered shared row.
// Writes L^-1 (unit lower), U^-1 and U^-T, BL x BL each.
constexpr int kDiagThreads = 1024;
constexpr int kSolveGroup = 8;  // panels per group of the N-RHS solves

// v[j] for a runtime j (unrolled selects keep v in registers)
__device__ __forceinline__ float pick32(const float (&v)[32], int j) {
    float x = 0.0f;
#pragma unroll
    for (int q = 0; q < 32; ++q) x = q == j ? v[q] : x;
    return x;
}

__global__ void __launch_bounds__(kDiagThreads) diag_lu_inv_kernel(const float *A, int64_t lda, float *Linv,
                                                                   float *Uinv, float *UinvT, int *status) {
    static_assert(BL == 128, "the thread layout assumes 128-row diagonal blocks");
    __shared__ float piv[2][2 * BL];
    const int t = threadIdx.x;
    const int r = t >> 3, sg = t & 7;  // row r, columns sg + 8 q (q < 16: A / U, q >= 16: right half)
    const int row_lane0 = (t & 31) & ~7;
    float v[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        const int c = sg + 8 * q;
        v[q] = c < BL ? A[static_cast<int64_t>(r) * lda + c] : (c - BL == r ? 1.0f : 0.0f);
    }
    // 1. [A | I] -> [U | L^-1]
    for (int k = 0; k < BL; ++k) {
        float *p = piv[k & 1];
        if (r == k) {
#pragma unroll
            for (int q = 0; q < 32; ++q) p[sg + 8 * q] = v[q];
        }
        __syncthreads();
        const float pk = p[k];
        if (pk == 0.0f) {  // zero pivot (the M-matrix has none): report and stop (uniform)
            if (t == 0) atomicOr(status, ST_BAD_INPUT);
            return;
        }
        const float ark = __shfl_sync(0xffffffffu, pick32(v, k >> 3), row_lane0 + (k & 7));  // a_rk
        if (r > k) {
            const float m = ark / pk;
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int c = sg + 8 * q;
                if (c > k) v[q] = fmaf(-m, p[c], v[q]);
            }
        }
    }
    // L^-1 is the right half now: write it, then start the right half over from I
#pragma unroll
    for (int q = 16; q < 32; ++q) {
        const int c = sg + 8 * (q - 16);
        Linv[r * BL + c] = c < r ? v[q] : (c == r ? 1.0f : 0.0f);
        v[q] = c == r ? 1.0f : 0.0f;
    }
    __syncthreads();
    // 2. [U | I] -> U^-1 on the right (only the right half is updated)
    for (int k = BL - 1; k >= 0; --k) {
        float *p = piv[k & 1];
        const float ukk = __shfl_sync(0xffffffffu, pick32(v, k >> 3), row_lane0 + (k & 7));  // used in row k
        if (r == k) {
            const float inv = 1.0f / ukk;
#pragma unroll
            for (int q = 16; q < 32; ++q) {
                v[q] *= inv;
                p[sg + 8 * (q - 16)] = v[q];
            }
        }
        __syncthreads();
        const float uik = __shfl_sync(0xffffffffu, pick32(v, k >> 3), row_lane0 + (k & 7));  // U's entry (r, k)
        if (r < k) {
#pragma unroll
            for (int q = 16; q < 32; ++q) v[q] = fmaf(-uik, p[sg + 8 * (q - 16)], v[q]);
        }
    }
#pragma unroll
    for (int q = 16; q < 32; ++q) {
        const int c = sg + 8 * (q - 16);
        const float x = c >= r ? v[q] : 0.0f;
        Uinv[r * BL + c] = x;
        UinvT[c * BL + r] = x;
    }
}

// Residual of the transposed system, one block per row j of Z, the row staged in shared
// memory:  R^T[j][i] = eps * sum_{k in succ(i)} (Z[j][k] + [k = j]) - Z[j][i]  (FP64),
// stored as FP32 (right-hand side of the correction solve); max |R| -> *rmax.
__global__ void __launch_bounds__(256) residual_t_kernel(const int *__restrict__ ptr, const int *__restrict__ col,
                                                         int n, int np, double eps, const double *__restrict__ Z,
                                                         float *__restrict__ R, unsigned long long *rmax) {
    extern __shared__ double zs[];
    const int j = blockIdx.x;
    const double *zrow = Z + static_cast<int64_t>(j) * np;
    for (int t = threadIdx.x; t < np; t += blockDim.x) zs[t] = zrow[t];
    __syncthreads();
    if (threadIdx.x == 0 && j < n) zs[j] += 1.0;  // the eps E[i][j] term, as k = j
    __syncthreads();
    double m = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        double r = 0.0;
        if (i < n && j < n) {
            double s = 0.0;
            for (int q = ptr[i]; q < ptr[i + 1]; ++q) s += zs[col[q]];
            r = eps * s - (zs[i] - (i == j ? 1.0 : 0.0));
        }
        R[static_cast<int64_t>(j) * np + i] = static_cast<float>(r);
        m = fmax(m, fabs(r));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0)
        atomicMax(rmax, static_cast<unsigned long long>(__double_as_longlong(m)));
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
                   const uint8_t *E, double eps, int *launches_io) {
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
        build_zt_kernel<<<tgrid, dim3(TT, 8), 0, s>>>(E, n, N, static_cast<float>(eps), Z32);
        MCK(cudaGetLastError());
        launches += 2;
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
    std::vector<Launch> lu, fwd, bwd;
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
    // The N-RHS solves run in groups of kSolveGroup panels: inside a group each panel is
    // solved with its diagonal inverse and updates the group's later (forward) or earlier
    // (backward) panels; one update with K = the group's width then carries the whole group to
    // the columns beyond it, so the trailing part of Z is read and written once per group.
    for (int g0 = 0; g0 < nb && ok; g0 += kSolveGroup) {
        const int g1 = std::min(nb, g0 + kSolveGroup), gs = g0 * BL, ge = g1 * BL;
        for (int k = g0; k < g1 && ok; ++k) {
            const int kb = k * BL;
            ok = add(fwd, EPI_STORE_F32, N, BL, BL, at(opZ, 0, kb), at(opL, kb, 0), Z32, np, 0, kb, false,
                     &flops_solve);
            if (ok && kb + BL < ge)
                ok = add(fwd, EPI_SUB_F32, N, ge - kb - BL, BL, at(opZ, 0, kb), at(opA, kb + BL, kb), Z32, np, 0,
                         kb + BL, false, &flops_solve);
        }
        if (ok && ge < N)
            ok = add(fwd, EPI_SUB_F32, N, N - ge, ge - gs, at(opZ, 0, gs), at(opA, ge, gs), Z32, np, 0, ge, false,
                     &flops_solve);
    }
    for (int g1 = nb; g1 > 0 && ok; g1 -= kSolveGroup) {
        const int g0 = std::max(0, g1 - kSolveGroup), gs = g0 * BL, ge = g1 * BL;
        for (int k = g1 - 1; k >= g0 && ok; --k) {
            const int kb = k * BL;
            ok = add(bwd, EPI_STORE_F32, N, BL, BL, at(opZ, 0, kb), at(opU, kb, 0), Z32, np, 0, kb, false,
                     &flops_solve);
            if (ok && kb > gs)
                ok = add(bwd, EPI_SUB_F32, N, kb - gs, BL, at(opZ, 0, kb), at(opA, gs, kb), Z32, np, 0, gs, false,
                         &flops_solve);
        }
        if (ok && gs > 0)
            ok = add(bwd, EPI_SUB_F32, N, gs, ge - gs, at(opZ, 0, gs), at(opA, 0, gs), Z32, np, 0, 0, false,
                     &flops_solve);
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
    for (int k = 0; k < nb; ++k) {
        const int64_t kb = static_cast<int64_t>(k) * BL;
        diag_lu_inv_kernel<<<1, kDiagThreads, 0, s>>>(A32 + kb * np + kb, np, Linv + kb * BL, Uinv + kb * BL,
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
    MCK(cudaEventRecord(ev[5], s));
    auto solve = [&]() -> cudaError_t {
        cudaError_t e;
        for (const Launch &L : fwd)
            if ((e = run(L)) != cudaSuccess) return e;
        for (const Launch &L : bwd)
            if ((e = run(L)) != cudaSuccess) return e;
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
    const size_t res_smem = sizeof(double) * static_cast<size_t>(np);
    MCK(cudaFuncSetAttribute(residual_t_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(res_smem)));
    unsigned long long *rmax_d = ws.scal + 20;
    double rmax = 0.0, best = 0.0;
    int it = 0, stall = 0;
    // The FP64 residual has a rounding floor of about (row length) * u * max|X|; refinement
    // stops at tol, or when it no longer halves the residual once that is below 1e-8 * eps.
    const double floor_ok = 1e-8 * eps;
    for (;;) {
        MCK(cudaMemsetAsync(rmax_d, 0, sizeof(unsigned long long), s));
        residual_t_kernel<<<static_cast<unsigned>(np), 256, res_smem, s>>>(csr_ptr, csr_col, n, N, eps, Z64, Z32,
                                                                           rmax_d);
        MCK(cudaGetLastError());
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
        st->gemm_launches = static_cast<int>(lu.size() + (fwd.size() + bwd.size()) * (1 + it));
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
