// dl_mixed.cu -- R~ = (I - eps E)^-1 eps E (Proposition 1) on the TF32 tensor cores, with FP64
// iterative refinement (DL_PATH_MIXED).
//
//   1. A = I - eps E in FP32 (padded with the identity).
//   2. Block LU of A without pivoting, blocks of b = 128 (A is strictly diagonally dominant by
//      rows, proof of Proposition 1, so every Schur complement is too and block elimination is
//      stable):  A = L U with L unit block lower (L_ik = A_ik S_kk^-1) and U block upper
//      (U_kj = A_kj after the eliminations before k, diagonal blocks S_kk).  Per block k:
//        diag:  S_kk^-1 by Gauss-Jordan on the CUDA cores (FP32, one CTA);
//        L21 = A21 S_kk^-1 (in place), T = A12^T;
//        look-ahead: the next block column and block row, A -= L21 U12 there;
//        bulk:  the rest of the trailing matrix, A22 -= L21 U12.
//      The look-ahead and the chain that needs it (the next diagonal block, its L21 and T) run
//      on a stream of the greatest priority, the bulk update on a stream of the least priority
//      and on all SMs but kReserve, so the chain of 128 x 128 steps proceeds while the bulk
//      update of the previous block streams through HBM.
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

namespace dl {

namespace {

constexpr int BL = 128;        // LU block size = GEMM tile
constexpr int TT = 32;         // transpose tile
constexpr int kSolveGroup = 8;  // blocks per group of the solves (1024 columns)
constexpr int kReserve = 16;   // SMs the bulk LU update leaves to the critical chain
constexpr size_t kResidualSmem = 227 * 1024;  // dynamic shared memory of one residual block

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

// S^-1 of the BL x BL block at A (row stride lda) by in-place Gauss-Jordan elimination without
// pivoting, FP32, one CTA of 256 threads.  Thread t holds an 8 x 8 tile of the block in
// registers: rows r0 .. r0 + 7 (r0 = 16 warp + 8 (lane / 16)), columns c0 .. c0 + 7
// (c0 = 8 (lane mod 16)).  Step k (p = 1 / S_kk, r = row k, c = column k before the step):
//     S_ij -= c_i r_j p (i, j != k),   S_kj = r_j p,   S_ik = -c_i p,   S_kk = p.
// The owners of row k and of column k publish them through shared memory (two buffers, so one
// barrier per step suffices: a buffer is rewritten two steps later, after every thread has
// passed the barrier between).  A is strictly diagonally dominant by rows and so is every
// Schur complement, hence every pivot is positive; a pivot that is not sets ST_BAD_INPUT.
// Writes S^-1 and S^-T (BL x BL, row-major).
constexpr int kDiagThreads = 256;

__global__ void __launch_bounds__(kDiagThreads) diag_inv_kernel(const float *__restrict__ A, int64_t lda,
                                                                float *__restrict__ Sinv, float *__restrict__ SinvT,
                                                                int *status) {
    static_assert(BL == 128 && kDiagThreads == 256, "8 x 8 tiles of a 128 x 128 block");
    __shared__ __align__(16) float rowbuf[2][BL];
    __shared__ __align__(16) float colbuf[2][BL];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r0 = 16 * warp + 8 * (lane >> 4);
    const int c0 = 8 * (lane & 15);
    float a[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float4 x = *reinterpret_cast<const float4 *>(A + (r0 + i) * lda + c0);
        const float4 y = *reinterpret_cast<const float4 *>(A + (r0 + i) * lda + c0 + 4);
        a[i][0] = x.x, a[i][1] = x.y, a[i][2] = x.z, a[i][3] = x.w;
        a[i][4] = y.x, a[i][5] = y.y, a[i][6] = y.z, a[i][7] = y.w;
    }
    bool bad = false;
#pragma unroll 1
    for (int kb = 0; kb < BL; kb += 8) {
        const bool row_owner = r0 == kb;  // rows kb .. kb + 7 are this thread's
        const bool col_owner = c0 == kb;  // columns kb .. kb + 7 are this thread's
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            const int k = kb + kk, buf = k & 1;
            if (row_owner) {
                *reinterpret_cast<float4 *>(&rowbuf[buf][c0]) = make_float4(a[kk][0], a[kk][1], a[kk][2], a[kk][3]);
                *reinterpret_cast<float4 *>(&rowbuf[buf][c0 + 4]) = make_float4(a[kk][4], a[kk][5], a[kk][6], a[kk][7]);
            }
            if (col_owner) {
                *reinterpret_cast<float4 *>(&colbuf[buf][r0]) = make_float4(a[0][kk], a[1][kk], a[2][kk], a[3][kk]);
                *reinterpret_cast<float4 *>(&colbuf[buf][r0 + 4]) = make_float4(a[4][kk], a[5][kk], a[6][kk], a[7][kk]);
            }
            __syncthreads();
            const float piv = rowbuf[buf][k];
            const float p = 1.0f / piv;
            bad |= !(piv > 0.0f) || !isfinite(p);
            float c[8], rp[8];
            {
                const float4 c_lo = *reinterpret_cast<const float4 *>(&colbuf[buf][r0]);
                const float4 c_hi = *reinterpret_cast<const float4 *>(&colbuf[buf][r0 + 4]);
                const float4 r_lo = *reinterpret_cast<const float4 *>(&rowbuf[buf][c0]);
                const float4 r_hi = *reinterpret_cast<const float4 *>(&rowbuf[buf][c0 + 4]);
                c[0] = c_lo.x, c[1] = c_lo.y, c[2] = c_lo.z, c[3] = c_lo.w;
                c[4] = c_hi.x, c[5] = c_hi.y, c[6] = c_hi.z, c[7] = c_hi.w;
                rp[0] = r_lo.x * p, rp[1] = r_lo.y * p, rp[2] = r_lo.z * p, rp[3] = r_lo.w * p;
                rp[4] = r_hi.x * p, rp[5] = r_hi.y * p, rp[6] = r_hi.z * p, rp[7] = r_hi.w * p;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float upd = fmaf(-c[i], rp[j], a[i][j]);
                    if (i == kk && j == kk) {
                        a[i][j] = row_owner && col_owner ? p : row_owner ? rp[j] : col_owner ? -c[i] * p : upd;
                    } else if (i == kk) {
                        a[i][j] = row_owner ? rp[j] : upd;
                    } else if (j == kk) {
                        a[i][j] = col_owner ? -c[i] * p : upd;
                    } else {
                        a[i][j] = upd;
                    }
                }
            }
        }
    }
    if (bad) atomicOr(status, ST_BAD_INPUT);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        *reinterpret_cast<float4 *>(Sinv + (r0 + i) * BL + c0) = make_float4(a[i][0], a[i][1], a[i][2], a[i][3]);
        *reinterpret_cast<float4 *>(Sinv + (r0 + i) * BL + c0 + 4) = make_float4(a[i][4], a[i][5], a[i][6], a[i][7]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        *reinterpret_cast<float4 *>(SinvT + (c0 + j) * BL + r0) = make_float4(a[0][j], a[1][j], a[2][j], a[3][j]);
        *reinterpret_cast<float4 *>(SinvT + (c0 + j) * BL + r0 + 4) = make_float4(a[4][j], a[5][j], a[6][j], a[7][j]);
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

// Z = I (np x np, zeroed before).
__global__ void identity_kernel(float *Z, int np) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < np) Z[static_cast<int64_t>(r) * np + r] = 1.0f;
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
    MCK(cudaStreamCreateWithPriority(&ws.mx_stream[0], cudaStreamNonBlocking, greatest));
    MCK(cudaStreamCreateWithPriority(&ws.mx_stream[1], cudaStreamNonBlocking, least));
    for (auto &e : ws.mx_ev) MCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return DL_OK;
}

}  // namespace

dl_status tc_mixed(dl_ctx *ctx, Workspace &ws, cudaStream_t s, const SolveArgs &a, dl_stats *st,
                   const uint8_t *E, double eps, unsigned long long dmax, int *launches_io) {
    const int32_t n = a.n;
    const int64_t np = round_up(std::max<int64_t>(n, 1), 256);
    const int nb = static_cast<int>(np / BL);
    const int N = static_cast<int>(np);
    int launches = 0;
    dl_status rc = mixed_streams(ws);
    if (rc) return rc;
    cudaStream_t P = ws.mx_stream[0], U = ws.mx_stream[1];
    auto *A32 = static_cast<float *>(ws.get("mx_A", np * np * 4));
    auto *W32 = static_cast<float *>(ws.get("mx_W", np * np * 4));   // Z = A^-T, then R
    auto *Wt = static_cast<float *>(ws.get("mx_Wt", np * np * 4));   // W = A^-1
    auto *D32 = static_cast<float *>(ws.get("mx_D", np * np * 4));
    auto *Z64 = static_cast<double *>(ws.get("mx_Z64", np * np * 8));
    auto *X64 = static_cast<double *>(ws.get("mx_X64", np * np * 8));
    auto *T2 = static_cast<float *>(ws.get("mx_T", 2 * np * BL * 4));  // two transposed row panels
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
    MCK(cudaEventRecord(ev[4], s));
    {
        dim3 grid(static_cast<unsigned>(std::min<int64_t>((np + 255) / 256, 64)), static_cast<unsigned>(np));
        build_a_kernel<<<grid, 256, 0, s>>>(E, n, N, static_cast<float>(eps), A32);
        MCK(cudaGetLastError());
        ++launches;
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

    // ---- GEMM table ---------------------------------------------------------------------
    Table tb;
    std::vector<Launch> l21, ahead, bulk, ginv, wfwd, wbwd, refine;
    double flops_lu = 0, flops_w = 0, flops_ref = 0;
    const Operand opA{A32, np, np, np, 0, 0};
    const Operand opS{Sinv, np, BL, BL, 0, 0}, opST{SinvT, np, BL, BL, 0, 0};
    bool ok = true;
    std::vector<int> has_bulk(nb, -1), has_ahead(nb, -1), has_l21(nb, -1);
    for (int k = 0; k < nb && ok; ++k) {
        const int kb = k * BL, rem = N - kb - BL;
        if (rem <= 0) break;
        const Operand opT{T2 + static_cast<int64_t>(k & 1) * np * BL, np, BL, BL, 0, 0};  // T = A12^T
        // L21 = A21 S^-1 (in place: each output tile reads only its own rows of A21)
        has_l21[k] = static_cast<int>(l21.size());
        ok = tb.add(l21, EPI_STORE_F32, BL, rem, BL, BL, at(opA, kb + BL, kb), at(opST, kb, 0), A32, np, kb + BL, kb,
                    false, &flops_lu);
        // look-ahead: block column k+1 (all rows below) and block row k+1 (columns beyond it)
        has_ahead[k] = static_cast<int>(ahead.size());
        ok = ok && tb.add(ahead, EPI_SUB_F32, BL, rem, BL, BL, at(opA, kb + BL, kb), opT, A32, np, kb + BL, kb + BL,
                          false, &flops_lu);
        if (ok && rem > BL) {
            ok = tb.add(ahead, EPI_SUB_F32, BL, BL, rem - BL, BL, at(opA, kb + BL, kb), at(opT, BL, 0), A32, np,
                        kb + BL, kb + 2 * BL, true, &flops_lu);
            has_bulk[k] = static_cast<int>(bulk.size());
            ok = ok && tb.add(bulk, EPI_SUB_F32, 256, rem - BL, rem - BL, BL, at(opA, kb + 2 * BL, kb),
                              at(opT, BL, 0), A32, np, kb + 2 * BL, kb + 2 * BL, false, &flops_lu);
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
    for (int kl = 0; kl < kSolveGroup && ok; ++kl) {
        bool first = true;  // step kl needs step kl - 1: a launch of its own
        for (int g = 0; g < ng && ok; ++g) {
            const int g0 = g * kSolveGroup, g1 = std::min(nb, g0 + kSolveGroup), gs = g0 * BL, ge = g1 * BL,
                      w = ge - gs, kb = gs + kl * BL;
            if (g0 + kl < g1 && kb + BL < ge) {
                ok = tb.add(ginv, EPI_SUB_F32, BL, w, ge - kb - BL, BL, at(opYL, gs, kl * BL), at(opA, kb + BL, kb), YL,
                            GW, gs, (kl + 1) * BL, !first, &flops_lu);
                first = false;
            }
        }
    }
    for (int kl = kSolveGroup - 1; kl >= 0 && ok; --kl) {
        bool first = true;
        for (int g = 0; g < ng && ok; ++g) {  // Y_k = Y_k S_kk^-T (in place: N = BL)
            const int g0 = g * kSolveGroup, g1 = std::min(nb, g0 + kSolveGroup), gs = g0 * BL, w = (g1 - g0) * BL;
            if (g0 + kl < g1) {
                ok = tb.add(ginv, EPI_STORE_F32, BL, w, BL, BL, at(opYU, gs, kl * BL), at(opS, gs + kl * BL, 0), YU,
                            GW, gs, kl * BL, !first, &flops_lu);
                first = false;
            }
        }
        first = true;
        for (int g = 0; g < ng && ok; ++g) {  // Y_{<k} -= Y_k U_{<k,k}^T
            const int g0 = g * kSolveGroup, g1 = std::min(nb, g0 + kSolveGroup), gs = g0 * BL, w = (g1 - g0) * BL,
                      kb = gs + kl * BL;
            if (g0 + kl < g1 && kb > gs) {
                ok = tb.add(ginv, EPI_SUB_F32, BL, w, kb - gs, BL, at(opYU, gs, kl * BL), at(opA, gs, kb), YU, GW, gs, 0,
                            !first, &flops_lu);
                first = false;
            }
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
    auto run = [&](const Launch &L, int max_grid, cudaStream_t on) -> cudaError_t {
        ++launches;
        return gemm_launch(KIND_TF32, true, L.bn, L.epi, dprob + L.first, L.count, L.tiles,
                           std::min(L.tiles, max_grid), ws.status, ctx->budget_ns, on);
    };
    const int sms = ctx->sms;

    // ---- LU with look-ahead --------------------------------------------------------------
    MCK(cudaEventRecord(ws.mx_ev[0], s));  // the table and A are ready on s
    MCK(cudaStreamWaitEvent(P, ws.mx_ev[0], 0));
    MCK(cudaStreamWaitEvent(U, ws.mx_ev[0], 0));
    cudaEvent_t evT[2] = {ws.mx_ev[0], ws.mx_ev[1]}, evB[2] = {ws.mx_ev[2], ws.mx_ev[3]};
    bool bulk_pending = false;  // the bulk update of the previous block is queued on U
    for (int k = 0; k < nb; ++k) {
        const int64_t kb = static_cast<int64_t>(k) * BL;
        const int rem = N - static_cast<int>(kb) - BL;
        diag_inv_kernel<<<1, kDiagThreads, 0, P>>>(A32 + kb * np + kb, np, Sinv + kb * BL, SinvT + kb * BL, ws.status);
        MCK(cudaGetLastError());
        ++launches;
        if (rem <= 0) break;
        // L21 runs beside the bulk update of block k - 1, which leaves it kReserve SMs
        const bool beside_bulk = k > 0 && has_bulk[k - 1] >= 0;
        MCK(run(l21[has_l21[k]], beside_bulk ? kReserve : sms, P));
        float *Tk = T2 + static_cast<int64_t>(k & 1) * np * BL;
        MCK(transpose(A32 + kb * np + kb + BL, np, BL, rem, Tk, BL, P));  // T = A12^T
        ++launches;
        MCK(cudaEventRecord(evT[k & 1], P));
        if (bulk_pending) MCK(cudaStreamWaitEvent(P, evB[(k - 1) & 1], 0));
        // the look-ahead launch (one or two problems)
        {
            Launch L = ahead[has_ahead[k]];
            MCK(run(L, sms, P));
        }
        bulk_pending = false;
        if (has_bulk[k] >= 0) {
            MCK(cudaStreamWaitEvent(U, evT[k & 1], 0));
            MCK(run(bulk[has_bulk[k]], std::max(1, sms - kReserve), U));
            MCK(cudaEventRecord(evB[k & 1], U));
            bulk_pending = true;
        }
    }
    MCK(cudaEventRecord(ws.mx_ev[0], U));  // (evT[0] is no longer needed)
    MCK(cudaStreamWaitEvent(P, ws.mx_ev[0], 0));
    MCK(cudaEventRecord(ws.mx_ev[1], P));
    MCK(cudaStreamWaitEvent(s, ws.mx_ev[1], 0));

    // group inverses: Y = I on each group's rows, the grouped steps, then G = Y^T per group
    MCK(cudaMemsetAsync(YL, 0, np * GW * 4, s));
    MCK(cudaMemsetAsync(YU, 0, np * GW * 4, s));
    group_identity_kernel<<<static_cast<unsigned>((np + 255) / 256), 256, 0, s>>>(YL, YU, N, static_cast<int>(GW));
    MCK(cudaGetLastError());
    ++launches;
    for (const Launch &L : ginv) MCK(run(L, sms, s));
    for (int64_t gs = 0; gs < np; gs += GW) {
        const int w = static_cast<int>(std::min<int64_t>(GW, np - gs));
        MCK(transpose(YL + gs * GW, GW, w, w, GL + gs * GW, GW, s));
        MCK(transpose(YU + gs * GW, GW, w, w, GU + gs * GW, GW, s));
        launches += 2;
    }
    MCK(cudaEventRecord(ev[5], s));

    // ---- W = A^-1 ------------------------------------------------------------------------
    MCK(cudaMemsetAsync(W32, 0, np * np * 4, s));
    identity_kernel<<<static_cast<unsigned>((np + 255) / 256), 256, 0, s>>>(W32, N);
    MCK(cudaGetLastError());
    ++launches;
    for (int pass = 0; pass < 2; ++pass) {
        const std::vector<Step> &steps = pass == 0 ? fwd_steps : bwd_steps;
        const std::vector<Launch> &list = pass == 0 ? wfwd : wbwd;
        for (const Step &sp : steps) {
            if (sp.launch >= 0) {
                MCK(run(list[sp.launch], sms, s));
            } else {
                MCK(cudaMemcpy2DAsync(W32 + sp.gs, np * 4, Tg, GW * 4, static_cast<size_t>(sp.w) * 4, sp.rows,
                                      cudaMemcpyDeviceToDevice, s));
            }
        }
    }
    MCK(transpose(W32, np, N, N, Wt, np, s));  // W = (A^-T)^T
    ++launches;
    MCK(cudaEventRecord(ev[6], s));

    // ---- refinement from Z = 0 -------------------------------------------------------------
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
                residual_fixed_kernel<3><<<grid, 1024, res_smem, s>>>(csr_ptr, csr_col, n, N, deg_bits, eps, Z64, R32,
                                                                     rmax_p, At);
                break;
            case 2:
                if ((e = cudaFuncSetAttribute(residual_fixed_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              static_cast<int>(res_smem))) != cudaSuccess)
                    return e;
                residual_fixed_kernel<2><<<grid, 1024, res_smem, s>>>(csr_ptr, csr_col, n, N, deg_bits, eps, Z64, R32,
                                                                     rmax_p, At);
                break;
            default:
                if ((e = cudaFuncSetAttribute(residual_fixed_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              static_cast<int>(res_smem))) != cudaSuccess)
                    return e;
                residual_fixed_kernel<1><<<grid, 1024, res_smem, s>>>(csr_ptr, csr_col, n, N, deg_bits, eps, Z64, R32,
                                                                     rmax_p, At);
        }
        return cudaGetLastError();
    };
    const int64_t cnt = np * np;
    const unsigned eblocks = static_cast<unsigned>(std::min<int64_t>((cnt + 255) / 256, 8 * 1024));
    unsigned long long *rmax_d = ws.scal + 20;
    double rmax = 0.0, best = 0.0;
    int products = 0, stall = 0;
    // The FP64 residual has a rounding floor of about (row length) * u * max|X|; refinement
    // stops at tol, or when it no longer halves the residual once that is below 1e-8 * eps.
    const double floor_ok = 1e-8 * eps;
    MCK(cudaMemsetAsync(Z64, 0, np * np * 8, s));
    for (;;) {
        MCK(cudaMemsetAsync(rmax_d, 0, sizeof(unsigned long long), s));
        MCK(residual(rmax_d));
        ++launches;
        unsigned long long h = 0;
        MCK(cudaMemcpyAsync(&h, rmax_d, sizeof(h), cudaMemcpyDeviceToHost, s));
        MCK(cudaStreamSynchronize(s));
        std::memcpy(&rmax, &h, sizeof(rmax));
        if (rmax <= tol * eps) break;
        if (products >= 1) {  // after the solve: refinement steps must keep halving the residual
            if (products == 1 || rmax < 0.5 * best) {
                best = rmax;
                stall = 0;
            } else if (++stall >= 2 && best <= floor_ok) {
                break;
            }
        }
        if (products > max_iters) {
            set_error("mixed path: refinement stopped at max|R|/eps = %.3g after %d steps", rmax / eps, products - 1);
            return DL_ENOTCONV;
        }
        MCK(run(refine[0], sms, s));  // D^T = R^T W^T
        add_f32_kernel<<<eblocks, 256, 0, s>>>(Z64, D32, cnt);
        MCK(cudaGetLastError());
        ++launches;
        ++products;
    }
    MCK(transpose(Z64, np, N, N, X64, np, s));  // X = Z^T
    ++launches;
    MCK(cudaEventRecord(ev[7], s));
    MCK(cudaEventSynchronize(ev[7]));
    if (st) {
        st->iters = std::max(products - 1, 0);  // refinement steps after the first product (the solve)
        st->final_resid = rmax / eps;
        st->gemm_flops = flops_lu + flops_w + flops_ref * products;
        st->gemm_launches = static_cast<int>(l21.size() + ahead.size() + bulk.size() + ginv.size() + wfwd.size() +
                                             wbwd.size()) + products;
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
