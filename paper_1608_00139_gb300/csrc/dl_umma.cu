// dl_umma.cu -- persistent tcgen05 GEMM for sm_103a with fused epilogues.
//
// The dense contractions of the method run here:
//   * boolean products on 0/1 matrices stored as FP8 e4m3 (1.0 = 0x38): the join
//     [[exists y r1(x,y) and r2(y,z)]] = min1(R1 R2) (Sec. 2, eq. denote:quant), the
//     squaring steps of the transitive closure and the same-generation doubling steps.
//     0/1 operands are exact in e4m3, products are 0/1 and FP32 sums of at most 2^24 ones are
//     exact, so the epilogue's test acc > 0 is the exact boolean OR of ANDs;
//   * TF32 products of the blocked LU of I - eps E and its triangular solves (Proposition 1),
//     C = A B^T or C -= A B^T with both operands K-major.
//
// Structure (one CTA per SM, persistent over output tiles of 128 x BN):
//   warp 0      TMA producer: A tile (128 rows x 128 bytes of K, 128-byte swizzle) and the
//               B tile (MN-major: BN/(128 B) boxes of BK k-rows; K-major: one box of BN rows)
//               into an S-stage shared-memory ring; mbarrier complete_tx.
//   warp 1      allocates 2*BN TMEM columns (two FP32 accumulators of 128 lanes x BN) and one
//               elected thread issues tcgen05.mma; tcgen05.commit releases smem stages and
//               signals a finished accumulator.
//   warps 2..9  epilogue: tcgen05.ld 32 lanes x 32 columns, fused min1/OR/bit-pack/popcount
//               (boolean) or read-modify-write of C (TF32 update), then release the
//               accumulator so the next tile's MMAs overlap this epilogue.  A warp may only
//               read the TMEM lane quarter (warp % 4), so two warps share each quarter and take
//               alternate 32-column chunks; the subtracting epilogue loads all of its chunks of
//               C before the accumulator is ready (a K = 128 update moves 8 bytes of C per 256
//               flops: it needs that many bytes in flight to run at HBM rate).
// Problems come from a device-memory table so that one launch can cover many independent
// problems (a grouped GEMM for the uneven batch).
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "dl_internal.h"
#include "dl_ptx.cuh"

namespace dl {

namespace {

constexpr int BM = 128;
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;

template <int KIND, int BN, int EPI>
struct Cfg {
    static constexpr int ELEM = KIND == KIND_F8 ? 1 : 4;      // bytes per element
    static constexpr int BK = 128 / ELEM;                      // elements per k-block
    static constexpr int KI = 32 / ELEM;                       // K of one MMA instruction
    static constexpr int A_BYTES = BM * 128;
    static constexpr int B_BYTES = BN * 128;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    // FP32 output: 32 x 32 float tiles per epilogue warp, taken from the pipeline's stages: two
    // for the subtracting epilogue (C of the next chunk in flight), one for the storing one
    static constexpr int EPI_TILES = KIND != KIND_TF32 ? 0 : EPI == EPI_SUB_F32 ? 2 : 1;
    static constexpr int EPI_STAGE = kEpiWarps * EPI_TILES * 32 * 32 * 4;
    static constexpr int S_FIT = (232448 - 1024 - 256 - EPI_STAGE) / STAGE;
    static constexpr int S = KIND == KIND_TF32 ? (S_FIT > 8 ? 8 : S_FIT) : ((196608 / STAGE) > 8 ? 8 : (196608 / STAGE));
    static constexpr int TMEM_COLS = 2 * BN;
    static constexpr int SMEM = 1024 + S * STAGE + 256 + EPI_STAGE;
};

template <int KIND, int BN, bool B_KMAJOR>
__host__ __device__ constexpr uint32_t make_idesc() {
    // D = F32 (bits 4-5 = 1); A/B format (bits 7-9, 10-12): E4M3 = 0, TF32 = 2;
    // A K-major (bit 15 = 0); B major (bit 16); N >> 3 (bits 17-22); M >> 4 (bits 24-28).
    return (1u << 4) | ((KIND == KIND_TF32 ? 2u : 0u) << 7) |
           ((KIND == KIND_TF32 ? 2u : 0u) << 10) | ((B_KMAJOR ? 0u : 1u) << 16) |
           (static_cast<uint32_t>(BN >> 3) << 17) | (static_cast<uint32_t>(BM >> 4) << 24);
}

__device__ __forceinline__ const GemmProblem *find_problem(const GemmProblem *probs, int nprob,
                                                           int tile) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (probs[mid].tile_start <= tile) lo = mid;
        else hi = mid - 1;
    }
    return probs + lo;
}

// A gated problem's tiles are skipped while its gate word is non-zero (finished batch
// instances).  Gates only change between launches, so all roles agree.
__device__ __forceinline__ bool gated_off(const GemmProblem *P) {
    return P->gate != nullptr && *reinterpret_cast<const volatile int *>(P->gate) != 0;
}

// Tile `tile` of the launch: its problem (null if gated off) and its index inside that
// problem.  With a device schedule the tile space is that of the listed problems only:
// sched[0] = count A, sched[1] = tiles, sched[2 + j] = problem of entry j (j < A), and
// sched[2 + nprob + j] = first tile of entry j.
__device__ __forceinline__ const GemmProblem *resolve_tile(const GemmProblem *probs, int nprob,
                                                           const int *sched, int tile, int *local) {
    if (sched == nullptr) {
        const GemmProblem *P = find_problem(probs, nprob, tile);
        *local = tile - P->tile_start;
        return gated_off(P) ? nullptr : P;
    }
    const int *start = sched + 2 + nprob;
    int lo = 0, hi = sched[0] - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= tile) lo = mid;
        else hi = mid - 1;
    }
    *local = tile - start[lo];
    return probs + sched[2 + lo];
}

// Output tile (mb, nb) of a problem's local tile index: groups of kGroupM row blocks, each
// swept column by column, so that the tiles a wave of CTAs works on (consecutive indices) share
// a few row blocks of A and a few column blocks of B that stay in L2 (walking all row blocks of a
// column first re-reads all of A from DRAM for every wave once A outgrows L2).
constexpr int kGroupM = 16;
__device__ __forceinline__ void tile_coords(const GemmProblem *P, int local, int &mb, int &nb) {
    const int per_group = kGroupM * P->tiles_n;
    const int g = local / per_group;
    const int first = g * kGroupM;
    const int rows = min(kGroupM, P->tiles_m - first);
    const int r = local - g * per_group;
    mb = first + r % rows;
    nb = r / rows;
}

// Does k-block kb of output tile (mb, nb) contribute?  (always, without occupancy maps)
template <int BN>
__device__ __forceinline__ bool kblock_live(const GemmProblem *P, int mb, int nb, int kb) {
    if (P->occ_a == nullptr) return true;
    if (!P->occ_a[mb * P->occ_ld + kb]) return false;
#pragma unroll
    for (int j = 0; j < BN / 128; ++j)
        if (P->occ_b[kb * P->occ_ld + nb * (BN / 128) + j]) return true;
    return false;
}

template <int BN>
__device__ __forceinline__ bool tile_live(const GemmProblem *P, int mb, int nb, int nkb) {
    if (P->occ_a == nullptr) return true;
    for (int kb = 0; kb < nkb; ++kb)
        if (kblock_live<BN>(P, mb, nb, kb)) return true;
    return false;
}

__device__ __forceinline__ uint32_t epi_bool_chunk(const GemmEpilogue &e, int row, int col,
                                                   const uint32_t (&v)[32], uint32_t &cnt) {
    uint32_t word = 0;
#pragma unroll
    for (int j = 0; j < 32; ++j) word |= (__uint_as_float(v[j]) > 0.0f ? 1u : 0u) << j;
    const int64_t r = static_cast<int64_t>(e.out_row0) + row;
    const int64_t c = static_cast<int64_t>(e.out_col0) + col;
    if (e.add8) {
        const uint4 *src = reinterpret_cast<const uint4 *>(e.add8 + r * e.ld_add8 + c);
        const uint4 a0 = src[0], a1 = src[1];
        const uint32_t w[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int b = 0; b < 4; ++b) word |= (((w[q] >> (8 * b)) & 0xFFu) != 0u ? 1u : 0u) << (4 * q + b);
    }
    if (e.out8) {
        uint32_t w[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            uint32_t x = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) x |= ((word >> (4 * q + b)) & 1u) * (0x38u << (8 * b));
            w[q] = x;
        }
        uint4 *dst = reinterpret_cast<uint4 *>(e.out8 + r * e.ld_out8 + c);
        dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
        dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
    }
    if (e.bits) e.bits[r * e.ld_bits32 + (c >> 5)] = word;
    cnt += __popc(word);
    return word;
}

template <int KIND, int BN, bool B_KMAJOR, int EPI>
__global__ void __launch_bounds__(kThreads, 1)
    umma_gemm_kernel(const GemmProblem *__restrict__ probs, int nprob, int total_tiles,
                     const int *__restrict__ sched, int *status, uint64_t budget_ns) {
    using C = Cfg<KIND, BN, EPI>;
    // A device schedule fixes the tile count; CTAs without a tile leave before any setup
    // (the value is the same for every thread of the CTA).
    if (sched != nullptr) {
        grid_dep_wait();  // the schedule is written by an earlier kernel
        total_tiles = sched[1];
        if (static_cast<int>(blockIdx.x) >= total_tiles) return;
    }
    constexpr uint32_t IDESC = make_idesc<KIND, BN, B_KMAJOR>();
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~static_cast<uintptr_t>(1023));
    uint8_t *sA = smem;
    uint8_t *sB = smem + C::S * C::A_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + C::S * C::STAGE);
    uint64_t *empty = full + C::S;
    uint64_t *accf = empty + C::S;
    uint64_t *acce = accf + 2;
    uint64_t *drain = acce + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    // FP32 epilogues: two 32 x 32 float tiles per epilogue warp
    float4 *epi_stage = reinterpret_cast<float4 *>(smem + C::S * C::STAGE + 256);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&accf[a], 1);
            mbar_init(&acce[a], 32 * kEpiWarps);
        }
        mbar_init(drain, 1);
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, C::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    // Under a programmatic launch the set-up above overlaps the predecessor's end; its outputs
    // (this launch's operands and C) are read only from here on.
    grid_dep_wait();

    if (warp == 0) {
        // ------------------------------ TMA producer ------------------------------------
        if (elect_one_sync()) {
            int stage = 0;
            uint32_t ph = 0;
            uint64_t issued = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < total_tiles && ok; tile += gridDim.x) {
                int local = 0;
                const GemmProblem *P = resolve_tile(probs, nprob, sched, tile, &local);
                if (P == nullptr) continue;
                int mb, nb;
                tile_coords(P, local, mb, nb);
                const int nkb = P->K / C::BK;
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!kblock_live<BN>(P, mb, nb, kb)) continue;
                    if (!mbar_wait_bounded(&empty[stage], ph ^ 1u, budget_ns, status,
                                           ST_TIMEOUT_EMPTY)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[stage], C::STAGE);
                    tma_load_2d(&P->tmA, sA + stage * C::A_BYTES, &full[stage],
                                P->a_col0 + kb * C::BK, P->a_row0 + mb * BM);
                    if (B_KMAJOR) {
                        tma_load_2d(&P->tmB, sB + stage * C::B_BYTES, &full[stage],
                                    P->b_col0 + kb * C::BK, P->b_row0 + nb * BN);
                    } else {
#pragma unroll
                        for (int j = 0; j < BN / C::BK; ++j)
                            tma_load_2d(&P->tmB, sB + stage * C::B_BYTES + j * (C::BK * 128),
                                        &full[stage], P->b_col0 + nb * BN + j * C::BK,
                                        P->b_row0 + kb * C::BK);
                    }
                    ++issued;
                    if (++stage == C::S) {
                        stage = 0;
                        ph ^= 1u;
                    }
                }
            }
            // Drain: every load issued must have landed before the CTA may exit.
            const uint64_t first = issued > static_cast<uint64_t>(C::S) ? issued - C::S : 0;
            for (uint64_t i = first; i < issued; ++i)
                mbar_wait_bounded(&full[i % C::S], static_cast<uint32_t>((i / C::S) & 1u),
                                  budget_ns, status, ST_TIMEOUT_DRAIN);
        }
        grid_dep_launch();  // (all lanes) no load left to issue: the successor may start launching
    } else if (warp == 1) {
        // ------------------------------ MMA issuer --------------------------------------
        if (elect_one_sync()) {
            int stage = 0;
            uint32_t ph = 0;
            int acc = 0;
            uint32_t acc_ph = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < total_tiles && ok; tile += gridDim.x) {
                int local = 0;
                const GemmProblem *P = resolve_tile(probs, nprob, sched, tile, &local);
                if (P == nullptr) continue;
                int mb, nb;
                tile_coords(P, local, mb, nb);
                const int nkb = P->K / C::BK;
                if (!mbar_wait_bounded(&acce[acc], acc_ph ^ 1u, budget_ns, status,
                                       ST_TIMEOUT_ACC_EMPTY)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(acc * BN);
                bool issued = false;
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!kblock_live<BN>(P, mb, nb, kb)) continue;
                    if (!mbar_wait_bounded(&full[stage], ph, budget_ns, status,
                                           ST_TIMEOUT_FULL)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA + stage * C::A_BYTES);
                    const uint32_t b0 = smem_u32(sB + stage * C::B_BYTES);
#pragma unroll
                    for (int kk = 0; kk < 128 / 32; ++kk) {
                        const uint64_t adesc = smem_desc_sw128(a0 + kk * 32, 16, 1024);
                        const uint64_t bdesc =
                            B_KMAJOR ? smem_desc_sw128(b0 + kk * 32, 16, 1024)
                                     : smem_desc_sw128(b0 + kk * C::KI * 128, C::BK * 128, 1024);
                        umma_issue<KIND>(d_tmem, adesc, bdesc, IDESC, (issued || kk != 0) ? 1u : 0u);
                    }
                    issued = true;
                    umma_commit(&empty[stage]);
                    if (++stage == C::S) {
                        stage = 0;
                        ph ^= 1u;
                    }
                }
                if (!ok) break;
                if (issued) umma_commit(&accf[acc]);
                else mbar_arrive(&accf[acc]);  // empty tile: the epilogue writes zeros
                acc ^= 1;
                if (acc == 0) acc_ph ^= 1u;
            }
            // Drain: no MMA may be in flight when TMEM is released.
            umma_commit(drain);
            mbar_wait_bounded(drain, 0u, budget_ns, status, ST_TIMEOUT_DRAIN);
        }
        grid_dep_launch();
    } else {
        // ------------------------------ epilogue (warps 2..9) ---------------------------
        const int quarter = warp & 3;       // TMEM lanes this warp may access
        const int half = (warp - 2) >> 2;   // this warp's chunks: half, half + 2, ...
        const int r_in_tile = quarter * 32 + lane;
        constexpr int kChunks = BN / 32;
        int acc = 0;
        uint32_t acc_ph = 0;
        for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
            if (tile + static_cast<int>(gridDim.x) >= total_tiles) grid_dep_launch();  // the CTA's last tile
            int local = 0;
            const GemmProblem *P = resolve_tile(probs, nprob, sched, tile, &local);
            if (P == nullptr) continue;
            int mb, nb;
            tile_coords(P, local, mb, nb);
            constexpr int kMine = kChunks / 2;  // chunks of this warp: half, half + 2, ...
            uint32_t cnt = 0;
            if constexpr (EPI == EPI_BOOL) {
                const int row = mb * BM + r_in_tile;
                const bool row_ok = row < P->M;
                if (!mbar_wait_bounded(&accf[acc], acc_ph, budget_ns, status, ST_TIMEOUT_ACC_FULL)) break;
                tc_fence_after();
                const bool live = tile_live<BN>(P, mb, nb, P->K / C::BK);  // warp-uniform
                const uint32_t tbase = tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) +
                                       static_cast<uint32_t>(acc * BN);
#pragma unroll
                for (int u = 0; u < kMine; ++u) {
                    const int c = half + 2 * u;
                    const int col = nb * BN + c * 32;
                    uint32_t v[32];
                    if (live) {
                        tmem_ld_32x32b_x32(tbase + c * 32, v);
                        tmem_ld_wait();
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = 0u;
                    }
                    uint32_t word = 0;
                    if (row_ok && col < P->N) word = epi_bool_chunk(P->epi, row, col, v, cnt);
                    if (P->epi.occ_out != nullptr) {
                        if (__any_sync(0xffffffffu, word != 0u) && lane == 0)
                            P->epi.occ_out[((P->epi.out_row0 + mb * BM + quarter * 32) >> 7) * P->epi.occ_ld +
                                           ((P->epi.out_col0 + col) >> 7)] = 1;
                    }
                }
            } else {
                // FP32 output, coalesced.  tcgen05.ld gives a lane one row's 32 columns of a chunk;
                // the chunk passes through a 32 x 32 shared-memory tile of the warp (16-byte granules
                // XOR-swizzled by row: conflict-free by rows and by granules), so that every load
                // and store of C moves whole 128-byte row segments.  The subtracting epilogue fetches
                // its first two chunks of C (cp.async) while the MMAs finish, and each later one
                // into the tile the chunk two before it has left (a K = 128 update is bound by
                // these bytes).
                float4 *tiles = epi_stage + (warp - 2) * C::EPI_TILES * 256;
                const int row0 = mb * BM + quarter * 32;  // the warp's rows: row0 .. row0 + 31
                const int rows = min(32, P->M - row0);
                const GemmEpilogue &E = P->epi;
                const int64_t ld = E.ld_c32;
                float *cbase = E.c32 + (static_cast<int64_t>(E.out_row0) + row0) * ld + E.out_col0 + nb * BN;
                auto gidx = [](int r, int g) { return r * 8 + (g ^ (r & 7)); };
                const int lr = lane >> 3, lg = lane & 7;  // coalesced transfers: rows 4 i + lr, granule lg
                auto chunk_ok = [&](int u) { return nb * BN + (half + 2 * u) * 32 < P->N; };
                auto fetch = [&](int u, float4 *t) {
                    if (chunk_ok(u) && rows > 0) {  // (src points into C only then)
                        const float *src = cbase + (half + 2 * u) * 32;
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int r = 4 * i + lr;
                            const bool ok = r < rows;
                            cp_async16(t + gidx(r, lg), ok ? src + r * ld + 4 * lg : src, ok ? 16u : 0u);
                        }
                    }
                    cp_async_commit();  // (empty for a chunk past N: the group count stays regular)
                };
                if constexpr (EPI == EPI_SUB_F32) {
                    fetch(0, tiles);
                    if (kMine > 1) fetch(1, tiles + 256);
                }
                if (!mbar_wait_bounded(&accf[acc], acc_ph, budget_ns, status, ST_TIMEOUT_ACC_FULL)) {
                    cp_async_wait<0>();  // no copy into shared memory may outlive the CTA
                    break;
                }
                tc_fence_after();
                const bool live = tile_live<BN>(P, mb, nb, P->K / C::BK);  // warp-uniform
                const uint32_t tbase = tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) +
                                       static_cast<uint32_t>(acc * BN);
#pragma unroll
                for (int u = 0; u < kMine; ++u) {
                    float4 *t = tiles + (EPI == EPI_SUB_F32 ? (u & 1) * 256 : 0);
                    uint32_t v[32];
                    if (live) {
                        tmem_ld_32x32b_x32(tbase + (half + 2 * u) * 32, v);
                        tmem_ld_wait();
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = 0u;
                    }
                    if constexpr (EPI == EPI_SUB_F32) {
                        if (u + 1 < kMine) cp_async_wait<1>();
                        else cp_async_wait<0>();
                        __syncwarp();
#pragma unroll
                        for (int g = 0; g < 8; ++g) {
                            const float4 c = t[gidx(lane, g)];
                            t[gidx(lane, g)] = make_float4(
                                c.x - __uint_as_float(v[4 * g + 0]), c.y - __uint_as_float(v[4 * g + 1]),
                                c.z - __uint_as_float(v[4 * g + 2]), c.w - __uint_as_float(v[4 * g + 3]));
                        }
                    } else {
#pragma unroll
                        for (int g = 0; g < 8; ++g)
                            t[gidx(lane, g)] = make_float4(__uint_as_float(v[4 * g + 0]), __uint_as_float(v[4 * g + 1]),
                                                           __uint_as_float(v[4 * g + 2]), __uint_as_float(v[4 * g + 3]));
                    }
                    __syncwarp();
                    if (chunk_ok(u)) {
                        float *dst = cbase + (half + 2 * u) * 32;
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int r = 4 * i + lr;
                            if (r < rows) *reinterpret_cast<float4 *>(dst + r * ld + 4 * lg) = t[gidx(r, lg)];
                        }
                    }
                    __syncwarp();
                    if constexpr (EPI == EPI_SUB_F32)
                        if (u + 2 < kMine) fetch(u + 2, t);
                }
            }
            tc_fence_before();
            mbar_arrive(&acce[acc]);
            if (EPI == EPI_BOOL && P->epi.count) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
                if (lane == 0 && cnt) atomicAdd(P->epi.count, static_cast<unsigned long long>(cnt));
            }
            acc ^= 1;
            if (acc == 0) acc_ph ^= 1u;
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem_base, C::TMEM_COLS);
}

// ---- host side ------------------------------------------------------------------------

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

bool make_map(CUtensorMap *m, CUtensorMapDataType dt, int elem, const Operand &op, uint32_t box_x,
              uint32_t box_y, std::string *err) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) {
        if (err) *err = "cuTensorMapEncodeTiled is not available from the driver";
        return false;
    }
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(op.cols), static_cast<cuuint64_t>(op.rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(op.ld) * elem};
    cuuint32_t box[2] = {box_x, box_y};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, dt, 2, const_cast<void *>(op.base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        if (err) {
            char buf[160];
            snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (%d) dims %llu x %llu ld %lld",
                     static_cast<int>(r), static_cast<unsigned long long>(op.cols),
                     static_cast<unsigned long long>(op.rows), static_cast<long long>(op.ld));
            *err = buf;
        }
        return false;
    }
    return true;
}

template <int KIND, int BN, bool BK_, int EPI>
cudaError_t prepare_t() {
    using C = Cfg<KIND, BN, EPI>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(umma_gemm_kernel<KIND, BN, BK_, EPI>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    });
    return attr_err;
}

template <int KIND, int BN, bool BK_, int EPI>
cudaError_t launch_t(const GemmProblem *d_probs, int nprob, int total_tiles, const int *sched, int grid,
                     int *status, uint64_t budget, cudaStream_t s, bool pdl) {
    using C = Cfg<KIND, BN, EPI>;
    const cudaError_t attr_err = prepare_t<KIND, BN, BK_, EPI>();
    if (attr_err != cudaSuccess) return attr_err;
    if (!pdl) {
        umma_gemm_kernel<KIND, BN, BK_, EPI><<<grid, kThreads, C::SMEM, s>>>(d_probs, nprob, total_tiles,
                                                                             sched, status, budget);
        return cudaGetLastError();
    }
    return launch_programmatic(umma_gemm_kernel<KIND, BN, BK_, EPI>, dim3(grid), dim3(kThreads), C::SMEM, s, d_probs,
                               nprob, total_tiles, sched, status, budget);
}

}  // namespace

bool tensor_map_2d(CUtensorMap *m, CUtensorMapDataType dt, int elem, const void *base, int64_t cols, int64_t rows,
                   int64_t ld, uint32_t box_x, uint32_t box_y, std::string *err) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) {
        if (err) *err = "cuTensorMapEncodeTiled is not available from the driver";
        return false;
    }
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * elem};
    cuuint32_t box[2] = {box_x, box_y};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(m, dt, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        if (err) *err = "cuTensorMapEncodeTiled failed";
        return false;
    }
    return true;
}

int gemm_tile_m() { return BM; }

cudaError_t gemm_prepare(GemmKind kind, bool b_kmajor, int bn, GemmEpi epi) {
    if (kind == KIND_F8 && epi == EPI_BOOL) {
        if (bn == 256) return b_kmajor ? prepare_t<KIND_F8, 256, true, EPI_BOOL>() : prepare_t<KIND_F8, 256, false, EPI_BOOL>();
        if (bn == 128) return b_kmajor ? prepare_t<KIND_F8, 128, true, EPI_BOOL>() : prepare_t<KIND_F8, 128, false, EPI_BOOL>();
    }
    // TF32 runs with K-major operands only (both operands row-major with K contiguous)
    if (kind == KIND_TF32 && b_kmajor && (bn == 128 || bn == 256)) {
        if (epi == EPI_SUB_F32)
            return bn == 256 ? prepare_t<KIND_TF32, 256, true, EPI_SUB_F32>() : prepare_t<KIND_TF32, 128, true, EPI_SUB_F32>();
        if (epi == EPI_STORE_F32)
            return bn == 256 ? prepare_t<KIND_TF32, 256, true, EPI_STORE_F32>()
                             : prepare_t<KIND_TF32, 128, true, EPI_STORE_F32>();
    }
    return cudaErrorInvalidValue;
}

bool gemm_make_problem(GemmProblem *p, GemmKind kind, bool b_kmajor, int bn, int M, int N, int K,
                       const Operand &A, const Operand &B, const GemmEpilogue &epi,
                       std::string *err) {
    std::memset(p, 0, sizeof(*p));
    const int elem = kind == KIND_F8 ? 1 : 4;
    const int bk = 128 / elem;
    if (M <= 0 || N <= 0 || K <= 0 || K % bk != 0 || N % 32 != 0 || (bn != 128 && bn != 256)) {
        if (err) *err = "unsupported GEMM shape";
        return false;
    }
    if (kind == KIND_TF32 && (reinterpret_cast<uintptr_t>(epi.c32) % 16 != 0 || epi.ld_c32 % 4 != 0 ||
                              epi.out_col0 % 4 != 0)) {
        if (err) *err = "FP32 output must be 16-byte aligned with a row stride of 4k elements";
        return false;
    }
    const CUtensorMapDataType dt =
        kind == KIND_F8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    if (!make_map(&p->tmA, dt, elem, A, static_cast<uint32_t>(bk), BM, err)) return false;
    if (b_kmajor) {
        if (!make_map(&p->tmB, dt, elem, B, static_cast<uint32_t>(bk), static_cast<uint32_t>(bn), err))
            return false;
    } else {
        if (!make_map(&p->tmB, dt, elem, B, static_cast<uint32_t>(bk), static_cast<uint32_t>(bk), err))
            return false;
    }
    p->M = M;
    p->N = N;
    p->K = K;
    p->tiles_m = (M + BM - 1) / BM;
    p->tiles_n = (N + bn - 1) / bn;
    p->tile_start = 0;
    p->a_row0 = A.row0;
    p->a_col0 = A.col0;
    p->b_row0 = B.row0;
    p->b_col0 = B.col0;
    p->epi = epi;
    return true;
}

cudaError_t gemm_launch(GemmKind kind, bool b_kmajor, int bn, GemmEpi epi, const GemmProblem *d_probs,
                        int nprob, int total_tiles, int grid, int *d_status, uint64_t budget_ns,
                        cudaStream_t stream, const int *d_sched, bool pdl) {
    if (total_tiles <= 0) return cudaSuccess;
    if (grid > total_tiles) grid = total_tiles;
    const int *sc = d_sched;
#define DL_GEMM_T(K_, BN_, BKM_, EPI_) \
    launch_t<K_, BN_, BKM_, EPI_>(d_probs, nprob, total_tiles, sc, grid, d_status, budget_ns, stream, pdl)
    if (kind == KIND_F8 && epi == EPI_BOOL) {
        if (bn == 256)
            return b_kmajor ? DL_GEMM_T(KIND_F8, 256, true, EPI_BOOL) : DL_GEMM_T(KIND_F8, 256, false, EPI_BOOL);
        if (bn == 128)
            return b_kmajor ? DL_GEMM_T(KIND_F8, 128, true, EPI_BOOL) : DL_GEMM_T(KIND_F8, 128, false, EPI_BOOL);
    }
    if (kind == KIND_TF32 && b_kmajor && (bn == 128 || bn == 256)) {
        if (epi == EPI_SUB_F32)
            return bn == 256 ? DL_GEMM_T(KIND_TF32, 256, true, EPI_SUB_F32) : DL_GEMM_T(KIND_TF32, 128, true, EPI_SUB_F32);
        if (epi == EPI_STORE_F32)
            return bn == 256 ? DL_GEMM_T(KIND_TF32, 256, true, EPI_STORE_F32)
                             : DL_GEMM_T(KIND_TF32, 128, true, EPI_STORE_F32);
    }
#undef DL_GEMM_T
    return cudaErrorInvalidValue;
}

}  // namespace dl
