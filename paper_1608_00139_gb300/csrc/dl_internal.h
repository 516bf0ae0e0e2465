// dl_internal.h -- declarations shared by the translation units of libdl (not installed).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <string>
#include <utility>

namespace dl {

// Every allocation of the library goes through these (dl_debug.cu): cudaMalloc / cudaMallocHost,
// or cudaErrorMemoryAllocation when the DL_FAULT plan says this allocation fails.
cudaError_t device_alloc(void **ptr, size_t bytes);
cudaError_t host_pinned_alloc(void **ptr, size_t bytes);

// An NVTX range for the lifetime of the object (a no-op unless a profiler is attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// Device status word bits (the host reads the word after a call).
enum : int {
    ST_TIMEOUT_FULL = 1,       // MMA warp: operand stage never arrived
    ST_TIMEOUT_EMPTY = 2,      // producer: stage never released
    ST_TIMEOUT_ACC_FULL = 4,   // epilogue: accumulator never completed
    ST_TIMEOUT_ACC_EMPTY = 8,  // MMA warp: accumulator never drained
    ST_TIMEOUT_DRAIN = 16,     // teardown drain expired
    ST_BAD_INPUT = 32,         // an input byte was not 0/1
    ST_TIMEOUT_DEP = 64,       // a dependency counter never reached its target
    ST_BAD_PAD = 128,          // a bit-packed input row had a bit at a column >= n
};

// ---------------------------------------------------------------------------------------
// tcgen05 GEMM (dl_umma.cu)
// ---------------------------------------------------------------------------------------
enum GemmKind : int { KIND_F8 = 0, KIND_TF32 = 1 };
enum GemmEpi : int { EPI_BOOL = 0, EPI_SUB_F32 = 1, EPI_STORE_F32 = 2 };

// Boolean epilogue: v = [acc > 0] OR [add8 != 0]; writes e4m3 1.0/0.0 bytes, packed bits,
// and adds the number of ones to *count.  SUB_F32 epilogue: c32 -= acc (in place);
// STORE_F32 epilogue: c32 = acc.
struct GemmEpilogue {
    uint8_t *out8;            // may be null
    int64_t ld_out8;          // bytes per row
    const uint8_t *add8;      // may be null
    int64_t ld_add8;
    uint32_t *bits;           // may be null; 32-bit words, bit j of word c/32 = column c+j
    int64_t ld_bits32;        // 32-bit words per row
    unsigned long long *count;  // may be null
    float *c32;               // SUB_F32 only
    int64_t ld_c32;           // floats per row
    int32_t out_row0, out_col0;  // output coordinates of the problem's (0, 0)
    uint8_t *occ_out;         // may be null: set to 1 for every 128 x 128 block with a one
    int32_t occ_ld;           // blocks per row of occ_out
};

// One GEMM problem D(MxN) = A(MxK) * B(KxN).  Lives in device memory (tensor maps are read
// by TMA from global memory; CUtensorMap carries the descriptor alignment).
struct GemmProblem {  // CUtensorMap members carry the TMA descriptor alignment
    CUtensorMap tmA;  // A: K-major (row-major M x K); box {128 bytes of K, 128 rows}
    CUtensorMap tmB;  // B: MN-major (row-major K x N; box {128 bytes of N, BK rows of K}) or
                      //    K-major (row-major N x K; box {128 bytes of K, BN rows})
    int32_t M, N, K;
    int32_t tiles_m, tiles_n, tile_start;
    int32_t a_row0, a_col0;  // A(0,0) at tensor coordinates (x = a_col0, y = a_row0)
    int32_t b_row0, b_col0;  // B: MN-major (x = n, y = k); K-major (x = k, y = n)
    const int *gate;         // may be null; tiles of this problem are skipped while *gate != 0
    // May be null (dense).  128 x 128 block occupancy of A (row-blocks x k-blocks) and of an
    // MN-major B (k-blocks x column-blocks), occ_ld blocks per row; FP8 only.  A k-block
    // whose A block or B blocks are all empty contributes nothing and is skipped.
    const uint8_t *occ_a, *occ_b;
    int32_t occ_ld;
    GemmEpilogue epi;
};

struct Operand {
    const void *base;   // start of the whole matrix (16-byte aligned)
    int64_t rows, cols; // extents of the whole matrix, elements
    int64_t ld;         // elements per row (row stride), ld*elem multiple of 16 bytes
    int32_t row0, col0; // where the operand starts inside that matrix
};

// Host: fill one problem (tensor maps + tiling).  bn: 128 or 256.  Returns false and sets
// *err on an unsupported shape.
bool gemm_make_problem(GemmProblem *p, GemmKind kind, bool b_kmajor, int bn, int M, int N, int K,
                       const Operand &A, const Operand &B, const GemmEpilogue &epi,
                       std::string *err);
// Launch over problems already in device memory.  total_tiles = sum of tiles.  With d_sched
// (device ints, written by an earlier kernel) only the problems it lists are computed:
// d_sched[0] = count A, d_sched[1] = their tiles, d_sched[2 + j] = problem index of entry j,
// d_sched[2 + nprob + j] = first tile of entry j; total_tiles and grid are then upper bounds.
// pdl: a programmatic launch (it may start while the previous kernel on the stream finishes;
// its set-up overlaps that kernel's end and it reads its operands only after that kernel is done).
cudaError_t gemm_launch(GemmKind kind, bool b_kmajor, int bn, GemmEpi epi,
                        const GemmProblem *d_probs, int nprob, int total_tiles, int grid,
                        int *d_status, uint64_t budget_ns, cudaStream_t stream,
                        const int *d_sched = nullptr, bool pdl = false);
// Launch kernel<<<grid, block, smem, s>>>(args...) with programmatic stream serialisation.
template <typename... Params, typename... Args>
cudaError_t launch_programmatic(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                Args &&...args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
int gemm_tile_m();
// A 2-D tensor map (no swizzle) of a row-major matrix (rows x cols elements, ld elements per
// row) with a box of box_y rows x box_x elements, for TMA loads outside the GEMM.
bool tensor_map_2d(CUtensorMap *m, CUtensorMapDataType dt, int elem, const void *base, int64_t cols, int64_t rows,
                   int64_t ld, uint32_t box_x, uint32_t box_y, std::string *err);
// Set the kernel's shared-memory attribute ahead of time (e.g. before a stream capture).
cudaError_t gemm_prepare(GemmKind kind, bool b_kmajor, int bn, GemmEpi epi);

// ---------------------------------------------------------------------------------------
// Boolean / streaming kernels (dl_bool.cu)
// ---------------------------------------------------------------------------------------
// Validate 0/1 input, reduce row sums (max into *dmax, total into *nnz), and write the
// e4m3 operand of size np x np: value 1.0 where src is 1, plus 1.0 on the diagonal if
// add_identity; zero padding outside n x n.  *count gets the number of ones written.
cudaError_t ingest_u8_to_e4m3(const uint8_t *src, int n, int np, uint8_t *dst, int add_identity,
                              unsigned long long *dmax, unsigned long long *nnz,
                              unsigned long long *count, int *status, cudaStream_t s);
// Load (under CUDA's lazy module loading) the kernels behind ingest_u8_to_e4m3 and bits_sweep.
cudaError_t load_ingest_and_sweep();
// One sweep of the certificate / recheck kernel on bits (64-bit words, wp words per row):
//   mode 0 (reflexive check):  out_i = OR_{k in succ(i)} M_k;  violation iff (out_i | e_i) != M_i
//   mode 1 (closure sweep):    out_i = M_i | E_i | OR_{k in succ(i)} M_k (in place allowed);
//                              violation iff out_i != M_i (row changed)
// E: n x n bytes (row stride lde).  stop_early: rows are skipped once a violation is seen.
cudaError_t bits_sweep(const uint8_t *E, int64_t lde, int n, const uint64_t *M, uint64_t *out,
                       int64_t wp, int mode, int stop_early, unsigned long long *violations,
                       unsigned long long *ones, cudaStream_t s);

// The sweep on the CSR (ptr, col) of E, edge-parallel: work units of up to 64 successors of
// one row, combined with atomicOr.  sweep_units builds unit_off (n + 1 entries; cnt is n ints
// of scratch) once per CSR.  mode 1: in place (out must be M), *violations += changed units;
// mode 0: out = E M (rows < n), *violations += rows with (out_i | e_i) != M_i, *ones += ones.
cudaError_t sweep_units(const int *ptr, int n, int *cnt, int *unit_off, cudaStream_t s);
// max_deg: ||E||_inf if known (rows of at most 256 successors take row-direct kernels, which
// need no unit_off), or -1.  skip_if_zero (mode 1): the previous sweep's counter; when it is
// zero on the device the sweep does nothing (that sweep already proved convergence).
// colmask (optional): the columns with an incoming edge.  Every row of E M lies inside it and
// every row of the reflexive closure inside it plus the row's own bit, so a row-direct sweep
// stops reading successors once a row covers that much (without it: all n columns).
// gate (row-direct only): when *gate != 0 on the device the launch does nothing.
cudaError_t bits_sweep_csr(const int *ptr, const int *col, const int *unit_off, int n, const uint64_t *M,
                           uint64_t *out, int64_t wp, int mode, unsigned long long *violations,
                           unsigned long long *ones, int *launches, cudaStream_t s, int max_deg,
                           const unsigned long long *skip_if_zero = nullptr, const uint64_t *colmask = nullptr,
                           const int *gate = nullptr);
// Whether bits_sweep_csr takes the row-direct kernels (then unit_off is not read).
bool row_direct(int max_deg, int64_t wp);
// Rows i < n of the reflexive closure by the Iteration on single rows (one warp per row,
// semi-naive frontier expansion over the CSR, row bits in shared memory): M_i gets every node
// reached; a row whose frontier outgrows 256 nodes keeps what it reached (a subset of its
// closure row) and counts in *open_rows.  Rows of at most 256 words (n <= 16384).
bool row_iteration_fits(int64_t wp);
// With gate: decided on the device; nothing but *open_rows += n if *gate != 0 or the graph
// has more than two facts per row.
cudaError_t row_iteration(const int *ptr, const int *col, int n, int64_t wp, uint64_t *M,
                          unsigned long long *open_rows, cudaStream_t s, const int *gate = nullptr);
// Bit-matrix helpers for same generation (np x np bits, wp = np / 64 words per row).
// dst = src^T (np a multiple of 64; dst distinct from src); nothing if *skip == 0.
cudaError_t bits_transpose(const uint64_t *src, uint64_t *dst, int np, int64_t wp, const unsigned long long *skip,
                           cudaStream_t s);
// Rows i < n: dst_i = [dst_i if accumulate] | OR_{k in succ(i)} src_k over the CSR (ptr, col);
// with accumulate *changed is non-zero iff a row changed; nothing if *skip == 0.  With unit_off
// (from sweep_units) rows are split into work units combined with atomicOr (heavy rows);
// without, one warp per row (wp <= 256).
cudaError_t bits_gather(const int *ptr, const int *col, const int *unit_off, int n, const uint64_t *src, uint64_t *dst,
                        int64_t wp, int accumulate, unsigned long long *changed, const unsigned long long *skip,
                        cudaStream_t s);
// *ones += ones in rows < n.
cudaError_t bits_count(const uint64_t *M, int n, int64_t wp, unsigned long long *ones, cudaStream_t s);
// M = identity on rows < n, zero elsewhere (np rows).
cudaError_t bits_identity(uint64_t *M, int n, int np, int64_t wp, cudaStream_t s);
// *diff += words where A and B differ.
cudaError_t bits_diff(const uint64_t *A, const uint64_t *B, int64_t words, unsigned long long *diff, cudaStream_t s);
// e4m3 0/1 operand (np x np, 1.0 = 0x38) from a bit matrix.
cudaError_t bits_to_e4m3(const uint64_t *bits, int64_t wp, int np, uint8_t *C, cudaStream_t s);

// ---------------------------------------------------------------------------------------
// Graph utilities (dl_graph.cu)
// ---------------------------------------------------------------------------------------
// CSR of a dense n x n 0/1 matrix: csr_build writes per-row counts and ptr (n + 1 entries,
// exclusive scan); after reading ptr[n] (= nnz) the caller sizes col and runs csr_fill.
cudaError_t csr_build(const uint8_t *E, int n, int *cnt, int *ptr, cudaStream_t s);
cudaError_t csr_fill(const uint8_t *E, int n, const int *ptr, int *col, cudaStream_t s);
// One pass over E: the bits of I + E into M (np rows of wp words; rows >= n hold only their
// diagonal bit), the CSR row pointers, and the ingest's checks: status |= ST_BAD_INPUT on a
// byte other than 0/1, *dmax = ||E||_inf, *nnz += facts, *diag += self-loops (counters zeroed
// by the caller), and colmask |= the columns with an incoming edge (wp words, zeroed by the
// caller; wp <= 6144).  E's rows may have any alignment.
cudaError_t csr_pack_checked(const uint8_t *E, int n, int np, int64_t wp, int *cnt, int *ptr, uint64_t *M,
                             unsigned long long *dmax, unsigned long long *nnz, unsigned long long *diag, int *status,
                             uint64_t *colmask, cudaStream_t s);
// The same from a bit-packed E (row r: ceil(n/64) words at Eb + r ceil(n/64), bit j mod 64 of
// word j/64 = E[r][j], the layout of the model bits): status |= ST_BAD_PAD if a bit at a
// column >= n is set (the bit is dropped).  wp <= 6144.
cudaError_t bits_ingest_checked(const uint64_t *Eb, int n, int np, int64_t wp, int *cnt, int *ptr, uint64_t *M,
                                unsigned long long *dmax, unsigned long long *nnz, unsigned long long *diag,
                                int *status, uint64_t *colmask, cudaStream_t s);
// The n x n bytes (row-major 0/1) of a bit-packed E, for the paths that start from bytes;
// status |= ST_BAD_PAD as above.
cudaError_t unpack_bits_u8(const uint64_t *Eb, int n, uint8_t *E, int *status, cudaStream_t s);
// Bits of E alone (np rows of wp words, rows >= n zero), status |= ST_BAD_INPUT on a byte other
// than 0/1.
cudaError_t pack_bits(const uint8_t *E, int n, int np, int64_t wp, uint64_t *M, int *status, cudaStream_t s);
// Column indices of E from the packed bits of I + E (as written by csr_pack_checked).
cudaError_t csr_fill_from_bits(const uint64_t *M, int n, int64_t wp, const int *ptr, int *col, cudaStream_t s);
// The same before the host knows the CSR's size: if the facts exceed cap entries or *dmax
// exceeds max_deg, nothing is written and *gate = 1, else *gate = 0.
cudaError_t csr_fill_from_bits_guarded(const uint64_t *M, int n, int64_t wp, const int *ptr, int *col, int64_t cap,
                                       const unsigned long long *dmax, int max_deg, int *gate, cudaStream_t s);
// out[0..n] = exclusive prefix sums of cnt[0..n-1] (out[n] = total); one CTA.
cudaError_t exclusive_scan(const int *cnt, int n, int *out, cudaStream_t s);
// The same with every SM taking part, for long arrays (scratch: 2 * (ceil(n / 1024) + 1) ints).
cudaError_t exclusive_scan_large(const int *cnt, int n, int *out, int *scratch, cudaStream_t s);

// ---------------------------------------------------------------------------------------
// FP64 path (dl_fp64.cu)
// ---------------------------------------------------------------------------------------
// G = [I - eps E | eps A] (np x 2np doubles, zero/identity padding; A = E for the closure).
cudaError_t fp64_build(const uint8_t *E, const uint8_t *A, int n, int np, double eps, double *G, int64_t ldg,
                       cudaStream_t s);
// The same with a real right-hand side: G = [I - eps E | eps F], F n x n FP64 (row stride n).
cudaError_t fp64_build_real(const uint8_t *E, const double *F, int n, int np, double eps, double *G, int64_t ldg,
                            cudaStream_t s);
cudaError_t fp64_solve(double *G, int64_t ldg, int np, int *launches, cudaStream_t s);
// threshold X > 0 into bits, count guard-band entries (|X| <= tau or X < 0)
cudaError_t thresh_pack_f64(const double *X, int64_t ldx, int n, int np, double tau, uint64_t *bits,
                            int64_t wp, unsigned long long *guard, cudaStream_t s);

int num_sms();

// ---------------------------------------------------------------------------------------
// Real same-generation solution S~ = eps (B + P S~ P^T) (dl_sgreal.cu)
// ---------------------------------------------------------------------------------------
// One FP64 step over the CSR of P (np x np row-major buffers, zero outside n x n; B: n x n
// bytes or NULL for the identity):  U = X P^T, V = eps (B + P U), D = V - X.  Xn (optional)
// <- V; R (optional) <- D in FP32.  *dmax (zeroed by the caller): with R, max |D| as the bit
// pattern of a non-negative double; without R (a series step, where V >= X), a bound coded as
// e + 4096 with max D < 2^e, or 0 when nothing changed (integer operations only).  np * 8 bytes
// of shared memory per block (np <= 29056).
// fused: one pass that sums X over (parent of i) x (parent of j) pairs, for P with at most 4
// parents per node and np <= 16384 (sg_real_fused); U is then unused.  dmax may be NULL (no
// change is measured and X is not read back).
cudaError_t sg_real_step(const int *ptr, const int *col, int n, int np, double eps, const uint8_t *B, const double *X,
                         double *U, double *Xn, float *R, unsigned long long *dmax, bool fused, cudaStream_t s);
bool sg_real_fused(int np, unsigned long long max_parents);
// A = scale P, NA = -A (FP32, np x np, zero padding).
cudaError_t sg_scaled_p(const uint8_t *P, int n, int np, float scale, float *A, float *NA, cudaStream_t s);
// *out = max_i sum_j |A[i][j]| as FP32 bits (zeroed by the caller).
cudaError_t row_abs_sum_max(const float *A, int np, unsigned *out, cudaStream_t s);
cudaError_t negate_f32(const float *a, float *b, int64_t count, cudaStream_t s);
cudaError_t add_f32_to_f64(double *x, const float *d, int64_t count, cudaStream_t s);
cudaError_t transpose_f32(const float *src, int64_t lds, int rows, int cols, float *dst, int64_t ldd, cudaStream_t s);
// One step of the transposed class's series (Sec. 6.2, eq. matrixeq:trans:1) over the CSR of R1:
// U = X^T, then Xn = eps (R1 + R1 U), i.e. Xn[i][j] = eps (R1[i][j] + sum_{y in succ(i)} X[j][y])
// (R1: n x n bytes; X, U, Xn: np x np, zero outside n x n); *dmax (zeroed by the caller) as
// for the same-generation series (a power-of-two bound on the step's largest change).
cudaError_t trans_real_step(const int *ptr, const int *col, int n, int np, double eps, const uint8_t *R1,
                            const double *X, double *U, double *Xn, unsigned long long *dmax, cudaStream_t s);
// dst |= src over `words` 64-bit words.
cudaError_t bits_or(uint64_t *dst, const uint64_t *src, int64_t words, cudaStream_t s);

}  // namespace dl
