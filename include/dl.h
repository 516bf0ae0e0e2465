/*
 * dl.h -- C ABI of libdl: least Herbrand models of linear Datalog programs over N constants
 * and binary predicates, computed on one GB300 GPU (sm_103a) the way Sato, "A Linear
 * Algebraic Approach to Datalog Evaluation" (TPLP) states the problem:
 *
 *   - constants are one-hot vectors and a binary relation r is its N x N adjacency matrix
 *     R with R[i][j] = 1 iff r(e_i, e_j) (Sec. 2);
 *   - the iff-completion of a program gives a matrix equation with the clamp
 *     min1(x) = min(x, 1) (Sec. 3), e.g. R2 = min1(R1 + R1 R2) for transitive closure;
 *   - its linearisation R~ = eps (R1 + R1 R~) (Sec. 4) has the least solution
 *     R~ = (I - eps R1)^-1 eps R1 when 0 < eps <= 1/(1 + ||R1||_inf) (Lemma 1,
 *     Proposition 1), and thresholding R~ at 0 gives the least model (Theorem 1).
 *
 * Conventions shared by every call:
 *   - Every call returns a dl_status; dl_last_error() gives a message for the last failed
 *     call on the calling thread.  No C++ exception crosses this boundary.
 *   - Matrices are dense, row-major, n*n bytes, each byte 0 or 1 (any other byte value is
 *     rejected with DL_EINVAL).  Bit matrices ("bits") hold ceil(n/64) uint64 words per row;
 *     entry (i, j) is bit (j mod 64) of word i*ceil(n/64) + j/64, least significant first.
 *   - dl_mem says where input and output pointers live: DL_MEM_HOST (ordinary host memory;
 *     the call copies in and out) or DL_MEM_DEVICE (device memory of the context's GPU,
 *     e.g. a torch CUDA tensor's data pointer).  Inputs and outputs of one call share it.
 *   - The caller owns every buffer.  Synchronous calls have read their inputs and written
 *     their outputs when they return (device outputs: complete on the context's stream,
 *     which the call synchronises before returning).
 *   - n == 0 returns DL_OK and writes nothing.  n < 0 or a NULL required pointer returns
 *     DL_EINVAL.
 *   - Calls on one context are serialised by the context; contexts are independent.
 */
#ifndef DL_H
#define DL_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DL_API __attribute__((visibility("default")))
#else
#define DL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dl_ctx dl_ctx;

typedef enum {
    DL_OK = 0,
    DL_EINVAL = 1,     /* bad argument (size, pointer, eps, threshold, non-0/1 input) */
    DL_ENOMEM = 2,     /* device or host allocation failed, or a request can never fit */
    DL_EDEVICE = 3,    /* CUDA error, or no usable sm_103 device */
    DL_ETIMEOUT = 4,   /* a bounded device-side wait expired, or dl_poll timed out */
    DL_EBUSY = 5,      /* dl_poll: the request is still running */
    DL_ENOTCONV = 6,   /* an iteration did not converge within its limit */
    DL_ECANCELED = 7,  /* the request was cancelled */
    DL_ENOTIMPL = 8    /* the requested path does not exist for this call */
} dl_status;

/* Which numerical route computes the model (all give the same, exact model). */
typedef enum {
    DL_PATH_AUTO = 0,      /* FP8 tensor-core squarings and bit sweeps (the Iteration step,
                              Sec. 7.1), whichever is cheaper for the graph */
    DL_PATH_FP64 = 1,      /* plain FP64 inverse of I - eps E (Prop. 1), threshold > 0 */
    DL_PATH_MIXED = 2,     /* TF32 tensor-core LU + FP64 iterative refinement + guard */
    DL_PATH_BOOL_FP8 = 3   /* boolean repeated squaring on FP8 e4m3 tensor cores */
} dl_path;

typedef enum { DL_MEM_HOST = 0, DL_MEM_DEVICE = 1 } dl_mem;

typedef struct {
    void *stream;              /* cudaStream_t to run on; NULL = the context's own stream */
    size_t hbm_budget_bytes;   /* serving admission budget; 0 = 90% of free device memory */
    int32_t max_slots;         /* serving: requests in flight at once; 0 = 4 */
    double refine_tol;         /* refinement of the real paths (closure, tail class, S~) and the
                                  S~ series: stop when max|R| <= tol * eps; 0 = 1e-13 */
    int32_t refine_max_iters;  /* refinement step limit of those paths; 0 = 30 */
    double guard_tau;          /* entries with |R~| <= tau are flagged for recheck; 0 = 1e-30 */
    double wait_timeout_s;     /* limit of every device-side wait; 0 = 2 s */
    int32_t autotune;          /* 1: tune each new size bucket on its first closure or same-generation
                                  call (dl_autotune); 0: the measured table only (cache or explicit
                                  dl_autotune calls), else the fixed rules */
    const char *tune_cache;    /* JSON cache of tuned choices, read at dl_create and written after
                                  each tuning run; NULL: the DL_TUNE_CACHE environment variable, if set */
} dl_config;

typedef struct {
    int32_t path_used;       /* dl_path that ran */
    double eps_used;         /* epsilon of the linearised equation (reported for every path) */
    int32_t iters;           /* squarings (FP8), doubling steps (SG), or refinement steps */
    double final_resid;      /* mixed/FP64: max|eps E - (I - eps E) X| / max|eps E| (-1: not formed) */
    int64_t guard_flagged;   /* entries in the guard band (|X| <= tau or X < 0) */
    int64_t rows_rechecked;  /* rows corrected by the exact boolean recheck */
    int32_t recheck_sweeps;  /* sweeps of the certificate/recheck kernel */
    int64_t model_ones;      /* number of 1 bits in the model */
    double ms_total;         /* device time of the call (CUDA events), ms */
    double ms_factor;        /* LU factorisation (FP64/mixed) or ingest (FP8) */
    double ms_solve;         /* triangular solves (FP64/mixed) or squarings (FP8/SG) */
    double ms_refine;        /* refinement (mixed) */
    double ms_epilogue;      /* threshold, bit packing, certificate and recheck */
    double tflops_equiv;     /* (8/3) n^3 / ms_total, TC only */
    int32_t gpu_launches;    /* kernels this call launched */
    int32_t gemm_launches;   /* tensor-core GEMM launches among them */
    double ms_gemm;          /* summed device time of those GEMM launches (CUDA events on the
                                launching stream), ms */
    double gemm_flops;       /* 2*M*N*K summed over those GEMM launches (padded sizes) */
    double ms_queue;         /* serving: dl_submit -> admission to the GPU (host clock), ms */
    double ms_latency;       /* serving: dl_submit -> completion (host clock), ms */
    int32_t sweep_launches;  /* bit-sweep kernels (AUTO path: Iteration steps and the final E M) */
    double ms_sweep;         /* their summed device time (CUDA events on the launching stream) */
    double sweep_bytes;      /* bytes every one of those sweeps must read at least: the CSR of E
                                and each row of the bit matrix once */
} dl_stats;

/* Create a context on CUDA device `device` (cfg may be NULL for defaults).  Fails with
 * DL_EDEVICE unless the device is compute capability 10.3 (GB300). */
DL_API dl_status dl_create(dl_ctx **out, int device, const dl_config *cfg);

/* Wait for outstanding work, free every device buffer of the context, free the context.  Every
 * program created on the context must be destroyed first (dl_program_destroy uses its context). */
DL_API dl_status dl_destroy(dl_ctx *ctx);

/* Message for the last failed call on this thread ("" if none).  Valid until the next call
 * on this thread. */
DL_API const char *dl_last_error(void);

/* Run subsequent synchronous calls on `stream` (a cudaStream_t of the context's device;
 * NULL = the context's own stream). */
DL_API dl_status dl_set_stream(dl_ctx *ctx, void *stream);

/*
 * Transitive closure, the program of Sec. 3 (eq. prog:trcl):
 *     r2(x,z) <- r1(x,z).     r2(x,z) <- r1(x,y), r2(y,z).
 * E: the n x n 0/1 matrix of r1.  Output: the least model of r2, i.e. the least solution
 * of R2 = min1(E + E R2) (eq. matrixeq:trcl), as bits (n * ceil(n/64) words).
 *
 * eps <= 0 selects eps = 1/(1 + ||E||_inf) (Sec. 4 after Prop. 1; Sec. 7.1); otherwise
 * 0 < eps <= 1/(1 + ||E||_inf) is required (Lemma 1), else DL_EINVAL.  The model does not
 * depend on eps (Theorem 1).
 * thr must be 0 (the threshold "> 0" of Theorem 1); other values return DL_EINVAL.
 * out_rtilde (optional, n*n doubles, NULL allowed): the real least solution
 * R~ = (I - eps E)^-1 eps E (Prop. 1); only the FP64 and mixed paths produce it (with
 * DL_PATH_BOOL_FP8 or DL_PATH_AUTO a non-NULL out_rtilde returns DL_EINVAL).  DL_PATH_MIXED
 * refines R~ (max|R| <= refine_tol * eps) only when out_rtilde is given; for the model alone it
 * stops after the solve, since X > 0 is already exact wherever X is positive (A is an M-matrix and
 * the factorisation keeps every sign) and the certificate and recheck settle entries lost to
 * underflow (stats: iters = 0, final_resid = -1).
 * stats (optional): filled on DL_OK.
 */
DL_API dl_status dl_tc_closure(dl_ctx *ctx, int32_t n, const uint8_t *E, dl_mem mem, double eps,
                        double thr, dl_path path, uint64_t *out_bits, double *out_rtilde,
                        dl_stats *stats);

/*
 * The same closure with E given bit-packed, in the layout of the output: row r of E is the
 * ceil(n/64) 64-bit words at E_bits + r * ceil(n/64), and bit (j mod 64) of word j/64 (least
 * significant bit first) is E[r][j].  mem says where E_bits and out_bits live (both host or
 * both device); the caller owns both.  A set bit at a column >= n in the last word of a row
 * returns DL_EINVAL.  eps, thr, path, out_rtilde and stats as for dl_tc_closure; the model is
 * the same as dl_tc_closure's on the unpacked bytes.  DL_PATH_AUTO reads the bits as they
 * are; the other paths expand them to bytes on the device first.  (The paper's base relations
 * are 0/1 matrices (Sec. 3); the packed form is this library's, an eighth of the bytes to
 * move.)
 */
DL_API dl_status dl_tc_closure_bits(dl_ctx *ctx, int32_t n, const uint64_t *E_bits, dl_mem mem, double eps,
                             double thr, dl_path path, uint64_t *out_bits, double *out_rtilde,
                             dl_stats *stats);

/*
 * Same generation, the right-hand program of Sec. 7.2 (Fig. "Tested programs"):
 *     sg(x,w) <- b(x,w).     sg(x,w) <- p(x,y), sg(y,z), p(w,z).
 * i.e. the least solution of S = min1(B + P S P^T) (two-sided class, Sec. 6.3;
 * Sec. 7.2 with B = I).  P: n x n 0/1; B: n x n 0/1, or NULL for the identity
 * (the paper's diag facts).  eps <= 0 selects 1/(1 + ||P||_inf^2) (Sec. 7.2; reported
 * only, the model does not depend on it); thr must be 0.  Only DL_PATH_BOOL_FP8 and
 * DL_PATH_AUTO exist (others: DL_ENOTIMPL).  Output: bits of S.
 */
DL_API dl_status dl_sg_least_model(dl_ctx *ctx, int32_t n, const uint8_t *P, const uint8_t *B,
                            dl_mem mem, double eps, double thr, dl_path path,
                            uint64_t *out_bits, dl_stats *stats);

/*
 * One equation of the tail recursive class (Sec. 6.1, eq. matrixeq:trec), the generalisation
 * of transitive closure to clauses r(x,z) <- s_1(x,y_1), ..., s_n(y_{n-1},z) and
 * r(x,z) <- s_1(x,y_1), ..., s_n(y_{n-1},y), t(y,z):
 *     R~ = eps (A + B0 R~),   R~ = (I - eps B0)^-1 eps A,
 * with the equation's non-recursive part A = A_1 + B_1 R_{j_1} + ... + B_q R_{j_q} already
 * formed from the lower equations (their models combined with dl_compose: the model depends
 * only on which entries are positive).  B0, A: n x n 0/1.  out_bits (required): the model, the
 * least R with R = min1(A + B0 R), i.e. min1((I + B0^+) A) with B0^+ the transitive closure.
 * eps <= 0 selects 1/(1 + ||B0||_inf) (inside the paper's uniqueness condition eps < 1/||B0||);
 * otherwise 0 < eps <= that value, else DL_EINVAL.  thr must be 0.  Paths: DL_PATH_AUTO and
 * DL_PATH_BOOL_FP8 give the model (the closure of B0 by that path, then one FP8 boolean
 * product); DL_PATH_FP64 and DL_PATH_MIXED also give R~ in out_rtilde (n x n doubles, optional)
 * by the closure's real paths with the right-hand side eps A, and report in rows_rechecked the
 * model entries that X > 0 missed (underflow; X > 0 never holds outside the model).
 * A = B0 = E is the closure program (dl_tc_closure).
 */
DL_API dl_status dl_tail_recursive(dl_ctx *ctx, int32_t n, const uint8_t *B0, const uint8_t *A, dl_mem mem,
                            double eps, double thr, dl_path path, uint64_t *out_bits, double *out_rtilde,
                            dl_stats *stats);

/*
 * One equation of the tail recursive class with the real solutions of the lower equations it
 * refers to (Sec. 6.1, eq. matrixeq:trec):
 *     R~ = eps (A1 + B0 R~ + B_1 R~_{j_1} + ... + B_q R~_{j_q}),
 *     R~ = (I - eps B0)^-1 eps F,   F = A1 + sum_k B_k R~_{j_k}.
 * B0, A1: n x n 0/1 or NULL (zero).  B[k] (n x n 0/1) and R[k] (n x n doubles, row-major: the
 * real solution of lower equation j_k) for k < nterms.  All inputs and outputs live in `mem`.
 * eps <= 0 selects 1/(1 + max_i (rowsum(B0)_i + sum_k rowsum(B_k)_i)), which makes
 * eps F[1,...,1] <= 1 (the condition of Theorem 2, with every R~_{j_k} <= 1) and eps < 1/||B0||
 * (the uniqueness condition of Sec. 6.1); a larger eps returns DL_EINVAL.
 * out_bits (required): the model, the least R with R = min1(A' + B0 R) where A' = [F > 0] is what
 * the lower models contribute (R~_{j_k} > 0 exactly on the lower models, Theorem 2; real values
 * that underflowed to 0 in the caller's R[k] would drop facts here: dl_tail_system forms A' from the
 * lower models instead).  out_rtilde (optional, n x n doubles): R~, by the closure's real
 * paths with the real right-hand side F: DL_PATH_FP64 (blocked LU in FP64) or DL_PATH_MIXED (TF32
 * LU, FP64 refinement; DL_PATH_AUTO takes it when out_rtilde is not NULL).  DL_PATH_BOOL_FP8: the
 * model only.  stats->rows_rechecked: model entries that R~ > 0 missed (underflow).
 */
DL_API dl_status dl_tail_recursive_real(dl_ctx *ctx, int32_t n, const uint8_t *B0, const uint8_t *A1, int32_t nterms,
                                        const uint8_t *const *B, const double *const *R, dl_mem mem, double eps,
                                        dl_path path, uint64_t *out_bits, double *out_rtilde, dl_stats *stats);

/* One equation of a layered tail recursive system (dl_tail_system). */
typedef struct {
    const uint8_t *A1;          /* n x n 0/1, or NULL */
    const uint8_t *B0;          /* n x n 0/1 coefficient of the equation's own R~, or NULL */
    int32_t nterms;             /* terms B_k R~_{j_k} of lower equations */
    const uint8_t *const *B;    /* nterms n x n 0/1 matrices */
    const int32_t *j;           /* nterms indices of lower equations: 0 <= j[k] < this equation's index */
    double eps;                 /* <= 0: the default of dl_tail_recursive_real */
} dl_tail_eq;

/*
 * A system of m tail recursive equations over the same n constants, solved in order
 * (Sec. 6.1: a solution is substituted into the equations above it, M solves in all):
 *     R~_h = eps_h (A1_h + B0_h R~_h + sum_k B_{h,k} R~_{j_{h,k}}),   j_{h,k} < h.
 * Equation h is what the clauses of one predicate r_h give when every predicate its clauses
 * read is defined in a lower layer or is r_h itself in the rightmost position.
 * out_bits[h] (required, n * ceil(n/64) words each): the model of equation h, always from the
 * lower models: A1_h + sum_k B_{h,k} R_{j_{h,k}} by FP8 products, then the equation's boolean
 * route (exact whatever the precision of R~).  out_rtilde (NULL, or m pointers each NULL or n x n
 * doubles): R~_h, on DL_PATH_FP64 or DL_PATH_MIXED; those paths keep every R~_h on the device for
 * the equations above it.  DL_PATH_AUTO / DL_PATH_BOOL_FP8 give the models only.  All matrices live in `mem`.  stats: sums over the equations (eps_used: the last
 * one's).
 */
DL_API dl_status dl_tail_system(dl_ctx *ctx, int32_t n, int32_t m, const dl_tail_eq *eqs, dl_mem mem, dl_path path,
                                uint64_t *const *out_bits, double *const *out_rtilde, dl_stats *stats);

/*
 * The real least solution of the same-generation equation (Sec. 7.2; the two-sided class of
 * Sec. 6.3, a discrete Stein/Sylvester equation):
 *     S~ = eps (B + P S~ P^T),
 * whose positive entries are the least model of sg (Theorem 2).  P: n x n 0/1; B: n x n 0/1,
 * or NULL for the identity.  eps <= 0 selects 1/(1 + ||P||_inf^2) (Sec. 7.2); otherwise
 * 0 < eps <= that bound is required (it makes eps ||P^T kron P||_inf < 1, the condition of
 * Sec. 6.3 for a unique solution), else DL_EINVAL.  out_stilde: n x n doubles, row-major
 * (required).  out_bits (optional, NULL allowed): the model, S~ > 0 made exact by the
 * boolean iteration (n * ceil(n/64) words).  mem: where P, B and both outputs live.
 * Paths: DL_PATH_FP64 -- the fixpoint series X <- eps (B + P X P^T) in FP64 until a step
 * changes nothing beyond refine_tol * eps (exact after depth + 1 steps when P is nilpotent);
 * DL_PATH_MIXED -- Smith's doubling on the TF32 tensor cores with FP64 refinement (device
 * workspace about (2K + 4) np^2 FP32 matrices, K the doubling steps, np = n rounded up to 256);
 * DL_PATH_AUTO -- the series, then the refinement if 64 steps did not converge.
 * DL_PATH_BOOL_FP8: DL_EINVAL (no real values).  n is limited to 29000 (a row of S~ in one
 * block's shared memory); DL_ENOTCONV if the series or the refinement does not converge.
 * stats: iters = series steps + refinement steps, final_resid = max|eps (B + P S P^T) - S|/eps
 * (after the series: a power-of-two bound on the last step's largest change, 0 if it changed
 * nothing),
 * path_used = DL_PATH_FP64 when the series alone sufficed, else DL_PATH_MIXED.
 */
DL_API dl_status dl_sg_real(dl_ctx *ctx, int32_t n, const uint8_t *P, const uint8_t *B, dl_mem mem, double eps,
                     dl_path path, double *out_stilde, uint64_t *out_bits, dl_stats *stats);

/*
 * The transposed class (Sec. 6.2), its program prog:2:
 *     r2(x,z) <- r1(x,z).     r2(x,z) <- r1(x,y), r2(z,y).
 * The recursive atom's arguments are interchanged, so the completion is R2 = min1(R1 + R1 R2^T)
 * and its linearisation R~2 = eps (R1 + R1 R~2^T) (eq. matrixeq:trans:1), with
 * 0 < eps <= 1/(1 + ||R1||_inf) (eps <= 0 selects that bound; a larger eps returns DL_EINVAL).
 * R1: n x n 0/1.  out_bits (required): the least model of r2.  The model is computed through
 * the paper's reduction to a two-sided equation (eq. matrixeq:trans:2):
 * R2 = min1(B + R1 R2 R1^T) with B = min1(R1 + R1 R1^T) (one FP8 tensor-core product), solved as
 * dl_sg_least_model does (boolean doubling or the Iteration on bits).
 * out_rtilde (optional, n x n doubles): the real least solution R~2, by the increasing series
 * X_{t+1} = eps (R1 + R1 X_t^T) from 0 in FP64 until a step changes no entry by more than
 * refine_tol * eps (DL_ENOTCONV after 100000 steps); stats->guard_flagged counts the 64-bit bit
 * words where R~2 > 0 differs from the model (nonzero only under FP64 underflow).
 * Paths: DL_PATH_AUTO (model; R~2 if out_rtilde is not NULL), DL_PATH_FP64 (model and the series,
 * out_rtilde optional), DL_PATH_BOOL_FP8 (model only: a non-NULL out_rtilde returns DL_EINVAL);
 * DL_PATH_MIXED returns DL_ENOTIMPL.  thr must be 0.
 * stats: eps_used, iters (series steps, or the model's steps), final_resid (a power-of-two bound
 * on the last step's largest change / eps), model_ones.
 */
DL_API dl_status dl_transposed(dl_ctx *ctx, int32_t n, const uint8_t *R1, dl_mem mem, double eps, double thr,
                               dl_path path, uint64_t *out_bits, double *out_rtilde, dl_stats *stats);

/*
 * Relational composition, the denotation of an existential join (Sec. 2,
 * eq. denote:quant):  [[exists y r1(x,y) and r2(y,z)]] = min1(R1 R2).
 * R1, R2: n x n 0/1.  Output: bits of min1(R1 R2).  Runs on the FP8 tensor-core path.
 */
DL_API dl_status dl_compose(dl_ctx *ctx, int32_t n, const uint8_t *R1, const uint8_t *R2,
                     dl_mem mem, uint64_t *out_bits, dl_stats *stats);

/* ---- autotuning ----------------------------------------------------------------------- */

/*
 * Measure, for problems of size n on this context's GPU, the choices the solvers otherwise take
 * from fixed rules, and keep them for n's size bucket (n rounded up to a power of two, at least
 * 256; measured up to 16384): the FP8 squaring's tile width (128 or 256) and its time per
 * squaring, the bytes per second of an unsaturated Iteration sweep (the AUTO path's cost model
 * between sweeps and squarings), the SMs the mixed path's LU leaves to its critical chain (16, 32
 * or 48) and how many of its steps go in units of 2 or 4 sharing one bulk update, and whether same
 * generation on AUTO takes the Iteration on bits or the doubling (when one is faster on both a
 * random forest and a heavy-tailed DAG; sg_iteration -1: the fixed size rule).  The sweep rate is
 * the faster of an ER digraph's and a heavy-tailed DAG's.  The inputs are synthetic (generated
 * on the device).  Every choice leaves every model exact; only
 * speed depends on it.  flags: 1 = measure again even if the bucket is known (from this context
 * or the cache).  report (cap bytes, may be NULL when cap is 0; *len gets the full length): JSON
 * {"key", "bucket", "source": "measured" | "cache" | "defaults ...", "entry": {sq_bn, t_sq_us,
 * sweep_gbs, mx_reserve, mx_pairs, mx_group, sg_iteration}}.  With a cache path (dl_config.tune_cache or
 * DL_TUNE_CACHE) the entry is written there, keyed by GPU name, driver version and bucket.
 * Takes from milliseconds (small buckets) to about a second (16384).
 */
DL_API dl_status dl_autotune(dl_ctx *ctx, int32_t n, int32_t flags, char *report, size_t cap, size_t *len);

/* ---- linear programs (the class C_lin of Sec. 5) ---------------------------------- */

/*
 * A Datalog program over binary predicates, evaluated layer by layer (Sec. 5).
 *
 * Text: clauses  head(X,Y) :- atom, ..., atom.  Variables start with an upper-case letter or
 * '_'; every predicate is binary; "not p(X,Y)" negates an atom; "%" starts a comment to the end
 * of the line; there are no facts or constants in the text (base relations come in through
 * dl_program_set).  The program must be in C_lin (Sec. 5):
 *   - every body is a chain between the head's two (different) variables: its atoms link
 *     X = x0, x1, ..., xk = Y in order, each atom in either argument order, no variable repeated;
 *   - linear: no body holds two atoms whose predicates lie in the head's strongly connected
 *     component of the dependency graph (Tarjan's algorithm);
 *   - a negated atom names a predicate of a lower layer or a base relation (stratified
 *     negation, Sec. 8: its matrix is 1 - R, over all n x n pairs).
 * Otherwise DL_EINVAL, with the reason and the clause in dl_last_error().
 *
 * Evaluation (dl_program_run): the SCCs in topological order are the layers; in each, a chain
 * is the FP8 tensor-core product of its atoms' matrices (transposed where an atom's arguments
 * are reversed), and the layer's equations R_h = min1(A_h + sum_q B_q R_{j_q}^o C_q)
 * (eq. matrixeq:gen0) go to the first solver that fits:
 *   - no recursive atom: the union of the products;
 *   - every recursive atom rightmost (C = I) and not reversed: the tail recursive class
 *     (Sec. 6.1), one equation by dl_tail_recursive's boolean route, several mutually recursive
 *     ones by the closure of their stacked system over m n constants;
 *   - every recursive atom leftmost (B = I), not reversed: the same on the transposes;
 *   - one predicate whose recursive atoms are all reversed with C = I (or all with B = I): the
 *     transposed class (Sec. 6.2) by the two-sided reduction, on the same-generation solver;
 *   - one predicate, one recursive clause B R B^T: the same-generation solver (Sec. 6.3, 7.2);
 *   - anything else: the series of Lemma 3, R^(k+1) = min1(F[R^(k)]) from 0, on FP8 products
 *     until it stops changing.
 * Every route gives the least model (exact, 0/1).
 */
typedef struct dl_program dl_program;

/* Parse and check `text` (a NUL-terminated string) into a program bound to ctx.  The context
   must outlive the program. */
DL_API dl_status dl_program_create(dl_ctx *ctx, const char *text, dl_program **out);
/* Free a program (NULL is a no-op); its context must still exist. */
DL_API dl_status dl_program_destroy(dl_program *prog);
/* Give base relation `pred` the n x n 0/1 matrix R (row-major bytes, in `mem`); the bytes are
   copied.  Every base relation of a program must have the same n (n >= 0).  DL_EINVAL if pred
   is not a base relation of the program or n differs from an earlier call's; a byte other than
   0/1 is reported by dl_program_run. */
DL_API dl_status dl_program_set(dl_program *prog, const char *pred, int32_t n, const uint8_t *R, dl_mem mem);
/* Evaluate every layer; DL_EINVAL if a base relation is unset or holds a byte other than 0/1.
   stats: iters = layers, gpu_launches / gemm_launches / ms_total summed over the solvers
   (ms_total: device time of the solver calls). */
DL_API dl_status dl_program_run(dl_program *prog, dl_stats *stats);
/* The least model of defined predicate `pred` after dl_program_run: n * ceil(n/64) words,
   row-major, bit (j mod 64) of word j / 64 of row i = [pred(i, j)], in `mem`. */
DL_API dl_status dl_program_get(dl_program *prog, const char *pred, uint64_t *out_bits, dl_mem mem);
/* A text account of the program: "base: ..." and "defined: ..." lines, one "layer k: ..." line
   per layer in evaluation order, and after a run "plan:" with the route each layer took.  Writes
   at most cap bytes (NUL-terminated when cap > 0) into buf (NULL allowed when cap is 0) and the
   full length without the NUL into *len (if not NULL). */
DL_API dl_status dl_program_describe(const dl_program *prog, char *buf, size_t cap, size_t *len);

/*
 * Batch of independent transitive-closure problems of uneven size, each with the model
 * dl_tc_closure gives (eps <= 0, thr = 0; the program of Sec. 3).  ns[k], Es[k], out_bits[k]
 * describe problem k; all live in `mem`.  Every problem follows the DL_PATH_AUTO scheme:
 * one packing pass over all inputs builds one CSR over all problems' rows (one host read
 * sizes it), then a captured CUDA graph runs problems of at most 1024 padded rows to their
 * fixpoint in shared memory (one CTA each), batched in-place Iteration sweeps (Sec. 7.1) over
 * the rows of every problem still changing, and rounds of one persistent grouped FP8
 * tensor-core squaring launch over exactly the problems still active, each followed by more
 * sweeps; a problem leaves the active lists when a sweep changes nothing, and its model and
 * certificate are written then.  A second captured graph with further rounds runs only if a
 * problem is still active after the first.  Every decision is taken on the device.
 * stats (optional, one for the whole batch): iters = squaring rounds launched.
 */
DL_API dl_status dl_tc_batch(dl_ctx *ctx, int32_t count, const int32_t *ns, const uint8_t *const *Es,
                      dl_mem mem, uint64_t *const *out_bits, dl_stats *stats);

/* ---- asynchronous serving (continuous batching) ------------------------------------ */

typedef struct {
    int32_t kind;            /* 0 = transitive closure, 1 = same generation */
    int32_t n;
    const uint8_t *base;     /* E (closure) or P (same generation), n*n bytes */
    const uint8_t *B;        /* same generation only: base relation or NULL (identity) */
    dl_mem mem;              /* where base, B and out_bits live */
    dl_path path;            /* DL_PATH_AUTO or DL_PATH_BOOL_FP8 */
    uint64_t *out_bits;      /* n * ceil(n/64) words */
} dl_request;

/* Queue a request.  The caller keeps base, B and out_bits alive until dl_poll returns
 * DL_OK or an error for it, or dl_cancel succeeds.  The request is admitted to the GPU
 * when a slot and its HBM footprint (n^2 bytes per dense operand plus workspace) are free;
 * DL_ENOMEM if it can never fit the budget. *ticket receives its id. */
DL_API dl_status dl_submit(dl_ctx *ctx, const dl_request *req, uint64_t *ticket);

/* Wait up to timeout_us microseconds (0 = just test, <0 = forever) for a request.
 * DL_EBUSY while it is queued or running; on completion returns its final status once
 * (later polls of the same ticket return DL_EINVAL).  stats may be NULL. */
DL_API dl_status dl_poll(dl_ctx *ctx, uint64_t ticket, int64_t timeout_us, dl_stats *stats);

/* Cancel a request that has not been admitted yet: DL_OK if cancelled (its ticket then
 * polls DL_ECANCELED), DL_EBUSY if it is already running or done. */
DL_API dl_status dl_cancel(dl_ctx *ctx, uint64_t ticket);

/*
 * Self-test of the device-side failure detection: launches one CTA that waits, through the
 * same bounded mbarrier wait every tcgen05 kernel of the library uses, on a barrier that no
 * thread ever arrives at.  The wait gives up after `seconds` (0 < seconds <= 10), the kernel
 * records the expiry in the context's status word and returns, and the call reports
 * DL_ETIMEOUT; the context stays usable.  Anything else (DL_OK, a hang) means the detection
 * is broken.  The paper has no counterpart.
 */
DL_API dl_status dl_selftest_wait_timeout(dl_ctx *ctx, double seconds);

/* ---- closure without device allocation ------------------------------------------- */

/* Largest n that dl_tc_closure_noalloc accepts. */
#define DL_NOALLOC_MAX_N 2048

/*
 * Transitive closure (as dl_tc_closure with eps <= 0, thr = 0, DL_PATH_BOOL_FP8) for callers
 * that cannot allocate device memory: it calls no cudaMalloc, cudaFree or other allocating
 * routine and needs no context.  The paper has no counterpart; it exists for callers whose
 * device memory is owned by someone else (another framework's pool, a host application
 * that forbids library allocations) or that cannot afford the device synchronisation a
 * cudaMalloc implies.
 *
 * E (n*n bytes, 0/1) and out_bits (n * ceil(n/64) words) are device pointers on the current
 * device; stream is a cudaStream_t (NULL = the legacy default stream); *squarings (may be
 * NULL) receives the number of tensor-core squarings.  n > DL_NOALLOC_MAX_N returns
 * DL_EINVAL.  The call is synchronous: it returns after its work on `stream` has finished,
 * and it must not be called while `stream` (or the legacy stream, under global capture mode)
 * is being captured into a CUDA graph.  A device-side wait that expires returns DL_ETIMEOUT.
 *
 * Its scratch is one fixed array (about 9 MiB) compiled into the library; every call looks up
 * its device address (cudaGetSymbolAddress) with the current device.  CUDA loads device code
 * lazily by default, so the array and the kernels this call launches are placed on a device
 * (a driver allocation) the first time they are needed there.  A caller that must allocate
 * nothing later makes one call with n = 0 on each device first (E and out_bits may be NULL):
 * it places the array and loads those kernels and writes nothing; with
 * CUDA_MODULE_LOADING=EAGER the driver does this when the library is loaded, and the array is
 * then held by every GPU that loads the library until the process exits.  All calls on a
 * device share the array and it keeps the previous call's contents (each call clears what it
 * needs zeroed); calls whose work overlaps on the GPU race on it and must be serialised by the
 * caller.
 */
DL_API dl_status dl_tc_closure_noalloc(int32_t n, const uint8_t *E, uint64_t *out_bits,
                                       void *stream, int32_t *squarings);

#ifdef __cplusplus
}
#endif
#endif /* DL_H */
