/*
 * oracle.c -- plain, slow, CPU reference for the least models of Sato, "A Linear Algebraic
 * Approach to Datalog Evaluation" (TPLP).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check of the package entry
 * file and the CPU-baseline leg of the benchmark load this library.  The CUDA library
 * shares no code, header, table or helper with it, and never calls it.
 *
 * What it computes (each function cites the passage it follows):
 *   - the least Herbrand model of the transitive-closure program (Sec. 3, eq. prog:trcl)
 *     and of the same-generation program (Sec. 7.2, Fig. "Tested programs", right), by
 *     symbolic semi-naive bottom-up evaluation of the T_DB fixpoint (Sec. 2) on bitsets;
 *   - the real solution R~ = (I - eps E)^-1 eps E of the linearised equation
 *     (Sec. 4, eq. matrixeq:trcl:epsilon; Proposition 1) by an FP64 LU factorisation and
 *     two triangular solves with N right-hand sides;
 *   - one column of R~ by the monotone series of Lemma 1 (eq. series:trcl:epsilon),
 *     for sampled checks at sizes where the full LU is too slow;
 *   - the paper's "Iteration" method (Sec. 7.1, eq. series:trcl) on 0/1 matrices.
 *
 * Layouts: matrices are dense row-major, n*n entries; E[i*n+j] = 1 iff r1(e_i, e_j)
 * (Sec. 2 adjacency encoding).  Bit matrices hold ceil(n/64) uint64 words per row, bit
 * (j mod 64) of word floor(j/64), least significant bit first.
 *
 * Return codes: 0 ok, -1 bad argument, -2 out of memory, -3 zero pivot, -4 not converged.
 * OpenMP parallelises the outer row loops only (the CPU baseline uses all host cores).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define WORDS(n) (((int64_t)(n) + 63) / 64)

int oracle_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
    return omp_get_max_threads();
#else
    (void)t;
    return 1;
#endif
}

/* ||A||_inf = max_i sum_j |a_ij| (Sec. 2): for a 0/1 matrix, the maximum out-degree. */
int64_t oracle_max_row_sum(int32_t n, const uint8_t *a)
{
    int64_t best = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t s = 0;
        for (int64_t j = 0; j < n; j++) s += a[i * n + j] ? 1 : 0;
        if (s > best) best = s;
    }
    return best;
}

/* eps = 1 / (1 + ||E||_inf): the largest value Lemma 1 allows, the one the paper uses
 * (Sec. 4 after Proposition 1; Sec. 7.1 "Matrix"). */
double oracle_tc_eps(int32_t n, const uint8_t *e)
{
    return 1.0 / (1.0 + (double)oracle_max_row_sum(n, e));
}

/* eps = 1 / (1 + ||P||_inf^2) for the same-generation equation (Sec. 7.2). */
double oracle_sg_eps(int32_t n, const uint8_t *p)
{
    double d = (double)oracle_max_row_sum(n, p);
    return 1.0 / (1.0 + d * d);
}

/* Successor lists of a dense 0/1 matrix (row i -> columns j with a[i][j] = 1). */
static int build_rows(int32_t n, const uint8_t *a, int64_t **ptr_out, int32_t **idx_out)
{
    int64_t *ptr = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!ptr) return -2;
    ptr[0] = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t c = 0;
        for (int64_t j = 0; j < n; j++) c += a[i * n + j] ? 1 : 0;
        ptr[i + 1] = ptr[i] + c;
    }
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ptr[n] > 0 ? ptr[n] : 1));
    if (!idx) { free(ptr); return -2; }
    for (int64_t i = 0; i < n; i++) {
        int64_t k = ptr[i];
        for (int64_t j = 0; j < n; j++)
            if (a[i * n + j]) idx[k++] = (int32_t)j;
    }
    *ptr_out = ptr;
    *idx_out = idx;
    return 0;
}

/*
 * Least model of  r2(x,z) <- r1(x,z);  r2(x,z) <- r1(x,y), r2(y,z)  (eq. prog:trcl),
 * by semi-naive evaluation of the T_DB fixpoint (Sec. 2):
 *   R_0 = D_0 = E;   D_{k+1}[x] = ( OR_{y : E[x][y]} D_k[y] ) minus R_k[x];
 *   R_{k+1} = R_k OR D_{k+1};   stop when D_{k+1} is empty.
 * D_{k+1} holds exactly the facts first derivable with one more application of the
 * recursive clause, so the loop computes I^infinity restricted to r2.
 * R: n * ceil(n/64) words (output).  *iters (may be NULL): number of D steps taken.
 */
int oracle_tc_seminaive(int32_t n, const uint8_t *e, uint64_t *r, int32_t *iters)
{
    if (n < 0 || (n > 0 && (!e || !r))) return -1;
    if (iters) *iters = 0;
    if (n == 0) return 0;
    const int64_t w = WORDS(n);
    int64_t *ptr;
    int32_t *idx;
    if (build_rows(n, e, &ptr, &idx)) return -2;
    uint64_t *delta = (uint64_t *)calloc((size_t)(n * w), 8);
    uint64_t *next = (uint64_t *)calloc((size_t)(n * w), 8);
    if (!delta || !next) { free(delta); free(next); free(ptr); free(idx); return -2; }
    memset(r, 0, (size_t)(n * w) * 8);
    for (int64_t i = 0; i < n; i++)
        for (int64_t k = ptr[i]; k < ptr[i + 1]; k++) {
            int64_t j = idx[k];
            r[i * w + j / 64] |= 1ull << (j % 64);
        }
    memcpy(delta, r, (size_t)(n * w) * 8);
    int32_t steps = 0;
    for (;;) {
        uint64_t any = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(| : any)
        for (int64_t x = 0; x < n; x++) {
            uint64_t *nx = next + x * w;
            memset(nx, 0, (size_t)w * 8);
            for (int64_t k = ptr[x]; k < ptr[x + 1]; k++) {
                const uint64_t *dy = delta + (int64_t)idx[k] * w;
                for (int64_t q = 0; q < w; q++) nx[q] |= dy[q];
            }
            for (int64_t q = 0; q < w; q++) {
                nx[q] &= ~r[x * w + q];
                any |= nx[q];
            }
        }
        if (!any) break;
        for (int64_t q = 0; q < n * w; q++) r[q] |= next[q];
        uint64_t *t = delta; delta = next; next = t;
        steps++;
    }
    if (iters) *iters = steps;
    free(delta); free(next); free(ptr); free(idx);
    return 0;
}

/*
 * The paper's "Iteration" method (Sec. 7.1; eq. series:trcl): R^(0) = 0,
 * R^(k+1) = min1(R1 + R1 R^(k)) on 0/1 matrices, until R^(k+1) = R^(k).
 * R: n*n bytes (output, 0/1).  Cost O(n^3) per step; for small n only.
 */
int oracle_tc_naive(int32_t n, const uint8_t *e, uint8_t *r, int32_t *iters)
{
    if (n < 0 || (n > 0 && (!e || !r))) return -1;
    if (iters) *iters = 0;
    if (n == 0) return 0;
    uint8_t *nx = (uint8_t *)malloc((size_t)n * n);
    if (!nx) return -2;
    memset(r, 0, (size_t)n * n);
    int32_t steps = 0;
    for (;;) {
        int changed = 0;
#pragma omp parallel for reduction(| : changed)
        for (int64_t i = 0; i < n; i++)
            for (int64_t j = 0; j < n; j++) {
                int64_t s = e[i * n + j] ? 1 : 0;
                for (int64_t m = 0; m < n && s == 0; m++)
                    s += (e[i * n + m] && r[m * n + j]) ? 1 : 0;
                uint8_t v = s >= 1 ? 1 : 0; /* min1 */
                nx[i * n + j] = v;
                changed |= (v != r[i * n + j]);
            }
        steps++;
        memcpy(r, nx, (size_t)n * n);
        if (!changed) break;
    }
    if (iters) *iters = steps;
    free(nx);
    return 0;
}

/*
 * R~ = (I - eps E)^-1 eps E  (Proposition 1), in FP64.
 * A = I - eps E is strictly diagonally dominant by rows when 0 < eps <= 1/(1+||E||_inf)
 * (proof of Proposition 1), so Gaussian elimination needs no pivoting: A = L U with L unit
 * lower triangular.  Then L Y = eps E (forward) and U X = Y (backward), column block by
 * column block.  X: n*n doubles (output, row-major).
 */
int oracle_tc_rtilde_lu(int32_t n, const uint8_t *e, double eps, double *x)
{
    if (n < 0 || (n > 0 && (!e || !x)) || !(eps > 0.0)) return -1;
    if (n == 0) return 0;
    const int64_t nn = n;
    double *a = (double *)malloc(sizeof(double) * (size_t)(nn * nn));
    if (!a) return -2;
    for (int64_t i = 0; i < nn; i++)
        for (int64_t j = 0; j < nn; j++) {
            double ev = e[i * nn + j] ? eps : 0.0;
            a[i * nn + j] = (i == j ? 1.0 : 0.0) - ev;
            x[i * nn + j] = ev;
        }
    /* A = L U, Doolittle, in place. */
    for (int64_t k = 0; k < nn; k++) {
        const double piv = a[k * nn + k];
        if (piv == 0.0) { free(a); return -3; }
#pragma omp parallel for schedule(static)
        for (int64_t i = k + 1; i < nn; i++) {
            double l = a[i * nn + k] / piv;
            a[i * nn + k] = l;
            if (l != 0.0)
                for (int64_t j = k + 1; j < nn; j++) a[i * nn + j] -= l * a[k * nn + j];
        }
    }
    /* Forward substitution L Y = eps E and backward U X = Y; columns are independent, so
     * threads split the columns. */
    const int64_t cb = 64;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c0 = 0; c0 < nn; c0 += cb) {
        const int64_t c1 = c0 + cb < nn ? c0 + cb : nn;
        for (int64_t i = 0; i < nn; i++)
            for (int64_t k = 0; k < i; k++) {
                const double l = a[i * nn + k];
                if (l != 0.0)
                    for (int64_t j = c0; j < c1; j++) x[i * nn + j] -= l * x[k * nn + j];
            }
        for (int64_t i = nn - 1; i >= 0; i--) {
            for (int64_t k = i + 1; k < nn; k++) {
                const double u = a[i * nn + k];
                if (u != 0.0)
                    for (int64_t j = c0; j < c1; j++) x[i * nn + j] -= u * x[k * nn + j];
            }
            const double d = a[i * nn + i];
            for (int64_t j = c0; j < c1; j++) x[i * nn + j] /= d;
        }
    }
    free(a);
    return 0;
}

/*
 * Column j of R~ by the series of Lemma 1 (eq. series:trcl:epsilon) restricted to one
 * column:  x^(0) = 0,  x^(k+1) = eps (E e_j + E x^(k)).
 * The sequence increases monotonically to the least solution (Lemma 1), which is column j
 * of (I - eps E)^-1 eps E (Proposition 1).  The loop stops when an update changes no
 * component (the FP64 fixed point) or after max_iter updates (returns -4).
 * xcol: n doubles (output).  *iters (may be NULL): updates taken.
 */
int oracle_tc_rtilde_series_col(int32_t n, const uint8_t *e, double eps, int32_t j,
                                double *xcol, int32_t max_iter, int32_t *iters)
{
    if (n < 0 || (n > 0 && (!e || !xcol)) || j < 0 || (n > 0 && j >= n) || !(eps > 0.0))
        return -1;
    if (iters) *iters = 0;
    if (n == 0) return 0;
    int64_t *ptr;
    int32_t *idx;
    if (build_rows(n, e, &ptr, &idx)) return -2;
    double *nx = (double *)malloc(sizeof(double) * (size_t)n);
    if (!nx) { free(ptr); free(idx); return -2; }
    for (int64_t i = 0; i < n; i++) xcol[i] = 0.0;
    int rc = -4;
    int32_t k;
    for (k = 0; k < max_iter; k++) {
        int changed = 0;
#pragma omp parallel for schedule(static) reduction(| : changed)
        for (int64_t i = 0; i < n; i++) {
            double s = e[(int64_t)i * n + j] ? 1.0 : 0.0;
            for (int64_t q = ptr[i]; q < ptr[i + 1]; q++) s += xcol[idx[q]];
            double v = eps * s;
            nx[i] = v;
            changed |= (v != xcol[i]);
        }
        memcpy(xcol, nx, sizeof(double) * (size_t)n);
        if (!changed) { rc = 0; k++; break; }
    }
    if (iters) *iters = k;
    free(nx); free(ptr); free(idx);
    return rc;
}

/*
 * Row i of R~ by the same series read along rows.  R~ = sum_{m >= 1} (eps E)^m, and the right
 * form of the equation, R~ = eps E + eps R~ E, has the same partial sums as Lemma 1's series,
 * so row i follows  x^(0) = 0,  x^(k+1) = eps (e_i^T E + x^(k) E):
 *     x^(k+1)[j] = eps (E[i][j] + sum_{q : E[q][j]} x^(k)[q]).
 * It increases monotonically to row i of (I - eps E)^-1 eps E.  Stops as the column series
 * does (no component changed; -4 after max_iter updates).  xrow: n doubles (output).
 */
int oracle_tc_rtilde_series_row(int32_t n, const uint8_t *e, double eps, int32_t i,
                                double *xrow, int32_t max_iter, int32_t *iters)
{
    if (n < 0 || (n > 0 && (!e || !xrow)) || i < 0 || (n > 0 && i >= n) || !(eps > 0.0))
        return -1;
    if (iters) *iters = 0;
    if (n == 0) return 0;
    /* predecessor lists: pred[pptr[j] .. pptr[j+1]) = {q : E[q][j]} */
    int64_t *pptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!pptr) return -2;
    for (int64_t q = 0; q < n; q++)
        for (int64_t j = 0; j < n; j++)
            if (e[q * n + j]) pptr[j + 1]++;
    for (int64_t j = 0; j < n; j++) pptr[j + 1] += pptr[j];
    int32_t *pred = (int32_t *)malloc(sizeof(int32_t) * (size_t)(pptr[n] > 0 ? pptr[n] : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    double *nx = (double *)malloc(sizeof(double) * (size_t)n);
    if (!pred || !fill || !nx) { free(pptr); free(pred); free(fill); free(nx); return -2; }
    for (int64_t j = 0; j < n; j++) fill[j] = pptr[j];
    for (int64_t q = 0; q < n; q++)
        for (int64_t j = 0; j < n; j++)
            if (e[q * n + j]) pred[fill[j]++] = (int32_t)q;
    for (int64_t j = 0; j < n; j++) xrow[j] = 0.0;
    int rc = -4;
    int32_t k;
    for (k = 0; k < max_iter; k++) {
        int changed = 0;
#pragma omp parallel for schedule(static) reduction(| : changed)
        for (int64_t j = 0; j < n; j++) {
            double s = e[(int64_t)i * n + j] ? 1.0 : 0.0;
            for (int64_t q = pptr[j]; q < pptr[j + 1]; q++) s += xrow[pred[q]];
            double v = eps * s;
            nx[j] = v;
            changed |= (v != xrow[j]);
        }
        memcpy(xrow, nx, sizeof(double) * (size_t)n);
        if (!changed) { rc = 0; k++; break; }
    }
    if (iters) *iters = k;
    free(nx); free(fill); free(pred); free(pptr);
    return rc;
}

/*
 * Least model of the same-generation program (Sec. 7.2, Fig. "Tested programs", right):
 *   sg(x,w) <- b(x,w);   sg(x,w) <- p(x,y), sg(y,z), p(w,z)
 * i.e. the least S with S = min1(B + P S P^T) (eq. matrixeq:two-sided:3 with B = I).
 * Semi-naive evaluation of the T_DB fixpoint (Sec. 2):
 *   S_0 = D_0 = B;  D_{k+1} = {(x,w) : P[x][y], D_k[y][z], P[w][z]} minus S_k;
 *   S_{k+1} = S_k OR D_{k+1};  stop when D_{k+1} is empty.
 * Evaluated row-wise:  T[y] = OR_{z in D_k[y]} C[z]  with C[z] = {w : P[w][z]},
 *                      D_{k+1}[x] = (OR_{y : P[x][y]} T[y]) minus S_k[x].
 * b may be NULL: then B = I (the diag(x,x) facts of the paper's program).
 * S: n * ceil(n/64) words (output).
 */
int oracle_sg_seminaive(int32_t n, const uint8_t *p, const uint8_t *b, uint64_t *s,
                        int32_t *iters)
{
    if (n < 0 || (n > 0 && (!p || !s))) return -1;
    if (iters) *iters = 0;
    if (n == 0) return 0;
    const int64_t w = WORDS(n);
    int64_t *ptr;
    int32_t *idx;
    if (build_rows(n, p, &ptr, &idx)) return -2;
    uint64_t *col = (uint64_t *)calloc((size_t)(n * w), 8);   /* C[z] = {w : P[w][z]} */
    uint64_t *delta = (uint64_t *)calloc((size_t)(n * w), 8);
    uint64_t *next = (uint64_t *)calloc((size_t)(n * w), 8);
    uint64_t *t = (uint64_t *)calloc((size_t)(n * w), 8);
    if (!col || !delta || !next || !t) {
        free(col); free(delta); free(next); free(t); free(ptr); free(idx);
        return -2;
    }
    for (int64_t wi = 0; wi < n; wi++)
        for (int64_t q = ptr[wi]; q < ptr[wi + 1]; q++) {
            int64_t z = idx[q];
            col[z * w + wi / 64] |= 1ull << (wi % 64);
        }
    memset(s, 0, (size_t)(n * w) * 8);
    for (int64_t x = 0; x < n; x++)
        for (int64_t y = 0; y < n; y++) {
            int on = b ? (b[x * n + y] != 0) : (x == y);
            if (on) s[x * w + y / 64] |= 1ull << (y % 64);
        }
    memcpy(delta, s, (size_t)(n * w) * 8);
    int32_t steps = 0;
    for (;;) {
#pragma omp parallel for schedule(dynamic, 8)
        for (int64_t y = 0; y < n; y++) {
            uint64_t *ty = t + y * w;
            memset(ty, 0, (size_t)w * 8);
            const uint64_t *dy = delta + y * w;
            for (int64_t q = 0; q < w; q++) {
                uint64_t bits = dy[q];
                while (bits) {
                    int bit = __builtin_ctzll(bits);
                    bits &= bits - 1;
                    const uint64_t *cz = col + (q * 64 + bit) * w;
                    for (int64_t r2 = 0; r2 < w; r2++) ty[r2] |= cz[r2];
                }
            }
        }
        uint64_t any = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(| : any)
        for (int64_t x = 0; x < n; x++) {
            uint64_t *nx = next + x * w;
            memset(nx, 0, (size_t)w * 8);
            for (int64_t q = ptr[x]; q < ptr[x + 1]; q++) {
                const uint64_t *ty = t + (int64_t)idx[q] * w;
                for (int64_t r2 = 0; r2 < w; r2++) nx[r2] |= ty[r2];
            }
            for (int64_t r2 = 0; r2 < w; r2++) {
                nx[r2] &= ~s[x * w + r2];
                any |= nx[r2];
            }
        }
        if (!any) break;
        for (int64_t q = 0; q < n * w; q++) s[q] |= next[q];
        uint64_t *tmp = delta; delta = next; next = tmp;
        steps++;
    }
    if (iters) *iters = steps;
    free(col); free(delta); free(next); free(t); free(ptr); free(idx);
    return 0;
}
