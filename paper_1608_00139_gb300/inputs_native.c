/*
 * inputs_native.c -- the preferential-attachment generator of inputs.pa_dag in C, for streams
 * that draw a fresh graph per request (the Python loop takes about 0.3 s at N = 16384).
 *
 * It makes the same draws in the same order as inputs.pa_dag and so writes the same matrix:
 * SplitMix64 as a counter-based generator (draw c of key k is mix64(k + (c + 1) GAMMA), a uniform
 * is (draw >> 11) 2^-53); node i >= 1 draws its out-degree k from the Zipf CDF the caller passes
 * (the first index whose CDF value exceeds the uniform, plus one), clipped to kmax and to i, and
 * then picks k distinct earlier nodes from an urn in which node j appears in_degree(j) + 1 times
 * (urn index floor(u m), m the urn's size, redrawn on a repeat); the chosen nodes go into the urn
 * in increasing order, followed by i.  No arithmetic of the evaluation method lives here.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double uniform(uint64_t key, uint64_t c)
{
    return (double)(mix64(key + (c + 1) * 0x9E3779B97F4A7C15ull) >> 11) * 0x1.0p-53;
}

static int cmp_i32(const void *a, const void *b)
{
    const int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/*
 * e: n rows of lde >= n bytes (the n x n block is overwritten; 1 at (i, j) for each edge).
 * key: the stream key of (seed, STREAM_PA); cdf: kmax doubles.  Returns 0, or -1 on bad
 * arguments, -2 when out of host memory.
 */
int inputs_pa_dag(int32_t n, uint64_t key, const double *cdf, int64_t kmax, uint8_t *e, int64_t lde)
{
    if (n < 0 || (n > 0 && (!e || lde < n)) || kmax < 1 || !cdf) return -1;
    for (int64_t r = 0; r < n; r++) memset(e + r * lde, 0, (size_t)n);
    if (n <= 1) return 0;
    int64_t cap = 8 * (int64_t)n + 16, len = 1;
    int32_t *urn = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *chosen = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!urn || !mark || !chosen) {
        free(urn); free(mark); free(chosen);
        return -2;
    }
    for (int32_t j = 0; j < n; j++) mark[j] = -1;
    urn[0] = 0;
    uint64_t c = 0;
    for (int32_t i = 1; i < n; i++) {
        const double u = uniform(key, c++);
        int64_t lo = 0, hi = kmax;  /* first index with cdf > u */
        while (lo < hi) {
            const int64_t mid = (lo + hi) / 2;
            if (cdf[mid] > u) hi = mid; else lo = mid + 1;
        }
        int64_t k = lo + 1;
        if (k > kmax) k = kmax;
        if (k > i) k = i;
        int32_t cnt = 0;
        if (k == i) {
            for (int32_t j = 0; j < i; j++) chosen[cnt++] = j;
        } else {
            while (cnt < k) {
                const int64_t m = len;
                int64_t idx = (int64_t)(uniform(key, c++) * (double)m);
                if (idx > m - 1) idx = m - 1;
                const int32_t j = urn[idx];
                if (mark[j] != i) {
                    mark[j] = i;
                    chosen[cnt++] = j;
                }
            }
            qsort(chosen, (size_t)cnt, sizeof(int32_t), cmp_i32);
        }
        if (len + cnt + 1 > cap) {
            int64_t ncap = 2 * cap + cnt + 1;
            int32_t *g = (int32_t *)realloc(urn, sizeof(int32_t) * (size_t)ncap);
            if (!g) {
                free(urn); free(mark); free(chosen);
                return -2;
            }
            urn = g;
            cap = ncap;
        }
        uint8_t *row = e + (int64_t)i * lde;
        for (int32_t q = 0; q < cnt; q++) {
            row[chosen[q]] = 1;
            urn[len++] = chosen[q];
        }
        urn[len++] = i;
    }
    free(urn); free(mark); free(chosen);
    return 0;
}
