/*
 * Seeded synthetic inputs for the column-row product workloads.
 *
 * This file produces input matrices only; it holds none of the product's
 * arithmetic (no hashing, no partitioning, no accumulation).  Both the CUDA
 * path and the CPU oracle consume the arrays it writes.
 *
 * Randomness: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC 2011), a counter-based generator, so every
 * transaction / column is drawn from its own counter block and the output is
 * independent of the thread count.
 *
 * Workload shapes (power-law item frequencies, short transactions, Poisson
 * lengths) stand in for the frequent-itemset and bag-of-words datasets of the
 * paper's case study (Section 6, Table 2).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Philox4x32-10                                                       */
/* ------------------------------------------------------------------ */
typedef struct { uint32_t v[4]; } ph_ctr;

static inline uint32_t mulhilo32(uint32_t a, uint32_t b, uint32_t *hi) {
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    return (uint32_t)p;
}

static inline ph_ctr philox4x32_10(ph_ctr c, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0, hi1;
        uint32_t lo0 = mulhilo32(M0, c.v[0], &hi0);
        uint32_t lo1 = mulhilo32(M1, c.v[2], &hi1);
        ph_ctr n;
        n.v[0] = hi1 ^ c.v[1] ^ k0;
        n.v[1] = lo1;
        n.v[2] = hi0 ^ c.v[3] ^ k1;
        n.v[3] = lo0;
        c = n;
        k0 += W0;
        k1 += W1;
    }
    return c;
}

/* A stream of uniform doubles in [0,1) addressed by (seed, stream, item). */
typedef struct {
    uint32_t k0, k1;
    ph_ctr ctr;
    uint32_t buf[4];
    int pos;
} ph_stream;

static void ph_init(ph_stream *s, uint64_t seed, uint32_t stream, uint64_t item) {
    s->k0 = (uint32_t)seed;
    s->k1 = (uint32_t)(seed >> 32);
    s->ctr.v[0] = 0;
    s->ctr.v[1] = stream;
    s->ctr.v[2] = (uint32_t)item;
    s->ctr.v[3] = (uint32_t)(item >> 32);
    s->pos = 4;
}

static inline uint32_t ph_u32(ph_stream *s) {
    if (s->pos == 4) {
        ph_ctr o = philox4x32_10(s->ctr, s->k0, s->k1);
        memcpy(s->buf, o.v, sizeof s->buf);
        s->ctr.v[0]++;
        s->pos = 0;
    }
    return s->buf[s->pos++];
}

static inline double ph_uniform(ph_stream *s) {
    uint64_t hi = ph_u32(s), lo = ph_u32(s);
    uint64_t x = (hi << 32) | lo;
    return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

/* Raw Philox block, exported so tests can check the generator alone. */
void crp_gen_philox_block(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                          uint32_t *out4) {
    ph_ctr c = {{c0, c1, c2, c3}};
    ph_ctr o = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    memcpy(out4, o.v, 4 * sizeof(uint32_t));
}

/* ------------------------------------------------------------------ */
/* Distributions                                                       */
/* ------------------------------------------------------------------ */

/* Poisson(lam) by sequential inverse transform; result clamped to [lo, hi]
 * when hi >= lo (hi < 0 means no clamp).  Truncation "to [a,b]" is read as a
 * clamp. */
static int64_t poisson_draw(ph_stream *s, double lam, int64_t lo, int64_t hi) {
    double u = ph_uniform(s);
    double p = exp(-lam), c = p;
    int64_t k = 0;
    while (u >= c && k < 100000) {
        ++k;
        p = p * lam / (double)k;
        c += p;
        if (p == 0.0 && (double)k > lam) break;
    }
    if (hi >= lo) {
        if (k < lo) k = lo;
        if (k > hi) k = hi;
    }
    return k;
}

/* Smallest r with cdf[r] > u (cdf strictly increasing to 1). */
static inline int32_t cdf_search(const double *cdf, int32_t n, double u) {
    int32_t lo = 0, hi = n - 1;
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (cdf[mid] > u) hi = mid; else lo = mid + 1;
    }
    return lo;
}

static double *zipf_cdf(int32_t n, double s) {
    double *cdf = (double *)malloc((size_t)n * sizeof(double));
    if (!cdf) return NULL;
    double acc = 0.0;
    for (int32_t r = 0; r < n; ++r) {
        acc += pow((double)(r + 1), -s);
        cdf[r] = acc;
    }
    for (int32_t r = 0; r < n; ++r) cdf[r] /= acc;
    cdf[n - 1] = 1.0;
    return cdf;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static void sort_small(int32_t *v, int64_t n) {
    if (n > 64) { qsort(v, (size_t)n, sizeof(int32_t), cmp_i32); return; }
    for (int64_t a = 1; a < n; ++a) {
        int32_t x = v[a];
        int64_t b = a - 1;
        while (b >= 0 && v[b] > x) { v[b + 1] = v[b]; --b; }
        v[b + 1] = x;
    }
}

/* Draw `len` distinct values into out[0..len) with `draw` and reject repeats.
 * Uses a small open-addressing set on the stack/heap. */
typedef struct { int32_t *slot; int64_t cap; } iset;

static int iset_insert(iset *st, int32_t x) {
    uint64_t h = ((uint64_t)(uint32_t)x * 0x9E3779B97F4A7C15ull) >> 20;
    int64_t m = st->cap - 1;
    for (int64_t p = (int64_t)(h & (uint64_t)m);; p = (p + 1) & m) {
        if (st->slot[p] == -1) { st->slot[p] = x; return 1; }
        if (st->slot[p] == x) return 0;
    }
}

/* ------------------------------------------------------------------ */
/* Transactions ({0,1} matrix T in CSR: rows = transactions)           */
/* ------------------------------------------------------------------ */

/* Lengths L_t ~ Poisson(lam) clamped to [lmin, lmax] (no clamp if lmax<lmin),
 * then capped at n (a transaction holds distinct items). */
int crp_gen_tx_lengths(uint64_t seed, int64_t m, int32_t n, double lam, int64_t lmin,
                       int64_t lmax, int64_t *len_out) {
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < m; ++t) {
        ph_stream s;
        ph_init(&s, seed, 0u, (uint64_t)t);
        int64_t L = poisson_draw(&s, lam, lmin, lmax);
        if (L > n) L = n;
        len_out[t] = L;
    }
    return 0;
}

/* Items of transaction t: Zipf(s) ranks over [n] (item id = rank - 1), drawn
 * by inverse CDF, repeats rejected until the row holds L_t distinct items;
 * each row is then sorted ascending. */
int crp_gen_tx_items(uint64_t seed, int64_t m, int32_t n, double zipf_s, const int64_t *rowptr,
                     int32_t *colidx) {
    double *cdf = zipf_cdf(n, zipf_s);
    if (!cdf) return 1;
    int err = 0;
#pragma omp parallel
    {
        int64_t cap = 256;
        int32_t *slots = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
#pragma omp for schedule(dynamic, 4096)
        for (int64_t t = 0; t < m; ++t) {
            int64_t b = rowptr[t], L = rowptr[t + 1] - b;
            if (L <= 0) continue;
            int64_t need = 4;
            while (need < 2 * L) need <<= 1;
            if (need > cap) {
                free(slots);
                cap = need;
                slots = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
            }
            if (!slots) { err = 1; continue; }
            iset st = {slots, need};
            for (int64_t q = 0; q < need; ++q) slots[q] = -1;
            ph_stream s;
            ph_init(&s, seed, 1u, (uint64_t)t);
            int64_t got = 0;
            while (got < L) {
                int32_t r = cdf_search(cdf, n, ph_uniform(&s));
                if (iset_insert(&st, r)) colidx[b + got++] = r;
            }
            sort_small(colidx + b, L);
        }
        free(slots);
    }
    free(cdf);
    return err;
}

/* ------------------------------------------------------------------ */
/* Column-stochastic real matrix (CSC), Markov-cluster expansion input  */
/* ------------------------------------------------------------------ */

/* Column nnz c_k from the discrete power law p(c) ~ c^-alpha on [cmin, cmax]. */
int crp_gen_powerlaw_counts(uint64_t seed, int64_t ncols, double alpha, int32_t cmin,
                            int32_t cmax, int64_t *cnt_out) {
    int32_t w = cmax - cmin + 1;
    double *cdf = (double *)malloc((size_t)w * sizeof(double));
    if (!cdf) return 1;
    double acc = 0.0;
    for (int32_t c = 0; c < w; ++c) { acc += pow((double)(cmin + c), -alpha); cdf[c] = acc; }
    for (int32_t c = 0; c < w; ++c) cdf[c] /= acc;
    cdf[w - 1] = 1.0;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < ncols; ++k) {
        ph_stream s;
        ph_init(&s, seed, 2u, (uint64_t)k);
        cnt_out[k] = cmin + cdf_search(cdf, w, ph_uniform(&s));
    }
    free(cdf);
    return 0;
}

/* Rows of column k uniform over [nrows] without replacement (sorted), values
 * lognormal(mu, sigma) drawn in fp64 (Box-Muller), normalised so the column
 * sums to 1 in fp64, stored as fp32. */
int crp_gen_stochastic_cols(uint64_t seed, int64_t ncols, int32_t nrows, double mu, double sigma,
                            const int64_t *colptr, int32_t *rowidx, float *val) {
    int err = 0;
#pragma omp parallel
    {
        int64_t cap = 256;
        int32_t *slots = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
        double *tmp = NULL;
        int64_t tcap = 0;
#pragma omp for schedule(dynamic, 256)
        for (int64_t k = 0; k < ncols; ++k) {
            int64_t b = colptr[k], L = colptr[k + 1] - b;
            if (L <= 0) continue;
            int64_t need = 4;
            while (need < 2 * L) need <<= 1;
            if (need > cap) {
                free(slots);
                cap = need;
                slots = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
            }
            if (L > tcap) {
                free(tmp);
                tcap = L;
                tmp = (double *)malloc((size_t)tcap * sizeof(double));
            }
            if (!slots || !tmp) { err = 1; continue; }
            iset st = {slots, need};
            for (int64_t q = 0; q < need; ++q) slots[q] = -1;
            ph_stream s;
            ph_init(&s, seed, 3u, (uint64_t)k);
            int64_t got = 0;
            while (got < L) {
                int32_t r = (int32_t)(ph_uniform(&s) * (double)nrows);
                if (r >= nrows) r = nrows - 1;
                if (iset_insert(&st, r)) rowidx[b + got++] = r;
            }
            sort_small(rowidx + b, L);
            ph_stream v;
            ph_init(&v, seed, 4u, (uint64_t)k);
            double sum = 0.0;
            for (int64_t q = 0; q < L; ++q) {
                double u1 = ph_uniform(&v), u2 = ph_uniform(&v);
                if (u1 <= 0.0) u1 = 1.0 / 9007199254740992.0;
                double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
                tmp[q] = exp(mu + sigma * z);
                sum += tmp[q];
            }
            for (int64_t q = 0; q < L; ++q) val[b + q] = (float)(tmp[q] / sum);
        }
        free(slots);
        free(tmp);
    }
    return err;
}

/* Transpose a compressed-sparse matrix: (ptr over `nmajor`, idx in [nminor])
 * -> (tptr over `nminor`, tidx in [nmajor]), values carried along (val may be
 * NULL).  Output minor indices come out sorted because the input is walked in
 * major order. */
int crp_gen_transpose(int64_t nmajor, int32_t nminor, const int64_t *ptr, const int32_t *idx,
                      const float *val, int64_t *tptr, int32_t *tidx, float *tval) {
    int64_t *fill = (int64_t *)calloc((size_t)nminor + 1, sizeof(int64_t));
    if (!fill) return 1;
    int64_t nnz = ptr[nmajor];
    for (int64_t q = 0; q < nnz; ++q) fill[idx[q] + 1]++;
    for (int32_t r = 0; r < nminor; ++r) fill[r + 1] += fill[r];
    memcpy(tptr, fill, ((size_t)nminor + 1) * sizeof(int64_t));
    for (int64_t k = 0; k < nmajor; ++k)
        for (int64_t q = ptr[k]; q < ptr[k + 1]; ++q) {
            int64_t d = fill[idx[q]]++;
            tidx[d] = (int32_t)k;
            if (val) tval[d] = val[q];
        }
    free(fill);
    return 0;
}

/* Uniform doubles and a Poisson draw for parameter sampling (batched
 * workload: per-problem sizes and exponents). */
double crp_gen_uniform(uint64_t seed, uint32_t stream, uint64_t item, int32_t which) {
    ph_stream s;
    ph_init(&s, seed, stream, item);
    double u = 0.0;
    for (int32_t q = 0; q <= which; ++q) u = ph_uniform(&s);
    return u;
}
