/*
 * Seeded synthetic input generators for the Boolean closure workloads.
 *
 * This file holds no part of the closure method: it only draws graphs and
 * query sets. Both the CPU oracle and the CUDA path are fed from here.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used counter-based:
 *   draw(key, c) = mix64(key + (c + 1) * 0x9E3779B97F4A7C15)
 * where mix64 is the SplitMix64 finaliser. A key is derived from
 * (seed, stream tag) with the same finaliser, so every generator and every
 * stream inside it is independent and reproducible.
 *
 * Determinism: the Erdos-Renyi generator uses only integer arithmetic plus
 * one correctly rounded division, so its graphs are bit-identical on every
 * IEEE-754 host. The Zipf tables use pow(), whose last-ulp rounding may
 * differ between C libraries; those graphs are reproducible per platform.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t draw(uint64_t key, uint64_t c) { return mix64(key + (c + 1) * GOLDEN); }

uint64_t wl_key(uint64_t seed, uint64_t tag) { return mix64(mix64(seed * GOLDEN + 0x632BE59BD9B4E019ULL) ^ (tag * 0xD1B54A32D192ED03ULL)); }

uint64_t wl_draw(uint64_t key, uint64_t c) { return draw(key, c); }

/* uniform integer in [0, m) from a 64-bit draw (multiply-high, bias < m / 2^64) */
static inline uint64_t below(uint64_t r, uint64_t m) { return (uint64_t)(((__uint128_t)r * (__uint128_t)m) >> 64); }

/* 53-bit integer threshold so that P[(draw >> 11) < thr] = p exactly up to 2^-53 */
static inline uint64_t thr53(double p) {
    if (p <= 0.0) return 0;
    if (p >= 1.0) return 1ULL << 53;
    return (uint64_t)(p * 9007199254740992.0); /* exact scaling by 2^53, truncation */
}

/* ---------------------------------------------------------------- ER -- */
/* Directed Erdos-Renyi: each ordered pair (i, j), i != j, is an edge with
 * probability p, decided by draw(key, i*n + j). Pass 1 counts per row. */
void wl_er_count(int64_t n, double p, uint64_t seed, int64_t* row_counts) {
    uint64_t key = wl_key(seed, 1), t = thr53(p);
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = 0;
        for (int64_t j = 0; j < n; ++j)
            if (j != i && (draw(key, (uint64_t)(i * n + j)) >> 11) < t) ++c;
        row_counts[i] = c;
    }
}

/* Pass 2 fills column indices into indices[indptr[i] .. indptr[i+1]). */
void wl_er_fill(int64_t n, double p, uint64_t seed, const int64_t* indptr, int32_t* indices) {
    uint64_t key = wl_key(seed, 1), t = thr53(p);
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int64_t o = indptr[i];
        for (int64_t j = 0; j < n; ++j)
            if (j != i && (draw(key, (uint64_t)(i * n + j)) >> 11) < t) indices[o++] = (int32_t)j;
    }
}

/* ------------------------------------------------------- Zipf tables -- */
/* cdf[k-1] = sum_{x=1..k} x^-alpha, k = 1..kmax */
static double* zipf_cdf(int64_t kmax, double alpha) {
    double* cdf = (double*)malloc(sizeof(double) * (size_t)kmax);
    double acc = 0.0;
    for (int64_t k = 1; k <= kmax; ++k) { acc += pow((double)k, -alpha); cdf[k - 1] = acc; }
    return cdf;
}

/* exact inverse CDF: smallest k with cdf[k-1] >= u * total */
static int64_t zipf_pick(const double* cdf, int64_t kmax, uint64_t r) {
    double u = (double)(r >> 11) * (1.0 / 9007199254740992.0);
    double target = u * cdf[kmax - 1];
    int64_t lo = 0, hi = kmax - 1;
    while (lo < hi) { int64_t mid = (lo + hi) / 2; if (cdf[mid] >= target) hi = mid; else lo = mid + 1; }
    return lo + 1;
}

/* ------------------------------------------------------ power law -- */
/* Out-degree k_i ~ Zipf(alpha) truncated to 1..kmax (and to n-1); targets by
 * preferential attachment on in-degree, P(j) proportional to in_j + 1, with an
 * urn that starts with every node once and gains a copy of j per edge into j.
 * Sources are taken in index order. Self-loops and duplicate targets in a row
 * are redrawn (at most 64 times, then the edge is dropped).
 * Returns nnz; indptr has n+1 entries; indices must hold n*min(kmax,n-1). */
int64_t wl_powerlaw(int64_t n, double alpha, int64_t kmax, uint64_t seed, int64_t* indptr, int32_t* indices) {
    if (kmax > n - 1) kmax = n - 1;
    indptr[0] = 0;
    if (n <= 1 || kmax < 1) { for (int64_t i = 0; i < n; ++i) indptr[i + 1] = 0; return 0; }
    double* cdf = zipf_cdf(kmax, alpha);
    uint64_t kdeg = wl_key(seed, 2), ktgt = wl_key(seed, 3);
    int64_t cap = n + n * kmax;
    int32_t* urn = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
    int64_t ulen = n;
    for (int64_t i = 0; i < n; ++i) urn[i] = (int32_t)i;
    uint64_t ctr = 0;
    int64_t nnz = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = zipf_pick(cdf, kmax, draw(kdeg, (uint64_t)i));
        int64_t row0 = nnz;
        for (int64_t e = 0; e < k; ++e) {
            for (int attempt = 0; attempt < 64; ++attempt) {
                int32_t j = urn[below(draw(ktgt, ctr++), (uint64_t)ulen)];
                if (j == i) continue;
                int dup = 0;
                for (int64_t x = row0; x < nnz; ++x) if (indices[x] == j) { dup = 1; break; }
                if (dup) continue;
                indices[nnz++] = j;
                urn[ulen++] = j;
                break;
            }
        }
        /* keep each row sorted */
        for (int64_t a = row0 + 1; a < nnz; ++a) {
            int32_t v = indices[a]; int64_t b = a - 1;
            while (b >= row0 && indices[b] > v) { indices[b + 1] = indices[b]; --b; }
            indices[b + 1] = v;
        }
        indptr[i + 1] = nnz;
    }
    free(urn); free(cdf);
    return nnz;
}

/* --------------------------------------------------------- queries -- */
/* q query rows; row r holds c_r ~ U[cmin, cmax] distinct uniform sources,
 * written LSB-first as packed uint64 rows of ld words (ld >= ceil(n/64)). */
void wl_query_rows(int64_t n, int64_t q, int64_t cmin, int64_t cmax, uint64_t seed, int64_t ld, uint64_t* rows) {
    uint64_t kc = wl_key(seed, 4), ks = wl_key(seed, 5);
    memset(rows, 0, sizeof(uint64_t) * (size_t)(q * ld));
    for (int64_t r = 0; r < q; ++r) {
        int64_t c = cmin + (int64_t)below(draw(kc, (uint64_t)r), (uint64_t)(cmax - cmin + 1));
        if (c > n) c = n;
        uint64_t* row = rows + r * ld;
        uint64_t ctr = (uint64_t)r << 20;
        int64_t got = 0;
        while (got < c) {
            int64_t s = (int64_t)below(draw(ks, ctr++), (uint64_t)n);
            uint64_t bit = 1ULL << (s & 63);
            if (row[s >> 6] & bit) continue;
            row[s >> 6] |= bit;
            ++got;
        }
    }
}

/* -------------------------------------------------- knowledge graph -- */
/* T draws of (head, relation, tail): relation rank ~ Zipf(alpha_r) over
 * 1..n_rel, head and tail uniform over n_ent with head != tail. Duplicates are
 * kept here and removed by the caller. */
void wl_kg_triples(int64_t n_ent, int64_t n_rel, int64_t T, double alpha_r, uint64_t seed,
                   int32_t* h, int32_t* r, int32_t* t) {
    double* cdf = zipf_cdf(n_rel, alpha_r);
    uint64_t kr = wl_key(seed, 6), kh = wl_key(seed, 7), kt = wl_key(seed, 8);
    for (int64_t x = 0; x < T; ++x) {
        r[x] = (int32_t)(zipf_pick(cdf, n_rel, draw(kr, (uint64_t)x)) - 1);
        int64_t hh = (int64_t)below(draw(kh, (uint64_t)x), (uint64_t)n_ent);
        uint64_t c = (uint64_t)x << 8;
        int64_t tt;
        do { tt = (int64_t)below(draw(kt, c++), (uint64_t)n_ent); } while (tt == hh && n_ent > 1);
        h[x] = (int32_t)hh; t[x] = (int32_t)tt;
    }
    free(cdf);
}

/* ----------------------------------------------------------- SBM --- */
/* Stochastic block model with nb equal blocks (block of i = i*nb/n): pair
 * (i, j), i != j, is an edge with probability p_in inside a block and p_out
 * across blocks. Same two-pass contract as the ER generator. */
void wl_sbm_count(int64_t n, int64_t nb, double p_in, double p_out, uint64_t seed, int64_t* row_counts) {
    uint64_t key = wl_key(seed, 9), ti = thr53(p_in), to = thr53(p_out);
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = 0, bi = i * nb / n;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            uint64_t t = (j * nb / n == bi) ? ti : to;
            if ((draw(key, (uint64_t)(i * n + j)) >> 11) < t) ++c;
        }
        row_counts[i] = c;
    }
}

void wl_sbm_fill(int64_t n, int64_t nb, double p_in, double p_out, uint64_t seed, const int64_t* indptr, int32_t* indices) {
    uint64_t key = wl_key(seed, 9), ti = thr53(p_in), to = thr53(p_out);
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int64_t o = indptr[i], bi = i * nb / n;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            uint64_t t = (j * nb / n == bi) ? ti : to;
            if ((draw(key, (uint64_t)(i * n + j)) >> 11) < t) indices[o++] = (int32_t)j;
        }
    }
}

/* --------------------------------------------- sparse skip sampling -- */
/* Bernoulli(p) trials over columns [lo, hi) of row i, by geometric gaps
 * (number of failures before a success = floor(log U / log(1 - p))), in
 * O(successes). Uses log(), so graphs are reproducible per platform only;
 * meant for large corpora. Writes at most cap columns (self-loop skipped). */
static int64_t skip_row(int64_t i, int64_t lo, int64_t hi, double p, uint64_t key, uint64_t* ctr, int32_t* out,
                        int64_t cap) {
    int64_t c = 0;
    if (p <= 0.0 || hi <= lo) return 0;
    if (p >= 1.0) {
        for (int64_t j = lo; j < hi && c < cap; ++j)
            if (j != i) { if (out) out[c] = (int32_t)j; ++c; }
        return c;
    }
    const double lq = log1p(-p);
    int64_t j = lo - 1;
    for (;;) {
        double u = ((double)(draw(key, (*ctr)++) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        double g = floor(log(u) / lq);
        if (g > (double)(hi - j)) break;
        j += (int64_t)g + 1;
        if (j >= hi) break;
        if (j == i) continue;
        if (c >= cap) break;
        if (out) out[c] = (int32_t)j;
        ++c;
    }
    return c;
}

/* Sparse directed ER / SBM in O(n + m): block of i = i*nb/n, probability
 * p_in inside a block and p_out across (nb = 1: plain ER). Two passes as the
 * dense generators; both passes draw the same numbers (per-row streams). */
static int64_t sbm_row(int64_t n, int64_t nb, double p_in, double p_out, uint64_t key, int64_t i, int32_t* out,
                       int64_t cap) {
    uint64_t ctr = (uint64_t)i << 32;
    int64_t bi = i * nb / n;
    int64_t b0 = (bi * n + nb - 1) / nb, b1 = ((bi + 1) * n + nb - 1) / nb; /* columns of block bi */
    int64_t c = 0;
    c += skip_row(i, 0, b0, p_out, key, &ctr, out ? out + c : 0, cap - c);
    c += skip_row(i, b0, b1, p_in, key, &ctr, out ? out + c : 0, cap - c);
    c += skip_row(i, b1, n, p_out, key, &ctr, out ? out + c : 0, cap - c);
    return c;
}

void wl_sbm_sparse_count(int64_t n, int64_t nb, double p_in, double p_out, uint64_t seed, int64_t* row_counts) {
    uint64_t key = wl_key(seed, 13);
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) row_counts[i] = sbm_row(n, nb, p_in, p_out, key, i, 0, n);
}

void wl_sbm_sparse_fill(int64_t n, int64_t nb, double p_in, double p_out, uint64_t seed, const int64_t* indptr,
                        int32_t* indices) {
    uint64_t key = wl_key(seed, 13);
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) sbm_row(n, nb, p_in, p_out, key, i, indices + indptr[i], indptr[i + 1] - indptr[i]);
}

/* CSR -> packed LSB-first rows of ld words (layout change only). */
void wl_csr_to_packed(int64_t n, const int64_t* indptr, const int32_t* indices, int64_t ld, uint64_t* rows) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        uint64_t* r = rows + i * ld;
        memset(r, 0, sizeof(uint64_t) * (size_t)ld);
        for (int64_t e = indptr[i]; e < indptr[i + 1]; ++e) r[indices[e] >> 6] |= 1ULL << (indices[e] & 63);
    }
}

/* uniform random pairs (i, j), i != j, count m: used for shortcut edges */
void wl_random_pairs(int64_t n, int64_t m, uint64_t seed, int32_t* src, int32_t* dst) {
    uint64_t ka = wl_key(seed, 10), kb = wl_key(seed, 11);
    for (int64_t x = 0; x < m; ++x) {
        int64_t a = (int64_t)below(draw(ka, (uint64_t)x), (uint64_t)n);
        uint64_t c = (uint64_t)x << 8;
        int64_t b;
        do { b = (int64_t)below(draw(kb, c++), (uint64_t)n); } while (b == a && n > 1);
        src[x] = (int32_t)a; dst[x] = (int32_t)b;
    }
}
