/*
 * CPU oracle for Boolean Matrix Logic Programming closures.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link or call
 * this file; it exists so that the tests, the smoke check and the benchmark's
 * CPU-baseline leg can check the CUDA library against an independent,
 * obviously correct definition. It shares no code with the CUDA library.
 *
 * What it computes (paper, Sec. 2 Eq. 1 and Sec. 3.3):
 *   R1+ = sum_{k>=1} R1^k   (Boolean sum = OR, Boolean product = OR of ANDs)
 * i.e. (R1+)_{ij} = 1 iff there is a directed path of length >= 1 from i to j.
 * The paper states (Sec. 3.3, correctness remark after Eq. 5) that BMLP-RMS
 * (Algorithm 1) and BMLP-SMP (Algorithm 2) reach exactly this closure, so the
 * oracle is that definition written out three independent ways:
 *   1. per-source breadth-first search from the successors of each source
 *      (rows of R1+; also the shortest-path depths that fix the number of
 *      squarings, Appendix C Prop. 1);
 *   2. semi-naive bottom-up evaluation of the linear program P2 of Sec. 3.3
 *      (r2 <- r1 ; r2 <- r1, r2) on sets of pairs, following Eq. 1;
 *   3. Warshall's triple loop (small n only).
 * Selective queries (Eq. 5): v* = v R1+, the union of the closure rows of the
 * sources. Composition (Sec. 3.4, Thm. 1) for p <- r1 ; p <- r2, p:
 *   P = (I + R2+) R1, evaluated by search and by semi-naive iteration.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

/* Threads of the parallel loops below (t <= 0: keep); returns the previous
 * setting. Used to time the oracle on one core and on all cores. */
int oracle_set_threads(int t) {
    const int prev = omp_get_max_threads();
    if (t > 0) omp_set_num_threads(t);
    return prev;
}

/* BFS over paths of length >= 1 from source s: dist[j] = shortest path
 * length s -> j (>= 1), -1 if j is not reached. The search starts at the
 * successors of s, so s is reached only if it lies on a cycle. queue holds
 * the reached nodes in BFS order; returns their count, *dmax the deepest. */
static int64_t bfs_from_successors(int64_t n, const int64_t* indptr, const int32_t* indices, int32_t s,
                                   int32_t* dist, int32_t* queue, int32_t* dmax_out) {
    for (int64_t j = 0; j < n; ++j) dist[j] = -1;
    int64_t head = 0, tail = 0;
    for (int64_t e = indptr[s]; e < indptr[s + 1]; ++e) {
        int32_t j = indices[e];
        if (dist[j] < 0) { dist[j] = 1; queue[tail++] = j; }
    }
    int32_t dmax = 0;
    while (head < tail) {
        int32_t u = queue[head++];
        if (dist[u] > dmax) dmax = dist[u];
        for (int64_t e = indptr[u]; e < indptr[u + 1]; ++e) {
            int32_t j = indices[e];
            if (dist[j] < 0) { dist[j] = dist[u] + 1; queue[tail++] = j; }
        }
    }
    *dmax_out = dmax;
    return tail;
}

/* Reach rows from a list of sources by BFS that starts at the successors of
 * each source (paths of length >= 1, so a source is in its own row only if
 * it lies on a cycle). For each requested source s:
 *   out[r*n + j] = 1 iff j is reachable from s = src[r] by >= 1 edge (if out)
 *   depth[r]     = max over reached j of the shortest path length s -> j,
 *                  0 if nothing is reached (if depth)
 *   count[r]     = number of reached j (if count)                         */
void oracle_reach_rows(int64_t n, const int64_t* indptr, const int32_t* indices,
                       const int32_t* src, int64_t nsrc,
                       uint8_t* out, int32_t* depth, int64_t* count) {
    #pragma omp parallel
    {
        int32_t* dist = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        #pragma omp for schedule(dynamic, 16)
        for (int64_t r = 0; r < nsrc; ++r) {
            int32_t dmax = 0;
            const int64_t reached = bfs_from_successors(n, indptr, indices, src[r], dist, queue, &dmax);
            if (out) {
                uint8_t* row = out + r * n;
                for (int64_t j = 0; j < n; ++j) row[j] = (uint8_t)(dist[j] > 0);
            }
            if (depth) depth[r] = dmax;
            if (count) count[r] = reached;
        }
        free(dist);
        free(queue);
    }
}

/* The same rows of R1+ as bit rows: bit j % 64 of word j / 64 of row r
 * (ldw words per row, least significant bit first) is 1 iff j is reachable
 * from src[r] by >= 1 edge; padding bits stay 0. Lets large closures be
 * compared word by word without an n x n byte matrix. */
void oracle_reach_rows_bits(int64_t n, const int64_t* indptr, const int32_t* indices,
                            const int32_t* src, int64_t nsrc, uint64_t* out, int64_t ldw) {
    #pragma omp parallel
    {
        int32_t* dist = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        #pragma omp for schedule(dynamic, 16)
        for (int64_t r = 0; r < nsrc; ++r) {
            int32_t dmax = 0;
            const int64_t reached = bfs_from_successors(n, indptr, indices, src[r], dist, queue, &dmax);
            uint64_t* row = out + r * ldw;
            memset(row, 0, sizeof(uint64_t) * (size_t)ldw);
            for (int64_t x = 0; x < reached; ++x) {
                const int32_t j = queue[x];
                row[j / 64] |= (uint64_t)1 << (j % 64);
            }
        }
        free(dist);
        free(queue);
    }
}

/* Selective query (Eq. 5, Algorithm 2): for query row q with source set S_q
 * (bit s of row q of the packed, LSB-first source matrix), out[q*n + j] = 1
 * iff j is reachable by >= 1 edge from some s in S_q. Multi-source BFS from
 * the successors of all sources. levels[q] = the deepest BFS level reached. */
void oracle_smp(int64_t n, const int64_t* indptr, const int32_t* indices,
                const uint64_t* src_rows, int64_t q, int64_t ld,
                uint8_t* out, int32_t* levels) {
    #pragma omp parallel
    {
        int32_t* dist = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        #pragma omp for schedule(dynamic, 4)
        for (int64_t r = 0; r < q; ++r) {
            const uint64_t* srow = src_rows + r * ld;
            for (int64_t j = 0; j < n; ++j) dist[j] = -1;
            int64_t head = 0, tail = 0;
            for (int64_t s = 0; s < n; ++s) {
                if (!((srow[s / 64] >> (s % 64)) & 1u)) continue;
                for (int64_t e = indptr[s]; e < indptr[s + 1]; ++e) {
                    int32_t j = indices[e];
                    if (dist[j] < 0) { dist[j] = 1; queue[tail++] = j; }
                }
            }
            int32_t dmax = 0;
            while (head < tail) {
                int32_t u = queue[head++];
                if (dist[u] > dmax) dmax = dist[u];
                for (int64_t e = indptr[u]; e < indptr[u + 1]; ++e) {
                    int32_t j = indices[e];
                    if (dist[j] < 0) { dist[j] = dist[u] + 1; queue[tail++] = j; }
                }
            }
            if (out) {
                uint8_t* row = out + r * n;
                for (int64_t j = 0; j < n; ++j) row[j] = (uint8_t)(dist[j] > 0);
            }
            if (levels) levels[r] = dmax;
        }
        free(dist);
        free(queue);
    }
}

/* Semi-naive evaluation of the linear program (Sec. 3.3 program P2, Eq. 1,
 * and its two-relation form of Sec. 3.4):
 *     p(X,Y) <- base(X,Y).
 *     p(X,Y) <- rec(X,Z), p(Z,Y).
 * on dense 0/1 relations (n x n bytes, nonzero = true):
 *     P = base; D = base;
 *     repeat: D' = { (x,y) : rec(x,z) and D(z,y) } \ P ; P = P u D' ; D = D'
 *     until D' is empty.
 * With base = rec = R1 this is the closure R1+; with base = R1, rec = R2 it
 * is the composition (I + R2+) R1. out receives P; the return value is the
 * number of rounds that derived new pairs (plus the final empty one). */
int32_t oracle_seminaive(int64_t n, const uint8_t* base, const uint8_t* rec, uint8_t* out) {
    size_t nn = (size_t)n * (size_t)n;
    uint8_t* D = (uint8_t*)malloc(nn ? nn : 1);
    uint8_t* Dn = (uint8_t*)malloc(nn ? nn : 1);
    for (size_t x = 0; x < nn; ++x) { out[x] = base[x] != 0; D[x] = out[x]; }
    int32_t rounds = 0;
    for (;;) {
        ++rounds;
        int64_t fresh = 0;
        #pragma omp parallel for schedule(dynamic, 8) reduction(+:fresh)
        for (int64_t x = 0; x < n; ++x) {
            uint8_t* dn = Dn + x * n;
            memset(dn, 0, (size_t)n);
            for (int64_t z = 0; z < n; ++z) {
                if (!rec[x * n + z]) continue;
                const uint8_t* dz = D + z * n;
                for (int64_t y = 0; y < n; ++y)
                    if (dz[y] && !out[x * n + y]) dn[y] = 1;
            }
            for (int64_t y = 0; y < n; ++y) fresh += dn[y];
        }
        if (fresh == 0) break;
        for (size_t x = 0; x < nn; ++x) out[x] |= Dn[x];
        uint8_t* t = D; D = Dn; Dn = t;
    }
    free(D);
    free(Dn);
    return rounds;
}

/* Warshall's algorithm: for k, for i with (i,k), row i |= row k. Leaves the
 * closure R1+ (paths of length >= 1) in out. O(n^3); for small n. */
void oracle_warshall(int64_t n, const uint8_t* in, uint8_t* out) {
    size_t nn = (size_t)n * (size_t)n;
    for (size_t x = 0; x < nn; ++x) out[x] = in[x] != 0;
    for (int64_t k = 0; k < n; ++k)
        for (int64_t i = 0; i < n; ++i)
            if (out[i * n + k])
                for (int64_t j = 0; j < n; ++j)
                    out[i * n + j] |= out[k * n + j];
}

/* Composition by search (Sec. 3.4, Thm. 1): p <- r1 ; p <- r2, p has the
 * least model P = (I + R2+) R1, i.e. P(i,j) = 1 iff some k with k = i or k
 * reachable from i through >= 1 r2 edge has r1(k, j). Rows rows[0..nr) of P
 * are written to out (nr x n). */
void oracle_compose_rows(int64_t n, const int64_t* ip1, const int32_t* ix1,
                         const int64_t* ip2, const int32_t* ix2,
                         const int32_t* rows, int64_t nr, uint8_t* out) {
    #pragma omp parallel
    {
        uint8_t* seen = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
        int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        #pragma omp for schedule(dynamic, 16)
        for (int64_t r = 0; r < nr; ++r) {
            int32_t i = rows[r];
            memset(seen, 0, (size_t)n);
            int64_t head = 0, tail = 0;
            seen[i] = 1; queue[tail++] = i;        /* k = i (the identity) */
            while (head < tail) {                  /* k reachable via r2   */
                int32_t u = queue[head++];
                for (int64_t e = ip2[u]; e < ip2[u + 1]; ++e) {
                    int32_t v = ix2[e];
                    if (!seen[v]) { seen[v] = 1; queue[tail++] = v; }
                }
            }
            uint8_t* row = out + r * n;
            memset(row, 0, (size_t)n);
            for (int64_t x = 0; x < tail; ++x) {
                int32_t k = queue[x];
                for (int64_t e = ip1[k]; e < ip1[k + 1]; ++e) row[ix1[e]] = 1;
            }
        }
        free(seen);
        free(queue);
    }
}
