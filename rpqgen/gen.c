/*
 * Seeded synthetic knowledge-graph generator (input preparation only).
 *
 * Produces the graph, edge labels, node keywords and keyword postings that
 * both the CPU oracle and the CUDA library consume.  Nothing here computes any
 * part of the search method: no edge weights, no activation levels, no
 * expansion.  The average-hops statistic used by the weighting scheme is an
 * input of the method (Section 3.1 and the dataset table of Section 5.1
 * estimate it by sampling node pairs); it is estimated here the same way.
 *
 * Every random draw is counter based (splitmix64 finaliser of a keyed
 * counter), so results do not depend on the number of OpenMP threads.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Counter-based generator: independent stream per (seed, stream id). */
static inline uint64_t crand(uint64_t seed, uint64_t stream, uint64_t i) {
    return mix64(mix64(seed ^ (stream * 0xD1B54A32D192ED03ull)) + i);
}

static inline double u01(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

enum { ST_RMAT = 1, ST_CL_SRC = 40, ST_CL_DST = 41, ST_PERM = 50, ST_LABEL = 60,
       ST_KWCOUNT = 70, ST_KWDRAW = 71, ST_ABAR = 80 };

/* ---------------------------------------------------------------- R-MAT -- */
/* Directed R-MAT edges (no noise): each of `scale` levels picks a quadrant. */
void gen_rmat_edges(int32_t scale, int64_t nedges, double a, double b, double c,
                    uint64_t seed, uint32_t *src, uint32_t *dst) {
    const double ab = a + b, abc = a + b + c;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nedges; ++i) {
        uint32_t u = 0, v = 0;
        for (int32_t k = 0; k < scale; ++k) {
            double r = u01(crand(seed, ST_RMAT + (uint64_t)k, (uint64_t)i));
            uint32_t bu, bv;
            if (r < a) { bu = 0; bv = 0; }
            else if (r < ab) { bu = 0; bv = 1; }
            else if (r < abc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        src[i] = u;
        dst[i] = v;
    }
}

/* ------------------------------------------------------------- Chung-Lu -- */
/* Endpoint sampling proportional to w_i = (i + i0)^(-1/(beta-1)), through a
 * Walker/Vose alias table (prob[n], alias[n]) built here. */
void gen_chunglu_alias(int64_t n, double beta, double i0, double *prob, uint32_t *alias) {
    const double ex = -1.0 / (beta - 1.0);
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) { prob[i] = pow((double)i + i0, ex); s += prob[i]; }
    uint32_t *small = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint32_t *large = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    int64_t ns = 0, nl = 0;
    for (int64_t i = 0; i < n; ++i) {
        prob[i] = prob[i] * (double)n / s;
        if (prob[i] < 1.0) small[ns++] = (uint32_t)i; else large[nl++] = (uint32_t)i;
    }
    while (ns > 0 && nl > 0) {
        uint32_t l = small[--ns], g = large[--nl];
        alias[l] = g;
        prob[g] = (prob[g] + prob[l]) - 1.0;
        if (prob[g] < 1.0) small[ns++] = g; else large[nl++] = g;
    }
    while (nl > 0) { uint32_t g = large[--nl]; prob[g] = 1.0; alias[g] = g; }
    while (ns > 0) { uint32_t l = small[--ns]; prob[l] = 1.0; alias[l] = l; }
    free(small); free(large);
}

static inline uint32_t alias_pick(const double *prob, const uint32_t *alias, int64_t n,
                                  uint64_t r1, uint64_t r2) {
    uint64_t i = r1 % (uint64_t)n;
    return u01(r2) < prob[i] ? (uint32_t)i : alias[i];
}

void gen_chunglu_edges(int64_t n, int64_t nedges, const double *prob, const uint32_t *alias,
                       uint64_t seed, uint32_t *src, uint32_t *dst) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nedges; ++i) {
        src[i] = alias_pick(prob, alias, n, crand(seed, ST_CL_SRC, 2 * (uint64_t)i),
                            crand(seed, ST_CL_SRC, 2 * (uint64_t)i + 1));
        dst[i] = alias_pick(prob, alias, n, crand(seed, ST_CL_DST, 2 * (uint64_t)i),
                            crand(seed, ST_CL_DST, 2 * (uint64_t)i + 1));
    }
}

/* Seeded node relabelling (Fisher-Yates over the counter generator), so that
 * degree is not correlated with node id. perm[old] = new. */
void gen_permutation(int64_t n, uint64_t seed, uint32_t *perm) {
    for (int64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)(crand(seed, ST_PERM, (uint64_t)i) % (uint64_t)(i + 1));
        uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

void gen_apply_permutation(int64_t m, const uint32_t *perm, uint32_t *x) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) x[i] = perm[x[i]];
}

/* ------------------------------------------------------------------ CSR -- */
static int cmp_u32(const void *x, const void *y) {
    uint32_t a = *(const uint32_t *)x, b = *(const uint32_t *)y;
    return (a > b) - (a < b);
}

/* Symmetrise the directed edge list, drop self-loops and duplicates and build
 * a CSR with ascending neighbour lists.  `col` must have room for 2*m
 * entries; row_ptr for n+1.  Returns the number of CSR entries kept. */
int64_t gen_build_csr(int64_t n, int64_t m, const uint32_t *src, const uint32_t *dst,
                      int64_t *row_ptr, uint32_t *col) {
    int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t i = 0; i < m; ++i) {
        if (src[i] == dst[i]) continue;
        deg[src[i]]++; deg[dst[i]]++;
    }
    int64_t *pos = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    pos[0] = 0;
    for (int64_t v = 0; v < n; ++v) pos[v + 1] = pos[v] + deg[v];
    memcpy(deg, pos, ((size_t)n + 1) * sizeof(int64_t));       /* deg = fill cursor */
    for (int64_t i = 0; i < m; ++i) {
        uint32_t u = src[i], v = dst[i];
        if (u == v) continue;
        col[deg[u]++] = v;
        col[deg[v]++] = u;
    }
    /* sort and dedupe each row in place; record new lengths */
    int64_t *len = deg;
    #pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t v = 0; v < n; ++v) {
        int64_t b = pos[v], e = pos[v + 1];
        if (e - b > 1) qsort(col + b, (size_t)(e - b), sizeof(uint32_t), cmp_u32);
        int64_t w = b;
        for (int64_t i = b; i < e; ++i)
            if (i == b || col[i] != col[i - 1]) col[w++] = col[i];
        len[v] = w - b;
    }
    /* compact */
    int64_t out = 0;
    row_ptr[0] = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t b = pos[v];
        if (out != b) memmove(col + out, col + b, (size_t)len[v] * sizeof(uint32_t));
        out += len[v];
        row_ptr[v + 1] = out;
    }
    free(pos); free(deg);
    return out;
}

/* --------------------------------------------------------------- labels -- */
static inline int64_t cdf_pick(const double *cdf, int64_t n, double u) {
    int64_t lo = 0, hi = n - 1;            /* smallest i with cdf[i] > u */
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (cdf[mid] > u) hi = mid; else lo = mid + 1;
    }
    return lo;
}

void gen_zipf_cdf(int64_t nvals, double s, double *cdf) {
    double acc = 0.0;
    for (int64_t r = 0; r < nvals; ++r) { acc += pow((double)(r + 1), -s); cdf[r] = acc; }
    for (int64_t r = 0; r < nvals; ++r) cdf[r] /= acc;
    cdf[nvals - 1] = 1.0;
}

/* One label per undirected edge, keyed by (min, max) so both CSR directions
 * carry the same label. */
void gen_edge_labels(int64_t n, const int64_t *row_ptr, const uint32_t *col,
                     const double *label_cdf, int64_t nlabels, uint64_t seed, uint16_t *label) {
    #pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            uint64_t v = col[e];
            uint64_t lo = (uint64_t)u < v ? (uint64_t)u : v, hi = (uint64_t)u < v ? v : (uint64_t)u;
            double r = u01(crand(seed, ST_LABEL, (lo << 32) | hi));
            label[e] = (uint16_t)cdf_pick(label_cdf, nlabels, r);
        }
    }
}

/* ------------------------------------------------------------- keywords -- */
/* Keyword count per node uniform in [kmin, kmax]; ids Zipf-distributed by
 * rank (id = rank - 1), distinct within a node. */
void gen_node_keyword_counts(int64_t n, int32_t kmin, int32_t kmax, uint64_t seed, int64_t *nk_ptr) {
    nk_ptr[0] = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t c = kmin + (int64_t)(crand(seed, ST_KWCOUNT, (uint64_t)v) % (uint64_t)(kmax - kmin + 1));
        nk_ptr[v + 1] = nk_ptr[v] + c;
    }
}

void gen_node_keywords(int64_t n, const int64_t *nk_ptr, const double *vocab_cdf, int64_t vocab,
                       uint64_t seed, int32_t *nk_ids) {
    #pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < n; ++v) {
        int64_t b = nk_ptr[v], e = nk_ptr[v + 1];
        uint64_t ctr = (uint64_t)v << 20;
        for (int64_t i = b; i < e; ++i) {
            for (;;) {
                int32_t id = (int32_t)cdf_pick(vocab_cdf, vocab, u01(crand(seed, ST_KWDRAW, ctr++)));
                int dup = 0;
                for (int64_t k = b; k < i; ++k) dup |= (nk_ids[k] == id);
                if (!dup) { nk_ids[i] = id; break; }
            }
        }
    }
}

/* Transpose node->keyword lists into keyword->node postings (ascending). */
void gen_postings(int64_t n, const int64_t *nk_ptr, const int32_t *nk_ids, int64_t vocab,
                  int64_t *kw_ptr, int32_t *kw_nodes) {
    memset(kw_ptr, 0, ((size_t)vocab + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < nk_ptr[n]; ++i) kw_ptr[nk_ids[i] + 1]++;
    for (int64_t k = 0; k < vocab; ++k) kw_ptr[k + 1] += kw_ptr[k];
    int64_t *cur = (int64_t *)malloc((size_t)vocab * sizeof(int64_t));
    memcpy(cur, kw_ptr, (size_t)vocab * sizeof(int64_t));
    for (int64_t v = 0; v < n; ++v)
        for (int64_t i = nk_ptr[v]; i < nk_ptr[v + 1]; ++i) kw_nodes[cur[nk_ids[i]]++] = (int32_t)v;
    free(cur);
}

/* ----------------------------------------------------------- average hops -- */
/* Mean unweighted hop distance from `nsrc` seeded sources (non-isolated nodes)
 * to every node they reach (source excluded).  Returns -1 if no pair. */
double gen_average_hops(int64_t n, const int64_t *row_ptr, const uint32_t *col,
                        int32_t nsrc, uint64_t seed) {
    double total = 0.0, pairs = 0.0;
    int64_t *srcs = (int64_t *)malloc((size_t)nsrc * sizeof(int64_t));
    int32_t found = 0;
    for (uint64_t t = 0; found < nsrc && t < (uint64_t)n * 64u + 1024u; ++t) {
        int64_t s = (int64_t)(crand(seed, ST_ABAR, t) % (uint64_t)n);
        if (row_ptr[s + 1] > row_ptr[s]) srcs[found++] = s;
    }
    #pragma omp parallel for schedule(dynamic, 1) reduction(+:total, pairs)
    for (int32_t si = 0; si < found; ++si) {
        int32_t *dist = (int32_t *)malloc((size_t)n * sizeof(int32_t));
        uint32_t *q = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
        for (int64_t v = 0; v < n; ++v) dist[v] = -1;
        int64_t qh = 0, qt = 0;
        dist[srcs[si]] = 0; q[qt++] = (uint32_t)srcs[si];
        double t_local = 0.0, p_local = 0.0;
        while (qh < qt) {
            uint32_t u = q[qh++];
            for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                uint32_t v = col[e];
                if (dist[v] < 0) { dist[v] = dist[u] + 1; q[qt++] = v; t_local += dist[v]; p_local += 1.0; }
            }
        }
        total += t_local; pairs += p_local;
        free(dist); free(q);
    }
    free(srcs);
    return pairs > 0 ? total / pairs : -1.0;
}
