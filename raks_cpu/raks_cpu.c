/*
 * RAKS-CPU: the paper's multi-core CPU implementation of the radial-pattern
 * search, as a parallel comparison point for the GPU library (Section 4.1:
 * OpenMP fork-join; Section 4.2.4 scheduling: one thread per frontier node
 * for all keywords, dynamic load balancing; Algorithm 1 with its per-level
 * re-scan of every neighbour; Section 4.2.2: sequential scan of F on the CPU;
 * Section 4.3: recovery parallel over CGs).
 *
 * Not part of the product path and not the oracle: it is a baseline that the
 * benchmark times next to the GPU.  Concurrent writes of Algorithm 1 store the
 * same value (Theorem 6); they are relaxed atomic stores here.  Activation
 * levels are computed here too (Section 3.1, Eq. 1-3), in parallel.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define INF 255u
#define ST8(p, v) __atomic_store_n((p), (uint8_t)(v), __ATOMIC_RELAXED)
#define LD8(p) __atomic_load_n((p), __ATOMIC_RELAXED)

/* Activation levels on a bi-directed CSR (each entry's reverse carries the
 * same label): count = same-label entries of u + same-label entries of v. */
int raks_activation(int32_t n, int64_t m2, const int64_t *row_ptr, const int32_t *col, const uint16_t *label,
                    int32_t n_labels, double alpha, double abar, uint8_t *a_out) {
    int64_t *dl = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m2 > 0 ? m2 : 1));
    #pragma omp parallel
    {
        int64_t *tally = (int64_t *)calloc((size_t)n_labels, sizeof(int64_t));
        #pragma omp for schedule(dynamic, 1024)
        for (int32_t u = 0; u < n; ++u) {
            for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) tally[label[e]]++;
            for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) dl[e] = tally[label[e]];
            for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) tally[label[e]] = 0;
        }
        free(tally);
    }
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m2 > 0 ? m2 : 1));
    int bad = 0;
    #pragma omp parallel for schedule(dynamic, 1024) reduction(|:bad)
    for (int32_t u = 0; u < n; ++u) {
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            const int32_t v = col[e];
            int64_t lo = row_ptr[v], hi = row_ptr[v + 1];
            while (lo < hi) { int64_t mid = (lo + hi) / 2; if (col[mid] < u) lo = mid + 1; else hi = mid; }
            if (lo >= row_ptr[v + 1] || col[lo] != u) { bad = 1; cnt[e] = 1; continue; }
            cnt[e] = dl[e] + dl[lo];
        }
    }
    if (bad) { free(dl); free(cnt); return -1; }
    double wmin = INFINITY, wmax = -INFINITY;
    #pragma omp parallel for reduction(min:wmin) reduction(max:wmax)
    for (int64_t e = 0; e < m2; ++e) {
        const double w = log((double)cnt[e]);
        if (w < wmin) wmin = w;
        if (w > wmax) wmax = w;
    }
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m2; ++e) {
        const double w = log((double)cnt[e]);
        const double ws = (wmax > wmin) ? (w - wmin) / (wmax - wmin) : 0.0;
        double x;
        if (ws <= alpha) { double reward = abar * (alpha - ws) / alpha; x = abar - reward; }
        else { double penalty = abar * (ws - alpha) / (1.0 - alpha); x = abar + penalty; }
        a_out[e] = (uint8_t)floor(x + 0.5);
    }
    free(dl); free(cnt);
    return 0;
}

typedef struct {
    int32_t n;
    const int64_t *row_ptr;
    const int32_t *col;
    const uint8_t *a;
    const int64_t *kw_ptr;
    const int32_t *kw_nodes;
} graph_t;

/* One run of the exploration phase; returns the CGs (central run) in cgs. */
static void explore(const graph_t *G, const int32_t *kws, int nt, int L, int central, int w, uint8_t *h,
                    uint8_t *stop, uint8_t *F, int32_t *Q, int64_t *ncg_out, int64_t *cg_node, int32_t *cg_score,
                    int32_t nsel, const int64_t *vc_ptr, const int32_t *vc_nodes, int32_t *matched, int32_t *s_m) {
    const int32_t n = G->n;
    memset(h, INF, (size_t)n * (size_t)nt);
    memset(stop, INF, (size_t)n);
    memset(F, 0, (size_t)n);
    for (int j = 0; j < nt; ++j)
        for (int64_t p = G->kw_ptr[kws[j]]; p < G->kw_ptr[kws[j] + 1]; ++p) {
            h[(int64_t)G->kw_nodes[p] * nt + j] = 0;
            F[G->kw_nodes[p]] = 1;
        }
    int64_t ncg = 0;
    for (int l = 0; l <= L; ++l) {
        int64_t nq = 0;
        for (int32_t v = 0; v < n; ++v) if (F[v]) { Q[nq++] = v; F[v] = 0; }  /* sequential scan (4.2.2) */
        /* identification (4.2.3) */
        if (central) {
            for (int64_t i = 0; i < nq; ++i) {
                const int32_t v = Q[i];
                if (stop[v] != INF) continue;
                int all = 1, mx = 0;
                for (int j = 0; j < nt; ++j) { int hv = h[(int64_t)v * nt + j]; if (hv == (int)INF) all = 0; else if (hv > mx) mx = hv; }
                if (all) { cg_node[ncg] = v; cg_score[ncg] = mx; ncg++; stop[v] = (uint8_t)l; }
            }
            if (ncg >= w || l == L) break;
        } else {
            if (nt >= 2)
                #pragma omp parallel for schedule(dynamic, 256)
                for (int64_t i = 0; i < nq; ++i) {
                    const int32_t v = Q[i];
                    if (stop[v] != INF) continue;
                    int all = 1;
                    for (int j = 0; j < nt; ++j) if (h[(int64_t)v * nt + j] == INF) all = 0;
                    if (all) stop[v] = (uint8_t)l;
                }
            int all_matched = 1;
            for (int32_t g = 0; g < nsel; ++g) {
                if (matched[g]) continue;
                int ok = 1, sm = 0;
                for (int j = 0; j < nt; ++j) {
                    int d = INF;
                    for (int64_t t = vc_ptr[g]; t < vc_ptr[g + 1]; ++t) { int hv = h[(int64_t)vc_nodes[t] * nt + j]; if (hv < d) d = hv; }
                    if (d == (int)INF) ok = 0; else if (d > sm) sm = d;
                }
                if (ok) { matched[g] = 1; s_m[g] = sm; } else all_matched = 0;
            }
            if (all_matched || l == L) break;
        }
        /* expansion (Algorithm 1): one thread per frontier node, all keywords */
        int any = 0;
        #pragma omp parallel for schedule(dynamic, 64) reduction(|:any)
        for (int64_t i = 0; i < nq; ++i) {
            const int32_t vf = Q[i];
            if (stop[vf] != INF) continue;
            for (int j = 0; j < nt; ++j) {
                if (LD8(&h[(int64_t)vf * nt + j]) > l) continue;
                for (int64_t e = G->row_ptr[vf]; e < G->row_ptr[vf + 1]; ++e) {
                    const int32_t vn = G->col[e];
                    if (G->a[e] > l) { ST8(&F[vf], 1); any = 1; continue; }
                    if (LD8(&h[(int64_t)vn * nt + j]) != INF) continue;
                    ST8(&h[(int64_t)vn * nt + j], l + 1);
                    ST8(&F[vn], 1);
                    any = 1;
                }
            }
        }
        if (!any) break;
    }
    if (ncg_out) *ncg_out = ncg;
}

typedef struct { int64_t node; double sr; int32_t sc, sm; } rec_t;

static int cmp_cg(const void *p, const void *q) {
    const int64_t *a = (const int64_t *)p, *b = (const int64_t *)q;
    if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
    return (a[1] > b[1]) - (a[1] < b[1]);
}
static int cmp_rec(const void *p, const void *q) {
    const rec_t *a = (const rec_t *)p, *b = (const rec_t *)q;
    if (a->sr != b->sr) return a->sr < b->sr ? -1 : 1;
    return (a->node > b->node) - (a->node < b->node);
}

/* Full query: central run, top-w CGs, recovery of V_C (parallel over CGs,
 * Section 4.3), marginal run, Eq. 6, top-k.  Results into out_* (k slots);
 * returns the number of results. */
int32_t raks_search(int32_t n, const int64_t *row_ptr, const int32_t *col, const uint8_t *a,
                    const int64_t *kw_ptr, const int32_t *kw_nodes, const int32_t *central, int32_t n_c,
                    const int32_t *marginal, int32_t n_m, int32_t k, int32_t L, double gamma,
                    int64_t *out_node, int32_t *out_sc, int32_t *out_sm, double *out_sr) {
    graph_t G = { n, row_ptr, col, a, kw_ptr, kw_nodes };
    for (int j = 0; j < n_c; ++j) if (kw_ptr[central[j] + 1] == kw_ptr[central[j]]) return 0;
    for (int j = 0; j < n_m; ++j) if (kw_ptr[marginal[j] + 1] == kw_ptr[marginal[j]]) return 0;
    const int nt = n_c > n_m ? n_c : n_m;
    uint8_t *h = (uint8_t *)malloc((size_t)n * (size_t)(nt > 0 ? nt : 1));
    uint8_t *stop = (uint8_t *)malloc((size_t)n), *F = (uint8_t *)malloc((size_t)n);
    int32_t *Q = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *cg_node = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int32_t *cg_score = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t ncg = 0;
    explore(&G, central, n_c, L, 1, k, h, stop, F, Q, &ncg, cg_node, cg_score, 0, NULL, NULL, NULL, NULL);
    int64_t *pairs = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)(ncg > 0 ? ncg : 1));
    for (int64_t i = 0; i < ncg; ++i) { pairs[2 * i] = cg_score[i]; pairs[2 * i + 1] = cg_node[i]; }
    qsort(pairs, (size_t)ncg, 2 * sizeof(int64_t), cmp_cg);
    const int32_t nsel = (int32_t)(ncg < k ? ncg : k);
    int64_t *vc_ptr = (int64_t *)calloc((size_t)nsel + 1, sizeof(int64_t));
    int32_t **vc_list = (int32_t **)calloc((size_t)(nsel > 0 ? nsel : 1), sizeof(int32_t *));
    int64_t *vc_len = (int64_t *)calloc((size_t)(nsel > 0 ? nsel : 1), sizeof(int64_t));
    if (n_m > 0 && nsel > 0) {
        /* in-neighbours = out-neighbours on the bi-directed graph; a(n->q) = a(q->n) */
        #pragma omp parallel for schedule(dynamic, 1)
        for (int32_t g = 0; g < nsel; ++g) {
            const int32_t vc = (int32_t)pairs[2 * g + 1];
            uint8_t *in_vc = (uint8_t *)calloc((size_t)n, 1);
            uint8_t *seen = (uint8_t *)malloc((size_t)n);
            int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
            int64_t cap = 64, cnt = 0;
            int32_t *nodes = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
            in_vc[vc] = 1; nodes[cnt++] = vc;
            for (int j = 0; j < n_c; ++j) {
                if (h[(int64_t)vc * n_c + j] == 0) continue;
                memset(seen, 0, (size_t)n);
                int64_t qh = 0, qt = 0;
                queue[qt++] = vc; seen[vc] = 1;
                while (qh < qt) {
                    const int32_t q = queue[qh++];
                    const int hq = h[(int64_t)q * n_c + j];
                    for (int64_t e = row_ptr[q]; e < row_ptr[q + 1]; ++e) {
                        const int32_t vn = col[e];
                        const int hn = h[(int64_t)vn * n_c + j];
                        if (hn == (int)INF) continue;
                        const int lam = a[e] > hn ? a[e] : hn;
                        if (hq != lam + 1 || !(lam < stop[vn])) continue;
                        if (!in_vc[vn]) {
                            in_vc[vn] = 1;
                            if (cnt == cap) { cap *= 2; nodes = (int32_t *)realloc(nodes, sizeof(int32_t) * (size_t)cap); }
                            nodes[cnt++] = vn;
                        }
                        if (hn != 0 && !seen[vn]) { seen[vn] = 1; queue[qt++] = vn; }
                    }
                }
            }
            int64_t w = 0;          /* keep nodes holding a central keyword */
            for (int64_t t = 0; t < cnt; ++t) {
                int holds = 0;
                for (int j = 0; j < n_c; ++j) if (h[(int64_t)nodes[t] * n_c + j] == 0) holds = 1;
                if (holds) nodes[w++] = nodes[t];
            }
            vc_list[g] = nodes; vc_len[g] = w;
            free(in_vc); free(seen); free(queue);
        }
    }
    for (int32_t g = 0; g < nsel; ++g) vc_ptr[g + 1] = vc_ptr[g] + vc_len[g];
    int32_t *vc_nodes = (int32_t *)malloc(sizeof(int32_t) * (size_t)(vc_ptr[nsel] > 0 ? vc_ptr[nsel] : 1));
    for (int32_t g = 0; g < nsel; ++g) {
        if (vc_len[g]) memcpy(vc_nodes + vc_ptr[g], vc_list[g], sizeof(int32_t) * (size_t)vc_len[g]);
        free(vc_list[g]);
    }
    int32_t *matched = (int32_t *)calloc((size_t)(nsel > 0 ? nsel : 1), sizeof(int32_t));
    int32_t *s_m = (int32_t *)calloc((size_t)(nsel > 0 ? nsel : 1), sizeof(int32_t));
    if (n_m > 0 && nsel > 0)
        explore(&G, marginal, n_m, L, 0, k, h, stop, F, Q, NULL, NULL, NULL, nsel, vc_ptr, vc_nodes, matched, s_m);
    rec_t *R = (rec_t *)malloc(sizeof(rec_t) * (size_t)(nsel > 0 ? nsel : 1));
    int32_t nr = 0;
    for (int32_t g = 0; g < nsel; ++g) {
        const int32_t sc = (int32_t)pairs[2 * g];
        if (n_m == 0) { R[nr].node = pairs[2 * g + 1]; R[nr].sc = sc; R[nr].sm = 0; R[nr].sr = sc; nr++; }
        else if (matched[g]) {
            R[nr].node = pairs[2 * g + 1]; R[nr].sc = sc; R[nr].sm = s_m[g];
            R[nr].sr = gamma * (double)sc + (1.0 - gamma) * (double)s_m[g]; nr++;
        }
    }
    qsort(R, (size_t)nr, sizeof(rec_t), cmp_rec);
    if (nr > k) nr = k;
    for (int32_t i = 0; i < nr; ++i) { out_node[i] = R[i].node; out_sc[i] = R[i].sc; out_sm[i] = R[i].sm; out_sr[i] = R[i].sr; }
    free(R); free(matched); free(s_m); free(vc_nodes); free(vc_ptr); free(vc_list); free(vc_len); free(pairs);
    free(h); free(stop); free(F); free(Q); free(cg_node); free(cg_score);
    return nr;
}

int raks_threads(void) { return omp_get_max_threads(); }
