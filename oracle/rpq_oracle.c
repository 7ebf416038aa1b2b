/*
 * Serial CPU oracle of radial-pattern keyword search (RAKS, arXiv 2001.06770).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA library: it is a plain, slow, single-threaded transcription of the
 * paper's definitions and algorithms, written for checking by eye.
 *
 *   orc_activation   Section 3.1, fine-grained weights and Eq. 1-3 (edge
 *                    activation levels), with min-max rescaling.
 *   orc_search       Section 4: exploration phase (initialisation 4.2.1,
 *                    frontier enqueue 4.2.2, result identification 4.2.3 with
 *                    Theorem 3, expansion Algorithm 1), recovering phase
 *                    (Algorithm 2, Lemma 3), the two runs of Fig. 3 (central
 *                    keywords -> top-w CGs, marginal keywords -> RPGs), the
 *                    scores of Eq. 4-6 and top-k selection (Definition 6);
 *                    result subgraphs G^c (V^c, E^c) and G^m = U SP(m_i, V_C)
 *                    (Definition 5, recovered with the two changes to
 *                    Algorithm 2 of Section 4.3) and the PTC check of
 *                    Definition 5 on each RPG.
 *
 * Readings taken where the paper is silent or ambiguous (each also listed in
 * the design notes of the repository):
 *   - w = natural log of the label count; when all weights are equal the
 *     rescaled weight is 0.
 *   - Eq. 1-2 are evaluated left to right as printed, in IEEE double:
 *     reward = abar*(alpha-w)/alpha, penalty = abar*(w-alpha)/(1-alpha);
 *     "Rounding" is round-half-up, floor(x+0.5) (Theorem 1's intervals are
 *     closed below and open above).
 *   - The first Glevel is 0; levels 0..L are identified and expansions run at
 *     levels 0..L-1 ("maximum allowed Glevel" L).
 *   - Inside one Glevel: frontier enqueue, then identification, then
 *     expansion (section order of 4.2.2 - 4.2.4).
 *   - The top-w CGs are the first w of all identified CGs ordered by
 *     (score, node id); w = k (Section 3.4); ties are broken by node id.
 *   - Recovery keeps an edge n->q only if n was still expanding at the level
 *     the edge was used (max(a_nq, h_n) < level at which n was stopped); this
 *     is the "expanded" condition of Lemma 3, which Algorithm 2 leaves out.
 *   - V_C is every CG node that holds a central keyword (h == 0 in a central
 *     column).
 *   - Marginal run: the PTC stop (a node reached by every marginal keyword
 *     stops expanding) applies only when |M| >= 2 (Definition 5 relaxes PTC
 *     for |M| = 1).  An RPG is identified for a CG when every marginal
 *     keyword has reached the union of its V_C; its marginal score is
 *     max_i min_{v in V_C} h^M[v][i].  The run ends when every selected CG is
 *     matched, at level L, or when the frontier empties.
 *   - |M| = 0: the results are the top-k CGs with S^m = 0 and S^r = S^c.
 *   - G^m of a matched CG: for each marginal keyword m_i the sweep starts at
 *     the nodes of V_C whose marginal hit level equals min_{v in V_C} h^M[v][i]
 *     and follows tight edges with the marginal run's stop levels.  Edges are
 *     CSR entries n -> q (n expanded to q); V^m includes those start nodes.
 *   - PTC check: the RPG is G^c U G^m as an undirected graph; marginal keyword
 *     nodes are its nodes holding a marginal keyword; the two nodes must be
 *     distinct and hold different marginal keywords (columns); a path "passes
 *     through" V_C when any of its nodes, endpoints included, is in V_C.
 *   - gamma defaults to 0.5; RPGs are ordered by (S^r, central node id).
 *   - Beam width w (top-w CGs, Section 3.4): w = k unless a larger w is
 *     given.  The marginal run then also stops by Theorem 4, applied with
 *     the smallest score a still unmatched CG g can reach,
 *     combine(S^c(g), l+1) at Glevel l (the printed bound uses S^m of the
 *     k-th RPG, which is <= l), and with ties decided by node id as in the
 *     ranking, so the stop never changes the top-k.
 *   - Multiplicative S^r (Section 3.3 allows one without a formula): the
 *     product S^c * S^m; gamma is not used then.
 *   - A central (marginal) keyword with no keyword node yields no result.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define INF 255u

/* ======================================================= activation levels */
/* Section 3.1: w_ij = log(|{e_ix : l_ix = l_ij, x in N_o(i)}| + |{e_xj : l_xj = l_ij, x in N_i(j)}|),
 * rescaled to [0,1], then coarsened by Eq. 1-3.  Out- and in-neighbour label
 * counts are taken literally from the CSR (in-edges from its transpose).
 * Outputs per CSR entry: a (uint8), and optionally cnt, w (rescaled), x (the
 * value before rounding).  amax[v] = largest a on v's out-edges (0 if none). */
int orc_activation(int32_t n, int64_t m2, const int64_t *row_ptr, const int32_t *col,
                   const uint16_t *label, int32_t n_labels, double alpha, double abar,
                   uint8_t *a_out, uint8_t *amax_out, int64_t *cnt_out, double *w_out, double *x_out) {
    if (n < 0 || m2 < 0 || n_labels <= 0 || !(alpha > 0.0 && alpha < 1.0) || !(abar > 0.0)) return -1;
    int64_t *outc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m2 > 0 ? m2 : 1));
    int64_t *inc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m2 > 0 ? m2 : 1));
    int64_t *tally = (int64_t *)calloc((size_t)n_labels, sizeof(int64_t));
    double *w = (double *)malloc(sizeof(double) * (size_t)(m2 > 0 ? m2 : 1));

    /* out-edges of u with the label of e */
    for (int32_t u = 0; u < n; ++u) {
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) tally[label[e]]++;
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) outc[e] = tally[label[e]];
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) tally[label[e]] = 0;
    }
    /* in-edges of v with the label of e: transpose the CSR (entry ids by target) */
    int64_t *tptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *tent = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m2 > 0 ? m2 : 1));
    for (int64_t e = 0; e < m2; ++e) tptr[col[e] + 1]++;
    for (int32_t v = 0; v < n; ++v) tptr[v + 1] += tptr[v];
    {
        int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
        memcpy(cur, tptr, sizeof(int64_t) * ((size_t)n + 1));
        for (int32_t u = 0; u < n; ++u)
            for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) tent[cur[col[e]]++] = e;
        free(cur);
    }
    for (int32_t v = 0; v < n; ++v) {
        for (int64_t t = tptr[v]; t < tptr[v + 1]; ++t) tally[label[tent[t]]]++;
        for (int64_t t = tptr[v]; t < tptr[v + 1]; ++t) inc[tent[t]] = tally[label[tent[t]]];
        for (int64_t t = tptr[v]; t < tptr[v + 1]; ++t) tally[label[tent[t]]] = 0;
    }

    double wmin = INFINITY, wmax = -INFINITY;
    for (int64_t e = 0; e < m2; ++e) {
        int64_t c = outc[e] + inc[e];
        if (cnt_out) cnt_out[e] = c;
        w[e] = log((double)c);
        if (w[e] < wmin) wmin = w[e];
        if (w[e] > wmax) wmax = w[e];
    }
    for (int64_t e = 0; e < m2; ++e) {
        double ws = (wmax > wmin) ? (w[e] - wmin) / (wmax - wmin) : 0.0;
        double x;
        if (ws <= alpha) {
            double reward = abar * (alpha - ws) / alpha;           /* Eq. 1 */
            x = abar - reward;                                     /* Eq. 3, first case */
        } else {
            double penalty = abar * (ws - alpha) / (1.0 - alpha);  /* Eq. 2 */
            x = abar + penalty;                                    /* Eq. 3, second case */
        }
        double r = floor(x + 0.5);                                 /* Rounding: half up */
        a_out[e] = (uint8_t)r;
        if (w_out) w_out[e] = ws;
        if (x_out) x_out[e] = x;
    }
    for (int32_t v = 0; v < n; ++v) {
        uint8_t mx = 0;
        for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) if (a_out[e] > mx) mx = a_out[e];
        amax_out[v] = mx;
    }
    free(outc); free(inc); free(tally); free(w); free(tptr); free(tent);
    return 0;
}

/* ============================================================== the search */
typedef struct {
    int32_t n;
    int64_t m2;
    const int64_t *row_ptr;
    const int32_t *col;
    const uint8_t *a;        /* activation level per CSR entry */
    int32_t n_kw;
    const int64_t *kw_ptr;
    const int32_t *kw_nodes;
    int64_t *tptr;           /* transpose: in-entries of each node */
    int64_t *tent;           /* ... their CSR entry ids */
    int32_t *tsrc;           /* ... and their source nodes */
} orc_graph;

typedef struct {                /* growable int64 list */
    int64_t *v;
    int64_t n, cap;
} vec;

static void vpush(vec *x, int64_t val) {
    if (x->n == x->cap) {
        x->cap = x->cap ? 2 * x->cap : 64;
        x->v = (int64_t *)realloc(x->v, sizeof(int64_t) * (size_t)x->cap);
    }
    x->v[x->n++] = val;
}

static int cmp_i64(const void *p, const void *q) {
    int64_t a = *(const int64_t *)p, b = *(const int64_t *)q;
    return (a > b) - (a < b);
}

/* splitmix64 for the order-shuffling test option (Theorem 6). */
static uint64_t sm_next(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void shuffle(int64_t *x, int64_t n, uint64_t *s) {
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)(sm_next(s) % (uint64_t)(i + 1));
        int64_t t = x[i]; x[i] = x[j]; x[j] = t;
    }
}

enum { RUN_CENTRAL = 0, RUN_MARGINAL = 1 };

/* State and trace of one run of the exploration phase. */
typedef struct {
    int32_t nt;              /* number of keyword columns */
    uint8_t *h;              /* Node-Keyword Matrix H, n x nt, row-major */
    uint8_t *stop;           /* level at which CF was set (INF = never) */
    uint8_t *ident;          /* central run: node already identified as a CG */
    int32_t last_level;      /* last Glevel that was identified */
    int32_t last_expanded;   /* last Glevel at which expansion ran (-1: none) */
    vec q_ptr, q_nodes;      /* per-level frontier Q_l (sorted) */
    vec cg_node, cg_score, cg_level;   /* identified CGs (central run) */
    int64_t e_act;           /* (column, edge) activations, see orc_e_act */
    int64_t new_hits;        /* number of h writes */
} run_state;

typedef struct {
    int32_t n_sel;
    int64_t *sel;            /* selected CG nodes, ordered by (S^c, id) */
    int64_t *sel_sc;
    vec *vc_all;             /* V^c per selected CG (sorted) */
    vec *vc_kw;              /* V_C per selected CG (sorted) */
    vec *ec;                 /* recovered CSR entries per selected CG (sorted) */
    vec *vm, *em;            /* RPG part G^m per matched CG: nodes, CSR entries (sorted) */
    int32_t *ptc;            /* Definition 5 check per selected CG: 1, 0, -1 = not an RPG */
    int32_t *matched;        /* marginal run: matched flag */
    int32_t *match_level;
    int32_t *s_m;
} cg_state;

typedef struct {
    int disable_stops;        /* test only: no CF and no early termination */
    int exhaustive_marginal;  /* test only: marginal run to L / empty frontier */
    uint64_t shuffle_seed;    /* test only: nonzero shuffles frontier and neighbour order */
    int record_frontiers;     /* keep every Q_l (the trace); off: results and counts only */
    int subgraphs;            /* G^m and the PTC check of each RPG */
} orc_options;

/* Result identification (Section 4.2.3). */
static void identify(run_state *R, int mode, int32_t l, const int64_t *Q, int64_t nq,
                     cg_state *S, const orc_options *opt) {
    const int32_t nt = R->nt;
    if (mode == RUN_CENTRAL) {
        /* Theorem 3: all central h finite -> central node, S^c = max_j h. */
        for (int64_t i = 0; i < nq; ++i) {
            int64_t v = Q[i];
            if (R->stop[v] != INF || R->ident[v]) continue;
            int all = 1, mx = 0;
            for (int32_t j = 0; j < nt; ++j) {
                uint8_t hv = R->h[v * nt + j];
                if (hv == INF) all = 0; else if (hv > mx) mx = hv;
            }
            if (!all) continue;
            vpush(&R->cg_node, v); vpush(&R->cg_score, mx); vpush(&R->cg_level, l);
            R->ident[v] = 1;
            if (!opt->disable_stops) R->stop[v] = (uint8_t)l;   /* stop expanding a central node */
        }
    } else {
        /* PTC: stop expanding a node reached by all marginal keywords (|M| >= 2). */
        if (nt >= 2 && !opt->disable_stops) {
            for (int64_t i = 0; i < nq; ++i) {
                int64_t v = Q[i];
                if (R->stop[v] != INF) continue;
                int all = 1;
                for (int32_t j = 0; j < nt; ++j) if (R->h[v * nt + j] == INF) all = 0;
                if (all) R->stop[v] = (uint8_t)l;
            }
        }
        /* RPG identification: every marginal keyword reaches some node of V_C. */
        for (int32_t g = 0; g < S->n_sel; ++g) {
            if (S->matched[g]) continue;
            int all = 1, sm = 0;
            for (int32_t j = 0; j < nt; ++j) {
                int d = INF;
                for (int64_t t = 0; t < S->vc_kw[g].n; ++t) {
                    uint8_t hv = R->h[S->vc_kw[g].v[t] * nt + j];
                    if (hv < d) d = hv;
                }
                if (d == (int)INF) all = 0; else if (d > sm) sm = d;
            }
            if (all) { S->matched[g] = 1; S->match_level[g] = l; S->s_m[g] = sm; }
        }
    }
}

/* Score of an RPG: Eq. 6 (weighted sum), or the multiplicative combination
 * that Section 3.3 allows, read as the product S^c * S^m. */
static double rpg_score(int64_t sc, int64_t sm, double gamma, int product) {
    if (product) return (double)(sc * sm);
    return gamma * (double)sc + (1.0 - gamma) * (double)sm;
}

typedef struct {
    int32_t w, k;             /* beam width (CGs kept) and number of results */
    double gamma;
    int product;              /* multiplicative S^r */
} score_params;

/* Theorem 4 at Glevel l of the marginal run: with at least k RPGs matched,
 * the search may stop when no CG still unmatched can give an RPG ranked
 * before the k-th one.  An unmatched CG g matches at level l+1 or later, so
 * its RPG scores at least combine(S^c(g), l+1) (both combinations grow with
 * S^m); the k-th RPG (S^r_k, id_k) is compared with that bound on
 * (score, node id), the ranking order. */
static int theorem4_stop(const cg_state *S, int32_t l, const score_params *sp) {
    int32_t nm = 0;
    for (int32_t g = 0; g < S->n_sel; ++g) nm += S->matched[g] != 0;
    if (nm < sp->k) return 0;
    double *sr = (double *)malloc(sizeof(double) * (size_t)nm);
    int64_t *id = (int64_t *)malloc(sizeof(int64_t) * (size_t)nm);
    int32_t t = 0;
    for (int32_t g = 0; g < S->n_sel; ++g)
        if (S->matched[g]) { sr[t] = rpg_score(S->sel_sc[g], S->s_m[g], sp->gamma, sp->product); id[t] = S->sel[g]; ++t; }
    /* k-th smallest (score, id): selection by repeated minimum */
    double srk = 0.0; int64_t idk = -1;
    uint8_t *used = (uint8_t *)calloc((size_t)nm, 1);
    for (int32_t r = 0; r < sp->k; ++r) {
        int32_t best = -1;
        for (int32_t i = 0; i < nm; ++i) {
            if (used[i]) continue;
            if (best < 0 || sr[i] < sr[best] || (sr[i] == sr[best] && id[i] < id[best])) best = i;
        }
        used[best] = 1; srk = sr[best]; idk = id[best];
    }
    int stop = 1;
    for (int32_t g = 0; g < S->n_sel && stop; ++g) {
        if (S->matched[g]) continue;
        double b = rpg_score(S->sel_sc[g], (int64_t)l + 1, sp->gamma, sp->product);
        if (!(b > srk || (b == srk && S->sel[g] > idk))) stop = 0;
    }
    free(sr); free(id); free(used);
    return stop;
}

static int terminate_run(const run_state *R, int mode, const cg_state *S, int32_t l, const score_params *sp,
                         const orc_options *opt) {
    if (opt->disable_stops) return 0;
    if (mode == RUN_CENTRAL) return R->cg_node.n >= sp->w;         /* at least w CGs collected */
    if (opt->exhaustive_marginal) return 0;
    int all = 1;
    for (int32_t g = 0; g < S->n_sel; ++g) if (!S->matched[g]) all = 0;
    if (all) return 1;                                              /* every selected CG matched */
    return theorem4_stop(S, l, sp);
}

/* Exploration phase of one run (Section 4.2, Algorithm 1). */
static void explore(const orc_graph *G, const int32_t *kws, int32_t nt, int32_t L, int mode, const score_params *sp,
                    run_state *R, cg_state *S, const orc_options *opt) {
    const int32_t n = G->n;
    R->nt = nt;
    R->h = (uint8_t *)malloc((size_t)n * (size_t)(nt > 0 ? nt : 1));
    memset(R->h, INF, (size_t)n * (size_t)(nt > 0 ? nt : 1));
    R->stop = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    memset(R->stop, INF, (size_t)(n > 0 ? n : 1));
    R->ident = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    R->last_level = -1; R->last_expanded = -1;
    uint8_t *F = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    uint64_t rs = opt->shuffle_seed;

    /* Initialisation: keyword nodes get h = 0 and become frontiers. */
    for (int32_t j = 0; j < nt; ++j)
        for (int64_t p = G->kw_ptr[kws[j]]; p < G->kw_ptr[kws[j] + 1]; ++p) {
            int64_t v = G->kw_nodes[p];
            R->h[v * nt + j] = 0;
            F[v] = 1;
        }
    if (opt->record_frontiers) vpush(&R->q_ptr, 0);
    int64_t *Q = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *nbr = NULL; int64_t nbr_cap = 0;
    for (int32_t l = 0; l <= L; ++l) {
        /* Frontier enqueue: sequential scan of F, then reset F. */
        int64_t nq = 0;
        for (int32_t v = 0; v < n; ++v) if (F[v]) { Q[nq++] = v; F[v] = 0; }
        if (opt->record_frontiers) {
            for (int64_t i = 0; i < nq; ++i) vpush(&R->q_nodes, Q[i]);
            vpush(&R->q_ptr, R->q_nodes.n);
        }
        R->last_level = l;
        identify(R, mode, l, Q, nq, S, opt);
        if (terminate_run(R, mode, S, l, sp, opt) || l == L) break;

        /* Expansion (Algorithm 1) at Glevel l. */
        if (opt->shuffle_seed) shuffle(Q, nq, &rs);
        int any = 0;
        for (int64_t i = 0; i < nq; ++i) {
            int64_t vf = Q[i];
            if (R->stop[vf] != INF) continue;                          /* CF = 1: skip */
            int64_t b = G->row_ptr[vf], e = G->row_ptr[vf + 1];
            if (e - b > nbr_cap) { nbr_cap = e - b; nbr = (int64_t *)realloc(nbr, sizeof(int64_t) * (size_t)nbr_cap); }
            for (int64_t t = b; t < e; ++t) nbr[t - b] = t;
            for (int32_t j = 0; j < nt; ++j) {
                if (R->h[vf * nt + j] > l) continue;                   /* not a frontier of t_j */
                if (opt->shuffle_seed) shuffle(nbr, e - b, &rs);
                for (int64_t t = 0; t < e - b; ++t) {
                    int64_t ent = nbr[t];
                    int64_t vn = G->col[ent];
                    if (G->a[ent] > l) { F[vf] = 1; any = 1; continue; } /* edge not yet active */
                    if (R->h[vn * nt + j] != INF) continue;              /* already reached */
                    R->h[vn * nt + j] = (uint8_t)(l + 1);
                    F[vn] = 1; any = 1;
                    R->new_hits++;
                }
            }
        }
        R->last_expanded = l;
        if (!any) break;
    }
    free(F); free(Q); free(nbr);

    /* Algorithmic work: (column, edge) pairs activated once, i.e. used at
     * level max(h_vj, a) by a node v still expanding at that level. */
    int64_t eact = 0;
    for (int32_t v = 0; v < n; ++v)
        for (int32_t j = 0; j < nt; ++j) {
            uint8_t hv = R->h[(int64_t)v * nt + j];
            if (hv == INF) continue;
            for (int64_t e = G->row_ptr[v]; e < G->row_ptr[v + 1]; ++e) {
                int lam = G->a[e] > hv ? G->a[e] : hv;
                if (lam <= R->last_expanded && lam < R->stop[v]) eact++;
            }
        }
    R->e_act = eact;
}

/* Backward sweep of Algorithm 2 for one keyword column j: from the start
 * nodes, follow every edge n -> q with h_q = max(a_nq, h_n) + 1 (Lemma 3)
 * whose source n was still expanding at level max(a_nq, h_n), down to the
 * keyword nodes (h = 0).  Appends new nodes to `nodes` (innodes marks them)
 * and the CSR entries n -> q of the recovered paths to `edges`. */
static void sweep(const orc_graph *G, const run_state *R, int32_t j, const int64_t *starts, int64_t ns,
                  uint8_t *innodes, vec *nodes, vec *edges) {
    const int32_t nt = R->nt, n = G->n;
    uint8_t *seen = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t qh = 0, qt = 0;
    for (int64_t i = 0; i < ns; ++i) {
        int64_t v = starts[i];
        if (!innodes[v]) { innodes[v] = 1; vpush(nodes, v); }
        if (!seen[v]) { seen[v] = 1; queue[qt++] = v; }
    }
    while (qh < qt) {
        int64_t q = queue[qh++];
        int hq = R->h[q * nt + j];
        if (hq == 0 || hq == (int)INF) continue;                     /* a keyword node: path start */
        for (int64_t t = G->tptr[q]; t < G->tptr[q + 1]; ++t) {      /* in-neighbours of q */
            int64_t e = G->tent[t];                                  /* entry vn -> q */
            int64_t vn = G->tsrc[t];
            int hn = R->h[vn * nt + j];
            if (hn == (int)INF) continue;
            int lam = G->a[e] > hn ? G->a[e] : hn;
            if (hq != lam + 1) continue;                             /* not a tight edge */
            if (!(lam < R->stop[vn])) continue;                      /* n never expanded at lam */
            vpush(edges, e);
            if (!innodes[vn]) { innodes[vn] = 1; vpush(nodes, vn); }
            if (!seen[vn]) { seen[vn] = 1; queue[qt++] = vn; }
        }
    }
    free(seen); free(queue);
}

static void sort_unique(vec *x) {
    qsort(x->v, (size_t)x->n, sizeof(int64_t), cmp_i64);
    int64_t w = 0;
    for (int64_t i = 0; i < x->n; ++i) if (i == 0 || x->v[i] != x->v[i - 1]) x->v[w++] = x->v[i];
    x->n = w;
}

/* Recovering phase for one CG (Algorithm 2 with Lemma 3's condition): the
 * union over central columns of all recovered shortest paths from the
 * keyword nodes to v_c, i.e. V^c and E^c. */
static void recover(const orc_graph *G, const run_state *R, int64_t vc, vec *nodes, vec *edges) {
    uint8_t *innodes = (uint8_t *)calloc((size_t)(G->n > 0 ? G->n : 1), 1);
    innodes[vc] = 1; vpush(nodes, vc);
    for (int32_t j = 0; j < R->nt; ++j) sweep(G, R, j, &vc, 1, innodes, nodes, edges);
    free(innodes);
    sort_unique(nodes);
    sort_unique(edges);                              /* an edge may serve several columns */
}

/* Recovering phase of an RPG (Section 4.3, the two changes to Algorithm 2):
 * the sweep of marginal column i starts from the nodes of V_C with the
 * smallest marginal hit level d_i = min_{v in V_C} h^M[v][i], so only the
 * smallest-score paths ending in V_C are kept: G^m = U_i SP(m_i, V_C)
 * (Definition 5).  The stop levels are those of the marginal run. */
static void recover_marginal(const orc_graph *G, const run_state *Rm, const vec *vck, vec *nodes, vec *edges) {
    uint8_t *innodes = (uint8_t *)calloc((size_t)(G->n > 0 ? G->n : 1), 1);
    int64_t *starts = (int64_t *)malloc(sizeof(int64_t) * (size_t)(vck->n > 0 ? vck->n : 1));
    for (int32_t i = 0; i < Rm->nt; ++i) {
        int d = INF;
        for (int64_t t = 0; t < vck->n; ++t) {
            int hv = Rm->h[vck->v[t] * Rm->nt + i];
            if (hv < d) d = hv;
        }
        if (d == (int)INF) continue;                 /* keyword i never reached V_C */
        int64_t ns = 0;
        for (int64_t t = 0; t < vck->n; ++t) if (Rm->h[vck->v[t] * Rm->nt + i] == d) starts[ns++] = vck->v[t];
        sweep(G, Rm, i, starts, ns, innodes, nodes, edges);
    }
    free(innodes); free(starts);
    sort_unique(nodes);
    sort_unique(edges);
}

/* Pass Through Constraint of Definition 5, checked on a finished RPG
 * G^r = G^c U G^m taken as an undirected graph.  A marginal keyword node is a
 * node of V^r that holds a marginal keyword (h^M = 0 in that column).  With
 * |M| >= 2 the constraint holds when two different such nodes x, y, holding
 * different marginal keywords, are joined only through V_C: x or y lies in
 * V_C, or y cannot be reached from x in G^r once the nodes of V_C are
 * removed.  With |M| = 1 it holds when some marginal keyword node is
 * connected to a node of V_C in G^r.  Returns 1 (holds) or 0 (violated). */
static int ptc_holds(const orc_graph *G, const run_state *Rm, const vec *vr, const vec *er, const vec *vck) {
    const int32_t n = G->n, nt = Rm->nt;
    uint8_t *in_vc = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    uint8_t *reach = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t t = 0; t < vck->n; ++t) in_vc[vck->v[t]] = 1;
    /* undirected adjacency of G^r: for each node of V^r the edges touching it */
    int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *ends = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)(er->n > 0 ? er->n : 1));
    for (int64_t t = 0; t < er->n; ++t) {
        int64_t e = er->v[t];
        int64_t u = 0, lo = 0, hi = n;               /* row of entry e */
        while (lo < hi) { int64_t mid = (lo + hi) / 2; if (G->row_ptr[mid + 1] <= e) lo = mid + 1; else hi = mid; }
        u = lo;
        ends[2 * t] = u; ends[2 * t + 1] = G->col[e];
        deg[u + 1]++; deg[G->col[e] + 1]++;
    }
    for (int32_t v = 0; v < n; ++v) deg[v + 1] += deg[v];
    int64_t *adj = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)(er->n > 0 ? er->n : 1));
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    memcpy(cur, deg, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t t = 0; t < er->n; ++t) {
        adj[cur[ends[2 * t]]++] = ends[2 * t + 1];
        adj[cur[ends[2 * t + 1]]++] = ends[2 * t];
    }
    int holds = 0;
    for (int64_t t = 0; t < vr->n && !holds; ++t) {
        int64_t x = vr->v[t];
        for (int32_t i = 0; i < nt && !holds; ++i) {
            if (Rm->h[x * nt + i] != 0) continue;    /* x does not hold m_i */
            /* BFS from x in G^r; with |M| >= 2 it may not enter V_C */
            memset(reach, 0, (size_t)(n > 0 ? n : 1));
            int64_t qh = 0, qt = 0;
            reach[x] = 1; queue[qt++] = x;
            int touches_vc = in_vc[x];
            while (qh < qt && !(nt >= 2 && in_vc[x])) {
                int64_t u = queue[qh++];
                for (int64_t p = deg[u]; p < deg[u + 1]; ++p) {
                    int64_t v = adj[p];
                    if (reach[v]) continue;
                    if (in_vc[v]) touches_vc = 1;
                    if (nt >= 2 && in_vc[v]) continue;
                    reach[v] = 1; queue[qt++] = v;
                }
            }
            if (nt == 1) { holds = touches_vc; continue; }
            for (int64_t s = 0; s < vr->n && !holds; ++s) {
                int64_t y = vr->v[s];
                if (y == x) continue;
                for (int32_t jj = 0; jj < nt; ++jj) {
                    if (jj == i || Rm->h[y * nt + jj] != 0) continue;
                    if (in_vc[x] || in_vc[y] || !reach[y]) { holds = 1; break; }
                }
            }
        }
    }
    free(in_vc); free(reach); free(queue); free(deg); free(ends); free(adj); free(cur);
    return holds;
}

/* ----------------------------------------------------------- public result */
typedef struct {
    int32_t status;
    int32_t n_c, n_m;
    run_state rc, rm;
    cg_state S;
    int32_t n_res;
    int64_t *res_node;
    int32_t *res_sc, *res_sm;
    double *res_sr;
} orc_result;

typedef struct { int64_t node; double sr; int32_t sc, sm; } rec;

static int cmp_cg(const void *p, const void *q) {
    const int64_t *a = (const int64_t *)p, *b = (const int64_t *)q;   /* (score, id) pairs */
    if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
    return (a[1] > b[1]) - (a[1] < b[1]);
}

static int cmp_rec(const void *p, const void *q) {
    const rec *a = (const rec *)p, *b = (const rec *)q;
    if (a->sr != b->sr) return a->sr < b->sr ? -1 : 1;
    return (a->node > b->node) - (a->node < b->node);
}

/* The graph a search reads, with the CSR transpose (the in-entries of every
 * node, used by the recovering phase) built once.  The caller's arrays are
 * referenced, not copied, and must outlive the handle.  Searches only read
 * it, so several may run on one prepared graph at the same time (one thread
 * each); every search keeps all of its own state. */
void *orc_graph_new(int32_t n, int64_t m2, const int64_t *row_ptr, const int32_t *col, const uint8_t *a,
                    int32_t n_kw, const int64_t *kw_ptr, const int32_t *kw_nodes) {
    if (n < 0 || m2 < 0 || n_kw < 0) return NULL;
    orc_graph *G = (orc_graph *)calloc(1, sizeof(orc_graph));
    *G = (orc_graph){ n, m2, row_ptr, col, a, n_kw, kw_ptr, kw_nodes, NULL, NULL, NULL };
    G->tptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    G->tent = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m2 > 0 ? m2 : 1));
    G->tsrc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m2 > 0 ? m2 : 1));
    for (int64_t e = 0; e < m2; ++e) G->tptr[col[e] + 1]++;
    for (int32_t v = 0; v < n; ++v) G->tptr[v + 1] += G->tptr[v];
    {
        int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
        memcpy(cur, G->tptr, sizeof(int64_t) * ((size_t)n + 1));
        for (int32_t u = 0; u < n; ++u)
            for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) { G->tsrc[cur[col[e]]] = u; G->tent[cur[col[e]]++] = e; }
        free(cur);
    }
    return G;
}

void orc_graph_free(void *graph) {
    orc_graph *G = (orc_graph *)graph;
    if (!G) return;
    free(G->tptr); free(G->tent); free(G->tsrc);
    free(G);
}

/* flags of orc_search_graph */
enum { ORC_TRACE = 1, ORC_SUBGRAPHS = 2 };

/* One radial-pattern query on a prepared graph.  flags: ORC_TRACE keeps every
 * frontier Q_l; ORC_SUBGRAPHS builds G^m and checks PTC for each RPG.  The
 * results and every other field do not depend on the flags. */
void *orc_search_graph(const void *graph, const int32_t *central, int32_t n_c, const int32_t *marginal, int32_t n_m,
                       int32_t k, int32_t max_depth, double gamma, int32_t w, int32_t product,
                       int32_t disable_stops, int32_t exhaustive_marginal, uint64_t shuffle_seed, int32_t flags) {
    const orc_graph G = *(const orc_graph *)graph;
    const int32_t n_kw = G.n_kw;
    const int64_t *kw_ptr = G.kw_ptr;
    orc_result *res = (orc_result *)calloc(1, sizeof(orc_result));
    res->n_c = n_c; res->n_m = n_m;
    if (n_c <= 0 || n_m < 0 || k <= 0 || max_depth < 0 || max_depth > 254 || (w != 0 && w < k)) { res->status = -1; return res; }
    for (int32_t j = 0; j < n_c; ++j) if (central[j] < 0 || central[j] >= n_kw) { res->status = -1; return res; }
    for (int32_t j = 0; j < n_m; ++j) if (marginal[j] < 0 || marginal[j] >= n_kw) { res->status = -1; return res; }
    orc_options opt = { disable_stops, exhaustive_marginal, shuffle_seed, (flags & ORC_TRACE) != 0,
                        (flags & ORC_SUBGRAPHS) != 0 };
    /* beam width: w = k unless given (Section 3.4 uses w = k; k <= w) */
    const score_params sp = { w > 0 ? w : k, k, gamma, product };
    const int32_t wb = sp.w;
    cg_state *S = &res->S;

    int empty_c = 0, empty_m = 0;
    for (int32_t j = 0; j < n_c; ++j) if (kw_ptr[central[j] + 1] == kw_ptr[central[j]]) empty_c = 1;
    for (int32_t j = 0; j < n_m; ++j) if (kw_ptr[marginal[j] + 1] == kw_ptr[marginal[j]]) empty_m = 1;

    if (!empty_c) {
        /* First run: central keywords -> CGs. */
        explore(&G, central, n_c, max_depth, RUN_CENTRAL, &sp, &res->rc, S, &opt);
        /* Top-w CGs by (S^c, id). */
        int64_t ncg = res->rc.cg_node.n;
        int64_t *pairs = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)(ncg > 0 ? ncg : 1));
        for (int64_t i = 0; i < ncg; ++i) { pairs[2 * i] = res->rc.cg_score.v[i]; pairs[2 * i + 1] = res->rc.cg_node.v[i]; }
        qsort(pairs, (size_t)ncg, 2 * sizeof(int64_t), cmp_cg);
        S->n_sel = (int32_t)(ncg < wb ? ncg : wb);
        S->sel = (int64_t *)malloc(sizeof(int64_t) * (size_t)(S->n_sel > 0 ? S->n_sel : 1));
        S->sel_sc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(S->n_sel > 0 ? S->n_sel : 1));
        for (int32_t g = 0; g < S->n_sel; ++g) { S->sel[g] = pairs[2 * g + 1]; S->sel_sc[g] = pairs[2 * g]; }
        free(pairs);
        /* Recovering phase: V^c, E^c and V_C of each selected CG. */
        S->vc_all = (vec *)calloc((size_t)(S->n_sel > 0 ? S->n_sel : 1), sizeof(vec));
        S->vc_kw = (vec *)calloc((size_t)(S->n_sel > 0 ? S->n_sel : 1), sizeof(vec));
        S->ec = (vec *)calloc((size_t)(S->n_sel > 0 ? S->n_sel : 1), sizeof(vec));
        S->matched = (int32_t *)calloc((size_t)(S->n_sel > 0 ? S->n_sel : 1), sizeof(int32_t));
        S->match_level = (int32_t *)malloc(sizeof(int32_t) * (size_t)(S->n_sel > 0 ? S->n_sel : 1));
        S->s_m = (int32_t *)calloc((size_t)(S->n_sel > 0 ? S->n_sel : 1), sizeof(int32_t));
        for (int32_t g = 0; g < S->n_sel; ++g) {
            S->match_level[g] = -1;
            recover(&G, &res->rc, S->sel[g], &S->vc_all[g], &S->ec[g]);
            for (int64_t t = 0; t < S->vc_all[g].n; ++t) {
                int64_t v = S->vc_all[g].v[t];
                int holds = 0;
                for (int32_t j = 0; j < n_c; ++j) if (res->rc.h[v * n_c + j] == 0) holds = 1;
                if (holds) vpush(&S->vc_kw[g], v);
            }
        }
        /* Second run: marginal keywords -> RPGs. */
        if (n_m > 0 && !empty_m && S->n_sel > 0)
            explore(&G, marginal, n_m, max_depth, RUN_MARGINAL, &sp, &res->rm, S, &opt);
        /* Recovering phase of the RPGs: G^m and the PTC check of each match. */
        S->vm = (vec *)calloc((size_t)(S->n_sel > 0 ? S->n_sel : 1), sizeof(vec));
        S->em = (vec *)calloc((size_t)(S->n_sel > 0 ? S->n_sel : 1), sizeof(vec));
        S->ptc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(S->n_sel > 0 ? S->n_sel : 1));
        for (int32_t g = 0; g < S->n_sel; ++g) {
            S->ptc[g] = -1;
            if (!S->matched[g] || !opt.subgraphs) continue;
            recover_marginal(&G, &res->rm, &S->vc_kw[g], &S->vm[g], &S->em[g]);
            vec vr = {0, 0, 0}, er = {0, 0, 0};
            for (int64_t t = 0; t < S->vc_all[g].n; ++t) vpush(&vr, S->vc_all[g].v[t]);
            for (int64_t t = 0; t < S->vm[g].n; ++t) vpush(&vr, S->vm[g].v[t]);
            for (int64_t t = 0; t < S->ec[g].n; ++t) vpush(&er, S->ec[g].v[t]);
            for (int64_t t = 0; t < S->em[g].n; ++t) vpush(&er, S->em[g].v[t]);
            sort_unique(&vr); sort_unique(&er);
            S->ptc[g] = ptc_holds(&G, &res->rm, &vr, &er, &S->vc_kw[g]);
            free(vr.v); free(er.v);
        }
    }

    /* Scoring (Eq. 6) and top-k (Definition 6). */
    rec *R = (rec *)malloc(sizeof(rec) * (size_t)(S->n_sel > 0 ? S->n_sel : 1));
    int32_t nr = 0;
    if (!empty_c && !(n_m > 0 && empty_m)) {
        for (int32_t g = 0; g < S->n_sel; ++g) {
            if (n_m == 0) {
                R[nr].node = S->sel[g]; R[nr].sc = (int32_t)S->sel_sc[g]; R[nr].sm = 0; R[nr].sr = (double)S->sel_sc[g];
                nr++;
            } else if (S->matched[g]) {
                R[nr].node = S->sel[g]; R[nr].sc = (int32_t)S->sel_sc[g]; R[nr].sm = S->s_m[g];
                R[nr].sr = rpg_score(S->sel_sc[g], S->s_m[g], gamma, product);
                nr++;
            }
        }
    }
    qsort(R, (size_t)nr, sizeof(rec), cmp_rec);
    if (nr > k) nr = k;
    res->n_res = nr;
    res->res_node = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nr > 0 ? nr : 1));
    res->res_sc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nr > 0 ? nr : 1));
    res->res_sm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nr > 0 ? nr : 1));
    res->res_sr = (double *)malloc(sizeof(double) * (size_t)(nr > 0 ? nr : 1));
    for (int32_t i = 0; i < nr; ++i) {
        res->res_node[i] = R[i].node; res->res_sc[i] = R[i].sc; res->res_sm[i] = R[i].sm; res->res_sr[i] = R[i].sr;
    }
    free(R);
    return res;
}

/* The same query on a graph prepared for this call alone, with the full trace
 * and the result subgraphs. */
void *orc_search(int32_t n, int64_t m2, const int64_t *row_ptr, const int32_t *col, const uint8_t *a,
                 int32_t n_kw, const int64_t *kw_ptr, const int32_t *kw_nodes,
                 const int32_t *central, int32_t n_c, const int32_t *marginal, int32_t n_m,
                 int32_t k, int32_t max_depth, double gamma, int32_t w, int32_t product,
                 int32_t disable_stops, int32_t exhaustive_marginal, uint64_t shuffle_seed) {
    void *G = orc_graph_new(n, m2, row_ptr, col, a, n_kw, kw_ptr, kw_nodes);
    if (!G) {
        orc_result *res = (orc_result *)calloc(1, sizeof(orc_result));
        res->status = -1;
        return res;
    }
    void *res = orc_search_graph(G, central, n_c, marginal, n_m, k, max_depth, gamma, w, product, disable_stops,
                                 exhaustive_marginal, shuffle_seed, ORC_TRACE | ORC_SUBGRAPHS);
    orc_graph_free(G);
    return res;
}

/* ----------------------------------------------------------- accessors */
/* Field ids for orc_get: copies the field into dst (if non-NULL) and returns
 * its element count.  Run r = 0 (central) or 1 (marginal); g = selected CG. */
enum {
    F_STATUS = 0, F_NRES, F_RES_NODE, F_RES_SC, F_RES_SM, F_RES_SR,
    F_QPTR, F_QNODES, F_LAST_LEVEL, F_LAST_EXPANDED, F_EACT, F_NEWHITS,
    F_CG_NODE, F_CG_SCORE, F_CG_LEVEL, F_NSEL, F_SEL, F_SEL_SC, F_VC_ALL, F_VC_KW, F_EC,
    F_MATCHED, F_MATCH_LEVEL, F_SM, F_RAN, F_VM, F_EM, F_PTC
};

static int64_t copy64(const int64_t *src, int64_t n, void *dst) { if (dst && n) memcpy(dst, src, sizeof(int64_t) * (size_t)n); return n; }
static int64_t copy32(const int32_t *src, int64_t n, void *dst) { if (dst && n) memcpy(dst, src, sizeof(int32_t) * (size_t)n); return n; }

int64_t orc_get(void *handle, int32_t field, int32_t r, int32_t g, void *dst) {
    orc_result *res = (orc_result *)handle;
    run_state *R = r == 0 ? &res->rc : &res->rm;
    cg_state *S = &res->S;
    switch (field) {
    case F_STATUS: if (dst) *(int32_t *)dst = res->status; return 1;
    case F_NRES: if (dst) *(int32_t *)dst = res->n_res; return 1;
    case F_RES_NODE: return copy64(res->res_node, res->n_res, dst);
    case F_RES_SC: return copy32(res->res_sc, res->n_res, dst);
    case F_RES_SM: return copy32(res->res_sm, res->n_res, dst);
    case F_RES_SR: if (dst && res->n_res) memcpy(dst, res->res_sr, sizeof(double) * (size_t)res->n_res); return res->n_res;
    case F_RAN: if (dst) *(int32_t *)dst = R->h != NULL; return 1;
    case F_QPTR: return copy64(R->q_ptr.v, R->q_ptr.n, dst);
    case F_QNODES: return copy64(R->q_nodes.v, R->q_nodes.n, dst);
    case F_LAST_LEVEL: if (dst) *(int32_t *)dst = R->last_level; return 1;
    case F_LAST_EXPANDED: if (dst) *(int32_t *)dst = R->last_expanded; return 1;
    case F_EACT: if (dst) *(int64_t *)dst = R->e_act; return 1;
    case F_NEWHITS: if (dst) *(int64_t *)dst = R->new_hits; return 1;
    case F_CG_NODE: return copy64(R->cg_node.v, R->cg_node.n, dst);
    case F_CG_SCORE: return copy64(R->cg_score.v, R->cg_score.n, dst);
    case F_CG_LEVEL: return copy64(R->cg_level.v, R->cg_level.n, dst);
    case F_NSEL: if (dst) *(int32_t *)dst = S->n_sel; return 1;
    case F_SEL: return copy64(S->sel, S->n_sel, dst);
    case F_SEL_SC: return copy64(S->sel_sc, S->n_sel, dst);
    case F_VC_ALL: return (g < S->n_sel) ? copy64(S->vc_all[g].v, S->vc_all[g].n, dst) : 0;
    case F_VC_KW: return (g < S->n_sel) ? copy64(S->vc_kw[g].v, S->vc_kw[g].n, dst) : 0;
    case F_EC: return (g < S->n_sel) ? copy64(S->ec[g].v, S->ec[g].n, dst) : 0;
    case F_MATCHED: return copy32(S->matched, S->n_sel, dst);
    case F_MATCH_LEVEL: return copy32(S->match_level, S->n_sel, dst);
    case F_SM: return copy32(S->s_m, S->n_sel, dst);
    case F_VM: return (g < S->n_sel && S->vm) ? copy64(S->vm[g].v, S->vm[g].n, dst) : 0;
    case F_EM: return (g < S->n_sel && S->em) ? copy64(S->em[g].v, S->em[g].n, dst) : 0;
    case F_PTC: return S->ptc ? copy32(S->ptc, S->n_sel, dst) : 0;
    }
    return -1;
}

/* H (n x nt) and the stop levels (n) of run r; returns nt, or -1 if the run did not execute. */
int32_t orc_get_h(void *handle, int32_t r, uint8_t *h_dst, uint8_t *stop_dst, int32_t n) {
    orc_result *res = (orc_result *)handle;
    run_state *R = r == 0 ? &res->rc : &res->rm;
    if (!R->h) return -1;
    if (h_dst) memcpy(h_dst, R->h, (size_t)n * (size_t)R->nt);
    if (stop_dst) memcpy(stop_dst, R->stop, (size_t)n);
    return R->nt;
}

static void free_run(run_state *R) {
    free(R->h); free(R->stop); free(R->ident);
    free(R->q_ptr.v); free(R->q_nodes.v); free(R->cg_node.v); free(R->cg_score.v); free(R->cg_level.v);
}

void orc_free(void *handle) {
    orc_result *res = (orc_result *)handle;
    if (!res) return;
    free_run(&res->rc); free_run(&res->rm);
    cg_state *S = &res->S;
    for (int32_t g = 0; g < S->n_sel; ++g) {
        free(S->vc_all[g].v); free(S->vc_kw[g].v); free(S->ec[g].v);
        if (S->vm) { free(S->vm[g].v); free(S->em[g].v); }
    }
    free(S->sel); free(S->sel_sc); free(S->vc_all); free(S->vc_kw); free(S->ec);
    free(S->vm); free(S->em); free(S->ptc);
    free(S->matched); free(S->match_level); free(S->s_m);
    free(res->res_node); free(res->res_sc); free(res->res_sm); free(res->res_sr);
    free(res);
}
