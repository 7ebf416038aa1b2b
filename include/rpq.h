/*
 * rpq.h - C ABI of the B300 radial-pattern keyword search library (librpq.so).
 *
 * Radial-pattern keyword search (RAKS, arXiv 2001.06770): a query Q = {C, M}
 * holds central keywords C (non-empty) and marginal keywords M (Definition 1).
 * The library returns the top-k radial pattern graphs (Definition 6), each
 * identified by its central node, with scores S^c (Eq. 4), S^m (Eq. 5) and
 * S^r = gamma*S^c + (1-gamma)*S^m (Eq. 6).  All search work runs in CUDA
 * kernels on one GPU; the knowledge graph stays resident in device memory.
 *
 * Conventions shared by every call:
 *   - Return value: RPQ_OK (0) on success, a negative RPQ_E* code otherwise;
 *     rpq_strerror() names the code and rpq_last_error() gives a message for
 *     the calling thread's last failure.
 *   - Host buffers are owned by the caller; the library never keeps a
 *     pointer to them after the call returns.
 *   - Device memory is allocated by the library (cudaMalloc) when a graph is
 *     loaded and when a search slot is first used; rpq_free_kg releases it.
 *   - Keyword ids index the postings given at load time; duplicate ids in a
 *     query are allowed and behave as identical columns (a repeated marginal
 *     keyword still counts towards |M|, which switches the PTC stop on).
 *   - Calls on the same rpq_kg from several threads must be serialised by the
 *     caller.
 */
#ifndef RPQ_H
#define RPQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- errors */
#define RPQ_OK         0
#define RPQ_EINVAL    (-1)  /* malformed graph or query, id out of range */
#define RPQ_ENOMEM    (-2)  /* device or pinned host allocation failed */
#define RPQ_ETIMEOUT  (-3)  /* a bounded device wait ran out */
#define RPQ_ECUDA     (-4)  /* a CUDA runtime call failed */
#define RPQ_ELIMIT    (-5)  /* input beyond a documented size limit */
#define RPQ_EINTERNAL (-6)  /* a device-side consistency check failed (in librpq_checked.so,
                               also an index that failed its bounds check) */
#define RPQ_ESIZE     (-7)  /* a caller buffer is too small; the call reports the size needed */

/* Documented limits of the library. */
#define RPQ_MAX_NODES    (1 << 26)  /* node ids are packed in 26 bits */
#define RPQ_MAX_LABELS   8192       /* edge labels must be < n_labels <= this */
#define RPQ_MAX_LEVEL    63         /* activation levels and max_depth <= 63 */
#define RPQ_MAX_KEYWORDS 8          /* per keyword set (central, marginal) */
#define RPQ_MAX_K        64         /* top-k (and beam width w = k) */

/* ------------------------------------------------------------------ graph */
typedef struct rpq_kg rpq_kg; /* opaque, device resident */

/* Knowledge graph handed to rpq_load_kg (Section 2: a bi-directed labelled
 * graph - every original edge has its reverse - stored as CSR, Section 4.1).
 *   n          number of nodes, 0 < n <= RPQ_MAX_NODES
 *   m2         number of CSR entries (both directions), 0 <= m2 < 2^32
 *   row_ptr    n+1 offsets, row_ptr[0] = 0, non-decreasing, row_ptr[n] = m2
 *   col        m2 neighbour ids; each row strictly ascending, no self-loop
 *   label      m2 edge labels < n_labels; the entry v->u carries the same
 *              label as u->v (the reverse edge of Section 2)
 *   n_labels   1 <= n_labels <= RPQ_MAX_LABELS
 *   n_kw       number of keywords; kw_ptr has n_kw+1 offsets into kw_nodes
 *   kw_nodes   node ids holding each keyword (V_t of Section 2), in [0, n)
 *   alpha      scaling parameter of Eq. 1-2, 0 < alpha < 1 (paper: 0.5)
 *   abar       average shortest hop count of the graph (Section 3.1), > 0
 * Symmetry (each u->v has v->u with the same label) is checked on the device;
 * a violation returns RPQ_EINVAL. */
typedef struct {
    int32_t n;
    int64_t m2;
    const int64_t *row_ptr;
    const int32_t *col;
    const uint16_t *label;
    int32_t n_labels;
    int32_t n_kw;
    const int64_t *kw_ptr;
    const int32_t *kw_nodes;
    double alpha;
    double abar;
} rpq_kg_desc;

/* Copy the graph to the current CUDA device and build the edge activation
 * levels there (Section 3.1: label counts, w = log count, min-max rescale,
 * Eq. 1-3 with round-half-up).  On success *out owns all device memory of the
 * graph.  Errors: RPQ_EINVAL (malformed CSR, asymmetric edge or label,
 * parameter out of range), RPQ_ELIMIT (a documented limit, or an activation
 * level above RPQ_MAX_LEVEL), RPQ_ENOMEM, RPQ_ECUDA. */
int rpq_load_kg(const rpq_kg_desc *desc, rpq_kg **out);

/* Release every device and host resource of the graph.  NULL is accepted. */
int rpq_free_kg(rpq_kg *kg);

/* Export the device adjacency for inspection: adj[m2] receives each row's
 * entries packed as (activation level << 26) | neighbour id, sorted ascending
 * (that is by level, then by neighbour id); amax[n] receives each node's
 * largest activation level (0 for an isolated node).  Either pointer may be
 * NULL.  Host buffers, caller owned. */
int rpq_kg_export(const rpq_kg *kg, uint32_t *adj, uint8_t *amax);

/* Graph size and device bytes held by the graph and its search slots. */
int rpq_kg_info(const rpq_kg *kg, int32_t *n, int64_t *m2, int64_t *device_bytes);

/* ------------------------------------------------------------------ query */
/* One radial pattern query (Definition 1; Table 2 parameters).
 *   central, n_c   1 <= n_c <= RPQ_MAX_KEYWORDS keyword ids
 *   marginal, n_m  0 <= n_m <= RPQ_MAX_KEYWORDS keyword ids (NULL if 0)
 *   k              1 <= k <= RPQ_MAX_K results
 *   max_depth      largest Glevel L, 0 <= L <= RPQ_MAX_LEVEL (paper: 20)
 *   gamma          weight of Eq. 6, 0 <= gamma <= 1 (default 0.5)
 *   w              CG beam width (top-w CGs, Section 3.4), k <= w <= RPQ_MAX_K;
 *                  0 means w = k, the paper's setting.  With w > k the
 *                  marginal run also stops by Theorem 4 (applied exactly:
 *                  it stops once no unmatched CG can still reach a score,
 *                  node id pair ranked before the k-th RPG's, so the top-k
 *                  equals that of a run to L)
 *   score          RPQ_SCORE_SUM: S^r of Eq. 6; RPQ_SCORE_PRODUCT: the
 *                  multiplicative combination Section 3.3 allows, taken as
 *                  S^r = S^c * S^m (gamma unused).  With M empty S^r = S^c.
 * A zero-initialised tail (w = 0, score = 0) gives the paper's defaults. */
#define RPQ_SCORE_SUM     0
#define RPQ_SCORE_PRODUCT 1
typedef struct {
    const int32_t *central;
    int32_t n_c;
    const int32_t *marginal;
    int32_t n_m;
    int32_t k;
    int32_t max_depth;
    double gamma;
    int32_t w;
    int32_t score;
} rpq_query;

/* One result: the central node of the RPG (or of the CG when M is empty) and
 * its scores.  With M empty, s_m = 0 and s_r = s_c. */
typedef struct {
    int32_t node;
    int32_t s_c;
    int32_t s_m;
    int32_t reserved;
    double s_r;
} rpq_result;

/* Per-query work counters. */
typedef struct {
    int64_t e_act_central;  /* (column, edge) activations, central run */
    int64_t e_act_marginal; /* same, marginal run */
    int64_t hits_central;   /* first hits ((node, column) pairs reached, seeds excluded), central run */
    int64_t hits_marginal;
    int32_t levels_central; /* last identified Glevel of each run (-1: not run) */
    int32_t levels_marginal;
    int32_t n_cg;           /* CGs identified in the central run */
    int32_t n_selected;     /* CGs kept (top-w) */
    int64_t work_units;     /* CSR entries read by the expansions (both runs) */
    int64_t work_items;     /* (frontier node, level) expansion items */
    int64_t frontier_nodes; /* sum over levels of |Q_l| (both runs) */
    int64_t kernels;        /* kernels the query launches when replayed from its CUDA graph */
    int64_t e_act_skipped;  /* part of e_act_marginal whose expansion was skipped: the last
                               marginal level, once its V_C nodes alone decide the outcome */
} rpq_stats;

/* Search one query (Sections 3-4): central run -> top-w CGs -> recovery of
 * each CG's central keyword nodes (Algorithm 2) -> marginal run with the PTC
 * stop -> RPG identification -> Eq. 6 scores -> top-k ordered by
 * (S^r, node id).  out must hold q->k records; *n_out receives how many are
 * valid (0 when no RPG exists, e.g. a keyword without keyword nodes).  stats
 * may be NULL.  Host buffers; synchronous.  Errors: RPQ_EINVAL, RPQ_ELIMIT,
 * RPQ_ENOMEM, RPQ_ECUDA, RPQ_EINTERNAL. */
int rpq_search(rpq_kg *kg, const rpq_query *q, rpq_result *out, int32_t *n_out, rpq_stats *stats);

/* Search nq independent queries.  out holds sum(k_i) records laid out in
 * query order (query i starts at sum_{j<i} k_j); n_out[i] and status[i]
 * receive each query's result count and return code; the call returns RPQ_OK
 * when it ran (individual failures are reported in status) or an error for
 * the whole batch.  Queries run concurrently on the device, each with its own
 * search state; results equal those of rpq_search one query at a time.
 * stats may be NULL or point to nq records. */
int rpq_search_batch(rpq_kg *kg, const rpq_query *qs, int32_t nq, rpq_result *out, int32_t *n_out,
                     int32_t *status, rpq_stats *stats);

/* The same contract as rpq_search_batch, with the whole batch in one
 * persistent kernel launch fed by a device work queue: up to
 * min(batch_slots, 32) queries are in flight, each offering the chunks of
 * its current phase (run clear, seeding, each Glevel's enqueue, V_C check
 * and expansion, top-w selection, each level of the recovery sweep) to the
 * resident blocks, and a slot whose query ends takes the next query of the
 * batch on the device, with no host step between queries.  Results and
 * stats equal those of rpq_search one query at a time, except
 * stats.kernels = 0 (the batch is a single launch).  The kernel's blocks
 * never wait for each other inside a phase; a watchdog ends the launch when
 * no phase finishes for about 1 s (RPQ_BARRIER_LIMIT clock cycles): the
 * queries not finished by then get RPQ_ETIMEOUT in status and the call
 * returns RPQ_ETIMEOUT (results of finished queries are kept).  Synchronous;
 * host buffers; temporary device memory of about 3 KB per query. */
int rpq_search_batch_persistent(rpq_kg *kg, const rpq_query *qs, int32_t nq, rpq_result *out, int32_t *n_out,
                                int32_t *status, rpq_stats *stats);

/* ---------------------------------------------------------------- tracing */
/* Debug trace of one query, for comparison with a reference implementation.
 * Every pointer may be NULL; sizes are in elements.
 *   h_central    n * n_c bytes, row-major: h[v][j] = hit level of node v for
 *                central keyword j, 255 when unreached (the Node-Keyword
 *                Matrix of Section 4.2.1)
 *   h_marginal   n * n_m bytes, same for the marginal run
 *   frontier_*   concatenated frontiers Q_0, Q_1, ... of each run (each level
 *                sorted ascending) with RPQ_MAX_LEVEL + 2 offsets in *_ptr;
 *                *_levels receives the number of levels; at most *_cap
 *                entries are written
 *   cgs          all identified CGs as (node << 8 | score), ascending; up to
 *                cg_cap entries; n_cgs receives the total
 *   vc           V_C of each selected CG as (selected index << 26 | node),
 *                ascending; up to vc_cap entries; n_vc receives the total
 *   selected     top-w CG nodes ordered by (S^c, id); n_selected of them */
typedef struct {
    uint8_t *h_central;
    uint8_t *h_marginal;
    int64_t *frontier_c_ptr;
    int32_t *frontier_c;
    int64_t frontier_c_cap;
    int32_t frontier_c_levels;
    int64_t *frontier_m_ptr;
    int32_t *frontier_m;
    int64_t frontier_m_cap;
    int32_t frontier_m_levels;
    int64_t *cgs;
    int64_t cg_cap;
    int64_t n_cgs;
    int64_t *vc;
    int64_t vc_cap;
    int64_t n_vc;
    int32_t selected[RPQ_MAX_K];
    int32_t n_selected;
} rpq_trace_buf;

/* Same search as rpq_search, also filling *trace (host buffers). */
int rpq_trace(rpq_kg *kg, const rpq_query *q, rpq_result *out, int32_t *n_out, rpq_stats *stats,
              rpq_trace_buf *trace);

/* ------------------------------------------------------ result subgraphs */
/* rpq_search_subgraphs: the search of rpq_search (same results, ranks and
 * scores) that also returns each result's subgraph and checks it.
 *
 * Per result r (ranked as in `out`) three node lists and two edge lists:
 *   V^c  the CG's nodes: every node on a recovered shortest path from a
 *        central keyword node to the central node (Definition 4; recovering
 *        phase, Algorithm 2 with Lemma 3), the central node included;
 *   V_C  the nodes of V^c that hold a central keyword;
 *   V^m  the nodes of G^m = U_i SP(m_i, V_C) (Definition 5): for each
 *        marginal keyword m_i, the recovered paths of the marginal run that
 *        end at the nodes of V_C with the smallest hit level
 *        min_{v in V_C} h^M[v][i] (the two changes to Algorithm 2 for RPGs,
 *        Section 4.3), those end nodes included; empty when M is empty;
 *   E^c, E^m  the edges of the same paths as (n, q) pairs of node ids, n
 *        expanded to q (h_q = max(h_n, a_nq) + 1, and n had not stopped).
 * Each list holds every element once, in no particular order.  ptc[r] is the
 * Pass Through Constraint of Definition 5 checked on G^r = G^c U G^m taken
 * as an undirected graph: 1 holds, 0 violated, -1 when M is empty.  With
 * |M| >= 2 it holds when two distinct nodes of V^c U V^m holding different
 * marginal keywords are joined only through V_C (one of them lies in V_C, or
 * they are disconnected once the nodes of V_C are removed); with |M| = 1
 * when a node holding the marginal keyword is connected to V_C.  The search
 * itself never uses the check: it is a diagnostic of the heuristic.
 *
 * Layout of the caller-owned host buffers: list l (RPQ_SG_VC, RPQ_SG_VCKW,
 * RPQ_SG_VM) of result r is nodes[node_off[3r+l] .. node_off[3r+l+1]); edge
 * list l (RPQ_SG_EC, RPQ_SG_EM) is the pairs edges[2e], edges[2e+1] for e in
 * [edge_off[2r+l], edge_off[2r+l+1]).  nodes_cap counts int32 entries of
 * nodes, edges_cap counts pairs (edges holds 2 * edges_cap int32).  When
 * nodes_total > nodes_cap or edges_total > edges_cap the call fills out,
 * n_out, stats, the offsets, ptc and both totals, copies no list and returns
 * RPQ_ESIZE: grow the buffers and call again (the search is deterministic).
 * NULL list pointers with zero capacity are allowed for that size query.
 *
 * Synchronous, on search slot 0.  The device scratch for the lists is
 * allocated on first use and grown when a query needs more; it is released
 * with the graph.  Errors: RPQ_EINVAL, RPQ_ELIMIT, RPQ_ESIZE, RPQ_ENOMEM,
 * RPQ_ECUDA, RPQ_EINTERNAL. */
#define RPQ_SG_VC   0
#define RPQ_SG_VCKW 1
#define RPQ_SG_VM   2
#define RPQ_SG_NODE_LISTS 3
#define RPQ_SG_EC   0
#define RPQ_SG_EM   1
#define RPQ_SG_EDGE_LISTS 2

typedef struct rpq_subgraphs {
    int32_t *nodes;       /* in: host array of nodes_cap entries (may be NULL if 0) */
    int64_t nodes_cap;
    int32_t *edges;       /* in: host array of 2 * edges_cap entries */
    int64_t edges_cap;
    int64_t node_off[RPQ_MAX_K * RPQ_SG_NODE_LISTS + 1];   /* out */
    int64_t edge_off[RPQ_MAX_K * RPQ_SG_EDGE_LISTS + 1];   /* out */
    int32_t ptc[RPQ_MAX_K];                                 /* out, per result */
    int64_t nodes_total;  /* out: entries needed in nodes */
    int64_t edges_total;  /* out: pairs needed in edges */
} rpq_subgraphs;

int rpq_search_subgraphs(rpq_kg *kg, const rpq_query *q, rpq_result *out, int32_t *n_out, rpq_stats *stats,
                         rpq_subgraphs *sg);

/* ------------------------------------------------- device-resident inputs */
/* rpq_search_device: the same search with the keyword ids already in device
 * memory and the results left in device memory, enqueued on the library's
 * stream of search slot 0 without a host synchronisation.  d_keywords holds
 * n_c central ids followed by n_m marginal ids (int32, device); d_out
 * receives k rpq_result records and d_n_out one int32 (both device).  Keyword
 * ids are checked on the device: an id outside [0, n_kw) sets the slot's
 * error word, the query returns no result and rpq_sync_device reports
 * RPQ_EINVAL.  The query shape (n_c, n_m, max_depth) selects a CUDA graph
 * captured on first use and replayed for every later query of that shape. */
int rpq_search_device(rpq_kg *kg, const int32_t *d_keywords, int32_t n_c, int32_t n_m, int32_t k,
                      int32_t max_depth, double gamma, rpq_result *d_out, int32_t *d_n_out);

/* Wait for searches issued with rpq_search_device and report the first
 * device-side error since the previous call. */
int rpq_sync_device(rpq_kg *kg);

/* ---------------------------------------------------------------- tuning */
/* Work-split parameters of the search (they change timings, never results).
 *   queue_div             a level's frontier is taken from a node queue while
 *                         it holds at most n / queue_div nodes (at least 4096),
 *                         otherwise from the frontier bit map (default 32)
 *   next_queue_mult       the next level's queue is kept while the current
 *                         level's work (CSR entries) is at most
 *                         next_queue_mult x that limit (default 16)
 *   batch_slots           concurrent search slots of rpq_search_batch (8; fewer
 *                         when device memory for more is not available)
 *   flat_levels           Glevels per run replayed as plain CUDA-graph nodes;
 *                         the rest run in a WHILE node that a run stopping
 *                         earlier never enters (4; 0 = all levels in the
 *                         loop, >= max_depth + 1 = no loop) */
typedef struct {
    int32_t queue_div;
    int32_t next_queue_mult;
    int32_t batch_slots;
    int32_t flat_levels;
} rpq_tuning;

int rpq_get_tuning(const rpq_kg *kg, rpq_tuning *out);
/* Values < 1 are rejected (RPQ_EINVAL); captured CUDA graphs are rebuilt. */
int rpq_set_tuning(rpq_kg *kg, const rpq_tuning *t);
/* Autotuner: times the one-at-a-time search of the nq sample queries for each
 * queue_div in {8, 32, 128} x next_queue_mult in {4, 16, 64}, then for
 * flat_levels in {2, 3, 4, 6, 64}, then rpq_search_batch for batch_slots in
 * {4, 8, 16, 32}, keeps the fastest setting
 * (the median of `repeats` timed passes after one warm-up pass decides) and
 * returns it in *best (may be NULL).  Results are the same under every
 * setting. */
int rpq_autotune(rpq_kg *kg, const rpq_query *qs, int32_t nq, int32_t repeats, rpq_tuning *best);

/* ------------------------------------------------------------- profiling */
/* CUDA stream (a cudaStream_t) on which search slot `slot` runs its kernels;
 * slot 0 serves rpq_search, rpq_trace and rpq_search_device.  The slot is
 * created if needed.  Useful to time searches with CUDA events. */
int rpq_slot_stream(rpq_kg *kg, int32_t slot, void **stream);

/* Kernel timing.  While enabled, searches launch their kernels directly (no
 * CUDA graph) and bracket each launch with CUDA events; rpq_profile_read
 * returns the accumulated device milliseconds and launch counts per kernel
 * class and, with reset != 0, clears them.  A search writes its results from
 * the kernel that ends it (the top-w selection, or the expansion that stops
 * the marginal run), so RPQ_PROF_RESULTS stays at zero (the trace and
 * subgraph calls launch a results kernel of their own, untimed). */
enum { RPQ_PROF_SETUP = 0, RPQ_PROF_ENQUEUE, RPQ_PROF_EXPAND, RPQ_PROF_TOPK, RPQ_PROF_RECOVER,
       RPQ_PROF_RESULTS, RPQ_PROF_CLASSES };
typedef struct {
    double ms[RPQ_PROF_CLASSES];
    int64_t launches[RPQ_PROF_CLASSES];
} rpq_profile;

int rpq_set_profiling(rpq_kg *kg, int32_t enable);
int rpq_profile_read(rpq_kg *kg, rpq_profile *out, int32_t reset);

/* Per-Glevel profile of the searches run while profiling is enabled: one
 * record per (query, run, Glevel) whose level kernels ran before the run
 * stopped, in launch order, with the device times of the level's frontier
 * enqueue (Section 4.2.2-4.2.3), V_C check and expansion (Algorithm 1), and
 * the level's work: |Q_l|, the expansion's work units (CSR entries of the
 * newly active segments) and items, the (column, edge) activations it
 * executed (its share of E_act) and the (node, column) claims it wrote
 * (h = l+1; racing writers of one pair each count).  rpq_profile_levels
 * copies up to `cap` records into `out` (caller-owned), sets *n_out to the
 * number held (which may exceed cap) and, with reset != 0, clears them.
 * Without profiling *n_out = 0.  Errors: RPQ_EINVAL (NULL n_out, cap < 0,
 * NULL out with cap > 0). */
#define RPQ_LVL_EXPANDED 1   /* the expansion ran */
#define RPQ_LVL_SKIPPED  2   /* the V_C check showed the expansion cannot change the results */
#define RPQ_LVL_STOP     4   /* the run stopped at this Glevel (no expansion) */
#define RPQ_LVL_QUEUE    8   /* the enqueue read the frontier queue, not the bit map */
typedef struct {
    int32_t run;            /* 0 central, 1 marginal */
    int32_t level;          /* Glevel l */
    int32_t flags;          /* RPQ_LVL_* */
    int32_t frontier;       /* |Q_l| */
    int32_t columns;        /* keyword columns of the run (|C| or |M|) */
    int32_t reserved;
    int64_t units, items, e_act, claims;
    double enqueue_ms, target_ms, expand_ms;
} rpq_level_profile;
int rpq_profile_levels(rpq_kg *kg, rpq_level_profile *out, int32_t cap, int32_t *n_out, int32_t reset);

/* --------------------------------------------------------------- serving */
/* A server runs queries with continuous batching (the serving pattern of
 * the problem statement, Section 4.1's server-side engine).  It owns search
 * slots, each the keyword-independent device state of one in-flight query
 * (visited bytes, frontier bit maps, work lists: about 45 bytes per graph
 * node, reported as slot_bytes) with its own stream, and two pools of column
 * pages: Node-Keyword Matrix pages (one byte per node: one hit-level column)
 * and recovery pages (12 bytes per node: the CG masks and node list of one
 * central column in Algorithm 2).  A query is admitted by its own hit-table
 * memory: it needs a free slot, max(|C|, |M|) matrix pages and |C| recovery
 * pages, which it holds until it completes; a query that does not fit waits,
 * and waiting queries are admitted in arrival order.  Queries in different
 * slots run concurrently on the device.  Each query runs the same kernels as
 * rpq_search, so its results equal those of rpq_search.
 *
 * rpq_server_create sizes the server from budget_bytes (checked before any
 * allocation): slots of slot_bytes with 6 matrix pages each and recovery
 * pages with the rest (at most 8 per slot), i.e. sized for queries of about
 * 4 central and 6 columns on average; at least one slot and 8 pages of each
 * kind are always created (every query fits), at most max_slots slots.
 * rpq_server_create_sized takes the counts directly (n_slots in [1, 4096],
 * pages in [8, 2^20]).  Errors: RPQ_EINVAL, RPQ_ENOMEM, RPQ_ECUDA. */
typedef struct rpq_server rpq_server;

typedef struct {
    uint64_t tag;                  /* the tag given at submit (replay: query index) */
    int32_t status;                /* RPQ_OK or the query's error */
    int32_t n_res;
    rpq_result res[RPQ_MAX_K];
    rpq_stats stats;
    double latency_s;              /* submit (or scheduled arrival) to completion */
} rpq_completion;

int rpq_server_create(rpq_kg *kg, int64_t budget_bytes, int32_t max_slots, rpq_server **out);
int rpq_server_create_sized(rpq_kg *kg, int32_t n_slots, int32_t h_pages, int32_t r_pages, rpq_server **out);
int rpq_server_info(const rpq_server *srv, int32_t *n_slots, int64_t *slot_bytes, int32_t *n_running,
                    int32_t *n_waiting);
/* Page pools of a server and the most queries it has had running at once.
 * Any output pointer may be NULL. */
int rpq_server_pages(const rpq_server *srv, int32_t *h_pages, int64_t *h_page_bytes, int32_t *r_pages,
                     int64_t *r_page_bytes, int32_t *peak_running);
/* Validate and enqueue one query (copied); admits it at once when a slot is
 * free.  Never waits for the device.  A query whose start fails completes
 * with that error as its status (its pages return to the pools, the queries
 * behind it are admitted as usual).  For tests of that path, the environment
 * variable RPQ_INJECT_START_FAILURE=k (read when the server is created) makes
 * the server's k-th query start fail on the host, before any launch. */
int rpq_server_submit(rpq_server *srv, const rpq_query *q, uint64_t tag);
/* Collect finished queries into out (up to max_done), admitting waiting ones
 * into freed slots.  wait != 0 blocks until at least one query has finished
 * (returns at once when nothing is running or waiting). */
int rpq_server_poll(rpq_server *srv, rpq_completion *out, int32_t max_done, int32_t *n_done, int32_t wait);
/* Serve an arrival schedule natively: query i is submitted at arrival_s[i]
 * seconds after the call starts (non-decreasing times).  latency_s[i] counts
 * from the scheduled arrival to completion; status[i], n_out[i] and (if out is
 * non-NULL) the results, laid out as in rpq_search_batch, are filled in;
 * *wall_s receives the elapsed time.  The server must be idle when the call
 * starts (every query submitted before has been polled), else RPQ_EINVAL. */
int rpq_server_replay(rpq_server *srv, const rpq_query *qs, const double *arrival_s, int32_t nq,
                      double *latency_s, int32_t *status, int32_t *n_out, rpq_result *out, double *wall_s);
/* Wait for running queries and release every slot of the server. */
int rpq_server_destroy(rpq_server *srv);

/* --------------------------------------------- selection without allocation */
/* rpq_topk_keys_noalloc: write the k smallest of n 32-bit keys, ascending, to
 * d_out and their count (min(k, n)) to *d_n_out.  The paper has no
 * counterpart; this is a service for callers that cannot allocate device
 * memory when they need a selection, e.g. code running while another
 * component captures a CUDA graph, or a serving loop whose device memory is
 * entirely held by a pre-planned pool.  It runs the same block-local top-K
 * merge as the search's CG selection, with its intermediate buffers in a
 * fixed device array compiled into the library (about 1.04 MB, held on every
 * GPU that loads the library until the process exits), and calls no
 * allocating routine.
 *   d_keys    n keys in device memory, each < 0xffffffff (that value pads)
 *   n         0 <= n <= 16,777,216 (2^24); larger inputs return RPQ_ELIMIT
 *   k         1 <= k <= RPQ_MAX_K
 *   d_out     k uint32 slots in device memory; d_n_out one uint32 (device)
 *   stream    cudaStream_t to enqueue on (NULL = legacy default stream); the
 *             call returns without waiting
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture that should contain later calls.  All calls on a device share the
 * one array: calls whose work overlaps on the GPU (different streams without
 * ordering, or several host threads) race and give wrong results.  Errors:
 * RPQ_EINVAL (NULL pointer, k out of range), RPQ_ELIMIT, RPQ_ECUDA. */
int rpq_topk_keys_noalloc(const uint32_t *d_keys, uint32_t n, int32_t k, uint32_t *d_out, uint32_t *d_n_out,
                          void *stream);

/* Host <-> device bytes of one rpq_search call with k results: *h2d is the
 * query record the launch carries (keyword ids and parameters), *d2h the one
 * copy that returns the control block with the results.  Either pointer may
 * be NULL.  Errors: RPQ_EINVAL (k out of range). */
int rpq_transfer_bytes(int32_t k, int64_t *h2d, int64_t *d2h);

/* -------------------------------------------------------------- messages */
const char *rpq_strerror(int code);
const char *rpq_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RPQ_H */
