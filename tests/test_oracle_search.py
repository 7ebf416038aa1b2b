"""Pins for the oracle's search (Section 4, Algorithms 1-2, Theorems 3, 5, 6, Lemma 3, Eq. 4-6).

Every check compares the oracle with something other than itself: hand-derived
golden micro-graphs, an independent bottleneck Dijkstra (Theorem 5), a textbook
BFS (all levels 0), a fixed-point formulation of the stop rules, brute-force
path enumeration on graphs of at most 20 nodes, and order shuffles (Theorem 6).
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import oracle
from tests import brute

INF = 255
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden_graph(n, edges, postings):
    g = brute.csr_from_undirected(n, [(u, v) for u, v, _ in edges])
    lv = {(min(u, v), max(u, v)): a for u, v, a in edges}
    a = np.zeros(g.m2, np.uint8)
    for u, v, e in g.edges():
        a[e] = lv[(min(u, v), max(u, v))]
    kw_ptr, kw_nodes = brute.postings_from_sets(len(postings), postings)
    return g, a, kw_ptr, kw_nodes


def run(g, a, kw_ptr, kw_nodes, C, M, k, L, **kw):
    return oracle.search(g, a, C, M, k, L, kw_ptr=kw_ptr, kw_nodes=kw_nodes, **kw)


def result_rows(r):
    return [[int(r.nodes[i]), int(r.s_c[i]), int(r.s_m[i]), float(r.s_r[i])] for i in range(len(r.nodes))]


# ------------------------------------------------------------------ golden
def test_golden_path8():
    fx = json.load(open(os.path.join(GOLDEN, "search_path8.json")))
    g, a, kp, kn = golden_graph(fx["n"], fx["edges"], fx["postings"])
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    for case in fx["cases"]:
        r = run(g, a, kp, kn, case["central"], case["marginal"], case["k"], case["L"])
        assert r.status == 0
        assert result_rows(r) == case["results"]
        if "h_central" in case:
            assert r.central.h.tolist() == case["h_central"]
        if "frontiers_central" in case:
            assert [f.tolist() for f in r.central.frontiers] == case["frontiers_central"]
        if "cgs" in case:
            assert [[int(x), int(s)] for x, s in zip(r.cg_node, r.cg_score)] == case["cgs"]
        if "vc_all" in case:
            assert r.vc_all[0].tolist() == case["vc_all"]
            assert r.vc_kw[0].tolist() == case["vc_kw"]
            assert sorted([int(src[e]), int(g.col[e])] for e in r.ec[0]) == sorted(case["ec_pairs"])
        if "h_marginal" in case:
            assert r.marginal.h.tolist() == case["h_marginal"]
            assert [f.tolist() for f in r.marginal.frontiers] == case["frontiers_marginal"]


def test_golden_ptc():
    fx = json.load(open(os.path.join(GOLDEN, "search_ptc.json")))
    for case in fx["cases"]:
        g, a, kp, kn = golden_graph(case["n"], case["edges"], case["postings"])
        r = run(g, a, kp, kn, case["central"], case["marginal"], case["k"], case["L"])
        assert [[int(x), int(s)] for x, s in zip(r.cg_node, r.cg_score)] == case["cgs"]
        assert r.vc_kw[0].tolist() == case["vc_kw"]
        assert result_rows(r) == case["results"]
        if "results_without_ptc" in case:
            r2 = run(g, a, kp, kn, case["central"], case["marginal"], case["k"], case["L"], disable_stops=True)
            assert result_rows(r2) == case["results_without_ptc"]


# ------------------------------------------------------- random small graphs
def random_case(seed, n=None, m=None, n_kw=6, amax=4):
    rng = np.random.default_rng(seed)
    n = n or int(rng.integers(6, 21))
    m = m or int(rng.integers(n, min(2 * n, n * (n - 1) // 2) + 1))
    g = brute.small_graph(rng, n, m)
    a = brute.random_levels_symmetric(g, rng, amax)
    sets = [list(rng.choice(n, size=int(rng.integers(1, 3)), replace=False)) for _ in range(n_kw)]
    kp, kn = brute.postings_from_sets(n_kw, sets)
    return rng, g, a, kp, kn, sets


@pytest.mark.parametrize("seed", range(40))
def test_theorem5_dijkstra_and_path_enumeration(seed):
    """With the stop rules off, h[v][j] = D(t_j, v) (Theorem 5) for every v
    with D <= L; checked against Dijkstra and against simple-path enumeration."""
    rng, g, a, kp, kn, sets = random_case(seed)
    L = int(rng.integers(2, 9))
    C = [0, 1, 2]
    r = run(g, a, kp, kn, C, [], 3, L, disable_stops=True)
    for j, kw in enumerate(C):
        d1 = brute.bottleneck_dijkstra(g, a, sets[kw], L)
        d2 = brute.path_enum_distance(g, a, sets[kw], L)
        assert (d1 == d2).all()
        assert (r.central.h[:, j].astype(np.int64) == d1).all(), (j, r.central.h[:, j], d1)


def test_theorem5_tiny_workload(tiny_ds, tiny_act):
    g = tiny_ds.graph
    C = [120, 377, 40]
    r = oracle.search(tiny_ds, tiny_act.a, C, [], 10, 7, disable_stops=True)
    for j, kw in enumerate(C):
        d = brute.bottleneck_dijkstra(g, tiny_act.a, tiny_ds.postings(kw), 7)
        assert (r.central.h[:, j].astype(np.int64) == d).all()


def test_all_zero_levels_is_textbook_bfs(tiny_ds):
    """All a = 0 reduces the path score to hop count: h is BFS distance."""
    g = tiny_ds.graph
    a0 = np.zeros(g.m2, np.uint8)
    A = sp.csr_matrix((np.ones(g.m2), g.col, g.row_ptr), shape=(g.n, g.n))
    C = [60, 200]
    r = oracle.search(tiny_ds, a0, C, [], 5, 12, disable_stops=True)
    for j, kw in enumerate(C):
        d = csg.shortest_path(A, method="D", unweighted=True, indices=tiny_ds.postings(kw)).min(axis=0)
        d = np.where(np.isfinite(d) & (d <= 12), d, INF).astype(np.int64)
        assert (r.central.h[:, j].astype(np.int64) == d).all()


@pytest.mark.parametrize("seed", range(40))
def test_fixed_point_with_stop_rules(seed):
    """The level loop with the central stop rule equals the fixed point of the
    simultaneous equations; likewise the marginal run with the PTC stop."""
    rng, g, a, kp, kn, sets = random_case(seed, amax=3)
    L = int(rng.integers(3, 9))
    k = int(rng.integers(1, 4))
    C, M = [0, 1], [2, 3]
    r = run(g, a, kp, kn, C, M, k, L)
    rc = r.central
    fp = brute.fixed_point(g, a, [sets[c] for c in C], rc.last_expanded, stop_rule=True)
    assert (rc.h.astype(np.int64) == fp).all()
    # the run ended at the first level with >= w CGs, else at L or an empty frontier
    fin = (fp != INF).all(axis=1)
    lev = np.where(fin, fp.max(axis=1), 10 ** 9)
    cnt_at = [int((lev <= x).sum()) for x in range(L + 1)]
    if rc.last_level < L and cnt_at[rc.last_level] >= k:
        assert rc.last_level == 0 or cnt_at[rc.last_level - 1] < k
    # the CG set is every node with all columns finite, with score max_j h (Theorem 3)
    assert sorted(r.cg_node.tolist()) == sorted(np.nonzero(fin)[0].tolist())
    assert all(int(s) == int(lev[v]) for v, s in zip(r.cg_node, r.cg_score))
    assert all(int(s) == int(l) for s, l in zip(r.cg_score, r.cg_level))
    if r.marginal is not None:
        rm = r.marginal
        fpm = brute.fixed_point(g, a, [sets[c] for c in M], rm.last_expanded, stop_rule=True)
        assert (rm.h.astype(np.int64) == fpm).all()


@pytest.mark.parametrize("seed", range(30))
def test_brute_force_first_level(seed):
    """Brute force on <= 20 nodes: the CGs found first are exactly the nodes
    minimising max_j D(c_j, v) (no stop has acted yet), their V^c is the set of
    nodes on prefix-shortest paths (Lemma 3), and with one marginal keyword the
    RPG score is max over... of min_{v in V_C} D(m, v) (Definition 5, Eq. 5-6)."""
    rng, g, a, kp, kn, sets = random_case(seed, amax=3)
    L = 8
    C, M = [0, 1], [2]
    D = {kw: brute.path_enum_distance(g, a, sets[kw], L) for kw in C + M}
    maxc = np.maximum(D[0], D[1])
    fin = (D[0] != INF) & (D[1] != INF)
    if not fin.any():
        r = run(g, a, kp, kn, C, M, 1, L)
        assert len(r.cg_node) == 0 and len(r.nodes) == 0
        return
    smin = int(maxc[fin].min())
    first = sorted(np.nonzero(fin & (maxc == smin))[0].tolist())
    k = len(first)
    r = run(g, a, kp, kn, C, M, k, L)
    assert r.selected.tolist() == first
    assert (r.selected_sc == smin).all()
    for gi, vc in enumerate(first):
        expect = {vc}
        for kw in C:
            expect |= brute.prefix_optimal_nodes(g, a, sets[kw], vc, D[kw])
        assert r.vc_all[gi].tolist() == sorted(expect)
        vck = sorted(v for v in expect if v in set(sets[0]) | set(sets[1]))
        assert r.vc_kw[gi].tolist() == vck
        dm = min(int(D[2][v]) for v in vck)
        if dm != INF:
            assert r.matched[gi] == 1 and r.sel_sm[gi] == dm
        else:
            assert r.matched[gi] == 0
    # results: matched CGs ranked by (S^r, id), S^r = 0.5 S^c + 0.5 S^m
    rows = sorted((0.5 * smin + 0.5 * int(r.sel_sm[i]), first[i]) for i in range(k) if r.matched[i])
    assert [int(x) for x in r.nodes] == [v for _, v in rows]
    assert r.s_r.tolist() == [s for s, _ in rows]
    # multiplicative S^r = S^c * S^m with the brute-force distances
    rp = run(g, a, kp, kn, C, M, k, L, product=True)
    dms = {vc: min(int(D[2][v]) for v in sorted(v for v in set(r.vc_kw[gi].tolist()))) for gi, vc in enumerate(first)}
    rows = sorted((smin * dms[v], v) for v in first if dms[v] != INF)
    assert [int(x) for x in rp.nodes] == [v for _, v in rows]
    assert rp.s_r.tolist() == [float(s) for s, _ in rows]


@pytest.mark.parametrize("seed", range(20))
def test_theorem6_order_independence(seed):
    """Shuffling frontier and neighbour processing order changes nothing."""
    rng, g, a, kp, kn, sets = random_case(seed, amax=3)
    base = run(g, a, kp, kn, [0, 1], [2, 3], 2, 7)
    for s in (1, 2, 3):
        r = run(g, a, kp, kn, [0, 1], [2, 3], 2, 7, shuffle_seed=1000 * seed + s)
        assert (r.central.h == base.central.h).all()
        assert result_rows(r) == result_rows(base)
        assert [f.tolist() for f in r.central.frontiers] == [f.tolist() for f in base.central.frontiers]
        if base.marginal is not None:
            assert (r.marginal.h == base.marginal.h).all()


def test_theorem6_tiny_workload(tiny_ds, tiny_act):
    q = dict(central=[124, 464], marginal=[375, 63], k=10, max_depth=6)
    base = oracle.search(tiny_ds, tiny_act.a, **q)
    r = oracle.search(tiny_ds, tiny_act.a, **q, shuffle_seed=77)
    assert (r.central.h == base.central.h).all() and (r.marginal.h == base.marginal.h).all()
    assert result_rows(r) == result_rows(base)


def test_lemma3_recovered_edges_are_tight(tiny_ds, tiny_act):
    g = tiny_ds.graph
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    C = [124, 464, 300]
    r = oracle.search(tiny_ds, tiny_act.a, C, [], 10, 6)
    h, stop = r.central.h.astype(int), r.central.stop.astype(int)
    for gi in range(len(r.selected)):
        nodes = set(r.vc_all[gi].tolist())
        for e in r.ec[gi]:
            u, v = int(src[e]), int(g.col[e])
            assert u in nodes and v in nodes
            ok = False
            for j in range(len(C)):
                if h[u, j] != INF and h[v, j] == max(h[u, j], int(tiny_act.a[e])) + 1:
                    ok |= max(h[u, j], int(tiny_act.a[e])) < stop[u]
            assert ok


def test_frontier_rule_invariant(tiny_ds, tiny_act):
    """Derived from Algorithm 1: Q_{l+1} = {nodes first hit at l} U {v in Q_l not
    stopped whose largest out-edge level exceeds l}."""
    q = dict(central=[124, 464], marginal=[375, 63], k=10, max_depth=6)
    r = oracle.search(tiny_ds, tiny_act.a, **q)
    for run_ in (r.central, r.marginal):
        h, stop = run_.h.astype(int), run_.stop.astype(int)
        newly = {l: set() for l in range(8)}
        for v in range(h.shape[0]):
            for j in range(h.shape[1]):
                if 0 < h[v, j] != INF:
                    newly[h[v, j] - 1].add(v)
        for l in range(len(run_.frontiers) - 1):
            ql = run_.frontiers[l].tolist()
            kept = {v for v in ql if stop[v] > l and tiny_act.amax[v] > l}
            assert set(run_.frontiers[l + 1].tolist()) == newly[l] | kept


# ------------------------------------------------------------- special cases
def test_single_central_keyword_no_marginal(tiny_ds, tiny_act):
    """|C| = 1, M empty: the central nodes are the keyword nodes, score 0."""
    kw = 30
    post = tiny_ds.postings(kw)
    r = oracle.search(tiny_ds, tiny_act.a, [kw], [], len(post) + 5, 6)
    assert sorted(r.cg_node.tolist()) == sorted(post.tolist())
    assert (r.cg_score == 0).all() and r.central.last_level == 0 or len(post) < len(post) + 5
    assert r.nodes.tolist() == sorted(post.tolist())
    assert (r.s_c == 0).all() and (r.s_r == 0).all()


def test_node_with_all_central_keywords():
    """A node holding every central keyword is a CG at level 0 with V^c = {v}."""
    g, a, kp, kn = golden_graph(4, [[0, 1, 0], [1, 2, 0], [2, 3, 0]], [[1, 3], [1], [0]])
    r = run(g, a, kp, kn, [0, 1], [2], 1, 4)
    assert r.cg_node.tolist() == [1] and r.cg_score.tolist() == [0]
    assert r.vc_all[0].tolist() == [1] and r.vc_kw[0].tolist() == [1]
    assert result_rows(r) == [[1, 0, 1, 0.5]]


def test_inactive_edges_never_used():
    """Edges with a > L-1 are never expanded: nothing beyond the seeds is hit."""
    rng, g, a, kp, kn, sets = random_case(5)
    L = 4
    a_hi = np.full_like(a, L)
    r = run(g, a_hi, kp, kn, [0, 1], [2], 3, L)
    for j, kw in enumerate([0, 1]):
        hit = set(np.nonzero(r.central.h[:, j] != INF)[0].tolist())
        assert hit == set(int(x) for x in sets[kw])
    assert r.central.e_act == 0


def test_empty_postings_give_no_result():
    g, a, kp, kn = golden_graph(3, [[0, 1, 0], [1, 2, 0]], [[0], [], [2]])
    assert len(run(g, a, kp, kn, [0, 1], [], 2, 4).nodes) == 0
    assert len(run(g, a, kp, kn, [0, 2], [1], 2, 4).nodes) == 0
    assert len(run(g, a, kp, kn, [0, 2], [], 2, 4).nodes) == 1


def test_invalid_queries_rejected():
    g, a, kp, kn = golden_graph(3, [[0, 1, 0], [1, 2, 0]], [[0], [1], [2]])
    assert run(g, a, kp, kn, [], [0], 1, 4).status != 0
    assert run(g, a, kp, kn, [5], [], 1, 4).status != 0
    assert run(g, a, kp, kn, [0], [], 0, 4).status != 0


@pytest.mark.parametrize("seed", range(15))
def test_marginal_early_stop_equals_exhaustive(seed):
    """With w = k, stopping once every selected CG is matched gives the same
    top-k as running the marginal run to L (Theorem 4 with w = k)."""
    rng, g, a, kp, kn, sets = random_case(seed, amax=3)
    r1 = run(g, a, kp, kn, [0, 1], [2, 3, 4], 3, 7)
    r2 = run(g, a, kp, kn, [0, 1], [2, 3, 4], 3, 7, exhaustive_marginal=True)
    assert result_rows(r1) == result_rows(r2)


@pytest.mark.parametrize("product", [False, True])
@pytest.mark.parametrize("gamma", [0.5, 0.3, 1.0, 0.0])
def test_theorem4_beam_wider_than_k(gamma, product):
    """k < w: the marginal run may stop by Theorem 4 before every selected CG
    is matched; the top-k it returns equals (a) the top-k of an exhaustive
    marginal run and (b) the first k results of the same query with k = w
    (every matched RPG, ranked).  The stop does fire on some queries."""
    fired = 0
    for seed in range(60):
        rng, g, a, kp, kn, sets = random_case(2000 + seed, amax=2)
        C, M = [0, 1], ([2, 3] if seed % 3 else [2])
        k, w = int(rng.integers(1, 3)), int(rng.integers(3, 6))
        r = run(g, a, kp, kn, C, M, k, 7, gamma=gamma, w=w, product=product)
        ex = run(g, a, kp, kn, C, M, k, 7, gamma=gamma, w=w, product=product, exhaustive_marginal=True)
        full = run(g, a, kp, kn, C, M, w, 7, gamma=gamma, w=w, product=product, exhaustive_marginal=True)
        assert result_rows(r) == result_rows(ex)
        assert result_rows(r) == result_rows(full)[:k]
        assert r.selected.tolist() == full.selected.tolist()        # the CG stage depends on w only
        if r.marginal is not None and not r.matched.all() and r.marginal.last_level < ex.marginal.last_level:
            fired += 1
    assert fired > 0


def test_product_score_ranks_by_product(tiny_ds, tiny_act):
    """Multiplicative S^r = S^c * S^m: the same RPGs as Eq. 6, ranked by the
    product of their integer scores, ties by node id."""
    q = dict(central=[124, 464], marginal=[375, 63], k=10, max_depth=6)
    add = oracle.search(tiny_ds, tiny_act.a, **q)
    mul = oracle.search(tiny_ds, tiny_act.a, **q, product=True)
    rows = sorted((int(c) * int(m), int(v), int(c), int(m)) for v, c, m in zip(add.nodes, add.s_c, add.s_m))
    assert [[v, c, m, float(p)] for p, v, c, m in rows] == result_rows(mul)


def test_duplicate_keywords_are_identical_columns(tiny_ds, tiny_act):
    """A repeated central keyword is an identical column and changes nothing.
    A repeated marginal keyword counts towards |M|: with |M| >= 2 the PTC stop
    applies, and every node reached by the keyword is reached by 'all' marginal
    columns at once, so nothing expands beyond the keyword nodes."""
    r1 = oracle.search(tiny_ds, tiny_act.a, [124, 464], [375], 10, 6)
    r2 = oracle.search(tiny_ds, tiny_act.a, [124, 464, 124], [375], 10, 6)
    assert (r2.central.h[:, 2] == r2.central.h[:, 0]).all()
    assert result_rows(r1) == result_rows(r2)
    r3 = oracle.search(tiny_ds, tiny_act.a, [124, 464], [375, 375], 10, 6)
    hit = np.nonzero(r3.marginal.h[:, 0] != INF)[0]
    assert sorted(hit.tolist()) == sorted(tiny_ds.postings(375).tolist())


def test_e_act_counts_rescan_free_work(tiny_ds, tiny_act):
    """E_act counts each (column, edge) once at level max(h, a); it is bounded
    by columns x CSR entries and equals the count recomputed from H."""
    g = tiny_ds.graph
    r = oracle.search(tiny_ds, tiny_act.a, [124, 464], [375, 63], 10, 6)
    rc = r.central
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    total = 0
    for j in range(rc.h.shape[1]):
        hv = rc.h[src, j].astype(int)
        lam = np.maximum(hv, tiny_act.a.astype(int))
        total += int(((hv != INF) & (lam <= rc.last_expanded) & (lam < rc.stop[src].astype(int))).sum())
    assert total == rc.e_act <= rc.h.shape[1] * g.m2


def test_golden_recovery_stop_guard():
    """An edge that is tight in H but leaves a node that had already stopped
    expanding is not an expansion edge (Lemma 3) and is not recovered."""
    fx = json.load(open(os.path.join(GOLDEN, "search_stop_guard.json")))
    g, a, kp, kn = golden_graph(fx["n"], fx["edges"], fx["postings"])
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    r = run(g, a, kp, kn, fx["central"], fx["marginal"], fx["k"], fx["L"])
    assert [[int(x), int(s)] for x, s in zip(r.cg_node, r.cg_score)] == fx["cgs"]
    assert [v.tolist() for v in r.vc_all] == fx["vc_all"]
    for gi, pairs in enumerate(fx["ec_pairs"]):
        assert sorted([int(src[e]), int(g.col[e])] for e in r.ec[gi]) == sorted(pairs)
    assert result_rows(r) == fx["results"]


# ------------------------------------------------------ result subgraphs
def pairs_of(g, entries):
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    return sorted([int(src[e]), int(g.col[e])] for e in entries)


def test_golden_subgraphs_and_ptc():
    """Hand-derived RPGs: V^c/E^c, G^m (Section 4.3 start nodes, several start
    nodes at an equal minimum) and the PTC check, held and violated."""
    fx = json.load(open(os.path.join(GOLDEN, "search_subgraphs.json")))
    for case in fx["cases"]:
        g, a, kp, kn = golden_graph(case["n"], case["edges"], case["postings"])
        r = run(g, a, kp, kn, case["central"], case["marginal"], case["k"], case["L"])
        assert result_rows(r) == case["results"], case["name"]
        assert r.vc_all[0].tolist() == case["vc_all"]
        assert pairs_of(g, r.ec[0]) == case["ec_pairs"]
        assert r.vc_kw[0].tolist() == case["vc_kw"]
        assert r.vm[0].tolist() == case["vm"]
        assert pairs_of(g, r.em[0]) == case["em_pairs"]
        assert int(r.ptc[0]) == case["ptc"]


def holders_of(sets, M, nodes):
    out = {}
    for i, kw in enumerate(M):
        for v in sets[kw]:
            if int(v) in nodes:
                out.setdefault(int(v), set()).add(i)
    return out


def check_rpg_parts_brute(g, a, sets, r, M, L):
    """G^m of each matched CG equals the union of the expansion paths from each
    marginal keyword to the nodes of V_C at its smallest hit level, found by
    forward path enumeration over the hit levels of an independent fixed point
    (|M| >= 2, PTC stop) or of simple-path distances (|M| = 1, no stop); the
    PTC flag equals simple-path enumeration of Definition 5.  Returns the
    PTC flags of the matched CGs."""
    rm = r.marginal
    if rm is None:
        return []
    if len(M) >= 2:
        h = brute.fixed_point(g, a, [sets[m] for m in M], rm.last_expanded, stop_rule=True)
        fin = (h != INF).all(axis=1)
        stop = np.where(fin, h.max(axis=1), 10 ** 9)
    else:
        h = brute.path_enum_distance(g, a, sets[M[0]], L)[:, None]
        stop = None
    flags = []
    for gi in range(len(r.selected)):
        if not r.matched[gi]:
            assert len(r.vm[gi]) == 0 and int(r.ptc[gi]) == -1
            continue
        vck = [int(v) for v in r.vc_kw[gi]]
        nodes, steps = set(), set()
        for i, kw in enumerate(M):
            d = min(int(h[v, i]) for v in vck)
            assert d != INF
            tg = [v for v in vck if int(h[v, i]) == d]
            nd, st = brute.recovered_paths(g, a, h[:, i], stop, sets[kw], tg)
            nodes |= nd | set(tg)
            steps |= st
        assert r.vm[gi].tolist() == sorted(nodes)
        assert pairs_of(g, r.em[gi]) == sorted([u, v] for u, v in steps)
        vr = set(r.vc_all[gi].tolist()) | nodes
        er = [tuple(p) for p in pairs_of(g, r.ec[gi])] + sorted(steps)
        flag = brute.ptc_by_paths(len(M), er, vck, holders_of(sets, M, vr))
        assert int(r.ptc[gi]) == flag
        flags.append(flag)
    return flags


@pytest.mark.parametrize("seed", range(40))
def test_marginal_recovery_and_ptc_brute_force(seed):
    rng, g, a, kp, kn, sets = random_case(seed, amax=3)
    L = int(rng.integers(3, 9))
    k = int(rng.integers(1, 4))
    M = [2, 3] if seed % 2 == 0 else [2]
    check_rpg_parts_brute(g, a, sets, run(g, a, kp, kn, [0, 1], M, k, L), M, L)


def test_ptc_brute_force_with_violations():
    """Seeds and shapes (|M| = 2, 3; few activation levels) where some RPGs
    violate the PTC: both outcomes occur and agree with path enumeration."""
    seen = set()
    for seed in range(1000, 1100):
        rng, g, a, kp, kn, sets = random_case(seed, amax=2)
        M = [2, 3, 4] if seed % 2 else [2, 3]
        seen.update(check_rpg_parts_brute(g, a, sets, run(g, a, kp, kn, [0, 1], M, 3, 6), M, 6))
    assert seen == {0, 1}


def test_no_marginal_keywords_gives_no_rpg_parts(tiny_ds, tiny_act):
    r = oracle.search(tiny_ds, tiny_act.a, [124, 464], [], 5, 6)
    assert len(r.selected) > 0
    assert all(len(x) == 0 for x in r.vm) and (r.ptc == -1).all()
