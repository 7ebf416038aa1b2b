"""Full-size checks on the large workload (Chung-Lu, 5e7 nodes, 7.6e8 CSR
entries, queries of 3 + 3 keywords, k = 20, L = 8, and the batched
workload's uneven shapes with head and tail keywords on the same graph).

Against the oracle (its own activation levels and a graph prepared once;
about half a minute of one host core per query, the sampled queries run in
parallel): two queries of the one-at-a-time workload element by element -
results, both runs' hit-level tables, the CG set, the selected CGs, V_C of
each, E_act and the stop levels - and two queries of the batched mix, one
with the most head keywords (postings over 10^5 nodes, rows of the hub
level index) and one of tail keywords only, by results, E_act and levels
through the one-at-a-time, batched and traced paths.

Properties that hold at any size, on the device's own trace, plus equality
between the search paths:

* hit levels (Theorem 5 with the stop rules): a sampled node's level h > 0 has
  a parent u with max(h_u, a) + 1 = h that had not stopped, no neighbour
  offers a smaller level, an unreached node has no neighbour that expanded to
  it, and h = 0 exactly on keyword nodes;
* Theorem 3: the CG set is every node whose central columns are all finite,
  with S^c = max h; the selected CGs are the w smallest by (S^c, node id);
* Eq. 6 and Definition 6: scores and the (S^r, id) order of the results;
* the graph-replayed search, the trace and the batch give the same results.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
import paper_2001_06770_b300 as rpq
import rpqgen
from tests.gpu_common import INF, check_levels, results_match

pytestmark = pytest.mark.gpu

HEAD_MIN = 100_000    # postings of a head keyword in the batched workload

@pytest.fixture(scope="module")
def large():
    ds = rpqgen.make_dataset("large")
    kg = rpq.KG.from_dataset(ds)
    adj, amax = kg.export()
    yield ds, kg, adj, rpqgen.workload_queries("large", ds)
    kg.close()


def test_large_trace_properties(large):
    ds, kg, adj, qs = large
    g = ds.graph
    q = qs[0]
    tr = kg.trace(q.central, q.marginal, q.k, q.max_depth, q.gamma)
    rng = np.random.default_rng(5)
    Hc = tr["h_central"]
    nc = Hc.shape[1]
    # Theorem 3: CGs = nodes with every central column finite, S^c = max h
    fin = (Hc != INF).all(axis=1)
    cg = {int(x) >> 8: int(x) & 0xff for x in tr["cgs"]}
    assert set(cg) == set(np.nonzero(fin)[0].tolist())
    for v, sc in list(cg.items())[:5000]:
        assert sc == int(Hc[v].max())
    # central stop levels: a CG stops at its identification level
    stop = np.full(g.n, 10 ** 9, np.int64)
    for v, sc in cg.items():
        stop[v] = sc
    # expansions ran up to one below the deepest level reached (a last
    # expansion that reached nothing is then simply not checked)
    check_levels(g, adj, Hc, stop, int(Hc[Hc != INF].max()) - 1, [ds.postings(k) for k in q.central], rng)
    # top-w selection
    order = sorted(cg.items(), key=lambda kv: (kv[1], kv[0]))[:q.k]
    assert tr["selected"].tolist() == [v for v, _ in order]
    # marginal run: PTC stop (|M| >= 2) at the level a node holds every marginal column
    Hm = tr["h_marginal"]
    if Hm is not None and len(q.marginal) >= 2:
        finm = (Hm != INF).all(axis=1)
        stopm = np.where(finm, Hm.max(axis=1).astype(np.int64), 10 ** 9)
        check_levels(g, adj, Hm, stopm, int(Hm[Hm != INF].max()) - 1, [ds.postings(k) for k in q.marginal], rng)
    # results: Eq. 6 and the (S^r, id) order
    res = tr["results"]
    sr = q.gamma * res["s_c"] + (1 - q.gamma) * res["s_m"]
    assert np.allclose(res["s_r"], sr, rtol=1e-12)
    keys = list(zip(res["s_r"].tolist(), res["node"].tolist()))
    assert keys == sorted(keys)


def test_large_paths_agree(large):
    """One-at-a-time queries and the mixed shapes of the batched workload
    (|C| 2-6, |M| 0-8, head and tail keywords, k in {5, 10, 20})."""
    ds, kg, adj, qs = large
    sample = [qs[i] for i in (0, 1, 2, 3)] + rpqgen.workload_queries("batched", ds)[:6]
    batch = kg.search_batch(sample)
    for q, (bres, _, status) in zip(sample, batch):
        assert status == 0
        res, st = kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)
        assert res.tobytes() == bres.tobytes()
    tr = kg.trace(sample[1].central, sample[1].marginal, sample[1].k, sample[1].max_depth, sample[1].gamma)
    res, _ = kg.search(sample[1].central, sample[1].marginal, sample[1].k, sample[1].max_depth, sample[1].gamma)
    assert res.tobytes() == tr["results"].tobytes()


def mixed_pair(ds):
    """From the first 400 queries of the batched workload: the one with the
    most head keywords (marginal keywords included) and one with tail keywords
    only, both with marginal keywords."""
    sizes = np.diff(ds.kw_ptr)
    mq = rpqgen.workload_queries("batched", ds)[:400]
    heads = [sum(int(sizes[k] > HEAD_MIN) for k in q.central + q.marginal) for q in mq]
    cand = [i for i in range(len(mq)) if mq[i].marginal]
    heavy = max(cand, key=lambda i: (heads[i], len(mq[i].central) + len(mq[i].marginal), -i))
    tail = next(i for i in cand if heads[i] == 0)
    return mq[heavy], mq[tail], heads[heavy]


@pytest.fixture(scope="module")
def large_oracle(large):
    """The oracle's answers for two one-at-a-time queries (with both runs'
    hit-level tables) and the two batched-mix queries, computed in parallel."""
    ds, kg, adj, qs = large
    act = oracle.dataset_activation(ds, detail=False)
    pg = oracle.PreparedGraph(ds, act.a)
    heavy, tail, nhead = mixed_pair(ds)
    jobs = [(qs[0], True), (qs[1], True), (heavy, False), (tail, False)]

    def one(job):
        q, tables = job
        return oracle.search(None, None, q.central, q.marginal, q.k, q.max_depth, q.gamma, prepared=pg,
                             trace=False, subgraphs=False, tables=tables)

    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        out = list(ex.map(one, jobs))
    pg.close()
    del act
    yield [q for q, _ in jobs], out, nhead


def test_large_trace_equals_oracle(large, large_oracle):
    """One-at-a-time queries of the large workload, element by element."""
    ds, kg, adj, qs = large
    queries, orcs, _ = large_oracle
    for q, orc in zip(queries[:2], orcs[:2]):
        tr = kg.trace(q.central, q.marginal, q.k, q.max_depth, q.gamma)
        results_match(tr["results"], orc)
        assert np.array_equal(tr["h_central"], orc.central.h), "central hit levels differ"
        gcg = sorted((int(x) >> 8, int(x) & 0xff) for x in tr["cgs"])
        assert gcg == sorted(zip(orc.cg_node.tolist(), orc.cg_score.tolist())), "CG sets differ"
        assert tr["selected"].tolist() == orc.selected.tolist()
        st = tr["stats"]
        assert st["e_act_central"] == orc.central.e_act
        assert st["levels_central"] == orc.central.last_level
        if orc.marginal is not None:
            for g in range(len(orc.selected)):
                assert tr["vc"][g].tolist() == orc.vc_kw[g].tolist(), f"V_C of CG {g} differs"
            assert np.array_equal(tr["h_marginal"], orc.marginal.h), "marginal hit levels differ"
            assert st["e_act_marginal"] == orc.marginal.e_act
            assert st["levels_marginal"] == orc.marginal.last_level
        # the graph-replayed search (it may skip the final marginal expansion)
        res, st1 = kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)
        results_match(res, orc)
        assert st1["e_act_central"] == orc.central.e_act
        if orc.marginal is not None:
            assert st1["e_act_marginal"] == orc.marginal.e_act


def test_large_mixed_shapes_equal_oracle(large, large_oracle):
    """Batched-mix queries (a head-heavy one reaching hub rows from posting
    lists of 10^5+ nodes, and a tail one): results, E_act and levels through
    the one-at-a-time, batched and persistent-batch paths."""
    ds, kg, adj, qs = large
    queries, orcs, nhead = large_oracle
    assert nhead >= 2
    batch = kg.search_batch(queries[2:])
    pers = kg.search_batch(queries[2:], persistent=True)
    for q, orc, (bres, bst, status), (pres, pst, pstatus) in zip(queries[2:], orcs[2:], batch, pers):
        assert status == 0 and pstatus == 0
        res, st = kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)
        results_match(res, orc)
        results_match(bres, orc)
        results_match(pres, orc)
        assert st["e_act_central"] == orc.central.e_act == bst["e_act_central"] == pst["e_act_central"]
        assert st["levels_central"] == orc.central.last_level == pst["levels_central"]
        if orc.marginal is not None:
            assert st["e_act_marginal"] == orc.marginal.e_act == bst["e_act_marginal"] == pst["e_act_marginal"]
            assert st["levels_marginal"] == orc.marginal.last_level == pst["levels_marginal"]
