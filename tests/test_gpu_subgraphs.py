"""GPU parity of the result subgraphs (Definition 5; Algorithm 2 with Lemma 3
and the RPG recovery of Section 4.3) and of the PTC check: for every result
the device lists V^c, V_C, V^m, E^c, E^m equal the oracle's as sets (the
library gives no order), and the PTC flag is identical.  Calls go through
rpq_search_subgraphs in the C ABI."""
import numpy as np
import pytest

import oracle
import paper_2001_06770_b300 as rpq
import rpqgen
from tests import brute
from tests.gpu_common import dataset_queries, oracle_query, results_match

pytestmark = pytest.mark.gpu


def entry_pairs(g, entries):
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    return sorted([int(src[e]), int(g.col[e])] for e in entries)


def rows(a):
    return sorted(map(list, np.asarray(a).reshape(-1, 2).tolist()))


def subgraphs_match(g, res, subs, orc):
    """Device subgraphs of each ranked result equal the oracle's for the same CG."""
    results_match(res, orc)
    pos = {int(v): i for i, v in enumerate(orc.selected)}
    assert len(subs) == len(res)
    ptcs = []
    for r, sub in enumerate(subs):
        gi = pos[int(res["node"][r])]
        assert sorted(sub["vc"].tolist()) == orc.vc_all[gi].tolist(), f"V^c of result {r}"
        assert sorted(sub["vc_kw"].tolist()) == orc.vc_kw[gi].tolist(), f"V_C of result {r}"
        assert rows(sub["ec"]) == entry_pairs(g, orc.ec[gi]), f"E^c of result {r}"
        assert sorted(sub["vm"].tolist()) == orc.vm[gi].tolist(), f"V^m of result {r}"
        assert rows(sub["em"]) == entry_pairs(g, orc.em[gi]), f"E^m of result {r}"
        assert sub["ptc"] == int(orc.ptc[gi]), f"PTC of result {r}"
        # every list holds each element once
        for key in ("vc", "vc_kw", "vm"):
            assert len(np.unique(sub[key])) == len(sub[key])
        ptcs.append(sub["ptc"])
    return ptcs


@pytest.fixture(scope="module", params=["tiny", "small", "cl_small", "mid"])
def bundle(request):
    ds = rpqgen.make_dataset(request.param)
    act = oracle.dataset_activation(ds)
    kg = rpq.KG.from_dataset(ds)
    yield request.param, ds, act, kg
    kg.close()


def test_subgraphs_match_oracle(bundle):
    name, ds, act, kg = bundle
    n = {"tiny": 8, "small": 8, "cl_small": 8, "mid": 4}[name]
    for q in dataset_queries(name, ds, n, seed=23):
        res, st, subs = kg.search_subgraphs(q.central, q.marginal, q.k, q.max_depth, q.gamma)
        subgraphs_match(ds.graph, res, subs, oracle_query(ds, act, q))
        # the same ranked results and counters as the plain search
        one, st1 = kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)
        assert res.tobytes() == one.tobytes()
        st.pop("kernels"), st1.pop("kernels")
        assert st == st1


def test_ptc_violations_found(bundle):
    """Queries with three and four marginal keywords on the power-law graph
    give RPGs that break the PTC; the device flags the same ones."""
    name, ds, act, kg = bundle
    if name != "cl_small":
        pytest.skip("violations are searched for on the Chung-Lu graph")
    seen = set()
    for q in dataset_queries(name, ds, 16, seed=3):
        res, _, subs = kg.search_subgraphs(q.central, q.marginal, q.k, q.max_depth, q.gamma)
        seen.update(subgraphs_match(ds.graph, res, subs, oracle_query(ds, act, q)))
    assert {0, 1, -1} <= seen


def test_small_buffers_grow():
    """A first call with too small buffers reports RPQ_ESIZE with the sizes;
    the binding grows them and repeats the (deterministic) search."""
    ds = rpqgen.make_dataset("tiny")
    act = oracle.dataset_activation(ds)
    kg = rpq.KG.from_dataset(ds)
    try:
        q = rpqgen.Query(central=[124, 464], marginal=[375, 63], k=10, max_depth=6)
        res, _, subs = kg.search_subgraphs(q.central, q.marginal, q.k, q.max_depth, nodes_cap=1, edges_cap=0)
        subgraphs_match(ds.graph, res, subs, oracle_query(ds, act, q))
        assert sum(len(s["vm"]) for s in subs) > 1
    finally:
        kg.close()


@pytest.mark.parametrize("seed", range(10))
def test_random_small_graphs(seed):
    """<= 20-node graphs with three labels: few activation levels, so stop
    rules and ties between start nodes of V_C are frequent."""
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(8, 21))
    g = brute.small_graph(rng, n, int(rng.integers(n, 2 * n)), n_labels=3)
    sets = [list(rng.choice(n, size=int(rng.integers(1, 4)), replace=False)) for _ in range(6)]
    kp, kn = brute.postings_from_sets(6, sets)
    act = oracle.activation(g.row_ptr, g.col, g.label, g.n_labels, 0.5, 2.5)
    kg = rpq.KG(g.row_ptr, g.col, g.label, g.n_labels, kp, kn, 0.5, 2.5)
    try:
        for C, M, k in [([0, 1], [2, 3], 3), ([0], [1], 2), ([0, 1], [], 3), ([3, 4], [5, 2, 1], 4)]:
            orc = oracle.search(g, act.a, C, M, k, 6, kw_ptr=kp, kw_nodes=kn)
            res, _, subs = kg.search_subgraphs(C, M, k, 6)
            subgraphs_match(g, res, subs, orc)
    finally:
        kg.close()


def test_medium_sampled_queries():
    """The full-size synthetic graph (2^21 nodes): sampled queries of the
    measured workload, subgraphs and PTC against the oracle."""
    ds = rpqgen.make_dataset("medium")
    act = oracle.dataset_activation(ds)
    kg = rpq.KG.from_dataset(ds)
    try:
        qs = rpqgen.workload_queries("medium", ds)
        for i in (0, 2):
            q = qs[i]
            res, _, subs = kg.search_subgraphs(q.central, q.marginal, q.k, q.max_depth, q.gamma)
            subgraphs_match(ds.graph, res, subs, oracle_query(ds, act, q))
    finally:
        kg.close()
