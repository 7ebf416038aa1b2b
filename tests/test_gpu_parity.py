"""GPU parity: the CUDA library against the CPU oracle (bit-exact hit levels,
frontiers, CG sets, top-w, V_C, top-k ids and integer scores; S^r within 1e-6
relative), on seeded synthetic knowledge graphs that span many tiles and a
ragged tail, plus edge cases.  Every call goes through the C ABI."""
import numpy as np
import pytest

import oracle
import paper_2001_06770_b300 as rpq
import rpqgen
from tests import brute
from tests.gpu_common import dataset_queries, oracle_query, results_match, trace_matches

pytestmark = pytest.mark.gpu

DATASETS = ["tiny", "small", "cl_small", "mid"]


@pytest.fixture(scope="module", params=DATASETS)
def bundle(request):
    ds = rpqgen.make_dataset(request.param)
    act = oracle.dataset_activation(ds)
    kg = rpq.KG.from_dataset(ds)
    yield request.param, ds, act, kg
    kg.close()


def test_activation_levels_bit_exact(bundle):
    """Device activation build (Section 3.1, Eq. 1-3) equals the oracle: every
    row holds (a << 26 | neighbour) sorted ascending, and amax matches."""
    name, ds, act, kg = bundle
    g = ds.graph
    adj, amax = kg.export()
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    expect = (act.a.astype(np.uint32) << 26) | g.col.astype(np.uint32)
    order = np.lexsort((expect, src))       # sort within each row
    assert np.array_equal(adj, expect[order])
    assert np.array_equal(amax, act.amax)


def test_trace_parity(bundle):
    name, ds, act, kg = bundle
    n = {"tiny": 8, "small": 8, "cl_small": 6, "mid": 4}[name]
    for q in dataset_queries(name, ds, n) + (rpqgen.workload_queries("tiny", ds) if name == "tiny" else []):
        orc = oracle_query(ds, act, q)
        tr = kg.trace(q.central, q.marginal, q.k, q.max_depth, q.gamma)
        trace_matches(tr, orc)


def test_search_matches_trace_and_oracle(bundle):
    """The graph-replayed search path gives the same results and counters."""
    name, ds, act, kg = bundle
    for q in dataset_queries(name, ds, 6, seed=11):
        orc = oracle_query(ds, act, q)
        res, st = kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)
        results_match(res, orc)
        if orc.central is not None:
            assert st["e_act_central"] == orc.central.e_act
            assert st["levels_central"] == orc.central.last_level
        if orc.marginal is not None:
            # E_act and the stop level stay exact when the V_C check skips the
            # last expansion and the last enqueue only counts the frontier
            assert st["e_act_marginal"] == orc.marginal.e_act
            assert st["levels_marginal"] == orc.marginal.last_level


def test_batch_equals_one_at_a_time(bundle):
    name, ds, act, kg = bundle
    qs = dataset_queries(name, ds, 12, seed=5)
    batch = kg.search_batch(qs)
    for q, (res, st, status) in zip(qs, batch):
        assert status == 0
        one, st1 = kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)
        assert res.tobytes() == one.tobytes()
        # the launch count depends on the launch mode (under RPQ_PERSISTENT=1
        # slot 0 runs each level loop as one persistent kernel, batch slots
        # never do), so only the search statistics must agree
        st.pop("kernels"), st1.pop("kernels")
        assert st == st1


def test_device_resident_path(bundle):
    import torch
    name, ds, act, kg = bundle
    for q in dataset_queries(name, ds, 4, seed=17):
        kw = torch.tensor(list(q.central) + list(q.marginal), dtype=torch.int32, device="cuda")
        out = torch.zeros(q.k * 24, dtype=torch.uint8, device="cuda")
        nout = torch.zeros(1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        kg.search_device(kw.data_ptr(), len(q.central), len(q.marginal), q.k, q.max_depth, q.gamma,
                         out.data_ptr(), nout.data_ptr())
        kg.sync_device()
        got = np.frombuffer(out.cpu().numpy().tobytes(), rpq.RESULT_DTYPE)[:int(nout.item())]
        host, _ = kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)
        assert got.tobytes() == host.tobytes()


# ------------------------------------------------------------------ edge cases
@pytest.fixture(scope="module")
def tiny():
    ds = rpqgen.make_dataset("tiny")
    act = oracle.dataset_activation(ds)
    kg = rpq.KG.from_dataset(ds)
    yield ds, act, kg
    kg.close()


@pytest.mark.parametrize("k,L", [(1, 6), (64, 6), (10, 0), (10, 1), (20, 12), (5, 63)])
def test_k_and_depth_extremes(tiny, k, L):
    ds, act, kg = tiny
    q = rpqgen.Query(central=[124, 464], marginal=[375, 63], k=k, max_depth=L)
    orc = oracle_query(ds, act, q)
    trace_matches(kg.trace(q.central, q.marginal, k, L), orc)
    # graph-replayed search: flat graph for L <= 12, WHILE-loop graph beyond
    res, st = kg.search(q.central, q.marginal, k, L)
    results_match(res, orc)
    assert st["e_act_central"] == orc.central.e_act


@pytest.mark.parametrize("C,M", [([30], []), ([124], [375]), ([124, 464, 124], [375]), ([124, 464], [375, 375]),
                                 ([1, 2, 3, 4, 5, 6, 7, 8], [9, 10, 11, 12, 13, 14, 15, 16]), ([0, 1], [2])])
def test_query_shapes(tiny, C, M):
    ds, act, kg = tiny
    q = rpqgen.Query(central=C, marginal=M, k=10, max_depth=6)
    trace_matches(kg.trace(C, M, 10, 6), oracle_query(ds, act, q))


def test_gamma_values(tiny):
    ds, act, kg = tiny
    for gamma in (0.0, 0.3, 1.0):
        q = rpqgen.Query(central=[124, 464], marginal=[375, 63], k=10, max_depth=6, gamma=gamma)
        res, _ = kg.search(q.central, q.marginal, q.k, q.max_depth, gamma)
        results_match(res, oracle_query(ds, act, q))


def test_empty_postings_and_invalid_queries(tiny):
    ds, act, kg = tiny
    sizes = np.diff(ds.kw_ptr)
    empty = int(np.nonzero(sizes == 0)[0][0]) if (sizes == 0).any() else None
    if empty is not None:
        assert len(kg.search([124, empty], [375], 10, 6)[0]) == 0
        assert len(kg.search([124, 464], [empty], 10, 6)[0]) == 0
    for bad in [dict(central=[], marginal=[1]), dict(central=[ds.n_kw], marginal=[]),
                dict(central=[1], marginal=[-1]), dict(central=[1], marginal=[], k=0),
                dict(central=[1], marginal=[], k=65), dict(central=[1], marginal=[], max_depth=64),
                dict(central=list(range(9)), marginal=[])]:
        args = dict(k=10, max_depth=6)
        args.update(bad)
        with pytest.raises(rpq.RPQError) as ei:
            kg.search(args["central"], args["marginal"], args["k"], args["max_depth"])
        assert ei.value.code == rpq.RPQ_EINVAL


def test_device_keyword_out_of_range_reported(tiny):
    import torch
    ds, act, kg = tiny
    kw = torch.tensor([124, ds.n_kw + 5], dtype=torch.int32, device="cuda")
    out = torch.zeros(10 * 24, dtype=torch.uint8, device="cuda")
    nout = torch.zeros(1, dtype=torch.int32, device="cuda")
    kg.search_device(kw.data_ptr(), 2, 0, 10, 6, 0.5, out.data_ptr(), nout.data_ptr())
    with pytest.raises(rpq.RPQError) as ei:
        kg.sync_device()
    assert ei.value.code == rpq.RPQ_EINVAL
    kg.sync_device()      # the error is reported once


@pytest.mark.parametrize("seed", range(12))
def test_random_small_graphs(seed):
    """<= 20-node graphs with few labels (so activation levels vary), isolated
    nodes and keyword nodes everywhere."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(6, 21))
    g = brute.small_graph(rng, n, int(rng.integers(n - 2, 2 * n)), n_labels=3)
    sets = [list(rng.choice(n, size=int(rng.integers(1, 3)), replace=False)) for _ in range(6)]
    kp, kn = brute.postings_from_sets(6, sets)
    abar = float(rng.uniform(1.0, 3.5))
    act = oracle.activation(g.row_ptr, g.col, g.label, g.n_labels, 0.5, abar)
    kg = rpq.KG(g.row_ptr, g.col, g.label, g.n_labels, kp, kn, 0.5, abar)
    try:
        adj, amax = kg.export()
        assert np.array_equal(amax, act.amax)
        for C, M, k in [([0, 1], [2, 3], 2), ([0], [1], 1), ([0, 1, 2], [], 3), ([3, 4], [5], 4)]:
            orc = oracle.search(g, act.a, C, M, k, 6, kw_ptr=kp, kw_nodes=kn)
            trace_matches(kg.trace(C, M, k, 6), orc)
    finally:
        kg.close()


def test_graph_rejected_on_device():
    """Asymmetric edges and unsorted rows are caught by the device checks."""
    kp = np.array([0, 1], np.int64)
    kn = np.array([0], np.int32)
    # 0->1 without 1->0
    with pytest.raises(rpq.RPQError) as ei:
        rpq.KG(np.array([0, 1, 1], np.int64), np.array([1], np.int32), np.zeros(1, np.uint16), 1, kp, kn)
    assert ei.value.code == rpq.RPQ_EINVAL
    # label mismatch between directions
    with pytest.raises(rpq.RPQError):
        rpq.KG(np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32), np.array([0, 1], np.uint16), 2, kp, kn)
    # unsorted row
    with pytest.raises(rpq.RPQError):
        rpq.KG(np.array([0, 2, 3, 4], np.int64), np.array([2, 1, 0, 0], np.int32), np.zeros(4, np.uint16), 1, kp, kn)


def test_graph_without_edges():
    kp = np.array([0, 1, 2], np.int64)
    kn = np.array([0, 1], np.int32)
    kg = rpq.KG(np.zeros(4, np.int64), np.zeros(0, np.int32), np.zeros(0, np.uint16), 1, kp, kn)
    try:
        res, st = kg.search([0, 1], [], 5, 4)
        assert len(res) == 0
        res, st = kg.search([0], [], 5, 4)
        assert res["node"].tolist() == [0] and res["s_c"].tolist() == [0]
    finally:
        kg.close()


@pytest.mark.parametrize("alpha", [0.2, 0.8])
def test_alpha_sweep(alpha):
    """Other values of the scaling parameter alpha (Eq. 1-2; Section 5.2 sweeps
    it): activation levels and results still equal the oracle's."""
    ds = rpqgen.make_dataset("small")
    g = ds.graph
    act = oracle.activation(g.row_ptr, g.col, g.label, g.n_labels, alpha, ds.abar)
    kg = rpq.KG(g.row_ptr, g.col, g.label, g.n_labels, ds.kw_ptr, ds.kw_nodes, alpha, ds.abar)
    try:
        adj, amax = kg.export()
        assert np.array_equal(amax, act.amax)
        src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
        expect = (act.a.astype(np.uint32) << 26) | g.col.astype(np.uint32)
        assert np.array_equal(adj, expect[np.lexsort((expect, src))])
        for q in dataset_queries("small", ds, 5, seed=61):
            orc = oracle.search(ds, act.a, q.central, q.marginal, q.k, q.max_depth, q.gamma)
            trace_matches(kg.trace(q.central, q.marginal, q.k, q.max_depth, q.gamma), orc)
    finally:
        kg.close()


def test_hub_rows_longer_than_the_16bit_level_index():
    """Two hubs with 100k and 70k neighbours (rows beyond 2^16 entries, whose
    level boundaries come from the 32-bit hub index) plus a sparse random
    graph; 8 Zipf labels spread the hubs' edges over several activation
    levels.  Keywords sit on hub neighbours and on random nodes."""
    n = 150_000
    rng = np.random.default_rng(7)
    src = np.concatenate([np.zeros(99_999, np.uint32), np.ones(70_000, np.uint32),
                          rng.integers(0, n, 300_000).astype(np.uint32)])
    dst = np.concatenate([np.arange(1, 100_000, dtype=np.uint32), np.arange(2, 70_002, dtype=np.uint32),
                          rng.integers(0, n, 300_000).astype(np.uint32)])
    g = rpqgen.build_graph(n, src, dst, seed=7, n_labels=8, permute=False)
    deg = np.diff(g.row_ptr)
    assert deg[0] > 65535 and deg[1] > 65535
    sets = [rng.choice(n, size=int(rng.integers(3, 40)), replace=False).tolist() for _ in range(8)]
    sets[0] += [5, 70_500]
    sets[1] += [99_000]
    kp, kn = brute.postings_from_sets(8, sets)
    abar = 3.0
    act = oracle.activation(g.row_ptr, g.col, g.label, g.n_labels, 0.5, abar)
    kg = rpq.KG(g.row_ptr, g.col, g.label, g.n_labels, kp, kn, 0.5, abar)
    try:
        adj, amax = kg.export()
        assert np.array_equal(amax, act.amax)
        # depth 12 also takes the binary search above the indexed levels 1..8
        for C, M, k, L in [([0, 1], [2, 3], 5, 8), ([0, 1, 2], [4], 10, 8), ([3], [5, 6], 3, 8),
                           ([4, 5], [6, 7, 0], 20, 8), ([0, 6], [1, 7], 20, 12), ([2, 3, 4], [5], 40, 12)]:
            orc = oracle.search(g, act.a, C, M, k, L, kw_ptr=kp, kw_nodes=kn)
            trace_matches(kg.trace(C, M, k, L), orc)
            res, _ = kg.search(C, M, k, L)
            results_match(res, orc)
    finally:
        kg.close()
