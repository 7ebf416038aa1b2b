"""The oracle on a prepared graph (transpose built once, searches from several
threads at once, trace and result subgraphs optional) gives exactly what the
one-call form gives: the same results, CG sets, V_C, counts and levels, and
with the trace on the same hit levels and frontiers."""
import numpy as np

import oracle
import rpqgen
from tests.gpu_common import dataset_queries


def _same(a, b, trace, subgraphs):
    assert a.status == b.status
    assert a.nodes.tolist() == b.nodes.tolist()
    assert a.s_c.tolist() == b.s_c.tolist() and a.s_m.tolist() == b.s_m.tolist()
    assert a.s_r.tobytes() == b.s_r.tobytes()
    assert a.cg_node.tolist() == b.cg_node.tolist() and a.cg_score.tolist() == b.cg_score.tolist()
    assert a.selected.tolist() == b.selected.tolist()
    assert [x.tolist() for x in a.vc_kw] == [x.tolist() for x in b.vc_kw]
    assert [x.tolist() for x in a.ec] == [x.tolist() for x in b.ec]
    assert a.matched.tolist() == b.matched.tolist() and a.sel_sm.tolist() == b.sel_sm.tolist()
    for ra, rb in ((a.central, b.central), (a.marginal, b.marginal)):
        assert (ra is None) == (rb is None)
        if ra is None:
            continue
        assert (ra.last_level, ra.last_expanded, ra.e_act, ra.new_hits) == \
            (rb.last_level, rb.last_expanded, rb.e_act, rb.new_hits)
        if trace:
            assert np.array_equal(ra.h, rb.h) and np.array_equal(ra.stop, rb.stop)
            assert len(ra.frontiers) == len(rb.frontiers)
            assert all(np.array_equal(x, y) for x, y in zip(ra.frontiers, rb.frontiers))
    if subgraphs:
        assert [x.tolist() for x in a.vm] == [x.tolist() for x in b.vm]
        assert [x.tolist() for x in a.em] == [x.tolist() for x in b.em]
        assert a.ptc.tolist() == b.ptc.tolist()


def test_prepared_graph_equals_one_call(tiny_ds, tiny_act):
    qs = dataset_queries("tiny", tiny_ds, 10, seed=41)
    ref = [oracle.search(tiny_ds, tiny_act.a, q.central, q.marginal, q.k, q.max_depth, q.gamma) for q in qs]
    pg = oracle.PreparedGraph(tiny_ds, tiny_act.a)
    try:
        for q, r in zip(qs, ref):
            got = oracle.search(None, None, q.central, q.marginal, q.k, q.max_depth, q.gamma, prepared=pg)
            _same(got, r, True, True)
        # hit-level tables without the frontier lists
        for q, r in zip(qs[:3], ref):
            got = oracle.search(None, None, q.central, q.marginal, q.k, q.max_depth, q.gamma, prepared=pg,
                                trace=False, subgraphs=False, tables=True)
            _same(got, r, False, False)
            for ra, rb in ((got.central, r.central), (got.marginal, r.marginal)):
                if ra is not None:
                    assert ra.frontiers is None
                    assert np.array_equal(ra.h, rb.h) and np.array_equal(ra.stop, rb.stop)
        # several threads on one prepared graph, counts only
        many = oracle.search_many(pg, qs, threads=4)
        for got, r in zip(many, ref):
            _same(got, r, False, False)
            assert got.central is None or got.central.h is None
            assert got.vm is None and got.ptc is None
    finally:
        pg.close()


def test_activation_without_detail(tiny_ds, tiny_act):
    act = oracle.dataset_activation(tiny_ds, detail=False)
    assert np.array_equal(act.a, tiny_act.a) and np.array_equal(act.amax, tiny_act.amax)
    assert act.cnt is None and act.w is None and act.x is None


def test_prepared_graph_variants():
    """Beam width, product score, shuffled orders and disabled stops pass
    through the prepared form unchanged."""
    ds = rpqgen.make_dataset("tiny")
    act = oracle.dataset_activation(ds, detail=False)
    pg = oracle.PreparedGraph(ds, act.a)
    try:
        for q in dataset_queries("tiny", ds, 4, seed=43):
            for kw in (dict(w=min(64, q.k + 7)), dict(product=True), dict(shuffle_seed=9),
                       dict(disable_stops=True), dict(exhaustive_marginal=True)):
                r = oracle.search(ds, act.a, q.central, q.marginal, q.k, q.max_depth, q.gamma, **kw)
                got = oracle.search(None, None, q.central, q.marginal, q.k, q.max_depth, q.gamma, prepared=pg, **kw)
                _same(got, r, True, True)
    finally:
        pg.close()
