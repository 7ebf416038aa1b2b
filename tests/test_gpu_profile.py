"""Kernel profiling (rpq_set_profiling, rpq_profile_levels): the per-Glevel
records of each query add up to its own statistics - work units, items,
frontier sizes, executed activations - list every level of each run in
order with the stop level last, carry the run's column count and the level
kernels' device times, and profiling changes no result."""
import pytest

import oracle
import paper_2001_06770_b300 as rpq
import rpqgen
from tests.gpu_common import dataset_queries, oracle_query, results_match

pytestmark = pytest.mark.gpu


def test_level_records_add_up_to_the_query_statistics():
    ds = rpqgen.make_dataset("cl_small")
    act = oracle.dataset_activation(ds)
    kg = rpq.KG.from_dataset(ds)
    try:
        qs = dataset_queries("cl_small", ds, 8, seed=71)
        kg.set_profiling(True)
        kg.profile_levels(reset=True)
        seen_levels = 0
        for q in qs:
            res, st = kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)
            recs = kg.profile_levels(reset=True)
            results_match(res, oracle_query(ds, act, q))
            if st["levels_central"] < 0:            # a keyword without keyword nodes: no device work
                assert recs == []
                continue
            assert sum(r["units"] for r in recs) == st["work_units"]
            assert sum(r["items"] for r in recs) == st["work_items"]
            assert sum(r["frontier"] for r in recs) == st["frontier_nodes"]
            assert sum(r["e_act"] for r in recs) == \
                st["e_act_central"] + st["e_act_marginal"] - st["e_act_skipped"]
            for run, cols in ((0, len(q.central)), (1, len(q.marginal))):
                mine = [r for r in recs if r["run"] == run]
                assert [r["level"] for r in mine] == list(range(len(mine)))
                if mine:
                    assert mine[-1]["flags"] & rpq.LVL_STOP
                    assert all(not (r["flags"] & rpq.LVL_STOP) for r in mine[:-1])
                    assert all(r["columns"] == cols for r in mine)
                    assert all(r["enqueue_ms"] > 0 and r["expand_ms"] > 0 for r in mine)
                    seen_levels += len(mine)
            # only an expanded level has work; a stop or skipped level has none
            assert all(r["units"] == 0 for r in recs if not (r["flags"] & rpq.LVL_EXPANDED))
            assert all(r["flags"] & rpq.LVL_EXPANDED for r in recs if r["units"] > 0)
        assert seen_levels > 0
        # the per-class totals count the same launches
        prof = kg.profile(reset=True)
        assert prof["expand"][1] > 0 and prof["enqueue"][1] > 0
    finally:
        kg.set_profiling(False)
        kg.close()
