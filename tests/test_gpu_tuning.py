"""Work-split tuning changes timings, never results: extreme queue
thresholds, next-queue bounds, batch slot counts and graph forms give the
oracle's results; the autotuner returns a valid setting."""
import pytest

import oracle
import paper_2001_06770_b300 as rpq
import rpqgen
from tests.gpu_common import dataset_queries, oracle_query, results_match

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    ds = rpqgen.make_dataset("small")
    act = oracle.dataset_activation(ds)
    kg = rpq.KG.from_dataset(ds)
    qs = dataset_queries("small", ds, 10, seed=51)
    orc = [oracle_query(ds, act, q) for q in qs]
    yield ds, kg, qs, orc
    kg.close()


@pytest.mark.parametrize("tune", [dict(queue_div=1, next_queue_mult=1000), dict(queue_div=1 << 30, next_queue_mult=1),
                                  dict(queue_div=4, next_queue_mult=1), dict(flat_levels=0), dict(flat_levels=2), dict(flat_levels=64),
                                  dict(batch_slots=1), dict(batch_slots=16)])
def test_results_do_not_depend_on_tuning(small, tune):
    ds, kg, qs, orc = small
    default = kg.tuning()
    try:
        kg.set_tuning(**tune)
        for q, o in zip(qs, orc):
            res, st = kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)
            results_match(res, o)
            if o.central is not None:
                assert st["e_act_central"] == o.central.e_act
        for (res, st, status), o in zip(kg.search_batch(qs), orc):
            assert status == 0
            results_match(res, o)
    finally:
        kg.set_tuning(**default)


def test_autotune(small):
    ds, kg, qs, orc = small
    t = kg.autotune(qs[:6], repeats=1)
    assert t["queue_div"] in (8, 32, 128) and t["next_queue_mult"] in (4, 16, 64)
    assert t["batch_slots"] in (4, 8, 16, 32) and t["flat_levels"] in (2, 3, 4, 6, 64)
    assert kg.tuning() == t
    for q, o in zip(qs, orc):
        results_match(kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)[0], o)
    with pytest.raises(rpq.RPQError):
        kg.set_tuning(queue_div=0)
