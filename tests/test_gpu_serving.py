"""Serving with continuous batching: queries submitted while others run are
admitted as slots free up, run concurrently, and each result equals the same
query run alone (rpq_search) - bit for bit, S^r included."""
import numpy as np
import pytest

import paper_2001_06770_b300 as rpq
import rpqgen
from tests.gpu_common import dataset_queries

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served():
    ds = rpqgen.make_dataset("small")
    kg = rpq.KG.from_dataset(ds)
    qs = dataset_queries("small", ds, 24, seed=21)
    alone = [kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)[0] for q in qs]
    yield ds, kg, qs, alone
    kg.close()


def test_submit_poll_mix_equals_alone(served):
    ds, kg, qs, alone = served
    slot_bytes = None
    srv = rpq.Server(kg, budget_bytes=1, max_slots=4)      # budget 1 byte: exactly one slot
    try:
        assert srv.info()["slots"] == 1
        slot_bytes = srv.info()["slot_bytes"]
    finally:
        srv.close()
    srv = rpq.Server(kg, budget_bytes=4 * slot_bytes, max_slots=64)
    try:
        assert srv.info()["slots"] == 4                     # admission by search-state memory
        got = {}
        for i, q in enumerate(qs):
            srv.submit(q, i)
            for tag, status, res, st, lat in srv.poll():
                got[tag] = (status, res)
        assert srv.info()["waiting"] >= 0
        while len(got) < len(qs):
            for tag, status, res, st, lat in srv.poll(wait=True):
                got[tag] = (status, res)
        for i in range(len(qs)):
            status, res = got[i]
            assert status == 0
            assert res.tobytes() == alone[i].tobytes(), i
    finally:
        srv.close()


def test_replay_poisson_mix_equals_alone(served):
    ds, kg, qs, alone = served
    srv = rpq.Server(kg, budget_bytes=1 << 40, max_slots=6)
    try:
        arrivals = rpqgen.poisson_arrivals(len(qs), 20000.0, seed=3)   # faster than service: queries overlap
        res, lat, status, wall = srv.replay(qs, arrivals)
        assert (status == 0).all()
        assert (lat > 0).all() and wall > 0
        for i in range(len(qs)):
            assert res[i].tobytes() == alone[i].tobytes(), i
        # the same queries, now in a different mix (reversed order, 2 slots)
        srv2 = rpq.Server(kg, budget_bytes=1 << 40, max_slots=2)
        try:
            res2, _, status2, _ = srv2.replay(qs[::-1], np.zeros(len(qs)))
            assert (status2 == 0).all()
            for i, r in enumerate(res2[::-1]):
                assert r.tobytes() == alone[i].tobytes()
        finally:
            srv2.close()
    finally:
        srv.close()


def test_server_rejects_bad_queries(served):
    ds, kg, qs, alone = served
    srv = rpq.Server(kg, budget_bytes=1 << 40, max_slots=2)
    try:
        with pytest.raises(rpq.RPQError):
            srv.submit(rpqgen.Query(central=[], marginal=[], k=5, max_depth=4), 1)
        with pytest.raises(rpq.RPQError):
            srv.replay([qs[0], qs[1]], np.array([1.0, 0.5]))      # decreasing arrivals
    finally:
        srv.close()
