"""Serving with continuous batching: queries submitted while others run are
admitted as slots free up, run concurrently, and each result equals the same
query run alone (rpq_search) - bit for bit, S^r included - and, for the
served workload's mix on the medium graph, the oracle's."""
import numpy as np
import pytest

import oracle
import paper_2001_06770_b300 as rpq
import rpqgen
from tests.gpu_common import dataset_queries, results_match

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
    srv = rpq.Server(kg, budget_bytes=1, max_slots=4)      # budget 1 byte: the minimum server
    try:
        info = srv.info()
        assert info["slots"] == 1 and info["h_pages"] == 8 and info["r_pages"] == 8
    finally:
        srv.close()
    srv = rpq.Server(kg, slots=4, h_pages=32, r_pages=32)
    try:
        assert srv.info()["slots"] == 4
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


def test_admission_by_column_pages(served):
    """Queries of 4 central keywords on a server with 6 slots but recovery
    pages for only two of them at a time: at most two run at once, the rest
    wait for pages, and every result equals the query run alone."""
    ds, kg, _, _ = served
    qs = rpqgen.queries_uniform(16, (4, 4), (0, 3), (20, 800), 10, 6, seed=61)
    alone = [kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)[0] for q in qs]
    srv = rpq.Server(kg, slots=6, h_pages=64, r_pages=8)
    try:
        res, lat, status, wall = srv.replay(qs, np.zeros(len(qs)))
        info = srv.info()
        assert (status == 0).all()
        assert 1 <= info["peak_running"] <= 2
        for i in range(len(qs)):
            assert res[i].tobytes() == alone[i].tobytes(), i
    finally:
        srv.close()
    # budget sizing: a budget with room for more slots than the fixed 8-column
    # worst case would allow, and at least 8 pages of each kind
    srv = rpq.Server(kg, budget_bytes=2 << 30, max_slots=256)
    try:
        info = srv.info()
        worst = info["slot_bytes"] + 8 * info["h_page_bytes"] + 8 * info["r_page_bytes"]
        assert info["slots"] > (2 << 30) // worst
        assert info["device_bytes"] <= (2 << 30)
        assert info["h_pages"] >= 8 and info["r_pages"] >= 8
    finally:
        srv.close()


def test_replay_poisson_mix_equals_alone(served):
    ds, kg, qs, alone = served
    srv = rpq.Server(kg, budget_bytes=1 << 33, max_slots=6)
    try:
        arrivals = rpqgen.poisson_arrivals(len(qs), 20000.0, seed=3)   # faster than service: queries overlap
        res, lat, status, wall = srv.replay(qs, arrivals)
        assert (status == 0).all()
        assert (lat > 0).all() and wall > 0
        for i in range(len(qs)):
            assert res[i].tobytes() == alone[i].tobytes(), i
        # the same queries, now in a different mix (reversed order, 2 slots)
        srv2 = rpq.Server(kg, budget_bytes=1 << 33, max_slots=2)
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
    srv = rpq.Server(kg, budget_bytes=1 << 33, max_slots=2)
    try:
        with pytest.raises(rpq.RPQError):
            srv.submit(rpqgen.Query(central=[], marginal=[], k=5, max_depth=4), 1)
        with pytest.raises(rpq.RPQError):
            srv.replay([qs[0], qs[1]], np.array([1.0, 0.5]))      # decreasing arrivals
        # a replay matches completions to its schedule by query index, so a
        # query submitted before it must have been polled first
        srv.submit(qs[0], 77)
        with pytest.raises(rpq.RPQError):
            srv.replay([qs[1]], np.zeros(1))
        got = []
        while not got:
            got = srv.poll(wait=True)
        assert got[0][0] == 77 and got[0][1] == 0 and got[0][2].tobytes() == alone[0].tobytes()
        res, _, status, _ = srv.replay([qs[1]], np.zeros(1))      # idle again
        assert status[0] == 0 and res[0].tobytes() == alone[1].tobytes()
    finally:
        srv.close()


def test_failed_start_completes_with_its_error():
    """Host-side fault injection (no GPU fault): the server's third query
    start fails before any launch.  That query alone completes with an error
    status, its column pages return to the pools (a server with only the
    minimum 8 pages of each kind still serves every later query), and every
    other result equals the query run alone."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    child = r"""
import os, sys
sys.path.insert(0, os.getcwd())
import rpqgen, paper_2001_06770_b300 as rpq
from tests.gpu_common import dataset_queries
ds = rpqgen.make_dataset("small")
kg = rpq.KG.from_dataset(ds)
qs = dataset_queries("small", ds, 24, seed=21)
alone = [kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)[0] for q in qs]
srv = rpq.Server(kg, slots=2, h_pages=8, r_pages=8)
got = {}
for i, q in enumerate(qs):
    srv.submit(q, i)
    for tag, status, res, st, lat in srv.poll():
        got[tag] = (status, res)
while len(got) < len(qs):
    for tag, status, res, st, lat in srv.poll(wait=True):
        got[tag] = (status, res)
    inf = srv.info()      # waiting queries with nothing running would mean lost pages
    assert inf["running"] > 0 or len(got) == len(qs), ("stuck", inf, len(got))
failed = [i for i, (status, _) in got.items() if status != 0]
assert len(failed) == 1 and got[failed[0]][0] == rpq.RPQ_EINTERNAL, failed
for i, (status, res) in got.items():
    if status == 0:
        assert res.tobytes() == alone[i].tobytes(), i
srv.close()
kg.close()
print("injected start failure handled")
"""
    env = dict(os.environ, RPQ_INJECT_START_FAILURE="3")
    r = subprocess.run([sys.executable, "-c", child], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "injected start failure handled" in r.stdout, (r.stdout[-2000:], r.stderr[-2000:])


def test_served_mix_equals_oracle():
    """The served workload's shapes (|C| 2-6, |M| 0-8, head and tail keywords,
    k in {5, 10, 20}) on the medium graph, arriving as a Poisson stream faster
    than the server drains it: every sampled result equals the oracle's."""
    ds = rpqgen.make_dataset("medium")
    qs = rpqgen.workload_queries("served", ds)[:400]
    pick = list(range(0, 400, 25))                       # 16 queries checked against the oracle
    kg = rpq.KG.from_dataset(ds)
    try:
        srv = rpq.Server(kg, budget_bytes=4 << 30, max_slots=16)
        try:
            res, lat, status, wall = srv.replay(qs, rpqgen.poisson_arrivals(len(qs), 20000.0, seed=5))
        finally:
            srv.close()
        assert (status == 0).all()
    finally:
        kg.close()
    act = oracle.dataset_activation(ds, detail=False)
    pg = oracle.PreparedGraph(ds, act.a)
    try:
        orcs = oracle.search_many(pg, [qs[i] for i in pick])
    finally:
        pg.close()
    for i, orc in zip(pick, orcs):
        results_match(res[i], orc)
