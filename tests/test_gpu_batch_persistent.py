"""The multi-query persistent kernel (the whole batch in one launch fed by a
device work queue, rpq_search_batch_persistent) against the oracle and the
one-at-a-time path: results bit for bit and equal search statistics, for
every graph of the parity suite, slot counts from one to the maximum,
variants, invalid and empty queries, and the watchdog that ends the launch
when no phase finishes."""
import os
import subprocess
import sys

import pytest

import oracle
import paper_2001_06770_b300 as rpq
import rpqgen
from tests.gpu_common import dataset_queries, oracle_query, results_match

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["tiny", "small", "cl_small", "mid"])
def bundle(request):
    ds = rpqgen.make_dataset(request.param)
    act = oracle.dataset_activation(ds)
    kg = rpq.KG.from_dataset(ds)
    yield request.param, ds, act, kg
    kg.close()


def equal_one_at_a_time(kg, qs, batch):
    for q, (res, st, status) in zip(qs, batch):
        assert status == 0
        one, st1 = kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma,
                             w=getattr(q, "w", 0), product=getattr(q, "product", False))
        assert res.tobytes() == one.tobytes()
        assert st.pop("kernels") == 0          # the batch is one launch
        st1.pop("kernels")
        assert st == st1


def test_persistent_batch_equals_oracle(bundle):
    name, ds, act, kg = bundle
    qs = dataset_queries(name, ds, 16, seed=23)
    batch = kg.search_batch(qs, persistent=True)
    for q, (res, st, status) in zip(qs, batch):
        assert status == 0
        orc = oracle_query(ds, act, q)
        results_match(res, orc)
        if orc.central is not None:
            assert st["e_act_central"] == orc.central.e_act
            assert st["levels_central"] == orc.central.last_level
        if orc.marginal is not None:
            assert st["e_act_marginal"] == orc.marginal.e_act
            assert st["levels_marginal"] == orc.marginal.last_level
    equal_one_at_a_time(kg, qs, batch)


@pytest.fixture(scope="module")
def small():
    ds = rpqgen.make_dataset("small")
    act = oracle.dataset_activation(ds)
    kg = rpq.KG.from_dataset(ds)
    yield ds, act, kg
    kg.close()


@pytest.mark.parametrize("slots", [1, 3, 32])
def test_persistent_batch_slot_counts(small, slots):
    """More queries than slots: every slot takes several queries in turn,
    with the variants (w > k, product scores) in the mix."""
    ds, act, kg = small
    qs = dataset_queries("small", ds, 30, seed=29)
    for i, q in enumerate(qs[::3]):
        if i % 2:
            q.product = True
        else:
            q.w = min(64, q.k + 7)
    default = kg.tuning()
    try:
        kg.set_tuning(batch_slots=slots)
        batch = kg.search_batch(qs, persistent=True)
    finally:
        kg.set_tuning(**default)
    for q, (res, st, status) in zip(qs, batch):
        assert status == 0
        results_match(res, oracle_query(ds, act, q))
    equal_one_at_a_time(kg, qs, batch)


def test_persistent_batch_invalid_and_empty(small):
    """Invalid queries and queries with a keyword on no node are answered on
    the host, as by rpq_search_batch; the others run in the kernel."""
    ds, act, kg = small
    qs = dataset_queries("small", ds, 6, seed=37)
    empty_kw = next((i for i in range(ds.n_kw) if ds.kw_ptr[i + 1] == ds.kw_ptr[i]), None)
    bad = rpqgen.Query(central=[0], marginal=[], k=0, max_depth=4, gamma=0.5)     # k = 0: invalid
    mixed = [qs[0], bad, qs[1]]
    if empty_kw is not None:
        mixed.append(rpqgen.Query(central=[empty_kw, qs[2].central[0]], marginal=[], k=5, max_depth=4, gamma=0.5))
    mixed += qs[2:]
    got = kg.search_batch(mixed, persistent=True)
    ref = kg.search_batch(mixed)
    for (r1, s1, st1), (r2, s2, st2) in zip(got, ref):
        assert st1 == st2
        assert r1.tobytes() == r2.tobytes()
    assert got[1][2] == rpq.RPQ_EINVAL
    assert kg.search_batch([], persistent=True) == []


WATCHDOG_CHILD = r"""
import sys
sys.path.insert(0, {root!r})
import oracle, rpqgen
import paper_2001_06770_b300 as rpq
from tests.gpu_common import dataset_queries, oracle_query, results_match
ds = rpqgen.make_dataset("small")
act = oracle.dataset_activation(ds)
kg = rpq.KG.from_dataset(ds)
qs = dataset_queries("small", ds, 12, seed=41)
try:
    kg.search_batch(qs, persistent=True)
    raise SystemExit("no timeout")
except rpq.RPQError as e:
    assert e.code == rpq.RPQ_ETIMEOUT, e
# the context stays usable, and the slots the stopped kernel left mid-query
# serve the next batch correctly
for q, (res, st, status) in zip(qs, kg.search_batch(qs)):
    assert status == 0
    results_match(res, oracle_query(ds, act, q))
kg.close()
print("watchdog ok")
"""


def test_persistent_batch_watchdog():
    """With a watchdog limit of one clock cycle, a block that finds no chunk
    twice with no phase finished in between ends the launch: the call returns
    RPQ_ETIMEOUT without any wait that does not end, and the next batch on
    the same slots gives the oracle's results."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RPQ_BARRIER_LIMIT="1")
    out = subprocess.run([sys.executable, "-c", WATCHDOG_CHILD.format(root=root)], env=env, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "watchdog ok" in out.stdout
