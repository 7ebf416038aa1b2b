"""Full-size checks on the large workload (Chung-Lu, 5e7 nodes, 7.6e8 CSR
entries, queries of 3 + 3 keywords, k = 20, L = 8).  The serial oracle needs
minutes per query there, so these tests check properties that hold at any
size, on the device's own trace, plus equality between the search paths:

* hit levels (Theorem 5 with the stop rules): a sampled node's level h > 0 has
  a parent u with max(h_u, a) + 1 = h that had not stopped, no neighbour
  offers a smaller level, an unreached node has no neighbour that expanded to
  it, and h = 0 exactly on keyword nodes;
* Theorem 3: the CG set is every node whose central columns are all finite,
  with S^c = max h; the selected CGs are the w smallest by (S^c, node id);
* Eq. 6 and Definition 6: scores and the (S^r, id) order of the results;
* the graph-replayed search, the trace and the batch give the same results.
"""
import numpy as np
import pytest

import paper_2001_06770_b300 as rpq
import rpqgen
from tests.gpu_common import INF, check_levels

pytestmark = pytest.mark.gpu

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
