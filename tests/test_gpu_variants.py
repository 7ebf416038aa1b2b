"""GPU parity of the search variants: beam width w > k with Theorem 4 early
termination of the marginal run, and the multiplicative RPG score.  The
trace comparison covers every frontier of both runs, so the device must stop
the marginal run at the same Glevel as the oracle."""
import dataclasses

import numpy as np
import pytest

import oracle
import paper_2001_06770_b300 as rpq
import rpqgen
from tests import brute
from tests.gpu_common import dataset_queries, oracle_query, results_match, trace_matches

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["tiny", "small", "cl_small"])
def bundle(request):
    ds = rpqgen.make_dataset(request.param)
    act = oracle.dataset_activation(ds)
    kg = rpq.KG.from_dataset(ds)
    yield request.param, ds, act, kg
    kg.close()


def variant_queries(name, ds, n, seed, product, gamma):
    rng = np.random.default_rng(seed)
    out = []
    for q in dataset_queries(name, ds, n, seed=seed):
        k = int(rng.integers(1, 6))
        w = int(rng.integers(k + 1, 21))
        out.append(dataclasses.replace(q, k=k, w=w, product=product, gamma=gamma))
    return out


@pytest.mark.parametrize("product,gamma", [(False, 0.5), (False, 1.0), (False, 0.3), (True, 0.5)])
def test_trace_parity_w_greater_than_k(bundle, product, gamma):
    name, ds, act, kg = bundle
    stops = 0
    for q in variant_queries(name, ds, 8, 41, product, gamma):
        orc = oracle_query(ds, act, q)
        tr = kg.trace(q.central, q.marginal, q.k, q.max_depth, q.gamma, w=q.w, product=q.product)
        trace_matches(tr, orc)
        res, _ = kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma, w=q.w, product=q.product)
        results_match(res, orc)
        if orc.marginal is not None and not orc.matched.all():
            stops += 1
    if name == "cl_small":
        assert stops > 0          # Theorem 4 ended some marginal runs early


def test_batch_with_variants(bundle):
    name, ds, act, kg = bundle
    qs = variant_queries(name, ds, 6, 7, False, 0.5) + variant_queries(name, ds, 6, 8, True, 0.5)
    for q, (res, st, status) in zip(qs, kg.search_batch(qs)):
        assert status == 0
        results_match(res, oracle_query(ds, act, q))


def test_invalid_beam_width_rejected(bundle):
    name, ds, act, kg = bundle
    for w in (3, 65):
        with pytest.raises(rpq.RPQError) as ei:
            kg.search([1], [2], 4, 6, w=w)
        assert ei.value.code == rpq.RPQ_EINVAL


@pytest.mark.parametrize("seed", range(8))
def test_random_small_graphs(seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(8, 21))
    g = brute.small_graph(rng, n, int(rng.integers(n, 2 * n)), n_labels=3)
    sets = [list(rng.choice(n, size=int(rng.integers(1, 3)), replace=False)) for _ in range(6)]
    kp, kn = brute.postings_from_sets(6, sets)
    act = oracle.activation(g.row_ptr, g.col, g.label, g.n_labels, 0.5, 2.0)
    kg = rpq.KG(g.row_ptr, g.col, g.label, g.n_labels, kp, kn, 0.5, 2.0)
    try:
        for C, M, k, w, prod in [([0, 1], [2, 3], 1, 4, False), ([0], [1, 2], 2, 5, True),
                                 ([0, 1], [2], 1, 3, False), ([3, 4], [5, 2], 2, 2, True)]:
            orc = oracle.search(g, act.a, C, M, k, 6, kw_ptr=kp, kw_nodes=kn, w=w, product=prod)
            trace_matches(kg.trace(C, M, k, 6, w=w, product=prod), orc)
    finally:
        kg.close()
