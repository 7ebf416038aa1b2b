"""The hit-level property check used at full size (tests/gpu_common.py
check_levels) accepts the oracle's hit levels and rejects planted mistakes
(run on CPU against the oracle)."""
import numpy as np
import pytest

import oracle
from tests.gpu_common import INF, check_levels


def packed_adj(g, a):
    """Rows as the device stores them: (a << 26) | neighbour, ascending."""
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    key = (a.astype(np.uint64) << np.uint64(26)) | g.col.astype(np.uint64)
    return key[np.lexsort((key, src))].astype(np.uint32)


@pytest.fixture(scope="module")
def case(tiny_ds, tiny_act):
    q = dict(central=[124, 464], marginal=[375, 63], k=10, max_depth=6)
    r = oracle.search(tiny_ds, tiny_act.a, **q)
    stop = np.full(tiny_ds.graph.n, 10 ** 9, np.int64)
    for v, sc in zip(r.cg_node, r.cg_score):
        stop[int(v)] = int(sc)
    H = r.central.h.copy()
    return tiny_ds, packed_adj(tiny_ds.graph, tiny_act.a), H, stop, r, q


def run(case, H):
    ds, adj, _, stop, r, q = case
    check_levels(ds.graph, adj, H, stop, int(H[H != INF].max()) - 1, [ds.postings(k) for k in q["central"]],
                 np.random.default_rng(1), nodes=np.arange(ds.graph.n))


def test_oracle_levels_pass(case):
    run(case, case[2])


@pytest.mark.parametrize("plant", ["raise", "lower", "unreach", "reach"])
def test_planted_mistakes_fail(case, plant):
    H = case[2].copy()
    j = 0
    fin = np.nonzero((H[:, j] != INF) & (H[:, j] > 1))[0]
    inf = np.nonzero(H[:, j] == INF)[0]
    if plant == "raise":
        H[fin[0], j] += 1
    elif plant == "lower":
        H[fin[0], j] -= 1
    elif plant == "unreach":
        H[fin[0], j] = INF
    else:
        H[inf[0], j] = 2
    with pytest.raises(AssertionError):
        run(case, H)
