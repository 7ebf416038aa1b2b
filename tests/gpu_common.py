"""Shared helpers of the GPU parity tests: compare the CUDA library with the
CPU oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle
import rpqgen

INF = 255
REL_TOL = 1e-6   # S^r (a double); everything else must match bit for bit


def results_match(gpu_res, orc):
    assert len(gpu_res) == len(orc.nodes), (gpu_res, orc.nodes)
    assert gpu_res["node"].tolist() == [int(x) for x in orc.nodes]
    assert gpu_res["s_c"].tolist() == orc.s_c.tolist()
    assert gpu_res["s_m"].tolist() == orc.s_m.tolist()
    assert np.allclose(gpu_res["s_r"], orc.s_r, rtol=REL_TOL, atol=0)


def trace_matches(tr, orc, check_stats=True):
    """Element-by-element comparison of a GPU trace with the oracle."""
    results_match(tr["results"], orc)
    if orc.central is None:
        assert len(tr["results"]) == 0
        return
    assert np.array_equal(tr["h_central"], orc.central.h), "central hit levels differ"
    assert len(tr["frontiers_central"]) == len(orc.central.frontiers)
    for l, (a, b) in enumerate(zip(tr["frontiers_central"], orc.central.frontiers)):
        assert np.array_equal(a, b), f"central frontier Q_{l} differs"
    gcg = sorted((int(x) >> 8, int(x) & 0xff) for x in tr["cgs"])
    ocg = sorted(zip(orc.cg_node.tolist(), orc.cg_score.tolist()))
    assert gcg == ocg, "CG sets differ"
    assert tr["selected"].tolist() == orc.selected.tolist()
    st = tr["stats"]
    if check_stats:
        assert st["e_act_central"] == orc.central.e_act
        assert st["levels_central"] == orc.central.last_level
    if orc.marginal is not None:
        for g in range(len(orc.selected)):
            assert tr["vc"][g].tolist() == orc.vc_kw[g].tolist(), f"V_C of CG {g} differs"
        assert np.array_equal(tr["h_marginal"], orc.marginal.h), "marginal hit levels differ"
        assert len(tr["frontiers_marginal"]) == len(orc.marginal.frontiers)
        for l, (a, b) in enumerate(zip(tr["frontiers_marginal"], orc.marginal.frontiers)):
            assert np.array_equal(a, b), f"marginal frontier Q_{l} differs"
        if check_stats:
            assert st["e_act_marginal"] == orc.marginal.e_act
            assert st["levels_marginal"] == orc.marginal.last_level


def oracle_query(ds, act, q):
    return oracle.search(ds, act.a, q.central, q.marginal, q.k, q.max_depth, q.gamma,
                         w=getattr(q, "w", 0), product=getattr(q, "product", False))


def dataset_queries(name, ds, n, seed=3):
    """Queries spread over each dataset's vocabulary: uniform shapes plus a
    head/tail mix."""
    vocab = ds.n_kw
    lo, hi = max(1, vocab // 400), max(2, vocab // 10)
    qs = rpqgen.queries_uniform(n, (1, 4), (0, 4), (lo, hi), 10, 6, seed)
    qs += rpqgen.queries_mixed(ds, max(2, n // 2), c_range=(2, 4), m_range=(0, 4), ks=(1, 5, 20),
                               max_depth=7, seed=seed, head_min=int(np.diff(ds.kw_ptr).max() // 4),
                               tail_max=20)
    return qs


def check_levels(g, adj, H, stop, last_expanded, postings, rng, n_sample=4000, nodes=None):
    """Fixed-point property of the hit levels (Theorem 5 with the stop rules)
    on sampled nodes and up to 300 nodes of each keyword's postings, or on
    `nodes`: h = 0 exactly on keyword nodes; h > 0 is one more than the
    smallest max(h_u, a) over neighbours u that expanded to the node (reached,
    not stopped by then, at a level <= last_expanded); an unreached node has
    no such neighbour.  `adj` holds the device's packed rows (a << 26 | u)."""
    rp = g.row_ptr
    if nodes is None:
        picks = [rng.choice(np.asarray(p), size=min(len(p), 300), replace=False) for p in postings if len(p)]
        nodes = np.unique(np.concatenate([rng.integers(0, g.n, size=n_sample)] + picks))
    for j in range(H.shape[1]):
        kw = set(int(x) for x in postings[j])
        h = H[:, j].astype(np.int64)
        for v in nodes:
            v = int(v)
            row = adj[rp[v]:rp[v + 1]]
            a = (row >> 26).astype(np.int64)
            u = (row & ((1 << 26) - 1)).astype(np.int64)
            hu = h[u]
            lam = np.maximum(hu, a)
            live = (hu != INF) & (lam < stop[u]) & (lam <= last_expanded)   # u expanded to v at level lam
            hv = int(h[v])
            if v in kw:
                assert hv == 0
                continue
            assert hv != 0
            if hv == INF:
                assert not live.any(), f"node {v} column {j}: reachable but unreached"
            else:
                assert live.any() and int((lam[live] + 1).min()) == hv, f"node {v} column {j}: level {hv}"
