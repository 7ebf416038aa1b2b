"""Pins for the oracle's activation levels (Section 3.1, Eq. 1-3, Theorem 1)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def stars_graph():
    pairs, labels = [], []
    nxt = 0
    for lab, leaves in enumerate([1, 2, 3, 4, 5, 6, 7]):
        c = nxt
        for i in range(leaves):
            pairs.append((c, c + 1 + i))
            labels.append(lab)
        nxt = c + 1 + leaves
    return brute.csr_from_undirected(nxt, pairs, labels, 7)


def test_golden_stars():
    fx = json.load(open(os.path.join(GOLDEN, "activation_stars.json")))
    g = stars_graph()
    for case in fx["cases"]:
        act = oracle.activation(g.row_ptr, g.col, g.label, g.n_labels, fx["alpha"], case["abar"])
        table = case.get("a_by_cnt") or case["a_by_cnt_partial"]
        seen = set()
        for e in range(g.m2):
            c = str(int(act.cnt[e]))
            if c in table:
                assert act.a[e] == table[c], (c, act.a[e], table[c])
                seen.add(c)
        assert seen == set(table)


def _theorem1_holds(a, w, alpha, abar, tol=1e-12):
    """Theorem 1: bounds on the rescaled weight given the activation level."""
    ra = math.floor(abar + 0.5)
    lo_r = alpha * (a - 0.5) / abar
    hi_r = alpha * (a + 0.5) / abar
    lo_p = 1 + (a - 0.5 - 2 * abar) * (1 - alpha) / abar
    hi_p = 1 + (a + 0.5 - 2 * abar) * (1 - alpha) / abar
    if a < ra:
        return lo_r - tol <= w < hi_r + tol
    if a == ra:
        return lo_r - tol <= w < hi_p + tol
    return lo_p - tol <= w < hi_p + tol


@pytest.mark.parametrize("alpha,abar", [(0.5, 2.9), (0.2, 3.87), (0.8, 3.68), (0.5, 3.25), (0.35, 1.6)])
def test_theorem1_bounds_tiny(tiny_ds, alpha, abar):
    g = tiny_ds.graph
    act = oracle.activation(g.row_ptr, g.col, g.label, g.n_labels, alpha, abar)
    bad = [e for e in range(0, g.m2, 7) if not _theorem1_holds(int(act.a[e]), act.w[e], alpha, abar)]
    assert not bad
    assert act.a.min() >= 0 and act.a.max() <= math.floor(2 * abar + 0.5)


def test_w_is_minmax_rescaled_log_count(tiny_ds, tiny_act):
    """w in [0,1], 0 exactly at the smallest count and 1 at the largest."""
    w, cnt = tiny_act.w, tiny_act.cnt
    assert w.min() == 0.0 and w.max() == 1.0
    assert (w[cnt == cnt.min()] == 0.0).all() and (w[cnt == cnt.max()] == 1.0).all()


def test_count_definition_brute(tiny_ds, tiny_act):
    """cnt(u->v) = out-edges of u with the label + in-edges of v with the label,
    counted directly from the edge list on a sample of entries."""
    g = tiny_ds.graph
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    rng = np.random.default_rng(3)
    for e in rng.integers(0, g.m2, size=300):
        u, v, lab = src[e], g.col[e], g.label[e]
        out_u = np.sum((src == u) & (g.label == lab))
        in_v = np.sum((g.col == v) & (g.label == lab))
        assert tiny_act.cnt[e] == out_u + in_v


def test_symmetric_and_monotone(tiny_ds, tiny_act):
    g = tiny_ds.graph
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    # symmetric: a(u->v) == a(v->u)
    key = src.astype(np.int64) * g.n + g.col
    rkey = g.col.astype(np.int64) * g.n + src
    order = np.argsort(key)
    pos = order[np.searchsorted(key[order], rkey)]
    assert (tiny_act.a == tiny_act.a[pos]).all()
    # monotone non-decreasing in the count
    o = np.argsort(tiny_act.cnt, kind="stable")
    assert (np.diff(tiny_act.a[o].astype(int)) >= 0).all()
    # amax is the row maximum
    for v in range(0, g.n, 97):
        b, e = g.row_ptr[v], g.row_ptr[v + 1]
        assert tiny_act.amax[v] == (tiny_act.a[b:e].max() if e > b else 0)


def test_constant_weights_give_zero_levels():
    """A cycle with one label: every count is 4, w_max = w_min, so w = 0 and a = 0."""
    n = 9
    g = brute.csr_from_undirected(n, [(i, (i + 1) % n) for i in range(n)], None, 1)
    act = oracle.activation(g.row_ptr, g.col, g.label, 1, 0.5, 3.0)
    assert (act.cnt == 4).all() and (act.a == 0).all() and (act.amax == 0).all()


def test_rounding_boundary_report(tiny_ds, tiny_act):
    """No edge of the tiny workload lies within 1e-9 of a rounding boundary, so
    the activation levels do not hinge on the last bit of the logarithm."""
    frac = tiny_act.x - np.floor(tiny_act.x)
    assert not np.any(np.abs(frac - 0.5) < 1e-9)


def test_rejects_bad_parameters():
    g = stars_graph()
    with pytest.raises(ValueError):
        oracle.activation(g.row_ptr, g.col, g.label, g.n_labels, 1.5, 3.0)
    with pytest.raises(ValueError):
        oracle.activation(g.row_ptr, g.col, g.label, g.n_labels, 0.5, 0.0)
