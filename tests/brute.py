"""Independent reference computations used to pin the oracle (test code only).

Nothing here calls the oracle's search: each function re-derives a quantity
from a different formulation of the paper's definitions.

* ``bottleneck_dijkstra``: D(t, v) of Definitions 2-3 under the path score of
  Definition 7 (F = max(F(prefix), a) + 1), by label-setting Dijkstra.
* ``path_enum_distance``: the same distance by enumerating every simple path.
* ``fixed_point``: the hit-level table with the stop rules, as the solution of
  simultaneous equations (Jacobi iteration), instead of the level loop.
* ``prefix_optimal_nodes``: nodes on paths whose every prefix is shortest,
  by forward path enumeration (what Algorithm 2 recovers, Lemma 3).
* ``recovered_paths``: the paths Algorithm 2 recovers (Lemma 3, the stop
  guard, the RPG start nodes of Section 4.3), by forward path enumeration.
* ``ptc_by_paths``: the Pass Through Constraint of Definition 5 by
  enumerating every simple path between marginal keyword nodes.
* ``small_graph``: random simple graphs of at most 20 nodes.
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass

import numpy as np

INF = 255


@dataclass
class SmallGraph:
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    label: np.ndarray
    n_labels: int

    @property
    def m2(self):
        return int(self.row_ptr[-1])

    def edges(self):
        for u in range(self.n):
            for e in range(self.row_ptr[u], self.row_ptr[u + 1]):
                yield u, int(self.col[e]), e


def csr_from_undirected(n, pairs, labels=None, n_labels=1):
    """Symmetric CSR (ascending rows) from undirected pairs; label per pair."""
    adj = [[] for _ in range(n)]
    for i, (u, v) in enumerate(pairs):
        lab = 0 if labels is None else labels[i]
        adj[u].append((v, lab))
        adj[v].append((u, lab))
    row_ptr = [0]
    col, lab = [], []
    for u in range(n):
        for v, l in sorted(adj[u]):
            col.append(v)
            lab.append(l)
        row_ptr.append(len(col))
    return SmallGraph(n, np.array(row_ptr, np.int64), np.array(col, np.int32),
                      np.array(lab, np.uint16), n_labels)


def small_graph(rng, n, m, n_labels=3):
    pairs = set()
    while len(pairs) < m:
        u, v = (int(x) for x in rng.integers(0, n, size=2))
        if u != v:
            pairs.add((min(u, v), max(u, v)))
    pairs = sorted(pairs)
    labels = [int(rng.integers(0, n_labels)) for _ in pairs]
    return csr_from_undirected(n, pairs, labels, n_labels)


def postings_from_sets(n_kw, node_sets):
    """Postings CSR from a list (per keyword) of node lists."""
    kw_ptr = [0]
    nodes = []
    for k in range(n_kw):
        s = sorted(set(node_sets[k]))
        nodes.extend(s)
        kw_ptr.append(len(nodes))
    return np.array(kw_ptr, np.int64), np.array(nodes, np.int32)


def random_levels_symmetric(g: SmallGraph, rng, amax):
    """Random activation level per undirected edge, same in both directions."""
    a = np.zeros(g.m2, np.uint8)
    lv = {}
    for u, v, e in g.edges():
        key = (min(u, v), max(u, v))
        if key not in lv:
            lv[key] = int(rng.integers(0, amax + 1))
        a[e] = lv[key]
    return a


def bottleneck_dijkstra(g, a, sources, cap):
    """min over paths of F(p), F(single node) = 0, F = max(F(prefix), a) + 1;
    values above cap become INF."""
    d = [10 ** 9] * g.n
    pq = []
    for s in sources:
        d[s] = 0
        pq.append((0, s))
    heapq.heapify(pq)
    while pq:
        du, u = heapq.heappop(pq)
        if du != d[u]:
            continue
        for e in range(g.row_ptr[u], g.row_ptr[u + 1]):
            v = int(g.col[e])
            cand = max(du, int(a[e])) + 1
            if cand < d[v]:
                d[v] = cand
                heapq.heappush(pq, (cand, v))
    return np.array([x if x <= cap else INF for x in d], np.int64)


def path_enum_distance(g, a, sources, cap):
    """Same distance by enumerating all simple paths from the sources."""
    best = [10 ** 9] * g.n
    nbrs = [[(int(g.col[e]), int(a[e])) for e in range(g.row_ptr[u], g.row_ptr[u + 1])] for u in range(g.n)]

    def dfs(u, score, onpath):
        if score < best[u]:
            best[u] = score
        for v, av in nbrs[u]:
            if v in onpath:
                continue
            s2 = max(score, av) + 1
            if s2 > cap:
                continue
            onpath.add(v)
            dfs(v, s2, onpath)
            onpath.remove(v)

    for s in sources:
        dfs(s, 0, {s})
    return np.array([x if x <= cap else INF for x in best], np.int64)


def fixed_point(g, a, col_sources, lam_max, stop_rule, max_iter=200):
    """Hit levels with the stop rule as a fixed point (Jacobi iteration):
    h[v][j] = 0 if v is a source of column j, else the least lam+1 over
    in-edges u->v with lam = max(h[u][j], a(u->v)) <= lam_max and
    lam < stop(u); stop(u) = max_j h[u][j] when every column is finite and
    stop_rule is set, else infinity."""
    nt = len(col_sources)
    h = np.full((g.n, nt), INF, np.int64)
    for j, srcs in enumerate(col_sources):
        for s in srcs:
            h[s, j] = 0
    ins = [[] for _ in range(g.n)]
    for u, v, e in g.edges():
        ins[v].append((u, int(a[e])))
    for _ in range(max_iter):
        stop = np.full(g.n, 10 ** 9, np.int64)
        if stop_rule:
            fin = (h != INF).all(axis=1)
            stop[fin] = h[fin].max(axis=1)
        new = np.full_like(h, INF)
        for j, srcs in enumerate(col_sources):
            for s in srcs:
                new[s, j] = 0
        for v in range(g.n):
            for j in range(nt):
                if new[v, j] == 0:
                    continue
                best = INF
                for u, av in ins[v]:
                    if h[u, j] == INF:
                        continue
                    lam = max(int(h[u, j]), av)
                    if lam <= lam_max and lam < stop[u] and lam + 1 < best:
                        best = lam + 1
                new[v, j] = best
        if (new == h).all():
            return h
        h = new
    raise RuntimeError("fixed point iteration did not converge")


def prefix_optimal_nodes(g, a, sources, target, dist):
    """Nodes lying on simple paths source -> target whose every prefix ending
    at x has score dist[x] (forward enumeration)."""
    nbrs = [[(int(g.col[e]), int(a[e])) for e in range(g.row_ptr[u], g.row_ptr[u + 1])] for u in range(g.n)]
    found = set()

    def dfs(u, score, path):
        if u == target:
            found.update(path)
            return
        for v, av in nbrs[u]:
            if v in path:
                continue
            s2 = max(score, av) + 1
            if s2 != dist[v]:
                continue
            path.append(v)
            dfs(v, s2, path)
            path.pop()

    for s in sources:
        if dist[s] == 0:
            dfs(s, 0, [s])
    return found


def recovered_paths(g, a, dist, stop, sources, targets):
    """Union of the simple paths from `sources` to `targets` along which every
    step u -> v (CSR entry e) is an expansion that happened: u was reached
    (dist[u] finite), lam = max(dist[u], a[e]) is below u's stop level and
    v was first hit at lam + 1 (forward enumeration).  Returns the node set
    and the set of (u, v) steps.  With `stop` None no node ever stopped."""
    nbrs = [[(int(g.col[e]), int(a[e])) for e in range(g.row_ptr[u], g.row_ptr[u + 1])] for u in range(g.n)]
    targets = set(int(t) for t in targets)
    nodes, steps = set(), set()

    def dfs(u, path):
        if u in targets:
            nodes.update(path)
            steps.update(zip(path[:-1], path[1:]))
            return
        for v, av in nbrs[u]:
            if v in path:
                continue
            lam = max(int(dist[u]), av)
            if stop is not None and not lam < int(stop[u]):
                continue
            if int(dist[v]) != lam + 1:
                continue
            path.append(v)
            dfs(v, path)
            path.pop()

    for s in sources:
        if int(dist[s]) == 0:
            dfs(int(s), [int(s)])
    return nodes, steps


def ptc_by_paths(n_m, pairs, vc, holders):
    """Pass Through Constraint of Definition 5 by enumerating simple paths of
    the undirected graph given by `pairs`.  `holders` maps each node holding
    a marginal keyword to the set of marginal columns it holds; `vc` is V_C.
    |M| >= 2: some two distinct holders of different columns are joined only
    by paths with a node (endpoints included) in V_C.  |M| = 1: some holder
    has a path to a node of V_C (or lies in V_C)."""
    adj = {}
    for u, v in pairs:
        adj.setdefault(u, set()).add(v)
        adj.setdefault(v, set()).add(u)
    vc = set(vc)

    def paths(x, y):
        out = []

        def dfs(u, path):
            if u == y:
                out.append(list(path))
                return
            for w in sorted(adj.get(u, ())):
                if w not in path:
                    path.append(w)
                    dfs(w, path)
                    path.pop()
        dfs(x, [x])
        return out

    hs = sorted(holders)
    if n_m == 1:
        for x in hs:
            if x in vc or any(paths(x, v) for v in vc):
                return 1
        return 0
    for x in hs:
        for y in hs:
            if x == y or not any(i != j for i in holders[x] for j in holders[y]):
                continue
            if all(any(w in vc for w in p) for p in paths(x, y)):
                return 1
    return 0
