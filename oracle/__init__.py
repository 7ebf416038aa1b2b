"""Python access to the serial CPU oracle (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never loads it.  The arithmetic lives in ``rpq_oracle.c``: a
plain, serial transcription of the paper's definitions (Section 3.1 and
Eq. 1-3 for activation levels; Section 4, Algorithms 1-2 and Eq. 4-6 for the
search).  This wrapper only marshals arrays.

Parity is pinned for every function by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (Theorem 1 bounds, Theorem 5 against an independent
bottleneck Dijkstra, a Bellman-Ford fixed point with the stop rules, brute
force path enumeration on graphs of 20 nodes or fewer, Theorem 6 order
independence, textbook BFS special case, hand-computed golden fixtures).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rpq_oracle.c")
_LIB = os.path.join(_HERE, "_rpq_oracle.so")
_lib = None
INF = 255

# field ids of orc_get (keep in step with the enum in rpq_oracle.c)
(F_STATUS, F_NRES, F_RES_NODE, F_RES_SC, F_RES_SM, F_RES_SR, F_QPTR, F_QNODES, F_LAST_LEVEL,
 F_LAST_EXPANDED, F_EACT, F_NEWHITS, F_CG_NODE, F_CG_SCORE, F_CG_LEVEL, F_NSEL, F_SEL, F_SEL_SC,
 F_VC_ALL, F_VC_KW, F_EC, F_MATCHED, F_MATCH_LEVEL, F_SM, F_RAN, F_VM, F_EM, F_PTC) = range(28)


def build_lib(force: bool = False) -> str:
    """Compile the oracle (plain C, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_lib())
        P = ctypes.c_void_p
        i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        _lib.orc_activation.argtypes = [i32, i64, P, P, P, i32, f64, f64, P, P, P, P, P]
        _lib.orc_activation.restype = ctypes.c_int
        _lib.orc_search.argtypes = [i32, i64, P, P, P, i32, P, P, P, i32, P, i32, i32, i32, f64,
                                    i32, i32, i32, i32, u64]
        _lib.orc_search.restype = P
        _lib.orc_get.argtypes = [P, i32, i32, i32, P]
        _lib.orc_get.restype = i64
        _lib.orc_get_h.argtypes = [P, i32, P, P, i32]
        _lib.orc_get_h.restype = i32
        _lib.orc_free.argtypes = [P]
        _lib.orc_graph_new.argtypes = [i32, i64, P, P, P, i32, P, P]
        _lib.orc_graph_new.restype = P
        _lib.orc_graph_free.argtypes = [P]
        _lib.orc_search_graph.argtypes = [P, P, i32, P, i32, i32, i32, f64, i32, i32, i32, i32, u64, i32]
        _lib.orc_search_graph.restype = P
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "arrays passed to the oracle must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Activation:
    a: np.ndarray      # uint8[m2] activation level per CSR entry
    amax: np.ndarray   # uint8[n]
    cnt: np.ndarray    # int64[m2] label count of Section 3.1
    w: np.ndarray      # float64[m2] rescaled fine-grained weight
    x: np.ndarray      # float64[m2] value before rounding (Eq. 3)


def activation(row_ptr, col, label, n_labels, alpha, abar) -> Activation:
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    label = np.ascontiguousarray(label, np.uint16)
    n = len(row_ptr) - 1
    m2 = int(row_ptr[-1])
    a = np.empty(m2, np.uint8)
    amax = np.empty(n, np.uint8)
    cnt = np.empty(m2, np.int64)
    w = np.empty(m2, np.float64)
    x = np.empty(m2, np.float64)
    rc = _L().orc_activation(n, m2, _p(row_ptr), _p(col), _p(label), int(n_labels), float(alpha),
                             float(abar), _p(a), _p(amax), _p(cnt), _p(w), _p(x))
    if rc != 0:
        raise ValueError("orc_activation rejected its arguments")
    return Activation(a, amax, cnt, w, x)


def dataset_activation(ds, detail: bool = True) -> Activation:
    """Activation levels of a dataset's graph.  With ``detail=False`` only
    ``a`` and ``amax`` are kept (the per-entry counts, weights and values before
    rounding take 24 bytes per CSR entry; they are None then)."""
    g = ds.graph
    if detail:
        return activation(g.row_ptr, g.col, g.label, g.n_labels, ds.alpha, ds.abar)
    row_ptr = np.ascontiguousarray(g.row_ptr, np.int64)
    col = np.ascontiguousarray(g.col, np.int32)
    label = np.ascontiguousarray(g.label, np.uint16)
    n = len(row_ptr) - 1
    a = np.empty(int(row_ptr[-1]), np.uint8)
    amax = np.empty(n, np.uint8)
    rc = _L().orc_activation(n, int(row_ptr[-1]), _p(row_ptr), _p(col), _p(label), int(g.n_labels),
                             float(ds.alpha), float(ds.abar), _p(a), _p(amax), None, None, None)
    if rc != 0:
        raise ValueError("orc_activation rejected its arguments")
    return Activation(a, amax, None, None, None)


class PreparedGraph:
    """A graph with its CSR transpose built once (``orc_graph_new``), for many
    searches.  The C side only reads it, so searches may run on it from several
    threads at once (the ctypes calls release the GIL).  Holds references to
    the arrays it was built from."""

    def __init__(self, ds_or_graph, a: np.ndarray, kw_ptr=None, kw_nodes=None):
        if hasattr(ds_or_graph, "graph"):
            g = ds_or_graph.graph
            kw_ptr, kw_nodes = ds_or_graph.kw_ptr, ds_or_graph.kw_nodes
        else:
            g = ds_or_graph
        self.row_ptr = np.ascontiguousarray(g.row_ptr, np.int64)
        self.col = np.ascontiguousarray(g.col, np.int32)
        self.a = np.ascontiguousarray(a, np.uint8)
        self.kw_ptr = np.ascontiguousarray(kw_ptr, np.int64)
        self.kw_nodes = np.ascontiguousarray(kw_nodes, np.int32)
        self.n = len(self.row_ptr) - 1
        self.handle = _L().orc_graph_new(self.n, int(self.row_ptr[-1]), _p(self.row_ptr), _p(self.col), _p(self.a),
                                         len(self.kw_ptr) - 1, _p(self.kw_ptr), _p(self.kw_nodes))
        if not self.handle:
            raise ValueError("orc_graph_new rejected its arguments")

    def close(self):
        if self.handle:
            _L().orc_graph_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class RunTrace:
    h: np.ndarray          # uint8[n, nt]
    stop: np.ndarray       # uint8[n] level at which the node stopped expanding (255 = never)
    frontiers: list        # list of sorted int64 arrays, Q_l for l = 0..last_level
    last_level: int
    last_expanded: int
    e_act: int
    new_hits: int


@dataclass
class SearchResult:
    status: int
    nodes: np.ndarray      # int64[n_res] central node of each RPG, ranked
    s_c: np.ndarray        # int32
    s_m: np.ndarray        # int32
    s_r: np.ndarray        # float64
    central: RunTrace | None
    marginal: RunTrace | None
    cg_node: np.ndarray    # all identified CGs (identification order)
    cg_score: np.ndarray
    cg_level: np.ndarray
    selected: np.ndarray   # top-w CG nodes, ordered by (S^c, id)
    selected_sc: np.ndarray
    vc_all: list           # V^c per selected CG
    vc_kw: list            # V_C per selected CG
    ec: list               # recovered CSR entries per selected CG
    matched: np.ndarray
    match_level: np.ndarray
    sel_sm: np.ndarray
    vm: list               # G^m nodes per selected CG (empty unless matched)
    em: list               # G^m CSR entries per selected CG
    ptc: np.ndarray        # Definition 5 check per selected CG: 1 holds, 0 violated, -1 not an RPG


def _get(L, h, field, r=0, g=0, dtype=np.int64):
    cnt = L.orc_get(h, field, r, g, None)
    out = np.empty(max(cnt, 0), dtype)
    if cnt > 0:
        L.orc_get(h, field, r, g, _p(out))
    return out


def _scalar(L, h, field, r=0, dtype=np.int32):
    out = np.zeros(1, dtype)
    L.orc_get(h, field, r, 0, _p(out))
    return int(out[0])


def _run(L, h, r, n, trace=True, tables=True) -> RunTrace | None:
    if not _scalar(L, h, F_RAN, r):
        return None
    H = stop = fr = None
    if tables:          # hit-level table and stop levels
        nt = L.orc_get_h(h, r, None, None, n)
        H = np.empty((n, max(nt, 1)), np.uint8)
        stop = np.empty(n, np.uint8)
        L.orc_get_h(h, r, _p(H), _p(stop), n)
        H = H[:, :nt]
    if trace:           # every frontier Q_l
        qptr = _get(L, h, F_QPTR, r)
        qn = _get(L, h, F_QNODES, r)
        fr = [qn[qptr[i]:qptr[i + 1]] for i in range(len(qptr) - 1)]
    return RunTrace(h=H, stop=stop, frontiers=fr, last_level=_scalar(L, h, F_LAST_LEVEL, r),
                    last_expanded=_scalar(L, h, F_LAST_EXPANDED, r),
                    e_act=_scalar(L, h, F_EACT, r, np.int64), new_hits=_scalar(L, h, F_NEWHITS, r, np.int64))


def search(ds_or_graph, a: np.ndarray, central, marginal, k: int, max_depth: int, gamma: float = 0.5,
           disable_stops: bool = False, exhaustive_marginal: bool = False, shuffle_seed: int = 0,
           kw_ptr=None, kw_nodes=None, w: int = 0, product: bool = False, prepared: PreparedGraph = None,
           trace: bool = True, subgraphs: bool = True, tables: bool = None) -> SearchResult:
    """Run the oracle on one query.  ``ds_or_graph`` is an ``rpqgen.Dataset`` or
    an ``rpqgen.Graph`` (then pass ``kw_ptr``/``kw_nodes``).  ``w`` is the CG
    beam width (0: w = k), ``product`` selects the multiplicative S^r.

    With ``prepared`` (a PreparedGraph of the same graph and levels) the
    graph arguments are ignored and the transpose is not rebuilt.
    ``trace=False`` keeps no frontiers and, unless ``tables=True``, no
    hit-level tables or stop levels (the runs' counts and levels remain);
    ``subgraphs=False`` builds no G^m and checks no PTC (vm, em and ptc are
    None).  None of these changes a result."""
    if tables is None:
        tables = trace
    if prepared is not None:
        return _search_prepared(prepared, central, marginal, k, max_depth, gamma, disable_stops,
                                exhaustive_marginal, shuffle_seed, w, product, trace, subgraphs, tables)
    if hasattr(ds_or_graph, "graph"):
        g = ds_or_graph.graph
        kw_ptr, kw_nodes = ds_or_graph.kw_ptr, ds_or_graph.kw_nodes
    else:
        g = ds_or_graph
    L = _L()
    row_ptr = np.ascontiguousarray(g.row_ptr, np.int64)
    col = np.ascontiguousarray(g.col, np.int32)
    a = np.ascontiguousarray(a, np.uint8)
    kw_ptr = np.ascontiguousarray(kw_ptr, np.int64)
    kw_nodes = np.ascontiguousarray(kw_nodes, np.int32)
    c = np.ascontiguousarray(central, np.int32)
    m = np.ascontiguousarray(marginal, np.int32)
    n = len(row_ptr) - 1
    h = L.orc_search(n, int(row_ptr[-1]), _p(row_ptr), _p(col), _p(a), len(kw_ptr) - 1, _p(kw_ptr),
                     _p(kw_nodes), _p(c), len(c), _p(m) if len(m) else None, len(m), int(k),
                     int(max_depth), float(gamma), int(w), int(bool(product)), int(disable_stops),
                     int(exhaustive_marginal), int(shuffle_seed))
    return _collect(L, h, n, True, True, True)


def _search_prepared(pg, central, marginal, k, max_depth, gamma, disable_stops, exhaustive_marginal,
                     shuffle_seed, w, product, trace, subgraphs, tables) -> SearchResult:
    L = _L()
    c = np.ascontiguousarray(central, np.int32)
    m = np.ascontiguousarray(marginal, np.int32)
    flags = (1 if trace else 0) | (2 if subgraphs else 0)
    h = L.orc_search_graph(pg.handle, _p(c), len(c), _p(m) if len(m) else None, len(m), int(k), int(max_depth),
                           float(gamma), int(w), int(bool(product)), int(disable_stops),
                           int(exhaustive_marginal), int(shuffle_seed), flags)
    return _collect(L, h, pg.n, trace, subgraphs, tables)


def _collect(L, h, n, trace, subgraphs, tables) -> SearchResult:
    try:
        nsel = _scalar(L, h, F_NSEL)
        res = SearchResult(
            status=_scalar(L, h, F_STATUS),
            nodes=_get(L, h, F_RES_NODE), s_c=_get(L, h, F_RES_SC, dtype=np.int32),
            s_m=_get(L, h, F_RES_SM, dtype=np.int32), s_r=_get(L, h, F_RES_SR, dtype=np.float64),
            central=_run(L, h, 0, n, trace, tables), marginal=_run(L, h, 1, n, trace, tables),
            cg_node=_get(L, h, F_CG_NODE, 0), cg_score=_get(L, h, F_CG_SCORE, 0),
            cg_level=_get(L, h, F_CG_LEVEL, 0),
            selected=_get(L, h, F_SEL), selected_sc=_get(L, h, F_SEL_SC),
            vc_all=[_get(L, h, F_VC_ALL, 0, g_) for g_ in range(nsel)],
            vc_kw=[_get(L, h, F_VC_KW, 0, g_) for g_ in range(nsel)],
            ec=[_get(L, h, F_EC, 0, g_) for g_ in range(nsel)],
            matched=_get(L, h, F_MATCHED, dtype=np.int32),
            match_level=_get(L, h, F_MATCH_LEVEL, dtype=np.int32),
            sel_sm=_get(L, h, F_SM, dtype=np.int32),
            vm=[_get(L, h, F_VM, 0, g_) for g_ in range(nsel)] if subgraphs else None,
            em=[_get(L, h, F_EM, 0, g_) for g_ in range(nsel)] if subgraphs else None,
            ptc=_get(L, h, F_PTC, dtype=np.int32) if subgraphs else None)
    finally:
        L.orc_free(h)
    return res


def search_many(pg: PreparedGraph, queries, threads: int = 0, trace: bool = False,
                subgraphs: bool = False) -> list:
    """The oracle on many queries of one prepared graph, query-parallel over
    ``threads`` threads (default: every host core).  Each search is the
    serial oracle on its own state; only the graph is shared.  Queries are
    ``rpqgen.Query``-like objects; results come back in query order."""
    from concurrent.futures import ThreadPoolExecutor

    qs = list(queries)
    nthreads = max(1, min(threads or (os.cpu_count() or 1), len(qs) or 1))

    def one(q):
        return search(None, None, q.central, q.marginal, q.k, q.max_depth, q.gamma,
                      w=getattr(q, "w", 0), product=getattr(q, "product", False), prepared=pg,
                      trace=trace, subgraphs=subgraphs)

    if nthreads == 1:
        return [one(q) for q in qs]
    with ThreadPoolExecutor(max_workers=nthreads) as ex:
        return list(ex.map(one, qs))
