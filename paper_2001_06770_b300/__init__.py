"""Python binding of librpq: radial-pattern keyword search on a B300 GPU.

Argument marshalling only.  Every step of the search runs in the CUDA
kernels of ``librpq.so`` (built from ``csrc/`` for sm_103a); there is no
CPU path.  If the library cannot be loaded the import of this binding's
functions raises.

Typical use::

    kg = KG(row_ptr, col, label, n_labels, kw_ptr, kw_nodes, alpha=0.5, abar=3.3)
    res, stats = kg.search(central=[12, 40], marginal=[7], k=20, max_depth=8)
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None

RPQ_OK, RPQ_EINVAL, RPQ_ENOMEM, RPQ_ETIMEOUT, RPQ_ECUDA, RPQ_ELIMIT, RPQ_EINTERNAL, RPQ_ESIZE = \
    0, -1, -2, -3, -4, -5, -6, -7
MAX_KEYWORDS, MAX_K, MAX_LEVEL, MAX_LABELS = 8, 64, 63, 8192
INF = 255
SYMBOLS = ["rpq_load_kg", "rpq_free_kg", "rpq_kg_export", "rpq_kg_info", "rpq_search", "rpq_search_batch",
           "rpq_search_batch_persistent",
           "rpq_trace", "rpq_search_subgraphs", "rpq_search_device", "rpq_sync_device", "rpq_slot_stream", "rpq_set_profiling",
           "rpq_profile_read", "rpq_profile_levels", "rpq_topk_keys_noalloc", "rpq_server_create", "rpq_server_create_sized", "rpq_server_info", "rpq_server_pages",
           "rpq_server_submit", "rpq_server_poll", "rpq_server_replay", "rpq_server_destroy",
           "rpq_get_tuning", "rpq_set_tuning", "rpq_autotune", "rpq_transfer_bytes",
           "rpq_strerror", "rpq_last_error"]
PROF_CLASSES = ["setup", "enqueue", "expand", "topk", "recover", "results"]


class RPQError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class KGDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m2", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("label", ctypes.c_void_p), ("n_labels", ctypes.c_int32),
                ("n_kw", ctypes.c_int32), ("kw_ptr", ctypes.c_void_p), ("kw_nodes", ctypes.c_void_p),
                ("alpha", ctypes.c_double), ("abar", ctypes.c_double)]


class Query(ctypes.Structure):
    _fields_ = [("central", ctypes.c_void_p), ("n_c", ctypes.c_int32), ("marginal", ctypes.c_void_p),
                ("n_m", ctypes.c_int32), ("k", ctypes.c_int32), ("max_depth", ctypes.c_int32),
                ("gamma", ctypes.c_double), ("w", ctypes.c_int32), ("score", ctypes.c_int32)]


SCORE_SUM, SCORE_PRODUCT = 0, 1


class Stats(ctypes.Structure):
    _fields_ = [("e_act_central", ctypes.c_int64), ("e_act_marginal", ctypes.c_int64),
                ("hits_central", ctypes.c_int64), ("hits_marginal", ctypes.c_int64),
                ("levels_central", ctypes.c_int32), ("levels_marginal", ctypes.c_int32),
                ("n_cg", ctypes.c_int32), ("n_selected", ctypes.c_int32),
                ("work_units", ctypes.c_int64), ("work_items", ctypes.c_int64), ("frontier_nodes", ctypes.c_int64),
                ("kernels", ctypes.c_int64), ("e_act_skipped", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class TraceBuf(ctypes.Structure):
    _fields_ = [("h_central", ctypes.c_void_p), ("h_marginal", ctypes.c_void_p),
                ("frontier_c_ptr", ctypes.c_void_p), ("frontier_c", ctypes.c_void_p),
                ("frontier_c_cap", ctypes.c_int64), ("frontier_c_levels", ctypes.c_int32),
                ("frontier_m_ptr", ctypes.c_void_p), ("frontier_m", ctypes.c_void_p),
                ("frontier_m_cap", ctypes.c_int64), ("frontier_m_levels", ctypes.c_int32),
                ("cgs", ctypes.c_void_p), ("cg_cap", ctypes.c_int64), ("n_cgs", ctypes.c_int64),
                ("vc", ctypes.c_void_p), ("vc_cap", ctypes.c_int64), ("n_vc", ctypes.c_int64),
                ("selected", ctypes.c_int32 * MAX_K), ("n_selected", ctypes.c_int32)]


class Completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int32), ("n_res", ctypes.c_int32),
                ("res", ctypes.c_uint8 * (24 * MAX_K)), ("stats", Stats), ("latency_s", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("queue_div", ctypes.c_int32), ("next_queue_mult", ctypes.c_int32),
                ("batch_slots", ctypes.c_int32), ("flat_levels", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 6), ("launches", ctypes.c_int64 * 6)]


class LevelProfile(ctypes.Structure):
    """rpq_level_profile of include/rpq.h."""
    _fields_ = [("run", ctypes.c_int32), ("level", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("frontier", ctypes.c_int32), ("columns", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("units", ctypes.c_int64), ("items", ctypes.c_int64),
                ("e_act", ctypes.c_int64), ("claims", ctypes.c_int64), ("enqueue_ms", ctypes.c_double),
                ("target_ms", ctypes.c_double), ("expand_ms", ctypes.c_double)]


LVL_EXPANDED, LVL_SKIPPED, LVL_STOP, LVL_QUEUE = 1, 2, 4, 8


class Subgraphs(ctypes.Structure):
    """rpq_subgraphs of include/rpq.h."""
    _fields_ = [("nodes", ctypes.c_void_p), ("nodes_cap", ctypes.c_int64),
                ("edges", ctypes.c_void_p), ("edges_cap", ctypes.c_int64),
                ("node_off", ctypes.c_int64 * (MAX_K * 3 + 1)), ("edge_off", ctypes.c_int64 * (MAX_K * 2 + 1)),
                ("ptc", ctypes.c_int32 * MAX_K), ("nodes_total", ctypes.c_int64), ("edges_total", ctypes.c_int64)]


RESULT_DTYPE = np.dtype([("node", np.int32), ("s_c", np.int32), ("s_m", np.int32), ("reserved", np.int32),
                         ("s_r", np.float64)])


def library_path() -> str:
    """librpq.so of this package, or the file named by RPQ_LIBRARY (to compare
    two builds of the library on the same inputs)."""
    return os.environ.get("RPQ_LIBRARY") or _build.LIB


def lib():
    """Load librpq.so, building it first when sources are newer."""
    global _lib
    if _lib is None:
        path = library_path()
        if path == _build.LIB and _build.stale():
            _build.build()
        L = ctypes.CDLL(path)
        P, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.rpq_load_kg.argtypes = [ctypes.POINTER(KGDesc), ctypes.POINTER(P)]
        L.rpq_free_kg.argtypes = [P]
        L.rpq_kg_export.argtypes = [P, P, P]
        L.rpq_kg_info.argtypes = [P, P, P, P]
        L.rpq_search.argtypes = [P, ctypes.POINTER(Query), P, P, P]
        L.rpq_search_batch.argtypes = [P, P, i32, P, P, P, P]
        L.rpq_search_batch_persistent.argtypes = [P, P, i32, P, P, P, P]
        L.rpq_trace.argtypes = [P, ctypes.POINTER(Query), P, P, P, ctypes.POINTER(TraceBuf)]
        L.rpq_search_subgraphs.argtypes = [P, ctypes.POINTER(Query), P, P, P, ctypes.POINTER(Subgraphs)]
        L.rpq_search_device.argtypes = [P, P, i32, i32, i32, i32, f64, P, P]
        L.rpq_sync_device.argtypes = [P]
        L.rpq_slot_stream.argtypes = [P, i32, ctypes.POINTER(P)]
        L.rpq_set_profiling.argtypes = [P, i32]
        L.rpq_profile_read.argtypes = [P, ctypes.POINTER(Profile), i32]
        L.rpq_profile_levels.argtypes = [P, P, i32, P, i32]
        L.rpq_topk_keys_noalloc.argtypes = [P, ctypes.c_uint32, i32, P, P, P]
        L.rpq_server_create.argtypes = [P, i64, i32, ctypes.POINTER(P)]
        L.rpq_server_create_sized.argtypes = [P, i32, i32, i32, ctypes.POINTER(P)]
        L.rpq_server_info.argtypes = [P, P, P, P, P]
        L.rpq_server_pages.argtypes = [P, P, P, P, P, P]
        L.rpq_server_submit.argtypes = [P, ctypes.POINTER(Query), ctypes.c_uint64]
        L.rpq_server_poll.argtypes = [P, P, i32, P, i32]
        L.rpq_server_replay.argtypes = [P, P, P, i32, P, P, P, P, P]
        L.rpq_server_destroy.argtypes = [P]
        L.rpq_get_tuning.argtypes = [P, ctypes.POINTER(Tuning)]
        L.rpq_set_tuning.argtypes = [P, ctypes.POINTER(Tuning)]
        L.rpq_autotune.argtypes = [P, P, i32, i32, ctypes.POINTER(Tuning)]
        L.rpq_transfer_bytes.argtypes = [i32, P, P]
        L.rpq_strerror.argtypes = [ctypes.c_int]
        L.rpq_strerror.restype = ctypes.c_char_p
        L.rpq_last_error.restype = ctypes.c_char_p
        for f in SYMBOLS[:-2]:
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc: int):
    if rc != RPQ_OK:
        raise RPQError(rc, lib().rpq_last_error().decode())


def _ptr(a):
    # the address as a Python int: every argument and field it feeds is c_void_p
    return None if a is None else a.ctypes.data


def transfer_bytes(k: int):
    """(host-to-device, device-to-host) bytes of one rpq_search with k results."""
    h, d = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().rpq_transfer_bytes(int(k), ctypes.byref(h), ctypes.byref(d)))
    return h.value, d.value


def topk_keys_noalloc(d_keys: int, n: int, k: int, d_out: int, d_n_out: int, stream: int = 0):
    """k smallest of n uint32 keys in device memory, without any allocation
    (raw device pointers; see rpq_topk_keys_noalloc in include/rpq.h)."""
    _check(lib().rpq_topk_keys_noalloc(ctypes.c_void_p(d_keys), n, k, ctypes.c_void_p(d_out),
                                       ctypes.c_void_p(d_n_out), ctypes.c_void_p(stream or None)))


@dataclass
class QuerySpec:
    central: list
    marginal: list
    k: int
    max_depth: int
    gamma: float = 0.5
    w: int = 0
    product: bool = False


def _query(central, marginal, k, max_depth, gamma, keep, w=0, product=False):
    c = np.ascontiguousarray(central, np.int32)
    m = np.ascontiguousarray(marginal, np.int32)
    keep.extend([c, m])
    return Query(_ptr(c), len(c), _ptr(m) if len(m) else None, len(m), int(k), int(max_depth), float(gamma),
                 int(w), SCORE_PRODUCT if product else SCORE_SUM)


def _query_of(q, keep):
    """rpq_query of a query object (central, marginal, k, max_depth and
    optional gamma, w, product attributes)."""
    return _query(q.central, q.marginal, q.k, q.max_depth, getattr(q, "gamma", 0.5), keep,
                  getattr(q, "w", 0), getattr(q, "product", False))


class KG:
    """A knowledge graph resident on the current CUDA device."""

    def __init__(self, row_ptr, col, label, n_labels, kw_ptr, kw_nodes, alpha=0.5, abar=3.0):
        self._h = ctypes.c_void_p()
        self._keep = [np.ascontiguousarray(row_ptr, np.int64), np.ascontiguousarray(col, np.int32),
                      np.ascontiguousarray(label, np.uint16), np.ascontiguousarray(kw_ptr, np.int64),
                      np.ascontiguousarray(kw_nodes, np.int32)]
        rp, cl, lb, kp, kn = self._keep
        self.n = len(rp) - 1
        self.m2 = int(rp[-1])
        d = KGDesc(self.n, self.m2, _ptr(rp), _ptr(cl), _ptr(lb), int(n_labels), len(kp) - 1, _ptr(kp), _ptr(kn),
                   float(alpha), float(abar))
        _check(lib().rpq_load_kg(ctypes.byref(d), ctypes.byref(self._h)))
        self._keep = None

    @classmethod
    def from_dataset(cls, ds):
        g = ds.graph
        return cls(g.row_ptr, g.col, g.label, g.n_labels, ds.kw_ptr, ds.kw_nodes, ds.alpha, ds.abar)

    def close(self):
        if self._h:
            lib().rpq_free_kg(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        n, m2, b = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().rpq_kg_info(self._h, ctypes.byref(n), ctypes.byref(m2), ctypes.byref(b)))
        return dict(n=n.value, m2=m2.value, device_bytes=b.value)

    def export(self):
        """Packed adjacency ((level << 26) | neighbour, rows ascending) and amax."""
        adj = np.empty(self.m2, np.uint32)
        amax = np.empty(self.n, np.uint8)
        _check(lib().rpq_kg_export(self._h, _ptr(adj), _ptr(amax)))
        return adj, amax

    def search(self, central, marginal, k, max_depth, gamma=0.5, w=0, product=False):
        keep = []
        q = _query(central, marginal, k, max_depth, gamma, keep, w, product)
        out = np.zeros(max(int(k), 1), RESULT_DTYPE)
        n_out = ctypes.c_int32()
        st = Stats()
        _check(lib().rpq_search(self._h, ctypes.byref(q), _ptr(out), ctypes.byref(n_out), ctypes.byref(st)))
        return out[:n_out.value].copy(), st.as_dict()

    def search_batch(self, queries, persistent=False):
        """queries: iterable of objects with central, marginal, k, max_depth
        (and optionally gamma).  Returns a list of (results, stats, status).
        persistent: the whole batch in one persistent kernel launch fed by a
        device work queue (rpq_search_batch_persistent) instead of concurrent
        per-query graphs on the batch slots."""
        queries = list(queries)
        keep = []
        arr = (Query * max(len(queries), 1))()
        for i, qs in enumerate(queries):
            arr[i] = _query_of(qs, keep)
        ks = [int(q.k) for q in queries]
        base = np.concatenate([[0], np.cumsum(ks)]).astype(np.int64)
        out = np.zeros(max(int(base[-1]), 1), RESULT_DTYPE)
        n_out = np.zeros(max(len(queries), 1), np.int32)
        status = np.zeros(max(len(queries), 1), np.int32)
        st = (Stats * max(len(queries), 1))()
        fn = lib().rpq_search_batch_persistent if persistent else lib().rpq_search_batch
        _check(fn(self._h, ctypes.cast(arr, ctypes.c_void_p), len(queries), _ptr(out),
                  _ptr(n_out), _ptr(status), ctypes.cast(st, ctypes.c_void_p)))
        return [(out[base[i]:base[i] + n_out[i]].copy(), st[i].as_dict(), int(status[i])) for i in range(len(queries))]

    def trace(self, central, marginal, k, max_depth, gamma=0.5, frontier_cap=None, w=0, product=False):
        """Search one query and return its intermediate state for inspection."""
        keep = []
        q = _query(central, marginal, k, max_depth, gamma, keep, w, product)
        nc, nm = len(central), len(marginal)
        cap = frontier_cap or self.n * (max_depth + 1)
        hc = np.empty((self.n, nc), np.uint8)
        hm = np.empty((self.n, max(nm, 1)), np.uint8)
        fcp = np.zeros(MAX_LEVEL + 2, np.int64)
        fmp = np.zeros(MAX_LEVEL + 2, np.int64)
        fc = np.empty(cap, np.int32)
        fm = np.empty(cap, np.int32)
        cgs = np.empty(self.n, np.int64)
        vc = np.empty(self.n * 4, np.int64)
        tb = TraceBuf(_ptr(hc), _ptr(hm) if nm else None, _ptr(fcp), _ptr(fc), cap, 0, _ptr(fmp), _ptr(fm), cap, 0,
                      _ptr(cgs), len(cgs), 0, _ptr(vc), len(vc), 0)
        out = np.zeros(max(int(k), 1), RESULT_DTYPE)
        n_out = ctypes.c_int32()
        st = Stats()
        _check(lib().rpq_trace(self._h, ctypes.byref(q), _ptr(out), ctypes.byref(n_out), ctypes.byref(st),
                               ctypes.byref(tb)))
        fr_c = [fc[fcp[l]:fcp[l + 1]].copy() for l in range(tb.frontier_c_levels)]
        fr_m = [fm[fmp[l]:fmp[l + 1]].copy() for l in range(tb.frontier_m_levels)]
        vcs = vc[:tb.n_vc]
        nsel = tb.n_selected
        return dict(results=out[:n_out.value].copy(), stats=st.as_dict(), h_central=hc,
                    h_marginal=hm[:, :nm] if nm else None, frontiers_central=fr_c, frontiers_marginal=fr_m,
                    cgs=cgs[:tb.n_cgs].copy(), selected=np.array(tb.selected[:nsel], np.int64),
                    vc=[np.sort(vcs[(vcs >> 26) == g] & ((1 << 26) - 1)) for g in range(nsel)])

    def search_subgraphs(self, central, marginal, k, max_depth, gamma=0.5, nodes_cap=1 << 16, edges_cap=1 << 16,
                         w=0, product=False):
        """Search one query and return (results, stats, subgraphs): one dict per
        result with the node lists ``vc`` (V^c), ``vc_kw`` (V_C), ``vm`` (V^m),
        the edge lists ``ec`` (E^c), ``em`` (E^m) as (n, q) rows, and ``ptc``
        (1 holds, 0 violated, -1 without marginal keywords).  Lists are in no
        particular order.  Buffers grow once when the library reports
        RPQ_ESIZE."""
        keep = []
        q = _query(central, marginal, k, max_depth, gamma, keep, w, product)
        out = np.zeros(max(int(k), 1), RESULT_DTYPE)
        n_out = ctypes.c_int32()
        st = Stats()
        for _ in range(2):
            nodes = np.empty(max(nodes_cap, 1), np.int32)
            edges = np.empty((max(edges_cap, 1), 2), np.int32)
            sg = Subgraphs(nodes.ctypes.data, nodes_cap, edges.ctypes.data, edges_cap)
            rc = lib().rpq_search_subgraphs(self._h, ctypes.byref(q), _ptr(out), ctypes.byref(n_out),
                                            ctypes.byref(st), ctypes.byref(sg))
            if rc != RPQ_ESIZE:
                break
            nodes_cap, edges_cap = max(nodes_cap, sg.nodes_total), max(edges_cap, sg.edges_total)
        _check(rc)
        no, eo = list(sg.node_off), list(sg.edge_off)
        subs = []
        for r in range(n_out.value):
            nl = [nodes[no[3 * r + i]:no[3 * r + i + 1]].copy() for i in range(3)]
            el = [edges[eo[2 * r + i]:eo[2 * r + i + 1]].copy() for i in range(2)]
            subs.append(dict(vc=nl[0], vc_kw=nl[1], vm=nl[2], ec=el[0], em=el[1], ptc=int(sg.ptc[r])))
        return out[:n_out.value].copy(), st.as_dict(), subs

    def search_device(self, d_keywords: int, n_c: int, n_m: int, k: int, max_depth: int, gamma: float,
                      d_out: int, d_n_out: int):
        """Enqueue a search whose keyword ids (int32) and outputs live in
        device memory (raw device pointers, e.g. ``tensor.data_ptr()``)."""
        _check(lib().rpq_search_device(self._h, ctypes.c_void_p(d_keywords), n_c, n_m, k, max_depth, gamma,
                                       ctypes.c_void_p(d_out), ctypes.c_void_p(d_n_out)))

    def sync_device(self):
        _check(lib().rpq_sync_device(self._h))

    def tuning(self):
        t = Tuning()
        _check(lib().rpq_get_tuning(self._h, ctypes.byref(t)))
        return t.as_dict()

    def set_tuning(self, **kw):
        t = Tuning(**{**self.tuning(), **kw})
        _check(lib().rpq_set_tuning(self._h, ctypes.byref(t)))

    def autotune(self, queries, repeats: int = 3):
        """Time the work-split settings on the sample queries and keep the
        fastest (rpq_autotune); returns the chosen tuning."""
        queries = list(queries)
        keep = []
        arr = (Query * len(queries))()
        for i, q in enumerate(queries):
            arr[i] = _query_of(q, keep)
        t = Tuning()
        _check(lib().rpq_autotune(self._h, ctypes.cast(arr, ctypes.c_void_p), len(queries), int(repeats),
                                  ctypes.byref(t)))
        return t.as_dict()

    def slot_stream(self, slot: int = 0) -> int:
        """Raw cudaStream_t of a search slot (for CUDA-event timing)."""
        st = ctypes.c_void_p()
        _check(lib().rpq_slot_stream(self._h, slot, ctypes.byref(st)))
        return st.value or 0

    def set_profiling(self, enable: bool):
        _check(lib().rpq_set_profiling(self._h, int(bool(enable))))

    def profile(self, reset: bool = False):
        """Accumulated device ms and launch counts per kernel class."""
        p = Profile()
        _check(lib().rpq_profile_read(self._h, ctypes.byref(p), int(bool(reset))))
        return {c: (p.ms[i], p.launches[i]) for i, c in enumerate(PROF_CLASSES)}

    def profile_levels(self, reset: bool = False):
        """Per-Glevel records of the profiled searches (rpq_profile_levels):
        a list of dicts with run, level, flags, frontier, units, items, e_act,
        claims and the enqueue / V_C check / expansion device milliseconds."""
        n = ctypes.c_int32()
        _check(lib().rpq_profile_levels(self._h, None, 0, ctypes.byref(n), 0))
        buf = (LevelProfile * max(n.value, 1))()
        _check(lib().rpq_profile_levels(self._h, ctypes.cast(buf, ctypes.c_void_p), n.value, ctypes.byref(n),
                                        int(bool(reset))))
        return [{f: getattr(buf[i], f) for f, _ in LevelProfile._fields_} for i in range(n.value)]


class Server:
    """Continuous-batching server over a loaded KG (rpq_server_* in rpq.h)."""

    def __init__(self, kg: KG, budget_bytes: int = 0, max_slots: int = 256, slots: int = 0, h_pages: int = 0,
                 r_pages: int = 0):
        """Sized from budget_bytes (rpq_server_create), or, with `slots`,
        from explicit slot and page counts (rpq_server_create_sized)."""
        self._h = ctypes.c_void_p()
        self.kg = kg
        if slots:
            _check(lib().rpq_server_create_sized(kg._h, int(slots), int(h_pages), int(r_pages),
                                                 ctypes.byref(self._h)))
        else:
            _check(lib().rpq_server_create(kg._h, int(budget_bytes), int(max_slots), ctypes.byref(self._h)))

    def info(self):
        n, b, r, w = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().rpq_server_info(self._h, ctypes.byref(n), ctypes.byref(b), ctypes.byref(r), ctypes.byref(w)))
        hp, hb, rp, rb, pk = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
        _check(lib().rpq_server_pages(self._h, ctypes.byref(hp), ctypes.byref(hb), ctypes.byref(rp), ctypes.byref(rb),
                                      ctypes.byref(pk)))
        return dict(slots=n.value, slot_bytes=b.value, running=r.value, waiting=w.value, h_pages=hp.value,
                    h_page_bytes=hb.value, r_pages=rp.value, r_page_bytes=rb.value, peak_running=pk.value,
                    device_bytes=n.value * b.value + hp.value * hb.value + rp.value * rb.value)

    def submit(self, q, tag: int):
        keep = []
        qq = _query_of(q, keep)
        _check(lib().rpq_server_submit(self._h, ctypes.byref(qq), ctypes.c_uint64(tag)))

    def poll(self, wait: bool = False, max_done: int = 256):
        """List of (tag, status, results, stats, latency_s) of finished queries."""
        buf = (Completion * max_done)()
        n = ctypes.c_int32()
        _check(lib().rpq_server_poll(self._h, ctypes.cast(buf, ctypes.c_void_p), max_done, ctypes.byref(n),
                                     int(bool(wait))))
        out = []
        for i in range(n.value):
            c = buf[i]
            res = np.frombuffer(bytes(c.res), RESULT_DTYPE)[:c.n_res].copy()
            out.append((int(c.tag), int(c.status), res, c.stats.as_dict(), float(c.latency_s)))
        return out

    def replay(self, queries, arrival_s):
        """Serve the queries at the given arrival times (seconds, non-decreasing)
        natively; returns (results list, latency_s array, status array, wall_s)."""
        queries = list(queries)
        nq = len(queries)
        keep = []
        arr = (Query * max(nq, 1))()
        for i, q in enumerate(queries):
            arr[i] = _query_of(q, keep)
        t = np.ascontiguousarray(arrival_s, np.float64)
        lat = np.zeros(max(nq, 1), np.float64)
        status = np.zeros(max(nq, 1), np.int32)
        n_out = np.zeros(max(nq, 1), np.int32)
        base = np.concatenate([[0], np.cumsum([int(q.k) for q in queries])]).astype(np.int64)
        out = np.zeros(max(int(base[-1]), 1), RESULT_DTYPE)
        wall = ctypes.c_double()
        _check(lib().rpq_server_replay(self._h, ctypes.cast(arr, ctypes.c_void_p), _ptr(t), nq, _ptr(lat),
                                       _ptr(status), _ptr(n_out), _ptr(out), ctypes.byref(wall)))
        res = [out[base[i]:base[i] + n_out[i]].copy() for i in range(nq)]
        return res, lat[:nq], status[:nq], wall.value

    def close(self):
        if self._h:
            lib().rpq_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
