"""Seeded synthetic inputs for radial-pattern keyword search (input preparation only).

This module is shared by the CPU oracle and the CUDA library's tests and
benchmark.  It holds none of the search method's arithmetic: it builds a
labelled, bi-directed graph (every original edge gets its reverse, Section 2),
node keyword sets, keyword postings, the average-hops statistic the weighting
scheme takes as input (Section 3.1; sampled as in Section 5.1), and queries.

The paper's datasets (Wikidata dumps, AAAI keyword lists) are not available;
these generators stand in for them with power-law graphs of the same kind.
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "_rpqgen.so")
_lib = None


def build_lib(force: bool = False) -> str:
    """Compile the generator core (gcc, OpenMP) next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_lib())
        P = ctypes.c_void_p
        i64, i32, u64, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
        _lib.gen_rmat_edges.argtypes = [i32, i64, f64, f64, f64, u64, P, P]
        _lib.gen_chunglu_alias.argtypes = [i64, f64, f64, P, P]
        _lib.gen_chunglu_edges.argtypes = [i64, i64, P, P, u64, P, P]
        _lib.gen_permutation.argtypes = [i64, u64, P]
        _lib.gen_apply_permutation.argtypes = [i64, P, P]
        _lib.gen_build_csr.argtypes = [i64, i64, P, P, P, P]
        _lib.gen_build_csr.restype = i64
        _lib.gen_zipf_cdf.argtypes = [i64, f64, P]
        _lib.gen_edge_labels.argtypes = [i64, P, P, P, i64, u64, P]
        _lib.gen_node_keyword_counts.argtypes = [i64, i32, i32, u64, P]
        _lib.gen_node_keywords.argtypes = [i64, P, P, i64, u64, P]
        _lib.gen_postings.argtypes = [i64, P, P, i64, P, P]
        _lib.gen_average_hops.argtypes = [i64, P, P, i32, u64]
        _lib.gen_average_hops.restype = f64
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------- graph
@dataclass
class Graph:
    n: int
    row_ptr: np.ndarray  # int64[n+1]
    col: np.ndarray      # int32[m2], ascending per row, symmetric, no self-loops
    label: np.ndarray    # uint16[m2], same label on both directions of an edge
    n_labels: int

    @property
    def m2(self) -> int:
        return int(self.row_ptr[-1])


@dataclass
class Dataset:
    name: str
    graph: Graph
    kw_ptr: np.ndarray    # int64[n_kw+1]
    kw_nodes: np.ndarray  # int32[...], ascending per keyword
    n_kw: int
    abar: float
    alpha: float = 0.5
    meta: dict = field(default_factory=dict)

    def postings(self, kw: int) -> np.ndarray:
        return self.kw_nodes[self.kw_ptr[kw]:self.kw_ptr[kw + 1]]


def rmat_edges(scale: int, nedges: int, seed: int, a=0.57, b=0.19, c=0.19):
    src = np.empty(nedges, np.uint32)
    dst = np.empty(nedges, np.uint32)
    _L().gen_rmat_edges(scale, nedges, a, b, c, seed, _p(src), _p(dst))
    return src, dst


def _chunglu_i0(n: int, nedges: int, beta: float, max_degree: float) -> float:
    """Offset i0 so that node 0's expected degree (2 E p_0) is about max_degree."""
    g = 1.0 / (beta - 1.0)

    def p0(i0):
        # sum_{i<n} (i+i0)^-g by the midpoint integral approximation
        tot = ((n + i0 - 0.5) ** (1 - g) - (i0 - 0.5) ** (1 - g)) / (1 - g) if i0 > 0.5 else None
        if tot is None:
            tot = sum((i + i0) ** -g for i in range(64)) + \
                ((n + i0 - 0.5) ** (1 - g) - (64 + i0 - 0.5) ** (1 - g)) / (1 - g)
        return i0 ** -g / tot

    target = max_degree / (2.0 * nedges)
    lo, hi = 1e-3, 1e9
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if p0(mid) > target:
            lo = mid
        else:
            hi = mid
    return math.sqrt(lo * hi)


def chunglu_edges(n: int, nedges: int, seed: int, beta=2.1, max_degree=1e6):
    i0 = _chunglu_i0(n, nedges, beta, max_degree)
    prob = np.empty(n, np.float64)
    alias = np.empty(n, np.uint32)
    _L().gen_chunglu_alias(n, beta, i0, _p(prob), _p(alias))
    src = np.empty(nedges, np.uint32)
    dst = np.empty(nedges, np.uint32)
    _L().gen_chunglu_edges(n, nedges, _p(prob), _p(alias), seed, _p(src), _p(dst))
    return src, dst


def build_graph(n: int, src: np.ndarray, dst: np.ndarray, seed: int, n_labels=64,
                label_zipf=1.2, permute=True) -> Graph:
    """Relabel nodes (seeded permutation), symmetrise, drop self-loops and
    duplicates, sort rows; draw one Zipf label per undirected edge."""
    L = _L()
    if permute:
        perm = np.empty(n, np.uint32)
        L.gen_permutation(n, seed, _p(perm))
        L.gen_apply_permutation(len(src), _p(perm), _p(src))
        L.gen_apply_permutation(len(dst), _p(perm), _p(dst))
        del perm
    row_ptr = np.empty(n + 1, np.int64)
    col = np.empty(2 * len(src), np.uint32)
    m2 = L.gen_build_csr(n, len(src), _p(src), _p(dst), _p(row_ptr), _p(col))
    col = np.ascontiguousarray(col[:m2]).view(np.int32)
    cdf = np.empty(n_labels, np.float64)
    L.gen_zipf_cdf(n_labels, label_zipf, _p(cdf))
    label = np.empty(m2, np.uint16)
    L.gen_edge_labels(n, _p(row_ptr), _p(col), _p(cdf), n_labels, seed, _p(label))
    return Graph(n=n, row_ptr=row_ptr, col=col, label=label, n_labels=n_labels)


def node_keywords(n: int, kmin: int, kmax: int, vocab: int, zipf_s: float, seed: int):
    L = _L()
    nk_ptr = np.empty(n + 1, np.int64)
    L.gen_node_keyword_counts(n, kmin, kmax, seed, _p(nk_ptr))
    cdf = np.empty(vocab, np.float64)
    L.gen_zipf_cdf(vocab, zipf_s, _p(cdf))
    nk_ids = np.empty(int(nk_ptr[-1]), np.int32)
    L.gen_node_keywords(n, _p(nk_ptr), _p(cdf), vocab, seed, _p(nk_ids))
    kw_ptr = np.empty(vocab + 1, np.int64)
    kw_nodes = np.empty(int(nk_ptr[-1]), np.int32)
    L.gen_postings(n, _p(nk_ptr), _p(nk_ids), vocab, _p(kw_ptr), _p(kw_nodes))
    return kw_ptr, kw_nodes


def average_hops(g: Graph, nsrc: int = 32, seed: int = 1) -> float:
    col = g.col.view(np.uint32)
    return float(_L().gen_average_hops(g.n, _p(g.row_ptr), _p(col), nsrc, seed))


# ------------------------------------------------------------------------- configs
# Workload shapes: R-MAT (a=.57,b=.19,c=.19) and Chung-Lu (exponent 2.1) graphs
# standing in for the WikiSmall/WikiLarge dumps; Zipf keyword vocabularies.
CONFIGS = {
    "tiny": dict(kind="rmat", scale=14, nedges=131072, kw=(1, 3), vocab=2000, kw_zipf=1.1),
    "medium": dict(kind="rmat", scale=21, nedges=33554432, kw=(1, 4), vocab=200000, kw_zipf=1.05),
    "large": dict(kind="chunglu", n=50_000_000, nedges=400_000_000, beta=2.1, max_degree=1e6,
                  kw=(1, 4), vocab=5_000_000, kw_zipf=1.0),
    # parity-test graphs: oracle finishes in seconds; several tiles plus a ragged tail
    "small": dict(kind="rmat", scale=16, nedges=600_000, kw=(1, 3), vocab=8000, kw_zipf=1.1),
    "mid": dict(kind="rmat", scale=18, nedges=3_000_000, kw=(1, 4), vocab=30000, kw_zipf=1.05),
    "cl_small": dict(kind="chunglu", n=300_000, nedges=2_000_000, beta=2.1, max_degree=2e4,
                     kw=(1, 4), vocab=40000, kw_zipf=1.0),
    # profiling case of the large graph's kind at a tenth of its size: the
    # adjacency (about 3e8 bytes) is still larger than L2
    "cl_5m": dict(kind="chunglu", n=5_000_000, nedges=40_000_000, beta=2.1, max_degree=1e5,
                  kw=(1, 4), vocab=500_000, kw_zipf=1.0),
}


def cache_dir() -> str:
    d = os.environ.get("RPQ_CACHE", "/tmp/rpq_cache")
    os.makedirs(d, exist_ok=True)
    return d


def _key(name: str, seed: int, spec: dict) -> str:
    src_hash = hashlib.sha1(open(_SRC, "rb").read()).hexdigest()
    h = hashlib.sha1(json.dumps([name, seed, spec, src_hash], sort_keys=True).encode()).hexdigest()[:12]
    return f"{name}_s{seed}_{h}"


def make_dataset(name: str, seed: int = 1, use_cache: bool = True, **overrides) -> Dataset:
    spec = dict(CONFIGS[name])
    spec.update(overrides)
    key = _key(name, seed, spec)
    path = os.path.join(cache_dir(), key)
    files = ["row_ptr", "col", "label", "kw_ptr", "kw_nodes"]
    if use_cache and os.path.exists(os.path.join(path, "meta.json")):
        meta = json.load(open(os.path.join(path, "meta.json")))
        arr = {f: np.load(os.path.join(path, f + ".npy"), mmap_mode="r") for f in files}
        g = Graph(n=meta["n"], row_ptr=np.ascontiguousarray(arr["row_ptr"]),
                  col=np.ascontiguousarray(arr["col"]), label=np.ascontiguousarray(arr["label"]),
                  n_labels=meta["n_labels"])
        return Dataset(name=name, graph=g, kw_ptr=np.ascontiguousarray(arr["kw_ptr"]),
                       kw_nodes=np.ascontiguousarray(arr["kw_nodes"]), n_kw=meta["n_kw"],
                       abar=meta["abar"], alpha=meta["alpha"], meta=meta)
    if spec["kind"] == "rmat":
        n = 1 << spec["scale"]
        src, dst = rmat_edges(spec["scale"], spec["nedges"], seed)
    else:
        n = spec["n"]
        src, dst = chunglu_edges(n, spec["nedges"], seed, spec["beta"], spec["max_degree"])
    g = build_graph(n, src, dst, seed)
    del src, dst
    kw_ptr, kw_nodes = node_keywords(n, spec["kw"][0], spec["kw"][1], spec["vocab"], spec["kw_zipf"], seed)
    abar = average_hops(g, 32, seed)
    meta = dict(name=name, seed=seed, spec=spec, n=n, m2=g.m2, n_labels=g.n_labels,
                n_kw=spec["vocab"], abar=abar, alpha=0.5, max_degree=int(np.diff(g.row_ptr).max()))
    ds = Dataset(name=name, graph=g, kw_ptr=kw_ptr, kw_nodes=kw_nodes, n_kw=spec["vocab"],
                 abar=abar, alpha=0.5, meta=meta)
    if use_cache:
        tmp = path + f".tmp{os.getpid()}"
        os.makedirs(tmp, exist_ok=True)
        for f, a in zip(files, [g.row_ptr, g.col, g.label, kw_ptr, kw_nodes]):
            np.save(os.path.join(tmp, f + ".npy"), a)
        json.dump(meta, open(os.path.join(tmp, "meta.json"), "w"))
        try:
            os.replace(tmp, path)
        except OSError:
            pass
    return ds


# ------------------------------------------------------------------------- queries
@dataclass
class Query:
    central: list
    marginal: list
    k: int
    max_depth: int
    gamma: float = 0.5
    w: int = 0                # CG beam width (0: w = k)
    product: bool = False     # multiplicative S^r


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed, stream]))


def _distinct_ranks(rng, lo, hi, count):
    out = []
    while len(out) < count:
        r = int(rng.integers(lo, hi + 1))
        if r not in out:
            out.append(r)
    return out


def queries_uniform(n_queries: int, c_range, m_range, rank_range, k, max_depth, seed, n_kw=None):
    """|C|, |M| uniform in the given inclusive ranges; keyword ranks uniform in
    rank_range (keyword id = rank - 1), all distinct within a query."""
    rng = _rng(seed, 7)
    qs = []
    for _ in range(n_queries):
        nc = int(rng.integers(c_range[0], c_range[1] + 1))
        nm = int(rng.integers(m_range[0], m_range[1] + 1))
        ranks = _distinct_ranks(rng, rank_range[0], rank_range[1], nc + nm)
        ids = [r - 1 for r in ranks]
        qs.append(Query(central=ids[:nc], marginal=ids[nc:], k=k, max_depth=max_depth))
    return qs


def queries_mixed(ds: Dataset, n_queries: int, c_range=(2, 6), m_range=(0, 8), ks=(5, 10, 20),
                  max_depth=8, seed=1, head_min=100_000, tail_max=100):
    """Uneven query shapes: each keyword is a head keyword (postings > head_min)
    or a tail keyword (0 < postings < tail_max) with equal probability."""
    sizes = np.diff(ds.kw_ptr)
    head = np.nonzero(sizes > head_min)[0]
    if len(head) == 0:
        head = np.argsort(-sizes)[:8]
    tail = np.nonzero((sizes > 0) & (sizes < tail_max))[0]
    rng = _rng(seed, 11)
    qs = []
    for _ in range(n_queries):
        nc = int(rng.integers(c_range[0], c_range[1] + 1))
        nm = int(rng.integers(m_range[0], m_range[1] + 1))
        ids = []
        while len(ids) < nc + nm:
            pool = head if rng.random() < 0.5 else tail
            kw = int(pool[int(rng.integers(0, len(pool)))])
            if kw not in ids:
                ids.append(kw)
        qs.append(Query(central=ids[:nc], marginal=ids[nc:], k=int(ks[int(rng.integers(0, len(ks)))]),
                        max_depth=max_depth))
    return qs


def workload_queries(name: str, ds: Dataset, seed: int = 1):
    """The query set of each named workload."""
    if name == "tiny":
        return queries_uniform(1, (2, 2), (2, 2), (50, 500), 10, 6, seed)
    if name == "medium":
        return queries_uniform(64, (2, 4), (0, 4), (100, 20000), 20, 8, seed)
    if name in ("large", "cl_5m"):
        return queries_uniform(256, (3, 3), (3, 3), (100, 20000), 20, 8, seed)
    if name == "batched":
        return queries_mixed(ds, 4096, seed=seed)
    if name == "served":
        return queries_mixed(ds, 20000, seed=seed)
    raise KeyError(name)


def poisson_arrivals(n: int, rate_per_s: float, seed: int = 1) -> np.ndarray:
    """Arrival times (seconds) of a Poisson stream."""
    rng = _rng(seed, 13)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
