"""The bounds-checked build of the library (librpq_checked.so, compiled with
-DRPQ_CHECKED): the search kernels test every index they derive from device
data - frontier queue and recovery list entries, CSR offsets, neighbour ids,
work-list and CG-list positions - before using it, and a failed test makes
the query fail with RPQ_EINTERNAL instead of touching memory outside a
buffer.  Over the parity graphs and every search path (traced and
graph-replayed searches, both batch forms, the server, result subgraphs) the
checked build must report no failed test and give the oracle's results.  It
runs in a child process because the binding loads one library per process."""
import os
import subprocess
import sys

import pytest

from paper_2001_06770_b300 import build as _build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import os, sys
sys.path.insert(0, os.getcwd())
import numpy as np
import oracle, rpqgen
import paper_2001_06770_b300 as rpq
from tests.gpu_common import dataset_queries, oracle_query, results_match, trace_matches

assert os.path.basename(rpq.library_path()) == "librpq_checked.so"
for name in ("small", "cl_small"):
    ds = rpqgen.make_dataset(name)
    act = oracle.dataset_activation(ds)
    kg = rpq.KG.from_dataset(ds)
    try:
        qs = dataset_queries(name, ds, 8, seed=29)
        orcs = [oracle_query(ds, act, q) for q in qs]
        for q, o in zip(qs, orcs):
            trace_matches(kg.trace(q.central, q.marginal, q.k, q.max_depth, q.gamma), o)
            res, _ = kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)
            results_match(res, o)
        for persistent in (False, True):
            for (res, st, status), o in zip(kg.search_batch(qs, persistent=persistent), orcs):
                assert status == 0, status
                results_match(res, o)
        srv = rpq.Server(kg, slots=3, h_pages=24, r_pages=24)
        try:
            res, lat, status, wall = srv.replay(qs, np.zeros(len(qs)))
            assert (status == 0).all(), status
            for r, o in zip(res, orcs):
                results_match(r, o)
        finally:
            srv.close()
        for q, o in zip(qs[:4], orcs[:4]):
            res, st, subs = kg.search_subgraphs(q.central, q.marginal, q.k, q.max_depth, q.gamma)
            results_match(res, o)
    finally:
        kg.close()
print("checked build: no failed bounds check")
'''


def test_checked_build_passes_every_search_path():
    lib = _build.build(checked=True)          # up to date after build(); compiled here otherwise
    env = dict(os.environ, RPQ_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0 and "no failed bounds check" in r.stdout, (r.stdout[-3000:], r.stderr[-3000:])
