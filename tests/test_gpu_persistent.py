"""The optional persistent run kernel (RPQ_PERSISTENT=1: one cooperative
launch per run with bounded grid barriers) gives the oracle's results.  Runs
in a child process because the switch is read once per process."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

CHILD = r"""
import sys
sys.path.insert(0, {root!r})
import oracle, rpqgen
import paper_2001_06770_b300 as rpq
from tests.gpu_common import dataset_queries, oracle_query, results_match
for name in ("tiny", "cl_small"):
    ds = rpqgen.make_dataset(name)
    act = oracle.dataset_activation(ds)
    kg = rpq.KG.from_dataset(ds)
    for q in dataset_queries(name, ds, 6, seed=31):
        res, st = kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)
        orc = oracle_query(ds, act, q)
        results_match(res, orc)
        if orc.central is not None:
            assert st["e_act_central"] == orc.central.e_act
            assert st["kernels"] > 0
        if orc.marginal is not None:
            assert st["e_act_marginal"] == orc.marginal.e_act
    kg.close()
print("persistent ok")
"""


def test_persistent_run_kernel_matches_oracle():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RPQ_PERSISTENT="1")
    out = subprocess.run([sys.executable, "-c", CHILD.format(root=root)], env=env, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "persistent ok" in out.stdout


TIMEOUT_CHILD = r"""
import sys
sys.path.insert(0, {root!r})
import numpy as np
import torch
import oracle, rpqgen
import paper_2001_06770_b300 as rpq
from tests.gpu_common import dataset_queries, oracle_query, results_match
ds = rpqgen.make_dataset("tiny")
kg = rpq.KG.from_dataset(ds)
q = dataset_queries("tiny", ds, 2, seed=33)[0]
try:
    kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)
    raise SystemExit("host path: no error")
except rpq.RPQError as e:
    assert e.code == rpq.RPQ_ETIMEOUT, e
try:                     # the host-path query also left its error in the sticky word: read and clear it
    kg.sync_device()
except rpq.RPQError as e:
    assert e.code == rpq.RPQ_ETIMEOUT, e
kw = torch.tensor(list(q.central) + list(q.marginal), dtype=torch.int32, device="cuda")
out = torch.zeros(q.k * 24, dtype=torch.uint8, device="cuda")
nout = torch.zeros(1, dtype=torch.int32, device="cuda")
kg.search_device(kw.data_ptr(), len(q.central), len(q.marginal), q.k, q.max_depth, q.gamma,
                 out.data_ptr(), nout.data_ptr())
try:
    kg.sync_device()
    raise SystemExit("device path: no error")
except rpq.RPQError as e:
    assert e.code == rpq.RPQ_ETIMEOUT, e
# the context stays usable: the traced search (kernel pairs, no grid barrier)
act = oracle.dataset_activation(ds)
tr = kg.trace(q.central, q.marginal, q.k, q.max_depth, q.gamma)
results_match(tr["results"], oracle_query(ds, act, q))
kg.close()
print("timeout ok")
"""


def test_persistent_barrier_timeout_reported():
    """A grid barrier of the persistent run kernel that waits longer than its
    limit ends the kernel with RPQ_ETIMEOUT, on the host path (control block)
    and on the device path (the slot's sticky error word, rpq_sync_device);
    the limit is set to a few cycles so that every wait gives up at once, and
    the context stays usable."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RPQ_PERSISTENT="1", RPQ_BARRIER_LIMIT="1")
    out = subprocess.run([sys.executable, "-c", TIMEOUT_CHILD.format(root=root)], env=env, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "timeout ok" in out.stdout
