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
