"""The multi-core CPU baseline (RAKS-CPU) returns the oracle's results."""
import numpy as np
import pytest

import oracle
import raks_cpu
import rpqgen
from tests.gpu_common import dataset_queries


@pytest.mark.parametrize("name", ["tiny", "small"])
def test_raks_cpu_matches_oracle(name):
    ds = rpqgen.make_dataset(name)
    act = oracle.dataset_activation(ds)
    a = raks_cpu.activation(ds)
    assert np.array_equal(a, act.a)
    qs = dataset_queries(name, ds, 8, seed=41) + rpqgen.workload_queries("tiny", ds)[:1]
    for q in qs:
        orc = oracle.search(ds, act.a, q.central, q.marginal, q.k, q.max_depth, q.gamma)
        node, sc, sm, sr = raks_cpu.search(ds, a, q.central, q.marginal, q.k, q.max_depth, q.gamma)
        assert node.tolist() == orc.nodes.tolist()
        assert sc.tolist() == orc.s_c.tolist() and sm.tolist() == orc.s_m.tolist()
        assert np.allclose(sr, orc.s_r, rtol=1e-6, atol=0)
