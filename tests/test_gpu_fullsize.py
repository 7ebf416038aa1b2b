"""Full-size parity on the benchmark workload (medium: R-MAT 2^21 nodes,
63.5M CSR entries, 64 queries, k = 20, L = 8) in the launch configuration the
benchmark times (graph-replayed rpq_search and the device-resident path):
a sample of the queries is checked against the oracle, results and work
counters bit for bit, S^r within 1e-6 relative."""
import numpy as np
import pytest

import oracle
import paper_2001_06770_b300 as rpq
import rpqgen
from tests.gpu_common import results_match

pytestmark = pytest.mark.gpu

SAMPLE = [0, 1, 2, 7, 19, 42, 63]


@pytest.fixture(scope="module")
def medium():
    ds = rpqgen.make_dataset("medium")
    act = oracle.dataset_activation(ds)
    kg = rpq.KG.from_dataset(ds)
    yield ds, act, kg, rpqgen.workload_queries("medium", ds)
    kg.close()


def test_medium_activation_levels(medium):
    ds, act, kg, qs = medium
    adj, amax = kg.export()
    assert np.array_equal(amax, act.amax)
    g = ds.graph
    rng = np.random.default_rng(0)
    for v in rng.integers(0, g.n, size=2000):
        b, e = g.row_ptr[v], g.row_ptr[v + 1]
        expect = np.sort((act.a[b:e].astype(np.uint32) << 26) | g.col[b:e].astype(np.uint32))
        assert np.array_equal(adj[b:e], expect)


def test_medium_sampled_queries(medium):
    import torch
    ds, act, kg, qs = medium
    for i in SAMPLE:
        q = qs[i]
        orc = oracle.search(ds, act.a, q.central, q.marginal, q.k, q.max_depth, q.gamma)
        res, st = kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)
        results_match(res, orc)
        assert st["e_act_central"] == orc.central.e_act
        if orc.marginal is not None:
            assert st["e_act_marginal"] == orc.marginal.e_act
            assert st["levels_marginal"] == orc.marginal.last_level
        assert st["levels_central"] == orc.central.last_level
        kw = torch.tensor(list(q.central) + list(q.marginal), dtype=torch.int32, device="cuda")
        out = torch.zeros(q.k * 24, dtype=torch.uint8, device="cuda")
        nout = torch.zeros(1, dtype=torch.int32, device="cuda")
        kg.search_device(kw.data_ptr(), len(q.central), len(q.marginal), q.k, q.max_depth, q.gamma,
                         out.data_ptr(), nout.data_ptr())
        kg.sync_device()
        got = np.frombuffer(out.cpu().numpy().tobytes(), rpq.RESULT_DTYPE)[:int(nout.item())]
        assert got.tobytes() == res.tobytes()
