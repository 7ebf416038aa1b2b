"""Query-sharded serving over graph replicas on real graphs: two ranks
(gloo), each with its own copy of the knowledge graph on cuda:0 and its own
share of the queries, gather every result on rank 0 in query order; the
gathered results equal the oracle's.  (One GPU serves both ranks here; the
ranks' kernels never wait on one another, only the host gather does.)"""
import os
import pickle
import socket

import pytest
import torch.multiprocessing as mp

import oracle
import rpqgen
from tests.gpu_common import dataset_queries, oracle_query, results_match

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), LOCAL_RANK="0", WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    import paper_2001_06770_b300 as rpq
    import rpqgen as gen
    from paper_2001_06770_b300 import replicas
    from tests.gpu_common import dataset_queries as dq
    torch.cuda.set_device(0)
    dist.init_process_group("gloo")
    ds = gen.make_dataset("small")
    kg = rpq.KG.from_dataset(ds)
    try:
        got = replicas.search_sharded(kg, dq("small", ds, 10, seed=51))
    finally:
        kg.close()
    if rank == 0:
        with open(out, "wb") as f:
            pickle.dump([(r.tobytes(), r.dtype.descr, st) for r, _, st in got], f)
    dist.destroy_process_group()


def test_sharded_replicas_equal_oracle(tmp_path):
    import numpy as np
    import paper_2001_06770_b300 as rpq
    out = str(tmp_path / "gathered.pkl")
    mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    got = pickle.load(open(out, "rb"))
    ds = rpqgen.make_dataset("small")
    act = oracle.dataset_activation(ds)
    qs = dataset_queries("small", ds, 10, seed=51)
    assert len(got) == len(qs)
    for q, (raw, _, status) in zip(qs, got):
        assert status == 0
        res = np.frombuffer(raw, rpq.RESULT_DTYPE)
        results_match(res, oracle_query(ds, act, q))
