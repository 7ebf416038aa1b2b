"""Multi-process host logic on CPU with the gloo backend, world size 2: the
benchmark's rank handling (barrier, max over ranks, rank 0 alone printing the
reference arm) and the query-sharded serving helper (round-robin shares,
results gathered in query order).  No GPU is involved."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))


def _dist_helpers(rank, world, port, out):
    _env(rank, world, port)
    sys.path.insert(0, ROOT)
    import bench
    ws, r, local = bench.dist_init()
    bench.barrier(ws)
    m = bench.allmax(ws, float(rank) + 0.5)
    with open(f"{out}.{rank}", "w") as f:
        json.dump({"ws": ws, "rank": r, "local": local, "max": m}, f)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_bench_rank_helpers(tmp_path):
    port = free_port()
    mp.start_processes(_dist_helpers, args=(2, port, str(tmp_path / "o")), nprocs=2, start_method="spawn")
    for rank in range(2):
        got = json.load(open(tmp_path / f"o.{rank}"))
        assert got == {"ws": 2, "rank": rank, "local": rank, "max": 1.5}


class FakeKG:
    """Stands in for a graph replica: answers each query with a record of
    which rank answered it."""

    def __init__(self, rank):
        self.rank = rank

    def search_batch(self, queries):
        return [({"query": q.k, "rank": self.rank}, {}, 0) for q in queries]


def _sharded(rank, world, port, out):
    _env(rank, world, port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import rpqgen
    from paper_2001_06770_b300 import replicas
    dist.init_process_group("gloo")
    qs = [rpqgen.Query(central=[1], marginal=[], k=i, max_depth=4) for i in range(11)]
    res = replicas.search_sharded(FakeKG(rank), qs)
    if rank == 0:
        with open(out, "w") as f:
            json.dump([r[0] for r in res], f)
    else:
        assert res is None
    dist.destroy_process_group()


def test_search_sharded_two_ranks(tmp_path):
    port = free_port()
    out = str(tmp_path / "res.json")
    mp.start_processes(_sharded, args=(2, port, out), nprocs=2, start_method="spawn")
    got = json.load(open(out))
    assert [g["query"] for g in got] == list(range(11))          # query order restored
    assert [g["rank"] for g in got] == [i % 2 for i in range(11)]  # round-robin shares


def test_shard_partitions_queries():
    from paper_2001_06770_b300 import replicas
    for n in (0, 1, 7, 64):
        for world in (1, 2, 3, 8):
            parts = [replicas.shard(n, r, world) for r in range(world)]
            assert sorted(i for p in parts for i in p) == list(range(n))
    with pytest.raises(ValueError):
        replicas.shard(4, 2, 2)


def test_reference_arm_under_torchrun():
    """Two ranks of bench.py's reference arm: rank 0 prints one JSON line,
    the other rank exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), "bench.py", "--impl", "reference",
           "--workload", "tiny", "--steps", "2", "--warmup", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
