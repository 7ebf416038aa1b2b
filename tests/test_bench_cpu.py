"""The benchmark's reference arm (the serial oracle on the host cores) runs
without a GPU and prints one JSON line of the benchmark contract."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "tiny", "--steps", "2", "--warmup", "1"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] and d["unit"] == "queries/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["config"]["workload"].startswith("tiny")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_level_bytes_worked_example():
    """The roofline numerator: algorithmic bytes of one Glevel's expansion
    (4 per work unit, 1 per executed activation, 2 per claim, 10 per item)
    and enqueue (the frontier read - the n-bit map, or 4 bytes per queued
    node - then 13 + |T| bytes per frontier node, 10 per item and 4 per
    128-unit warp tile), on a level worked out by hand."""
    sys.path.insert(0, ROOT)
    import bench
    rec = dict(units=1000, e_act=1500, claims=100, items=20, frontier=50, flags=0, columns=3)
    # expansion 4000 + 1500 + 200 + 200; bit-map enqueue 128 (1024 bits) + 50 * 16 + 200 + 8 tiles * 4
    assert bench.level_bytes(rec, 1024) == (5900, 1160)
    # read from the frontier queue (flag 8): 50 nodes * 4 bytes in place of the bit map
    assert bench.level_bytes(dict(rec, flags=8), 1024) == (5900, 1232)
    # a ragged bit map: 1,001 nodes take 126 bytes
    assert bench.level_bytes(dict(rec, units=0, items=0), 1001)[1] == 126 + 50 * 16


def test_sample_indices_spread():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.sample_indices(5, 8) == [0, 1, 2, 3, 4]
    assert bench.sample_indices(256, 16)[0] == 0 and bench.sample_indices(256, 16)[-1] == 255
    assert len(bench.sample_indices(4096, 16)) == 16
