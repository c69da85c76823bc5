"""Host-side pieces of the benchmark (no GPU): the entry counts behind the
metric and the compulsory-bytes model of the build kernels."""
import math
import os

import bench


def test_live_entries_per_node():
    # r_h C(k-1, h-1) summed over h: the colour-relative row widths
    assert [bench.live_entries_per_node(k) for k in range(4, 9)] == [14, 42, 131, 420, 1376]


def test_geometry_widths():
    Wc, Ws = bench.geometry(8)
    assert sum(Wc.values()) == 1376 and sum(Ws.values()) == 615
    Wc, Ws = bench.geometry(5)
    assert [Wc[h] for h in range(1, 6)] == [1, 4, 12, 16, 9]
    assert [Ws[h] for h in range(1, 5)] == [4, 6, 8, 4]


def test_gather_and_merge_bytes():
    import paper_2009_03052_gb300 as M
    M.load()
    n, nnz, B = 1000, 8000, 8
    csr = 8 * (n + 1) + 4 * nnz + n
    assert bench.algorithmic_bytes("gather_h3", n, nnz, 5, B) == n * (12 + 8) * B + csr
    # merge of level 5: reads c rows of the T' sizes and S rows of the T''
    # sizes the level's decompositions use, writes the level-5 row
    Wc, Ws = bench.geometry(5)
    used1, used2 = set(), set()
    for s in M.shape_info(5)["code"]:
        bits = format(int(s), "08b")
        depth = 0
        for i, ch in enumerate(bits):
            depth += 1 if ch == "1" else -1
            if depth == 0:
                used2.add((i + 1) // 2)
                used1.add(5 - (i + 1) // 2)
                break
    want = n * (sum(Wc[x] for x in used1 if x > 1) + sum(Ws[x] for x in used2) + Wc[5]) * B
    assert bench.algorithmic_bytes("merge_h5", n, nnz, 5, B) == want
    assert math.isclose(want / n / B, 63)  # c2 4 + c3 12 + c4 16 + S1 4 + S2 6 + S3 8 + S4 4 + out 9


def test_job_throughput_single_rank():
    ms, v = bench.job_throughput(1000.0, 2.0, 1)
    assert ms == 2.0 and v == 1000.0 / 0.002


def test_traffic_only_for_the_captured_source(monkeypatch):
    # an ncu traffic figure is reported while the kernel's source file hashes
    # to the value recorded with the capture, and dropped once it changes
    h = bench.source_hash("sample")
    assert len(h) == 16
    monkeypatch.setitem(bench.TRAFFIC, ("w", "sample"), (123, h))
    assert bench.traffic_of("w", "sample") == 123
    monkeypatch.setitem(bench.TRAFFIC, ("w", "sample"), (123, "0" * 16))
    assert bench.traffic_of("w", "sample") is None
    assert bench.traffic_of("w", "gather_h3") is None
    monkeypatch.setitem(bench.TRAFFIC, ("w", "gather_h3"), (7, bench.source_hash("gather_h3"), 4))
    assert bench.traffic_of("w", "gather_h3", 4) == 7
    assert bench.traffic_of("w", "gather_h3", 6) is None
    assert bench.source_hash("gather_h3") == bench.source_hash("gather_h4") != ""


def test_reference_arm_line_on_the_small_case():
    # the reference arm (the oracle on host cores) prints the contract's line
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--small", "--steps", "1",
                          "--warmup", "3"], cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "data", "config"):
        assert key in line, key
    assert line["steps"] == 1 and line["warmup"] == 3 and line["value"] > 0
    assert line["config"]["workload"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
