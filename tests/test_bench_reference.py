"""The reference arm of bench.py on the host (no GPU): `--impl reference` times
the oracle, as it stands, on the host cores over a bounded sample of the
workload's walk ids, and prints one JSON line with the contract's keys
(impl, metric, value, unit, n_gpus, steps, warmup, higher_is_better, scaling,
config, cpu_baseline, e2e with zero copy bytes).  The small ER workload keeps
the run to a few seconds.  Also the bench's host helpers: step counting and
the row signature that checks the Elias-Fano leg's rows."""
import json
import os
import subprocess
import sys

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "er1k", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup",
                "higher_is_better", "scaling", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"]
    assert "er1k" in d["config"]["workload"] or "Erdos" in d["config"]["workload"]


def test_step_count_and_row_signature():
    sys.path.insert(0, ROOT)
    import bench
    rows = torch.tensor([[3, 4, 5, -1], [7, -1, -1, -1], [-1, -1, -1, -1], [1, 2, 3, 4]],
                        dtype=torch.int32)
    # transitions: 2 + 0 + 0 (bad start) + 3
    assert bench.count_steps(rows) == 5
    sig = bench.row_signature(rows)
    assert sig == bench.row_signature(rows.clone())
    for (i, j) in [(0, 0), (1, 1), (3, 3), (2, 0)]:
        other = rows.clone()
        other[i, j] += 1
        assert bench.row_signature(other) != sig
    swapped = rows[[1, 0, 2, 3]].contiguous()
    assert bench.row_signature(swapped) != sig


def test_pinned_arena_carves_and_coalesces():
    """The served rows' host arena: first-fit slices rounded to 64 entries,
    given back and merged with their neighbours, a buffer of its own when full."""
    sys.path.insert(0, ROOT)
    import bench
    a = bench.PinnedArena(1024, pin=False)
    k1, b1 = a.take(100)               # 128 entries
    k2, b2 = a.take(300)               # 320
    k3, b3 = a.take(64)
    assert (k1[1], k1[2]) == (0, 128) and (k2[1], k2[2]) == (128, 320) and k3[1] == 448
    assert b1.data_ptr() == a.buf.data_ptr() and b2.numel() == 320
    a.give(k2)
    k4, _ = a.take(200)                # fits the hole at 128
    assert k4[1] == 128
    a.give(k1)
    a.give(k4)
    a.give(k3)
    assert a.free == [(0, 1024)]       # everything merged back
    k5, b5 = a.take(2000)              # larger than the arena: its own buffer
    assert k5[0] == "own" and b5.numel() >= 2000 and a.extra == 1
    a.give(k5)
    assert a.free == [(0, 1024)]


def test_job_steps_and_byte_models():
    """Steps of a whole-graph job on an undirected graph (a walk from a
    non-isolated start takes walk_len - 1 transitions), and the per-step byte
    model and sector counts the roofline is built from."""
    sys.path.insert(0, ROOT)
    import bench

    class Job:
        walk_len, walks_per_node = 5, 3

    deg = torch.tensor([2, 0, 1, 4], dtype=torch.int64)
    assert bench.job_steps(deg, Job) == 3 * 3 * 4
    c = {"steps": 10, "trials": 30, "gathers": 12, "searches": 4, "probes": 5, "walks": 2}
    assert bench.model_bytes(c, weighted=False) == 36 * 10 + 32 * 30 + 32 * 5
    assert bench.model_bytes(c, weighted=True) == 36 * 10 + 64 * 30 + 32 * 5
    assert bench.sector_minimal_bytes(c, rows=2, walk_len=6) == 32 * (12 + 4 + 2) + 4 * 12
    assert bench.random_sectors(c) == 12 + 5 + 2
    r = bench.roofline(dict(c, filtered=0, fallbacks=0), 2, 6, False, 1000.0, 100.0, "measured",
                       None, 1e9)
    assert abs(r["achieved"] - bench.model_bytes(c, False) / 1e9) < 1e-9
    assert abs(r["frac_of_random_sector_peak"] - 19 / 1e9) < 1e-15
