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
