"""The benchmark's CPU arm (the oracle timed on the host cores, `bench.py
--impl reference`) runs without a GPU and prints the contract's JSON line,
on the same `config` as the GPU arm."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["value"] > 0 and line["unit"] == "queries/s" and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 3 and line["n_gpus"] == 1
    # the GPU arm's configuration: the serving workload, its per-index budgets
    assert line["config"]["workload"].startswith("serving: 3 resident indexes")
    assert line["config"]["P"] == [256, 3072, 2048] and line["config"]["k"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == (os.cpu_count() or 1)
    assert line["e2e"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_both_arms_share_one_config():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.serve_config(1) == bench.serve_config(1)
    assert bench.serve_config(1)["P"] == list(bench.SERVE_P)
    sizes, which, offs, _ = bench.serve_trace()
    assert sizes.min() >= 1 and sizes.max() <= 4096 and len(sizes) == bench.SERVE_REQUESTS
    assert ((offs >= 0) & (offs + sizes <= bench.SERVE_POOL)).all()
    assert set(np.unique(which)) == {0, 1, 2}
