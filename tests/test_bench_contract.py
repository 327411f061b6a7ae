"""The benchmark's command-line contract, on the CPU.

The reference arm (`--impl reference`) times the oracle on the host, so its
JSON line can be checked without a GPU: the keys and types the line must
carry, rank 0 alone printing under a multi-rank launch, and the warm-up rule.
A tiny oracle grid (`--ref-n 8`) keeps it to a second or two.
"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args, env=None):
    e = dict(os.environ, OMP_NUM_THREADS="2")
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=e,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_json_line():
    r = _bench("--impl", "reference", "--steps", "2", "--warmup", "3", "--ref-n", "8")
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1  # one JSON line
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "cell-updates/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 3 and d["ms_per_step"] > 0
    assert d["scaling"] in ("weak", "strong") and d["vs_baseline"] is None
    assert d["data"] == "synthetic" and d["dtype"] == "f64"
    assert isinstance(d["config"], dict) and "workload" in d["config"]
    assert "metric" in d and "TGV 256^3" in d["metric"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert isinstance(cb["cores"], int) and cb["cores"] >= 1 and "8^3" in cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_do_no_work():
    r = _bench("--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--ref-n", "8",
               env={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_fewer_than_three_warmup_steps_rejected():
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "2", "--ref-n", "8")
    assert r.returncode == 2 and "warm-up" in r.stderr
