"""bench.py's reference arm on CPU: the FP64 oracle timed on a bounded sample of the workload, one
JSON line with the contract's keys (no GPU needed, none used). A rank other than 0 prints nothing
and exits 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                       capture_output=True, text=True, timeout=300, env=env, cwd=ROOT)
    return r


def test_reference_arm_prints_one_contract_line():
    r = _run(None, "--steps", "1", "--warmup", "3", "--workload", "sod400x4")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "GLUPS" and d["unit"] == "GLUPS"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["warmup"] >= 3
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert cb["single_core"]["cores"] == 1 and cb["single_core"]["value"] > 0
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == "GLUPS"
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "sod400x4"


def test_reference_arm_other_ranks_do_no_work():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"}, "--steps", "1", "--warmup", "3")
    assert r.returncode == 0 and r.stdout.strip() == ""
