"""CPU tests of bench.py's reference arm (the FP64 oracle timed on the host
cores): it picks nprobe by the library arm's recall rule, prints one JSON
line of the contract, and under a multi-rank launch only rank 0 works."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--workload", "tiny_window", "--steps", "2", "--warmup", "1", *args]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]


def test_reference_line_and_recall_rule():
    lines = _run()
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["unit"] == "queries/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    # nprobe: the smallest of the sweep whose recall@10 reaches 0.95
    rec = {int(p): r for p, r in d["recall_by_nprobe"].items()}
    chosen = d["config"]["nprobe"]
    assert rec[chosen] >= 0.95 and d["recall_at_10"] == rec[chosen]
    assert all(r < 0.95 for p, r in rec.items() if p < chosen)
    assert d["e2e"] == {"value": d["value"], "unit": "queries/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert f"nprobe={chosen}" in cb["sample"]


def test_reference_fixed_nprobe_skips_the_sweep():
    d = _run(None, "--nprobe", "3")[0]
    assert d["config"]["nprobe"] == 3 and d["recall_by_nprobe"] == {}


def test_reference_other_ranks_do_no_work():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []
