"""bench.py's output contract, on the CPU: the reference arm's JSON line (the
FP64 oracle timed on the host cores), its silence on ranks other than 0, and
the rule that a DRAM-traffic figure is reported only for the sources it was
captured from."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

ARGS = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "plain",
        "--steps", "1", "--warmup", "0", "--n-therm", "3", "--n-meas", "3"]


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run(ARGS, capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)


def test_reference_arm_prints_one_line_with_the_contract_keys():
    r = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "attempts/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "attempts/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == bench.WORKLOADS["plain"]["text"]


def test_reference_arm_is_silent_on_other_ranks():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_traffic_is_reported_only_for_the_captured_sources(monkeypatch):
    monkeypatch.setitem(bench.TRAFFIC, "probe", {"sources": "0123456789abcdef", "bytes": 1.5e9})
    monkeypatch.setattr(bench, "sources_hash", lambda: "0123456789abcdef")
    assert bench.launch_traffic("probe") == 1.5e9
    monkeypatch.setattr(bench, "sources_hash", lambda: "fedcba9876543210")
    assert bench.launch_traffic("probe") is None
    assert bench.launch_traffic("no-such-workload") is None


def test_attempt_counts_follow_the_lattice_kind():
    assert bench.sites((16, 1.0, 4)) == 4096
    assert bench.sites((64, 1.0, 4, "chain")) == 64
    assert bench.sites((60, 2.0, 4, "ising")) == 3600
    assert bench.attempts_of([(16, 1.0, 4), (60, 2.0, 2, "ising")], 10) == (4096 * 4 + 3600 * 2) * 10
