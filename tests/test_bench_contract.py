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


def test_reference_sample_deals_one_path_per_core_round_robin(monkeypatch):
    import oracle

    seen = {}

    def fake_run(systems, n_therm, n_meas, **kw):
        seen["counts"] = [(s.T, s.path_begin, s.path_count) for s in systems]
        seen["threads"] = kw.get("threads")
        return [None] * len(systems)

    monkeypatch.setattr(oracle, "run", fake_run)
    w = bench.WORKLOADS["sc16"]
    att, _ = bench.oracle_sample(w, 0, 16, total_paths=16)
    assert seen["threads"] == 16
    assert [c for _, _, c in seen["counts"]] == [1] * 16  # systems 0..15, one path each
    assert att == 16 * 4096 * 4000
    bench.oracle_sample(w, 0, 16, total_paths=32)
    assert [c for _, _, c in seen["counts"]] == [2] * 11 + [1] * 10


def test_paired_difference_and_estimates():
    import numpy as np

    rng = np.random.default_rng(1)
    rec = rng.uniform(0.1, 1.0, size=(200, 20))
    # identical runs differ by exactly zero, with zero standard error
    for key in ("e", "m", "chi", "cv", "binder"):
        assert bench.paired_difference(rec, rec.copy(), key, 64, 0.7) == (0.0, 0.0)
    # a constant shift of every path's <e> is the difference, known exactly
    sh = rec.copy()
    sh[:, 0] += 1e-3
    d, se = bench.paired_difference(sh, rec, "e", 64, 0.7)
    assert abs(d - 1e-3) < 1e-15 and se < 1e-15
    # Eq. (cv) and Eq. (kum) from pooled means
    mu = rec.mean(axis=0)
    import pytest

    assert bench._estimate("chi", mu, 64, 0.7) == pytest.approx(64 * 0.7 * (mu[3] - mu[2] ** 2), rel=1e-13)
    assert bench._estimate("cv", mu, 64, 0.7) == pytest.approx(64 * 0.49 * (mu[1] - mu[0] ** 2), rel=1e-13)
    assert bench._estimate("binder", mu, 64, 0.7) == pytest.approx(1 - mu[4] / (3 * mu[3] ** 2), rel=1e-13)
    # an independent run: the jackknife SE of a mean difference is the SE of the paired differences
    other = rng.uniform(0.1, 1.0, size=(200, 20))
    d, se = bench.paired_difference(rec, other, "e", 64, 0.7)
    diff = rec[:, 0] - other[:, 0]
    assert abs(se - diff.std(ddof=1) / np.sqrt(200)) < 1e-12
