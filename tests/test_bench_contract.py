"""bench.py on the CPU: the reference (oracle) arm's JSON line and the source-digest rule that
decides whether a committed ncu profile may supply roofline.traffic."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _run_reference(env_extra):
    env = dict(os.environ, **env_extra)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "1",
           "--L", "12", "--chi", "4", "--ref-sites", "12"]
    return subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)


def test_reference_arm_prints_one_contract_line():
    r = _run_reference({"RANK": "0"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1, r.stdout
    out = json.loads(lines[0])
    assert out["impl"] == "reference"
    assert out["metric"] == bench.METRIC and out["unit"] == bench.UNIT
    assert out["value"] > 0 and out["ms_per_step"] > 0
    assert out["steps"] == 1 and out["warmup"] == 1 and out["n_gpus"] == 1
    assert out["higher_is_better"] is True and out["dtype"] == "f64" and out["data"] == "synthetic"
    assert out["config"]["workload"].startswith("xxx_L12_chi4")
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == out["value"] and cb["sample"]
    assert out["e2e"] == {"value": out["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_print_nothing():
    r = _run_reference({"RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_profile_traffic_only_for_matching_sources(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2501_17913_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("__global__ void k() {}\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    digest = bench.csrc_digest()
    prof = tmp_path / "profiles" / "p.md"
    prof.write_text("csrc digest: %s\ndram bytes per unit: 1000\n" % digest)
    traffic, src = bench.profiled_traffic("p.md", 256)
    assert traffic == pytest.approx(256000.0) and "scaled by units" in src
    (csrc / "k.cu").write_text("__global__ void k() { }\n")      # the kernel changed
    assert bench.csrc_digest() != digest
    traffic, src = bench.profiled_traffic("p.md", 256)
    assert traffic is None and "changed" in src
    assert bench.profiled_traffic("missing.md", 256) == (None, "no profile")
