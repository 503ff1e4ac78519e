"""Host-side checks of bench.py's contract (no GPU): the L2 note of each workload,
the committed traffic summaries it reads, the hash guard that turns a changed
kernel source into null traffic, and the reference arm's JSON line."""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _args(config, n_samples=None):
    return argparse.Namespace(config=config, n_samples=n_samples, precision="mixed", tol=1e-10)


def test_l2_note_follows_the_pointing_size():
    # 12 bytes of pointing per sample against the 129 MB L2
    assert bench.config_dict(_args(1))["l2"].startswith("L2-resident")
    assert bench.config_dict(_args(4))["l2"].startswith("inputs larger than L2")
    assert bench.config_dict(_args(4, 1_000_000))["l2"].startswith("L2-resident")
    assert bench.config_dict(_args(4, 1_000_000))["workload"].endswith("-prefix1000000")


def test_committed_traffic_summaries_parse():
    files = [f for f in os.listdir(os.path.join(ROOT, "profiles")) if f.endswith("_traffic.md")]
    assert files
    for f in files:
        text = open(os.path.join(ROOT, "profiles", f)).read()
        m = re.search(r"(\w+\.cu) sha256\[:16\]:\s*([0-9a-f]{16})", text)
        assert m, f
        assert os.path.exists(os.path.join(ROOT, "paper_1309_5609_gb300", "csrc", m.group(1))), f
        figures = re.findall(r"dram bytes per sample \[([\w.-]+)\]:\s*([0-9.]+)", text)
        assert figures and all(float(v) > 0 for _, v in figures), f


def test_traffic_is_null_once_the_source_changes(tmp_path, monkeypatch):
    src_dir = tmp_path / "paper_1309_5609_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = src_dir / "k.cu"
    src.write_bytes(b"__global__ void k_x() {}\n")
    h = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles" / "k_x_traffic.md").write_text(
        f"k.cu sha256[:16]: {h}\ndram bytes per sample [work]: 12.5\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic(1000, "k_x", "work-prefix5") == pytest.approx(12500.0)
    assert bench.kernel_traffic(1000, "k_x", "other") is None   # no figure for it
    assert bench.kernel_traffic(1000, "k_y", "work") is None    # no summary
    src.write_bytes(b"__global__ void k_x() { }\n")               # the kernel changed
    assert bench.kernel_traffic(1000, "k_x", "work") is None


def test_reference_arm_prints_its_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--config", "1", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("qu-nside64-2^20-L500")
