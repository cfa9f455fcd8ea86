"""Host logic of bench.py, on the CPU: the committed ncu summaries are read
only while they match the kernel sources (and, for DRAM traffic, the
captured size), the precision check's strata cover the range one pick
each, and the reference arm prints the contract's JSON line."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _write(path, text):
    with open(path, "w") as f:
        f.write(text)


def test_recorded_traffic_follows_hash_and_size(tmp_path, monkeypatch):
    f = tmp_path / "traffic.txt"
    h = bench.kernel_hash()
    _write(f, f"# comment: 1\nkernel_source_sha256_16: {h}\nn_captured: 1024\n"
              "dram_bytes_read: 10\ndram_bytes_write: 32\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.recorded_traffic(1024) == 42.0
    assert bench.recorded_traffic(2048) is None  # captured for another size
    _write(f, "kernel_source_sha256_16: 0000000000000000\nn_captured: 1024\n"
              "dram_bytes_read: 10\ndram_bytes_write: 32\n")
    assert bench.recorded_traffic(1024) is None  # kernel changed since


def test_recorded_pipes_quote_the_busiest(tmp_path, monkeypatch):
    f = tmp_path / "pipes.txt"
    h = bench.kernel_hash()
    _write(f, f"kernel_source_sha256_16: {h}\nn_captured: 64\n"
              "index.fmaheavy_pct: 70.0\nindex.alu_pct: 50.0\nindex.issue_pct: 60.0\n"
              "packed.fmaheavy_pct: 40.0\npacked.alu_pct: 45.0\npacked.issue_pct: 63.0\n")
    monkeypatch.setattr(bench, "PIPES_FILE", str(f))
    a, b = bench.recorded_pipes("index"), bench.recorded_pipes("packed")
    assert a["pipe"] == "fmaheavy" and a["frac"] == pytest.approx(0.70)
    assert b["pipe"] == "issue" and b["frac"] == pytest.approx(0.63)
    _write(f, "kernel_source_sha256_16: 0000000000000000\n")
    assert bench.recorded_pipes("index") is None


def test_committed_summaries_parse():
    """The committed files hold every key the readers need (values are
    used only while their hash matches the sources)."""
    for path, keys in ((bench.TRAFFIC_FILE, ("kernel_source_sha256_16", "n_captured",
                                             "dram_bytes_read", "dram_bytes_write")),
                       (bench.PIPES_FILE, ("kernel_source_sha256_16", "n_captured",
                                           "index.fmaheavy_pct", "packed.issue_pct"))):
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        for k in keys:
            assert k in kv, (path, k)
        assert len(kv["kernel_source_sha256_16"]) == 16


def test_kernel_hash_covers_only_device_sources(tmp_path, monkeypatch):
    a = tmp_path / "a.cu"
    _write(a, "device code\n// Host side\nhost code v1\n")
    monkeypatch.setattr(bench, "KERNEL_SRCS", [str(a)])
    h1 = bench.kernel_hash()
    _write(a, "device code\n// Host side\nhost code v2\n")
    assert bench.kernel_hash() == h1  # host part is not hashed
    _write(a, "device code changed\n// Host side\nhost code v2\n")
    assert bench.kernel_hash() != h1


def test_stratified_positions_one_per_stratum():
    n, m = 1 << 20, 1 << 10
    idx = bench.stratified_positions(n, m)
    assert idx.dtype == np.uint64 and idx.size == m
    width = n // m
    assert np.array_equal(idx // np.uint64(width), np.arange(m, dtype=np.uint64))
    assert int(idx.max()) < n


def test_reference_arm_prints_the_contract_line():
    """`--impl reference` (the CPU oracle) prints one JSON line with the
    contract's keys, marked as the reference arm, without a GPU."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "dtype", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["config"]["workload"] == bench.DEFAULT_WORKLOAD
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
