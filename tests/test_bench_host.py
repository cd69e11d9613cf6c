"""Host logic of bench.py that needs no GPU: the traffic lookup keyed by the
kernel source's digest, the peak denominators, the clock summary, and that the
committed traffic record matches the current kernel sources."""
import io
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _tree(tmp_path, src_text, entry):
    csrc = tmp_path / "paper_1808_03374_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text(src_text)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"wl": {"k_x": entry}}))


def test_traffic_only_while_the_source_is_unchanged(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    import hashlib
    sha = hashlib.sha256(b"kernel v1").hexdigest()[:16]
    _tree(tmp_path, "kernel v1", {"dram_bytes_per_launch": 1234, "source": "k.cu", "source_sha": sha})
    assert bench.ncu_traffic("k_x", "wl") == 1234
    assert bench.ncu_traffic("k_y", "wl") is None          # no record for that kernel
    assert bench.ncu_traffic("k_x", "other") is None       # nor for that workload
    (tmp_path / "paper_1808_03374_gb300" / "csrc" / "k.cu").write_text("kernel v2")
    assert bench.ncu_traffic("k_x", "wl") is None          # source changed since the capture


def test_peaks_measured_else_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")
    assert bench.measured_e4m3_peak()[1].startswith("fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6783.1, "bf16_tflops": 1964.0}))
    assert bench.measured_peaks() == (6783.1, "measured")
    assert bench.measured_e4m3_peak() == (3928.0, "measured bf16 burst x 2")


def test_clock_summary_median_and_reasons():
    c = bench.ClockSampler(0)
    c.proc = object()
    c.file = io.StringIO("0, 2070, 2070, 900, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                         "0, 1900, 2070, 1390, 0x4, Not Active, Not Active, Not Active, Active\n"
                         "0, 2070, 2070, 1000, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                         "garbled\n")
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_committed_traffic_matches_the_sources():
    """profiles/traffic.json must describe the kernels as committed: every
    entry's source digest is the current file's (else the benchmark would
    report no traffic), and its traffic is within 10% of the algorithmic bytes
    for the single-vector products."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    with open(p) as f:
        d = json.load(f)
    entries = d["large_200k_x_1m"]
    alg = 1_000_000 * 50_000 + 4 * 1_000_000 + 4 * 200_000
    for k, e in entries.items():
        assert bench.source_digest(e["source"]) == e["source_sha"], k
    for k in ("k_mv_pair", "k_rmv_tc"):
        assert 1.0 <= entries[k]["dram_bytes_per_launch"] / alg <= 1.1, k
    assert bench.ncu_traffic("k_mv_pair", bench.WORKLOAD) == entries["k_mv_pair"]["dram_bytes_per_launch"]


@pytest.mark.parametrize("units,ms,expect", [(345.0, 7529.5, 345.0 / 7.5295)])
def test_throughput_single_process(units, ms, expect):
    v, t = bench.job_throughput(units, ms)
    assert t == ms and abs(v - expect) < 1e-12
