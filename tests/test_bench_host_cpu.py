"""bench.py's host helpers, on the CPU: the clock sampler's parsing of nvidia-smi
lines (median SM clock under load, throttle reasons seen during the timed region
only) and the gate that reports DRAM traffic only for the kernel sources it was
captured on."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _line(sm, mx, hw="Not Active", cap="Not Active"):
    return f"2026/01/01 00:00:00.000, {sm}, {mx}, 900.0, 0x0, {hw}, Not Active, Not Active, {cap}"


def test_clock_sampler_keeps_the_timed_region_only(monkeypatch):
    c = bench.ClockSampler("0")
    c.proc = _DoneProc()
    c.t0 = 100.0
    c.lines = [(99.0, _line(1000, 2070, hw="Active")),  # before the timed region: ignored
               (100.1, _line(2070, 2070)), (100.3, _line(2055, 2070, cap="Active")), (100.5, _line(2070, 2070)),
               (100.6, "garbage"), (100.7, _line("[N/A]", 2070))]
    monkeypatch.setattr(bench.time, "time", lambda: 100.6)
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    out = c.stop()
    assert out["samples"] == 3 and out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]  # hw_slowdown came before t0


def test_clock_sampler_without_nvidia_smi_says_so():
    c = bench.ClockSampler("0")
    c.t0 = 0.0
    out = c.stop()
    assert out["samples"] == 0 and out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


def test_traffic_is_reported_only_for_the_sources_it_was_captured_on(tmp_path, monkeypatch):
    with open(os.path.join(ROOT, "profiles", "stage_traffic.json")) as fh:
        committed = json.load(fh)
    # the committed capture matches the committed kernel sources
    assert committed["source_hash"] == bench.kernel_source_hash()
    assert bench.ncu_traffic("pass2", 1) == committed["bytes_per_launch"]["ts1"]["pass2"]
    # a capture of other sources is not reported
    root = tmp_path / "r"
    (root / "profiles").mkdir(parents=True)
    stale = dict(committed, source_hash="0" * 16)
    (root / "profiles" / "stage_traffic.json").write_text(json.dumps(stale))
    csrc = root / "paper_2603_24370_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for fn in ("ss_flow_kernel.cuh", "ss_flow.cu", "ss_device.cuh", "ss_flow_cm.cu", "ss_pack.cuh"):
        with open(os.path.join(ROOT, "paper_2603_24370_gb300", "csrc", fn), "rb") as src:
            (csrc / fn).write_bytes(src.read())
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.ncu_traffic("pass2", 1) is None
