"""Host logic of bench.py that needs no GPU: the clock/throttle sampler (against a fake
nvidia-smi) and the roofline peak source."""
import json
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

FAKE = """#!/bin/sh
cat <<'CSV'
0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active
0, 1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active
0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active
garbage line
0, [N/A], 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active
CSV
exec sleep 30
"""


def _fake_smi(tmp_path, body):
    p = tmp_path / "nvidia-smi"
    p.write_text(body)
    p.chmod(p.stat().st_mode | stat.S_IEXEC)
    return str(tmp_path)


def test_clock_sampler_parses_clocks_and_reasons(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, FAKE) + os.pathsep + os.environ.get("PATH", ""))
    s = bench.ClockSampler(0)
    s.start()
    t0 = time.time()
    while len(s.lines) < 5 and time.time() - t0 < 10:
        time.sleep(0.05)
    out = s.stop()
    assert out["samples"] == 3                  # the malformed and N/A lines are skipped
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench.ClockSampler(0)
    s.start()
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_peaks_measured_or_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, src = bench._peaks()
    assert src == "fallback" and peaks["hbm_gbs"] == 6800.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6674.2, "bf16_tflops": 2100.0}))
    peaks, src = bench._peaks()
    assert src == "measured" and peaks["hbm_gbs"] == 6674.2
