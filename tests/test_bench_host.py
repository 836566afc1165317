"""Host logic of bench.py that needs no GPU: the clock/throttle sampler (against a fake
nvidia-smi), the roofline peak source and the roofline arithmetic, the workload's
right-hand sides, and the reference arm's JSON line (the oracle on the host)."""
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


class _FakeStats:
    def __init__(self, ms, nbytes, n):
        self.kernel_ms = [0.0, ms, 0.0]
        self.kernel_bytes = [0.0, nbytes, 0.0]
        self.kernel_launches = [0, n, 0]


def test_kernel_roofline_is_algorithmic_bytes_over_event_time():
    # two RHS entries of one batch share its totals: 3 launches of 7.26 GB in 4.0 ms in all
    stats = [_FakeStats(2.0, 3 * 7.26e9 / 2, 2), _FakeStats(2.0, 3 * 7.26e9 / 2, 1)]
    peaks = {"hbm_gbs": 6776.3}
    r = bench.kernel_roofline(stats, 1, peaks, "measured", "k", traffic=8.3e9, traffic_src="ncu")
    assert r["launches_timed"] == 3
    assert abs(r["avg_launch_ms"] - 4.0 / 3) < 1e-5          # reported to 5 decimals
    assert abs(r["bytes_per_launch"] - 7.26e9) < 1
    assert abs(r["achieved"] - 7.26e9 / (4.0e-3 / 3) / 1e9) < 0.1
    assert abs(r["frac"] - r["achieved"] / 6776.3) < 1e-4
    assert r["traffic"] == 8.3e9 and r["bound"] == "hbm" and r["unit"] == "GB/s"
    # no timed launch of that kind: no roofline
    assert bench.kernel_roofline([_FakeStats(0.0, 0.0, 0)], 1, peaks, "measured", "k") is None


def test_workload_inputs_subset_equals_the_full_list():
    # the legs that need one right-hand side make only that one; it is the same vector
    import numpy as np

    import synth
    _, dims, _, _, B = bench.workload_inputs(name=bench.C2)
    _, _, _, _, S = bench.workload_inputs(name=bench.C2, rhs=(7, 0))
    assert B.shape[0] == bench.workload_rhs_count(bench.C2) == 12
    assert np.array_equal(S, B[[7, 0]])
    _, _, _, _, E = bench.workload_inputs(name=bench.C2, rhs=())
    assert E.shape == (0,) + B.shape[1:]
    assert bench.workload_rhs_count() == 49
    small = "wilson_4x4x4x4"
    w = synth.WORKLOADS[small]
    _, dims, _, _, G = bench.workload_inputs(name=small)
    assert G.shape[0] == bench.workload_rhs_count(small) == 5
    assert np.array_equal(G[0], synth.gaussian_spinor(dims, w["first_rhs_seed"]))
    assert np.array_equal(G[1:], synth.gaussian_spinors(dims, w["rhs_seeds"]))
    _, _, _, _, one = bench.workload_inputs(name=small, rhs=(1,))
    assert np.array_equal(one, G[1:2])


def test_reference_arm_line_on_rank_zero(monkeypatch, capsys):
    # one oracle CGNR iteration on the 24^3x48 workload: the line the contract asks for
    import argparse
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    bench.run_reference(argparse.Namespace(steps=1, warmup=1, ref_iters=1, kappa=None))
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["metric"] == bench.METRIC and out["unit"] == bench.UNIT
    assert out["value"] > 0 and out["higher_is_better"] is True and out["n_gpus"] == 1
    assert out["steps"] == 1 and out["warmup"] == 1 and out["dtype"] == "f64"
    assert out["config"]["workload"] == bench.WORKLOAD and out["config"]["rhs"] == 49
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == out["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = out["e2e"]
    assert e2e["value"] == out["value"] and e2e["unit"] == out["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def _profile_commands():
    """Every `python bench.py ...` command line in the ncu summaries under profiles/
    (continuation lines joined; redirections and what follows `&&` cut off)."""
    import glob
    import shlex
    out = []
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        text = open(path).read().replace("\\\n", " ")
        for line in text.splitlines():
            i = line.find("python bench.py")
            while i >= 0:
                rest = line[i + len("python bench.py"):]
                for stop in ("&&", ">", "|", "`"):
                    j = rest.find(stop)
                    if j >= 0:
                        rest = rest[:j]
                out.append((os.path.basename(path), shlex.split(rest)))
                i = line.find("python bench.py", i + 1)
    return out


def test_profile_commands_parse_with_the_current_command_line():
    cmds = _profile_commands()
    # each summary that times a bench case gives its command
    assert {name for name, _ in cmds} >= {
        "k_cg_wilson_24x24x24x48_n16.md", "k_eo_cgnr_wilson_16x16x16x32_n16.md",
        "k_tc_combine_dots_wilson_16x16x16x32.md", "launches_wilson_24x24x24x48_step.md"}
    for name, argv in cmds:
        bench.parser().parse_args(argv)
