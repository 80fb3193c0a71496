"""bench.py's clock sampler (host logic, no GPU): nvidia-smi's CSV samples, here printed by a stand-in
process, give the median SM clock under load, the maximum clock and the throttle reasons that were active in
any sample ("Not Active" counts as inactive); without nvidia-smi the line says so."""
import subprocess
import sys
import time

import bench

SAMPLES = [
    "0, 2070, 2070, 910.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "0, 2055, 2070, 1380.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
    "0, 2070, 2070, 1395.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
    "0, 1980, 2070, 1400.1, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
    "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
]


def _fake_popen(real):
    def popen(cmd, **kw):
        assert cmd[0] == "nvidia-smi" and "--format=csv,noheader,nounits" in cmd
        script = "import sys, time\nfor l in %r:\n    print(l, flush=True)\ntime.sleep(60)\n" % (SAMPLES,)
        return real([sys.executable, "-c", script], **kw)
    return popen


def test_clock_summary_from_samples(monkeypatch):
    monkeypatch.setattr(bench.subprocess, "Popen", _fake_popen(subprocess.Popen))
    cs = bench.ClockSampler(0)
    cs.start()
    t = time.time()
    while len(cs.samples) < len(SAMPLES) and time.time() - t < 30:
        time.sleep(0.05)
    out = cs.stop()
    assert out["samples"] == len(SAMPLES)
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0          # median of 1980 2055 2070 2070 2070
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert cs.proc.poll() is not None                                       # the sampler process was ended


def test_missing_nvidia_smi_is_reported(monkeypatch):
    def popen(cmd, **kw):
        raise FileNotFoundError(cmd[0])
    monkeypatch.setattr(bench.subprocess, "Popen", popen)
    cs = bench.ClockSampler(0)
    cs.start()
    assert cs.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
