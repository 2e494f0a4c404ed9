"""The integer-ALU rates the roofline rests on, re-measured on the device:
tests/alu_peak_probe.cu is compiled and run, and the ratios between operations
must show what the peak assumes -- 32-bit adds at the issue rate (one per issue
slot, 128 lane-ops per SM per clock), the max family (max, three-input max,
fused add-max) at half of it, the fused forms doing two operations each."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_alu_rates(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = tmp_path / "alu_peak_probe"
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", str(exe),
                           os.path.join(HERE, "alu_peak_probe.cu")])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    rate = {}
    for line in out.stdout.splitlines()[1:]:
        name, ops, _ms = line.split()
        rate[name] = float(ops)
    # adds near the issue rate (128 lane-ops per SM per clock at the maximum clock)
    assert 90 <= rate["add"] <= 135, rate
    # single maxes at about half the add rate; fused pairs retire two operations per slot
    assert 0.4 <= rate["max"] / rate["add"] <= 0.7, rate
    assert 1.6 <= rate["max3"] / rate["max"] <= 2.2, rate
    assert 1.6 <= rate["addmax"] / rate["max"] <= 2.2, rate
    # two adds and one three-input max per pair of candidates beat single maxes
    assert rate["relax"] > 1.6 * rate["max"], rate
