"""Host side of the serving loop, without a GPU: the device arena's first-fit
bookkeeping (compiled C++ check) and the checks msa_submit / msa_poll /
msa_cancel / msa_wait_any / msa_drain make before any device work."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import inputs
import paper_2311_17530_gb300 as msa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2311_17530_gb300", "csrc")


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_arena_first_fit_and_coalescing(tmp_path):
    exe = tmp_path / "arena_check"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "arena_check.cpp"),
                           "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout


def code_of(fn):
    with pytest.raises(msa.MsaError) as ei:
        fn()
    return ei.value.code


def test_submit_refuses_bad_requests_before_device_work():
    dna = inputs.dna_table()
    assert code_of(lambda: msa.msa_submit(["ACGT"], inputs.DNA, dna, -8)) == msa.MSA_EINVAL  # k = 1
    assert code_of(lambda: msa.msa_submit(["ACGX", "AC"], inputs.DNA, dna, -8)) == msa.MSA_EINVAL
    asym = dna.copy()
    asym[0, 1] = 3
    assert code_of(lambda: msa.msa_submit(["ACG", "AC"], inputs.DNA, asym, -8)) == msa.MSA_EINVAL
    assert code_of(lambda: msa.msa_submit(["AC", "A"], "AA", np.zeros((2, 2), np.int32), -8)) == msa.MSA_EINVAL
    # footprint above the device budget (27 GB of traceback bytes, default budget 16 GiB)
    assert code_of(lambda: msa.msa_submit(["A" * 3000] * 3, inputs.DNA, dna, -8)) == msa.MSA_ETOOBIG


def test_unknown_handles_and_empty_queue():
    assert code_of(lambda: msa.msa_poll(987654321, 2, 4)) == msa.MSA_EBADHANDLE
    assert code_of(lambda: msa.msa_cancel(987654321)) == msa.MSA_EBADHANDLE
    assert msa.msa_wait_any(0) is None
    msa.msa_drain()  # nothing queued or running: returns at once


def test_serving_without_a_device_fails_cleanly():
    """With no usable GPU, serving fails cleanly: either msa_submit refuses the
    request at once, or the loop's device set-up fails and the queued request
    completes with that error (no hang); later submits are refused too. Runs in
    its own process, since a failed loop stays failed for the process."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the serving loop would start")
    code = r'''
import sys
sys.path.insert(0, %r)
import inputs
import paper_2311_17530_gb300 as msa
dna = inputs.dna_table()
try:
    h = msa.msa_submit(["ACGT", "AGT"], inputs.DNA, dna, -8)
except msa.MsaError as e:  # no device at all: refused before the loop starts
    assert e.code == msa.MSA_ECUDA, e
    h = None
if h is not None:  # the loop started and its device set-up failed
    got = msa.msa_wait_any(20 * 1000 * 1000)
    assert got == h, (got, h)
    try:
        msa.msa_poll(h, 2, 7)
        raise SystemExit("poll succeeded without a device")
    except msa.MsaError as e:
        assert e.code in (msa.MSA_ECUDA, msa.MSA_ENOMEM), e
try:
    msa.msa_submit(["ACGT", "AGT"], inputs.DNA, dna, -8)
    raise SystemExit("submit accepted without a device")
except msa.MsaError as e:
    assert e.code in (msa.MSA_ECUDA, msa.MSA_ENOMEM), e
assert msa.msa_wait_any(0) is None
msa.msa_drain()
print("ok")
''' % ROOT
    import sys
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", (out.stdout, out.stderr)
