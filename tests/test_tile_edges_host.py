"""Tile-edge settings (host only): the compiled candidates per k, validation,
and the tile shape the planner reports for a chosen edge (section 3.2's
partition size S; Eq. 2 and 3 count the waves and tiles of the resulting grid)."""
import math
import os
import shutil
import subprocess

import pytest

import paper_2311_17530_gb300 as msa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2311_17530_gb300", "csrc")
CANDIDATES = {2: [16, 32, 64], 3: [8, 12, 16], 4: [4, 5, 6], 5: [3, 4, 5], 6: [2, 3, 4], 7: [2, 3], 8: [2]}
DEFAULT = {2: 32, 3: 12, 4: 6, 5: 4, 6: 3, 7: 2, 8: 2}


@pytest.fixture(autouse=True)
def restore():
    yield
    for k in CANDIDATES:
        msa.msa_set_tile_edge(k, 0)
    msa.msa_config("fill_kernel", 0)


def test_defaults_and_validation():
    for k, edges in CANDIDATES.items():
        assert msa.msa_get_tile_edge(k) == DEFAULT[k]
        for e in edges:
            msa.msa_set_tile_edge(k, e)
            assert msa.msa_get_tile_edge(k) == e
        for bad in (1, 7, 100, -3):
            if bad not in edges:
                with pytest.raises(msa.MsaError) as ei:
                    msa.msa_set_tile_edge(k, bad)
                assert ei.value.code == msa.MSA_EINVAL
        msa.msa_set_tile_edge(k, 0)
        assert msa.msa_get_tile_edge(k) == DEFAULT[k]
    for k in (1, 9):
        with pytest.raises(msa.MsaError):
            msa.msa_set_tile_edge(k, 2)


def test_tile_shape_follows_the_edge():
    msa.msa_config("fill_kernel", 1)  # generic kernel for every k
    for k, edges in CANDIDATES.items():
        lens = [37 + 3 * i for i in range(k)] if k <= 4 else [9 + i for i in range(k)]
        for e in edges:
            msa.msa_set_tile_edge(k, e)
            ext, grid = msa.msa_tile_shape(lens)
            want = [2 * e if (k == 2 and i == 1) else e for i in range(k)]
            assert ext == want
            assert grid == [math.ceil((n + 1) / x) for n, x in zip(lens, want)]
            sizes = msa.msa_wave_sizes(grid)
            assert len(sizes) == sum(grid) - k + 1 and sum(sizes) == math.prod(grid)  # Eq. 2, Eq. 3


def test_planner_refuses_tensors_beyond_32_bit_tile_blocks():
    msa.msa_config("fill_kernel", 1)
    with pytest.raises(msa.MsaError) as ei:
        msa.msa_tile_shape([400, 400, 400, 400])  # 2.6e10 cells: tile-major scratch offsets exceed 32 bits
    assert ei.value.code == msa.MSA_ETOOBIG


def _nvcc():
    for c in ("/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    return None


@pytest.mark.skipif(_nvcc() is None, reason="needs nvcc")
def test_padded_tile_layout_is_a_bijection(tmp_path):
    # every compiled tile shape: halo'd cells at distinct offsets inside the
    # buffer, predecessor offsets = sums of strides, halo-cell count (host program)
    exe = tmp_path / "tile_geometry_check"
    subprocess.check_call([_nvcc(), "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC, "-I",
                           os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "tile_geometry_check.cu"),
                           "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_planner_ticket_order_is_by_wave(tmp_path):
    # every tile once, by wave (tile index sum, decoded by division) and by
    # increasing linear index within a wave; wave offsets; column plans by a + b
    exe = tmp_path / "plan_order_check"
    cuda_inc = "/usr/local/cuda/include"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-I", cuda_inc,
                           os.path.join(ROOT, "tests", "plan_order_check.cpp"), os.path.join(CSRC, "plan.cpp"),
                           "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout
