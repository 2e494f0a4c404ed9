"""Host-side checks of libmsadp that need no GPU: the library loads, exports every
entry point include/msadp.h declares, its planner reproduces the paper's wave
tables (section 3.1 Eq. 2 and Eq. 3, section 3.2 Tables 1 and 2), and argument
validation rejects bad calls before any CUDA work.
"""
import json
import math
import os
import re

import numpy as np
import pytest

import inputs
import paper_2311_17530_gb300 as msa
from paper_2311_17530_gb300 import msadp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "msadp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(msa_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = msa.library()
    declared = _declared_functions()
    assert declared, "no declarations parsed"
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in include/msadp.h but not exported"
    assert set(msadp.EXPORTED) == set(declared)


def test_paper_table2_wave_sizes_and_eq2_eq3():
    t2 = json.load(open(os.path.join(GOLDEN, "paper_tables.json")))["table2"]
    # Eq. 3: p_i = (rho_i - 1) / (S - 1) partitions per axis
    p = [(r - 1) // (t2["S"] - 1) for r in t2["shape"]]
    sizes = msa.msa_wave_sizes(p)
    assert sizes == t2["sizes"]
    assert len(sizes) == t2["waves"]                       # Eq. 2
    assert sum(sizes) == math.prod(p) == t2["partitions"]  # Eq. 3
    assert math.prod(t2["shape"]) == t2["cells"]
    # Eq. 2 as printed: t = (rho_0-1)/(S-1) + sum_{i>=1} ((rho_i-1)/(S-1) - 1)
    S = t2["S"]
    eq2 = (t2["shape"][0] - 1) // (S - 1) + sum((r - 1) // (S - 1) - 1 for r in t2["shape"][1:])
    assert eq2 == t2["waves"]


def test_paper_table1_unbounded_waves():
    t1 = json.load(open(os.path.join(GOLDEN, "paper_tables.json")))["table1"]["rows"]
    for k, row in t1.items():
        k = int(k)
        if k > msadp.MAX_K:
            continue
        sizes = msa.msa_wave_sizes([len(row)] * k)  # grid large enough for 9 waves
        assert sizes[: len(row)] == row


def test_tile_shape_covers_the_tensor():
    for lens in ([128, 128, 128], [700, 760, 800], [110, 118, 124, 130], [23, 24, 24, 21, 24, 24],
                 [0, 5], [1, 1, 1, 1, 1, 1, 1, 1]):
        ext, grid = msa.msa_tile_shape(lens)
        for n, e, g in zip(lens, ext, grid):
            assert e >= 1 and g == -(-(n + 1) // e)


@pytest.mark.parametrize("bad", [
    dict(seqs=["ACG"], err="k=1"),
    dict(seqs=["ACG"] * 9, err="k=9"),
    dict(seqs=["ACG", "AXG"], err="residue"),
    dict(seqs=["ACG", "ACG"], alphabet="", err="alphabet size"),
    dict(seqs=["ACG", "ACG"], alphabet="ACGA", err="repeats"),
    dict(seqs=["ACG", "ACG"], subst="asym", err="symmetric"),
])
def test_msa_align_rejects_bad_arguments_before_cuda(bad):
    alphabet = bad.get("alphabet", "ACGT")
    subst = inputs.dna_table()
    if bad.get("subst") == "asym":
        subst = subst.copy()
        subst[0, 1] = 3
    with pytest.raises(msa.MsaError) as ei:
        msa.msa_align(bad["seqs"], alphabet, subst if alphabet else np.zeros((1, 1)), -8)
    assert ei.value.code == msa.MSA_EINVAL
    assert bad["err"] in str(ei.value)


def test_config_validation():
    with pytest.raises(msa.MsaError):
        msa.msa_config("no_such_key", 1)
    with pytest.raises(msa.MsaError):
        msa.msa_config("spin_timeout_ms", 0)
    msa.msa_config("spin_timeout_ms", 5000)


def test_wave_shuffle_hook_is_validated_and_keeps_plans_valid():
    with pytest.raises(msa.MsaError):
        msa.msa_config("test_shuffle_waves", -1)
    msa.msa_config("test_shuffle_waves", 99)
    try:
        ext, grid = msa.msa_tile_shape([120, 90, 100])  # planning under the hook still succeeds
        assert all(g >= 1 for g in grid)
    finally:
        msa.msa_config("test_shuffle_waves", 0)


def test_automatic_kernel_choice_by_k_and_last_axis():
    """The planner's automatic choice, read through the tile shape it reports: the
    streamed line kernel sweeps the whole last axis in one tile (k = 4, 5, and at
    k = 6 only while the whole-column form holds the axis: 25 positions), the line
    kernel cuts it into equal segments (k = 6 beyond 25 positions: at most 25, the
    compiled length not above it)."""
    for lens in ([9, 13, 10, 70], [4, 5, 3, 6, 40], [5, 4, 3, 3, 2, 20], [5, 4, 3, 3, 2, 24]):
        ext, grid = msa.msa_tile_shape(lens)
        assert ext[-1] == lens[-1] + 1 and grid[-1] == 1, lens
    for lens in ([5, 4, 3, 3, 2, 25], [5, 4, 3, 3, 2, 30], [3, 3, 3, 3, 3, 60]):
        ext, grid = msa.msa_tile_shape(lens)
        assert ext[-1] <= 25 and grid[-1] >= 2 and ext[-1] * grid[-1] >= lens[-1] + 1, lens
