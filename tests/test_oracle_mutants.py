"""The oracle pins are strong enough: each plausible mistake, planted in a copy of
the oracle's C source on the CPU, is caught by at least one pin.
"""
import os
import subprocess

import numpy as np
import pytest

import inputs
import oracle
from tests._independent import brute_force, needleman_wunsch

SRC = os.path.join(os.path.dirname(oracle.__file__), "msa_oracle.c")

MUTANTS = {
    "tie_break_ge": ("cand > best", "cand >= best"),
    "residue_index_off_by_one": ("int b = seq[j][x[j] - 1];", "int b = seq[j][x[j] > 1 ? x[j] - 2 : 0];"),
    "gap_sign": ("sp += gap;", "sp -= gap;"),
    "gap_term_dropped": ("sp += gap;", "sp += 0;"),
    "transposed_table": ("sp += sub[a * A + b];", "sp += sub[b * A + a];"),
    "pair_dropped": ("for (int j = i + 1; j < k; ++j)", "for (int j = i + 2; j < k; ++j)"),
    "origin_not_zero": ("H[0] = 0;", "H[0] = 1;"),
    "columns_not_reversed": ("for (int32_t a = 0, b = ncols - 1; a < b; ++a, --b)",
                             "for (int32_t a = 0, b = ncols - 1; a < 0; ++a, --b)"),
    "gap_gap_charged": ("} else if (in_i || in_j) {", "} else {"),
    "full_move_skipped": ("for (int m = 1; m <= nmoves; ++m) {", "for (int m = 1; m < nmoves; ++m) {"),
    "score_not_from_corner": ("*out_score = H[N - 1];", "*out_score = H[N > 1 ? N - 2 : 0];"),
    "traceback_not_from_corner": ("int64_t l = N - 1;", "int64_t l = N > 1 ? N - 2 : 0;"),
}


def _pins(lib):
    """A reduced battery of the pins in test_oracle_pins.py; raises on the first miss."""
    rng = np.random.default_rng(3)
    asym = rng.integers(-5, 6, size=(3, 3)).astype(np.int32)
    for lens in [(2, 3), (3, 1, 2), (2, 2, 2), (0, 2, 1)]:
        seqs = [inputs.random_seq(rng, "ACG", n) for n in lens]
        for table, gap in [(asym, -2), (np.eye(3, dtype=np.int32), -1)]:
            bs, bm = brute_force(seqs, "ACG", table, gap)
            r = oracle.align(seqs, "ACG", table, gap, lib=lib)
            assert (r.score, r.masks) == (bs, bm)
    for rep in range(5):
        a = inputs.random_seq(rng, "ACGT", int(rng.integers(3, 20)))
        b = inputs.random_seq(rng, "ACGT", int(rng.integers(3, 20)))
        assert (oracle.align([a, b], "ACGT", inputs.dna_table(), -8, lib=lib).masks
                == needleman_wunsch(a, b, "ACGT", inputs.dna_table(), -8)[1])


def test_unmutated_oracle_passes_the_battery():
    _pins(None)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = src.replace(old, new, 1)
    cpath = tmp_path / "mutant.c"
    cpath.write_text(mutated)
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", str(so), str(cpath)])
    lib = oracle.load_library(str(so))
    with pytest.raises(AssertionError):
        _pins(lib)
