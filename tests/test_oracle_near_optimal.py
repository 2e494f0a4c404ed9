"""Pins for the oracle of optimal and near-optimal alignment enumeration (the
paper's section 6: further optimal or near-optimal solutions by forking at
equally ranked paths, or within a user threshold).

Checked against brute-force enumeration of every alignment (the set within the
threshold and its order: increasing lexicographic order of the reversed column
sequence), against the single-alignment oracle (the first optimal one), against
independent rescoring, and by planted mistakes.
"""
import os
import subprocess

import numpy as np
import pytest

import inputs
import oracle
from tests._independent import column_score, rescore_rows

SRC = os.path.join(os.path.dirname(oracle.__file__), "msa_oracle.c")
PAPER_TABLE = np.eye(4, dtype=np.int32)  # section 5.2: +1 match, 0 mismatch (gap -1)


def all_alignments(seqs, alphabet, table, gap):
    """Every alignment as (score, masks first column first), by enumeration."""
    k = len(seqs)
    out = []
    path = []

    def rec(x, acc):
        if all(v == 0 for v in x):
            out.append((acc, list(reversed(path))))
            return
        for m in range(1, 1 << k):
            if any(((m >> i) & 1) and x[i] == 0 for i in range(k)):
                continue
            chars = [seqs[i][x[i] - 1] if (m >> i) & 1 else None for i in range(k)]
            path.append(m)
            rec([x[i] - ((m >> i) & 1) for i in range(k)], acc + column_score(chars, alphabet, table, gap))
            path.pop()

    rec([len(s) for s in seqs], 0)
    return out


def expected(seqs, alphabet, table, gap, delta):
    al = all_alignments(seqs, alphabet, table, gap)
    opt = max(s for s, _ in al)
    keep = [(s, m) for s, m in al if s >= opt - delta]
    keep.sort(key=lambda t: list(reversed(t[1])))
    return keep


def _cases():
    rng = np.random.default_rng(51)
    cases = []
    for lens in [(3, 4), (4, 4), (2, 3, 3), (3, 2, 3), (0, 3, 2), (1, 1, 1, 1)]:
        seqs = [inputs.random_seq(rng, "ACGT", n) for n in lens]
        cases.append((seqs, PAPER_TABLE, -1))
        asym = rng.integers(-4, 5, size=(4, 4)).astype(np.int32)
        cases.append((seqs, asym, -2))
    return cases


@pytest.mark.parametrize("delta", [0, 1, 3])
def test_enumeration_equals_brute_force(delta):
    for seqs, table, gap in _cases():
        want = expected(seqs, "ACGT", table, gap, delta)
        got, more = oracle.align_near_optimal(seqs, "ACGT", table, gap, delta, max_count=100000)
        assert not more
        assert [(r.score, r.masks) for r in got] == want, (seqs, delta)


def test_first_optimal_is_the_single_alignment_and_scores_rescore():
    rng = np.random.default_rng(52)
    for k, n in [(2, 30), (3, 12), (4, 6)]:
        p = inputs.random_problem(int(rng.integers(1000)), k, [n] * k, table=PAPER_TABLE, gap=-1)
        best = oracle.align_problem(p)
        opt, _ = oracle.align_near_optimal(p.seqs, p.alphabet, p.subst, p.gap, 0, max_count=50)
        assert opt[0].masks == best.masks and all(r.score == best.score for r in opt)
        got, _ = oracle.align_near_optimal(p.seqs, p.alphabet, p.subst, p.gap, 2, max_count=50)
        for r in got:
            assert rescore_rows(r.rows, p.alphabet, p.subst, p.gap) == r.score >= best.score - 2
            assert [row.replace("-", "") for row in r.rows] == p.seqs
        order = [list(reversed(r.masks)) for r in got]
        assert order == sorted(order) and len({tuple(o) for o in order}) == len(order)


def test_truncation_at_max_count():
    seqs, table, gap = ["ACGTA", "AGTC", "CGTA"], PAPER_TABLE, -1
    full, more = oracle.align_near_optimal(seqs, "ACGT", table, gap, 2, max_count=100000)
    assert not more and len(full) > 3
    part, more = oracle.align_near_optimal(seqs, "ACGT", table, gap, 2, max_count=len(full) - 1)
    assert more and [r.masks for r in part] == [r.masks for r in full[:-1]]
    exact, more = oracle.align_near_optimal(seqs, "ACGT", table, gap, 2, max_count=len(full))
    assert not more and len(exact) == len(full)


def test_empty_sequences():
    got, more = oracle.align_near_optimal(["", ""], "ACGT", PAPER_TABLE, -1, 0, 4)
    assert not more and [(r.score, r.masks) for r in got] == [(0, [])]
    got, _ = oracle.align_near_optimal(["", "AC"], "ACGT", PAPER_TABLE, -1, 5, 4)
    assert [(r.score, r.masks) for r in got] == [(-2, [2, 2])]


NEAR_MUTANTS = {
    "threshold_strict": ("H[pred] + sp + acc[d] >= threshold", "H[pred] + sp + acc[d] > threshold"),
    "suffix_score_not_accumulated": ("acc[d + 1] = acc[d] + sp;", "acc[d + 1] = acc[d];"),
    "columns_not_reversed": ("dst[c] = path[d - 1 - c];", "dst[c] = path[c];"),
    "delta_ignored": ("const int64_t threshold = score - delta;", "const int64_t threshold = score;"),
}


def _near_pins(lib):
    for seqs, table, gap in _cases()[:6]:
        for delta in (0, 2):
            want = expected(seqs, "ACGT", table, gap, delta)
            got, more = oracle.align_near_optimal(seqs, "ACGT", table, gap, delta, max_count=100000, lib=lib)
            assert [(r.score, r.masks) for r in got] == want


def test_unmutated_enumeration_passes_the_battery():
    _near_pins(None)


@pytest.mark.parametrize("name", sorted(NEAR_MUTANTS))
def test_planted_enumeration_mistake_is_caught(name, tmp_path):
    old, new = NEAR_MUTANTS[name]
    src = open(SRC).read()
    marker = "int oracle_msa_near_optimal("
    head, tail = src.split(marker, 1)  # mutate the enumeration code only
    assert tail.count(old) == 1, f"mutation anchor for {name} not unique"
    cpath = tmp_path / "mutant.c"
    cpath.write_text(head + marker + tail.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", str(so), str(cpath)])
    lib = oracle.load_library(str(so))
    with pytest.raises(AssertionError):
        _near_pins(lib)
