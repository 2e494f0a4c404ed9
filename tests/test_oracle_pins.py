"""Pins for the CPU oracle, against facts fixed by the paper and by mathematics.

None of these re-types the oracle's own loop: brute-force enumeration of every
alignment, the textbook pairwise recurrence (Eq. 1), a closed form for identical
sequences, permutation invariance of the sum-of-pairs score (section 5.2), and
structural invariants of any global alignment. The paper's 6-sequence example
(section 5.2, score -5) cannot be used: its sequences are not published.
"""
import itertools
import math

import numpy as np
import pytest

import inputs
import oracle
from tests._independent import brute_force, needleman_wunsch, rescore_rows

# The paper's own SP scheme, section 5.2: +1 match, 0 mismatch, -1 gap, 0 gap-gap.
PAPER_SCHEME = (np.array([[1 if a == b else 0 for b in range(4)] for a in range(4)], dtype=np.int32), -1)


def _asym_table(seed, n=4):
    rng = np.random.default_rng(seed)
    return rng.integers(-5, 6, size=(n, n)).astype(np.int32)


def _check_vs_brute(seqs, alphabet, table, gap):
    bs, bm = brute_force(seqs, alphabet, table, gap)
    r = oracle.align(seqs, alphabet, table, gap)
    assert r.score == bs, (seqs, r.score, bs)
    assert r.masks == bm, (seqs, r.masks, bm)


@pytest.mark.parametrize("table_kind", ["paper", "dna", "asym"])
def test_brute_force_k2_all_lengths_0_to_4(table_kind):
    rng = np.random.default_rng(11)
    for la in range(5):
        for lb in range(5):
            for rep in range(2):
                seqs = [inputs.random_seq(rng, "ACGT", la), inputs.random_seq(rng, "ACGT", lb)]
                if table_kind == "paper":
                    table, gap = PAPER_SCHEME
                elif table_kind == "dna":
                    table, gap = inputs.dna_table(), -8
                else:
                    table, gap = _asym_table(la * 10 + lb + rep), -3
                _check_vs_brute(seqs, "ACGT", table, gap)


@pytest.mark.parametrize("table_kind", ["paper", "asym"])
def test_brute_force_k3_all_lengths_0_to_3(table_kind):
    rng = np.random.default_rng(12)
    for lens in itertools.product(range(4), repeat=3):
        seqs = [inputs.random_seq(rng, "ACG", n) for n in lens]
        if table_kind == "paper":
            table, gap = PAPER_SCHEME[0][:3, :3], PAPER_SCHEME[1]
        else:
            table, gap = _asym_table(sum(lens), 3), -2
        _check_vs_brute(seqs, "ACG", table, gap)


def test_brute_force_k3_length_4():
    p = inputs.random_problem(7, 3, [4, 4, 4])
    _check_vs_brute(p.seqs, p.alphabet, p.subst, p.gap)
    rng = np.random.default_rng(5)
    seqs = [inputs.random_seq(rng, "AC", n) for n in (4, 3, 4)]
    _check_vs_brute(seqs, "AC", PAPER_SCHEME[0][:2, :2], -1)


def test_brute_force_k4_small():
    rng = np.random.default_rng(13)
    for lens in [(2, 2, 2, 2), (1, 2, 0, 2), (2, 1, 2, 1)]:
        seqs = [inputs.random_seq(rng, "AC", n) for n in lens]
        _check_vs_brute(seqs, "AC", _asym_table(3, 2), -2)


def test_brute_force_every_cell_of_tb_and_H():
    """tb(x) and H(x) of the full tensor equal brute force on the prefix problem x."""
    rng = np.random.default_rng(21)
    seqs = [inputs.random_seq(rng, "ACG", n) for n in (3, 2, 3)]
    table, gap = _asym_table(9, 3), -2
    r = oracle.align(seqs, "ACG", table, gap, want_tb=True, want_H=True)
    for x in itertools.product(*[range(len(s) + 1) for s in seqs]):
        pre = [s[:n] for s, n in zip(seqs, x)]
        bs, bm = brute_force(pre, "ACG", table, gap)
        assert r.H[x] == bs
        assert r.tb[x] == (bm[-1] if bm else 0)


def test_textbook_needleman_wunsch_k2():
    rng = np.random.default_rng(31)
    prot = inputs.protein_table(np.random.default_rng(2))
    for rep in range(40):
        la, lb = int(rng.integers(0, 40)), int(rng.integers(0, 40))
        if rep % 2:
            alphabet, table, gap = "ACGT", inputs.dna_table(), -8
        else:
            alphabet, table, gap = inputs.PROTEIN, prot, -6
        a = inputs.random_seq(rng, alphabet, la)
        b = inputs.random_seq(rng, alphabet, lb)
        ns, nm = needleman_wunsch(a, b, alphabet, table, gap)
        r = oracle.align([a, b], alphabet, table, gap)
        assert (r.score, r.masks) == (ns, nm)


@pytest.mark.parametrize("k,L", [(2, 15), (3, 12), (4, 9), (5, 6), (6, 5)])
def test_closed_form_identical_sequences(k, L):
    """k copies of one sequence: score C(k,2) * sum_x sub(s_x, s_x), all-diagonal path."""
    rng = np.random.default_rng(k * 100 + L)
    for alphabet, table, gap in [("ACGT", inputs.dna_table(), -8),
                                 (inputs.PROTEIN, inputs.protein_table(rng), -6)]:
        s = inputs.random_seq(rng, alphabet, L)
        idx = {c: i for i, c in enumerate(alphabet)}
        expect = math.comb(k, 2) * sum(int(table[idx[c], idx[c]]) for c in s)
        r = oracle.align([s] * k, alphabet, table, gap)
        assert r.score == expect
        assert r.masks == [(1 << k) - 1] * L


def test_permutation_invariance_of_score():
    rng = np.random.default_rng(41)
    for k, lens_hi, nperm in [(3, 12, None), (4, 7, None), (5, 4, 10)]:
        for rep in range(3):
            lens = [int(x) for x in rng.integers(0, lens_hi + 1, size=k)]
            p = inputs.random_problem(int(rng.integers(1 << 30)), k, lens,
                                      alphabet=inputs.PROTEIN if rep % 2 else inputs.DNA)
            base = oracle.align_problem(p).score
            perms = list(itertools.permutations(range(k)))
            if nperm is not None:
                perms = [perms[int(i)] for i in rng.choice(len(perms), size=nperm, replace=False)]
            for perm in perms:
                seqs = [p.seqs[i] for i in perm]
                assert oracle.align(seqs, p.alphabet, p.subst, p.gap).score == base


def test_alignment_invariants():
    rng = np.random.default_rng(51)
    for rep in range(30):
        k = int(rng.integers(2, 6))
        hi = {2: 40, 3: 14, 4: 8, 5: 5}[k]
        lens = [int(x) for x in rng.integers(0, hi + 1, size=k)]
        p = inputs.random_problem(1000 + rep, k, lens,
                                  alphabet=inputs.PROTEIN if rep % 3 == 0 else inputs.DNA,
                                  related=bool(rep % 2))
        r = oracle.align_problem(p)
        # rescoring the emitted alignment column by column gives the score
        assert rescore_rows(r.rows, p.alphabet, p.subst, p.gap) == r.score
        # de-gapping each row gives its sequence
        assert [row.replace("-", "") for row in r.rows] == p.seqs
        # no column is all gaps; all rows have ncols characters
        assert all(m != 0 for m in r.masks)
        assert all(len(row) == len(r.masks) for row in r.rows)
        # ncols lies between the longest sequence and the total length
        assert max(lens) <= len(r.masks) <= sum(lens)
        # SP score is bounded by the sum of optimal pairwise scores
        pair_sum = sum(needleman_wunsch(p.seqs[i], p.seqs[j], p.alphabet, p.subst, p.gap)[0]
                       for i in range(k) for j in range(i + 1, k))
        assert r.score <= pair_sum
        if k == 2:
            assert r.score == pair_sum


def test_empty_sequences():
    t = inputs.dna_table()
    r = oracle.align(["", "ACGTA"], "ACGT", t, -8)
    assert r.score == -8 * 5 and r.masks == [2] * 5
    r = oracle.align(["ACG", ""], "ACGT", t, -8)
    assert r.score == -8 * 3 and r.masks == [1] * 3
    r = oracle.align(["", "", ""], "ACGT", t, -8)
    assert r.score == 0 and r.masks == [] and r.rows == ["", "", ""]
    # k=3 with one empty row: each column also pays one residue/gap pair per residue
    r = oracle.align(["ACG", "", "AG"], "ACGT", t, -8)
    assert rescore_rows(r.rows, "ACGT", t, -8) == r.score


@pytest.mark.parametrize("k", [2, 3, 4])
def test_paper_scheme_brute_force(k):
    """The paper's +1/0/-1/0 scoring (section 5.2) against exhaustive enumeration."""
    rng = np.random.default_rng(40 + k)
    lens = [int(x) for x in rng.integers(0, 4 if k < 4 else 3, size=k)]
    seqs = [inputs.random_seq(rng, "ACGT", n) for n in lens]
    table = inputs.paper_table(4)
    bs, bm = brute_force(seqs, "ACGT", table, inputs.PAPER_GAP)
    r = oracle.align(seqs, "ACGT", table, inputs.PAPER_GAP)
    assert (r.score, r.masks) == (bs, bm)


@pytest.mark.parametrize("k", [7, 8])
def test_paper_scheme_identical_sequences_closed_form(k):
    """k copies of one sequence under +1/0/-1/0: C(k,2) * L, all-diagonal."""
    s = "ACGTTGCA"[: 9 - k]
    r = oracle.align([s] * k, "ACGT", inputs.paper_table(4), inputs.PAPER_GAP)
    assert r.score == k * (k - 1) // 2 * len(s)
    assert r.masks == [(1 << k) - 1] * len(s)
