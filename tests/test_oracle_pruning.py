"""Pins for the oracle of exact search-space pruning (the paper's future work,
section 6; the bound of Carrillo and Lipman).

The oracle's pairwise tables are checked against the textbook recurrence (Eq. 1)
on every prefix and suffix pair; its bound against brute-force enumeration of
every alignment through every cell; its pruned DP against the unpruned oracle
(score and alignment, for every lower bound up to the optimum) and against an
independent count of the cells the bound leaves out. Planted mistakes in the
pruning code are caught by these pins.
"""
import itertools
import os
import subprocess

import numpy as np
import pytest

import inputs
import oracle
from tests._independent import column_score, needleman_wunsch, rescore_rows

SRC = os.path.join(os.path.dirname(oracle.__file__), "msa_oracle.c")


def _asym(seed, n):
    return np.random.default_rng(seed).integers(-5, 6, size=(n, n)).astype(np.int32)


def _pair_bound(seqs, alphabet, table, gap):
    """U(x) for every cell, from textbook NW on prefixes and suffixes (independent of the oracle)."""
    k = len(seqs)
    shape = tuple(len(s) + 1 for s in seqs)
    U = np.zeros(shape, dtype=np.int64)
    for i in range(k):
        for j in range(i + 1, k):
            a, b = seqs[i], seqs[j]
            pq = np.zeros((len(a) + 1, len(b) + 1), dtype=np.int64)
            for p in range(len(a) + 1):
                for q in range(len(b) + 1):
                    pq[p, q] = (needleman_wunsch(a[:p], b[:q], alphabet, table, gap)[0]
                                + needleman_wunsch(a[p:], b[q:], alphabet, table, gap)[0])
            for x in itertools.product(*[range(n) for n in shape]):
                U[x] += pq[x[i], x[j]]
    return U


def _best_through_each_cell(seqs, alphabet, table, gap):
    """Best alignment score over every alignment through each cell, by enumeration."""
    k = len(seqs)
    shape = tuple(len(s) + 1 for s in seqs)
    best = np.full(shape, np.iinfo(np.int64).min, dtype=np.int64)
    cells = []

    def rec(x, acc):
        cells.append(tuple(x))
        if all(v == 0 for v in x):
            for c in cells:
                best[c] = max(best[c], acc)
        else:
            for m in range(1, 1 << k):
                if any(((m >> i) & 1) and x[i] == 0 for i in range(k)):
                    continue
                chars = [seqs[i][x[i] - 1] if (m >> i) & 1 else None for i in range(k)]
                rec([x[i] - ((m >> i) & 1) for i in range(k)], acc + column_score(chars, alphabet, table, gap))
        cells.pop()

    rec([len(s) for s in seqs], 0)
    return best


def test_pair_tables_are_prefix_and_suffix_nw_scores():
    rng = np.random.default_rng(41)
    for rep in range(6):
        table, gap = (_asym(rep, 4), -3) if rep % 2 else (inputs.dna_table(), -8)
        a = inputs.random_seq(rng, "ACGT", int(rng.integers(0, 8)))
        b = inputs.random_seq(rng, "ACGT", int(rng.integers(0, 8)))
        fwd, bwd = oracle.pair_tables(a, b, "ACGT", table, gap)
        for p in range(len(a) + 1):
            for q in range(len(b) + 1):
                assert fwd[p, q] == needleman_wunsch(a[:p], b[:q], "ACGT", table, gap)[0]
                assert bwd[p, q] == needleman_wunsch(a[p:], b[q:], "ACGT", table, gap)[0]
        assert fwd[-1, -1] == bwd[0, 0]


def test_bound_is_at_least_every_alignment_through_the_cell():
    rng = np.random.default_rng(42)
    for lens in [(2, 3, 2), (3, 1, 3), (3, 3, 2)]:
        seqs = [inputs.random_seq(rng, "ACG", n) for n in lens]
        table, gap = _asym(sum(lens), 3), -2
        U = _pair_bound(seqs, "ACG", table, gap)
        best = _best_through_each_cell(seqs, "ACG", table, gap)
        assert (U >= best).all()
        # every alignment passes through the origin: the enumeration's best there is the optimum
        assert best[(0,) * 3] == oracle.align(seqs, "ACG", table, gap).score


@pytest.mark.parametrize("k,lens", [(2, [40, 37]), (3, [25, 22, 27]), (4, [9, 11, 8, 10]), (5, [6, 5, 7, 6, 5])])
def test_pruned_dp_equals_the_full_dp_for_every_bound_up_to_the_optimum(k, lens):
    for rep in range(3):
        p = inputs.random_problem(300 + 10 * k + rep, k, lens, alphabet=inputs.PROTEIN if rep % 2 else inputs.DNA,
                                  related=rep != 2)
        full = oracle.align_problem(p)
        # a feasible alignment: every sequence left-aligned, padded with gaps
        width = max(lens)
        feasible = rescore_rows([s + "-" * (width - len(s)) for s in p.seqs], p.alphabet, p.subst, p.gap)
        assert feasible <= full.score
        prev = None
        for L in sorted({full.score, full.score - 1, full.score - 7, (full.score + feasible) // 2, feasible},
                        reverse=True):
            r, excluded = oracle.align_pruned(p.seqs, p.alphabet, p.subst, p.gap, L)
            assert (r.score, r.masks) == (full.score, full.masks), (p.name, L)
            assert prev is None or excluded <= prev  # a lower bound keeps at least as many cells
            prev = excluded
        assert excluded >= 0


def test_cells_left_out_match_an_independent_count():
    rng = np.random.default_rng(43)
    for lens in [(3, 4, 3), (4, 2, 4), (2, 5)]:
        seqs = [inputs.random_seq(rng, "ACG", n) for n in lens]
        table, gap = _asym(7 + sum(lens), 3), -2
        U = _pair_bound(seqs, "ACG", table, gap)
        opt = oracle.align(seqs, "ACG", table, gap).score
        for L in (opt, opt - 2, opt - 10):
            _, excluded = oracle.align_pruned(seqs, "ACG", table, gap, L)
            assert excluded == int((U < L).sum()), (lens, L)


def test_related_sequences_prune_most_of_the_tensor():
    p = inputs.random_problem(5, 3, [40, 42, 38], alphabet=inputs.PROTEIN, related=True)
    full = oracle.align_problem(p)
    r, excluded = oracle.align_pruned(p.seqs, p.alphabet, p.subst, p.gap, full.score)
    assert r.score == full.score and excluded > 0.9 * p.cells


def test_bound_above_the_optimum_is_reported():
    p = inputs.random_problem(8, 3, [12, 10, 11])
    full = oracle.align_problem(p)
    with pytest.raises(oracle.BoundAboveOptimum):
        oracle.align_pruned(p.seqs, p.alphabet, p.subst, p.gap, full.score + 1)


PRUNING_MUTANTS = {
    "bound_uses_forward_twice": ("U += fwd[i][j][idx] + bwd[i][j][idx];", "U += fwd[i][j][idx] + fwd[i][j][idx];"),
    "backward_residue_off_by_one": ("bwd[(p + 1) * W + q + 1] + sub[a[p] * A + b[q]] > best",
                                    "bwd[(p + 1) * W + q + 1] + sub[a[p > 0 ? p - 1 : 0] * A + b[q]] > best"),
    "bound_compared_with_ge": ("if (U < lower_bound) {", "if (U <= lower_bound) {"),
    "forward_residue_off_by_one": ("sub[a[p - 1] * A + b[q - 1]]", "sub[a[p - 1] * A + b[q > 1 ? q - 2 : 0]]"),
    "forward_gap_dropped": ("fwd[p * W + q - 1] + gap", "fwd[p * W + q - 1] + 0"),
}


def _pruning_pins(lib):
    rng = np.random.default_rng(44)
    for lens in [(3, 4, 3), (2, 5)]:
        seqs = [inputs.random_seq(rng, "ACG", n) for n in lens]
        table, gap = _asym(11 + sum(lens), 3), -2
        U = _pair_bound(seqs, "ACG", table, gap)
        full = oracle.align(seqs, "ACG", table, gap)
        for L in (full.score, full.score - 3):
            r, excluded = oracle.align_pruned(seqs, "ACG", table, gap, L, lib=lib)
            assert (r.score, r.masks) == (full.score, full.masks)
            assert excluded == int((U < L).sum())
        a, b = seqs[0], seqs[1]
        fwd, bwd = oracle.pair_tables(a, b, "ACG", table, gap, lib=lib)
        for p in range(len(a) + 1):
            for q in range(len(b) + 1):
                assert fwd[p, q] == needleman_wunsch(a[:p], b[:q], "ACG", table, gap)[0]
                assert bwd[p, q] == needleman_wunsch(a[p:], b[q:], "ACG", table, gap)[0]


def test_unmutated_pruning_passes_the_battery():
    _pruning_pins(None)


@pytest.mark.parametrize("name", sorted(PRUNING_MUTANTS))
def test_planted_pruning_mistake_is_caught(name, tmp_path):
    old, new = PRUNING_MUTANTS[name]
    src = open(SRC).read()
    head, tail = src.split("#define ORACLE_NEG", 1)  # mutate the pruning code only
    assert tail.count(old) >= 1, f"mutation anchor for {name} not found"
    cpath = tmp_path / "mutant.c"
    cpath.write_text(head + "#define ORACLE_NEG" + tail.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", str(so), str(cpath)])
    lib = oracle.load_library(str(so))
    with pytest.raises((AssertionError, oracle.BoundAboveOptimum)):
        _pruning_pins(lib)


# --- whole tiles: the per-tile bound and the DP with cells left out -------------

def _expand_tiles(mask, extents, shape):
    out = mask
    for ax, e in enumerate(extents):
        out = np.repeat(out, e, axis=ax)
    return out[tuple(slice(0, n) for n in shape)]


def test_tile_bound_is_never_below_the_cells_inside():
    rng = np.random.default_rng(45)
    for lens, ext in [((4, 5, 3), (2, 2, 2)), ((5, 3, 4), (3, 2, 4)), ((6, 7), (3, 2)), ((3, 3, 2, 3), (2, 2, 2, 2))]:
        seqs = [inputs.random_seq(rng, "ACG", n) for n in lens]
        table, gap = _asym(13 + sum(lens), 3), -2
        U = _pair_bound(seqs, "ACG", table, gap)
        tb = oracle.tile_bounds(seqs, "ACG", table, gap, ext)
        for t in itertools.product(*[range(g) for g in tb.shape]):
            cells = U[tuple(slice(c * e, (c + 1) * e) for c, e in zip(t, ext))]
            assert tb[t] >= cells.max(), (lens, ext, t)
            if len(lens) == 2:  # one pair: the bound is the tile's largest cell bound
                assert tb[t] == cells.max()


def test_skipping_tiles_below_the_bound_keeps_the_result():
    for k, lens, ext in [(3, [30, 28, 33], (8, 8, 8)), (4, [9, 10, 8, 11], (3, 3, 3, 3)), (2, [60, 55], (16, 16))]:
        p = inputs.random_problem(60 + k, k, lens, alphabet=inputs.PROTEIN, related=True)
        full = oracle.align_problem(p)
        shape = tuple(n + 1 for n in lens)
        for L in (full.score, full.score - 4):
            skip = oracle.tile_bounds(p.seqs, p.alphabet, p.subst, p.gap, ext) < L
            assert skip.any()
            r = oracle.align_excluding(p.seqs, p.alphabet, p.subst, p.gap, _expand_tiles(skip, ext, shape))
            assert (r.score, r.masks) == (full.score, full.masks), (p.name, L)


def test_any_subset_of_prunable_cells_keeps_the_result():
    rng = np.random.default_rng(46)
    for lens in [(4, 5, 4), (6, 5)]:
        seqs = [inputs.random_seq(rng, "ACG", n) for n in lens]
        table, gap = _asym(17 + sum(lens), 3), -2
        U = _pair_bound(seqs, "ACG", table, gap)
        full = oracle.align(seqs, "ACG", table, gap)
        plain = oracle.align_excluding(seqs, "ACG", table, gap, np.zeros(U.shape, dtype=bool))
        assert (plain.score, plain.masks) == (full.score, full.masks)
        for rep in range(5):
            ex = (U < full.score - rep) & (rng.random(U.shape) < 0.6)
            r = oracle.align_excluding(seqs, "ACG", table, gap, ex)
            assert (r.score, r.masks) == (full.score, full.masks)


def test_leaving_out_a_cell_of_the_optimal_path_changes_the_path():
    p = inputs.random_problem(9, 3, [12, 11, 13], related=True)
    full = oracle.align_problem(p)
    x = [0, 0, 0]
    for m in full.masks[: len(full.masks) // 2]:  # walk half of the path from the origin
        x = [x[i] + ((m >> i) & 1) for i in range(3)]
    ex = np.zeros(tuple(n + 1 for n in p.lens), dtype=bool)
    ex[tuple(x)] = True
    try:
        r = oracle.align_excluding(p.seqs, p.alphabet, p.subst, p.gap, ex)
        assert r.masks != full.masks and r.score <= full.score
    except oracle.BoundAboveOptimum:
        pass


TILE_MUTANTS = {
    "tile_bound_keeps_last_pair_only": ("out_bound[t] += blk[ci * G[j] + cj];", "out_bound[t] = blk[ci * G[j] + cj];"),
    "tile_bound_takes_minimum": ("if (v > blk[b])", "if (blk[b] == ORACLE_NEG || v < blk[b])"),
    "exclusions_ignored": ("if (excluded[l]) {", "if (0) {"),
}


def _tile_pins(lib):
    rng = np.random.default_rng(47)
    seqs = [inputs.random_seq(rng, "ACG", n) for n in (5, 3, 4)]
    table, gap = _asym(19, 3), -2
    U = _pair_bound(seqs, "ACG", table, gap)
    tb = oracle.tile_bounds(seqs, "ACG", table, gap, (2, 2, 2), lib=lib)
    for t in itertools.product(*[range(g) for g in tb.shape]):
        assert tb[t] >= U[tuple(slice(2 * c, 2 * c + 2) for c in t)].max()
    full = oracle.align(seqs, "ACG", table, gap)
    x = [0, 0, 0]
    for m in full.masks[:3]:
        x = [x[i] + ((m >> i) & 1) for i in range(3)]
    ex = np.zeros(U.shape, dtype=bool)
    ex[tuple(x)] = True
    try:
        r = oracle.align_excluding(seqs, "ACG", table, gap, ex, lib=lib)
        assert r.masks != full.masks
    except oracle.BoundAboveOptimum:
        pass


def test_unmutated_tile_pruning_passes_the_battery():
    _tile_pins(None)


@pytest.mark.parametrize("name", sorted(TILE_MUTANTS))
def test_planted_tile_pruning_mistake_is_caught(name, tmp_path):
    old, new = TILE_MUTANTS[name]
    src = open(SRC).read()
    marker = "int oracle_tile_bounds("
    head, tail = src.split(marker, 1)
    assert tail.count(old) == 1, f"mutation anchor for {name} not unique"
    cpath = tmp_path / "mutant.c"
    cpath.write_text(head + marker + tail.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", str(so), str(cpath)])
    lib = oracle.load_library(str(so))
    with pytest.raises(AssertionError):
        _tile_pins(lib)
