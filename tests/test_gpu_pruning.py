"""Exact search-space pruning on the device (section 6: search only the
partitions where an optimal alignment can lie) against the oracle:

* the device's tile bounds equal oracle_tile_bounds element by element, for
  several extents and k = 2 .. 5;
* the pruned fill gives the full oracle's score and alignment (the same tie
  rule), with the device's own lower bound, with the optimum itself as the
  bound, and with a bound too low to leave anything out;
* the tiles it leaves out are those whose bound is below L, and the oracle's DP
  with exactly those cells left out gives the same result;
* the device's lower bound never exceeds the optimum, and related sequences get
  tiles left out;
* a bound above the optimum is reported, not answered."""
import numpy as np
import pytest

import inputs
import oracle
import paper_2311_17530_gb300 as msa
from paper_2311_17530_gb300 import msadp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PAPER_TABLE = np.eye(4, dtype=np.int32)  # section 5.2: +1 match, 0 mismatch, gap -1


def _problems():
    out = []
    shapes = [(40, 37), (150, 170), (20, 24, 22), (45, 40, 50), (9, 11, 10, 12), (14, 13, 15, 12), (6, 7, 5, 6, 7)]
    for i, lens in enumerate(shapes):
        out.append(inputs.random_problem(9000 + i, len(lens), list(lens), alphabet=inputs.PROTEIN, related=True))
        out.append(inputs.random_problem(9100 + i, len(lens), list(lens), alphabet=inputs.DNA, related=False))
    out.append(inputs.random_problem(9200, 3, [30, 28, 33], table=PAPER_TABLE, gap=-1))
    return out


def plan_extents(k, lens):
    """Tile extents of the generic tile kernel for this shape (the pruned fill's tiles)."""
    msa.msa_config("fill_kernel", 1)
    try:
        ext, grid = msa.msa_tile_shape(lens)
    finally:
        msa.msa_config("fill_kernel", 0)
    return ext, grid


@pytest.mark.parametrize("p", _problems(), ids=lambda p: p.name)
def test_tile_bounds_match_oracle(p):
    for ext in ([3] * p.k, [5] * p.k, [1] + [4] * (p.k - 1), plan_extents(p.k, p.lens)[0]):
        got = msadp.msa_tile_bounds(p.seqs, p.alphabet, p.subst, p.gap, ext)
        want = oracle.tile_bounds(p.seqs, p.alphabet, p.subst, p.gap, ext).reshape(-1)
        np.testing.assert_array_equal(got, want, err_msg=f"{p.name} {ext}")


@pytest.mark.parametrize("p", _problems(), ids=lambda p: p.name)
def test_pruned_fill_matches_full_oracle(p):
    want = oracle.align_problem(p)
    score, rows, st = msadp.msa_align_pruned(p.seqs, p.alphabet, p.subst, p.gap)
    assert (score, rows) == (want.score, want.rows), p.name
    assert st["lower_bound"] <= want.score
    assert 0 <= st["tiles_skipped"] <= st["tiles"] and 0 <= st["cells_skipped"] <= st["cells"]
    # the same with the optimum as the bound (the tightest exact bound)
    score2, rows2, st2 = msadp.msa_align_pruned(p.seqs, p.alphabet, p.subst, p.gap, lower_bound=want.score)
    assert (score2, rows2) == (want.score, want.rows)
    assert st2["tiles_skipped"] >= st["tiles_skipped"]
    # a bound below every tile's: nothing left out
    score3, rows3, st3 = msadp.msa_align_pruned(p.seqs, p.alphabet, p.subst, p.gap, lower_bound=-(1 << 40))
    assert (score3, rows3) == (want.score, want.rows) and st3["tiles_skipped"] == 0


@pytest.mark.parametrize("p", _problems()[::3], ids=lambda p: p.name)
def test_left_out_tiles_are_those_below_the_bound(p):
    """Rebuild the set of left-out cells from the device bounds and L, and run the
    oracle's DP without them: the same score and alignment, and the same count."""
    want = oracle.align_problem(p)
    score, rows, st = msadp.msa_align_pruned(p.seqs, p.alphabet, p.subst, p.gap, lower_bound=want.score)
    ext, grid = plan_extents(p.k, p.lens)
    bounds = msadp.msa_tile_bounds(p.seqs, p.alphabet, p.subst, p.gap, ext).reshape(grid)
    out_tiles = bounds < want.score
    assert int(out_tiles.sum()) == st["tiles_skipped"]
    ex = np.zeros([n + 1 for n in p.lens], dtype=np.uint8)
    for t in zip(*np.nonzero(out_tiles)):
        ex[tuple(slice(c * e, (c + 1) * e) for c, e in zip(t, ext))] = 1
    assert int(ex.sum()) == st["cells_skipped"]
    got = oracle.align_excluding(p.seqs, p.alphabet, p.subst, p.gap, ex)
    assert (got.score, got.rows) == (want.score, want.rows) == (score, rows)


def test_related_sequences_leave_tiles_out():
    """Related sequences: the device's feasible alignment is close to the optimum
    and most of the tensor lies below it."""
    for seed, lens in [(9300, [120, 110, 130]), (9301, [40, 42, 38, 41])]:
        p = inputs.random_problem(seed, len(lens), lens, alphabet=inputs.PROTEIN, related=True)
        want = oracle.align_problem(p)
        score, rows, st = msadp.msa_align_pruned(p.seqs, p.alphabet, p.subst, p.gap)
        assert (score, rows) == (want.score, want.rows)
        assert st["cells_skipped"] > st["cells"] // 4, st


def test_bound_above_the_optimum_is_reported():
    p = inputs.random_problem(9400, 3, [25, 22, 27], alphabet=inputs.PROTEIN, related=True)
    want = oracle.align_problem(p)
    with pytest.raises(msa.MsaError) as ei:
        msadp.msa_align_pruned(p.seqs, p.alphabet, p.subst, p.gap, lower_bound=want.score + 1000)
    assert ei.value.code == msa.MSA_EINVAL
