"""Optimal and near-optimal alignment enumeration on the device (section 6:
further solutions by forking at equally ranked paths or within a user
threshold) against the oracle's enumeration, item by item: the same alignments
(move masks), in the same order, with the same scores, the same count and the
same "more left" flag, for thresholds 0, 1 and 3 and several caps; k = 2 .. 5
(row-major kept scores for k <= 3, tile-major for k >= 4), the paper's
ties-heavy +1/0/-1/0 scheme and random tables."""
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
    for i, lens in enumerate([(5, 6), (12, 9), (4, 5, 4), (7, 6, 8), (3, 4, 3, 4), (6, 5, 7, 6), (3, 2, 3, 3, 2)]):
        out.append(inputs.random_problem(8000 + i, len(lens), list(lens), table=PAPER_TABLE, gap=-1))
        out.append(inputs.random_problem(8100 + i, len(lens), list(lens), alphabet=inputs.PROTEIN, related=True))
    return out


def check(p, delta, max_count):
    got, more = msadp.msa_near_optimal(p.seqs, p.alphabet, p.subst, p.gap, delta, max_count)
    want, wmore = oracle.align_near_optimal(p.seqs, p.alphabet, p.subst, p.gap, delta, max_count)
    assert more == wmore, (p.name, delta, max_count)
    assert len(got) == len(want), (p.name, delta, max_count, len(got), len(want))
    for a, (g, w) in enumerate(zip(got, want)):
        assert g[1] == w.masks, (p.name, delta, a)
        assert g[0] == w.score, (p.name, delta, a)
        assert g[2] == w.rows, (p.name, delta, a)
    return got


@pytest.mark.parametrize("p", _problems(), ids=lambda p: p.name)
@pytest.mark.parametrize("delta,max_count", [(0, 200), (1, 200), (3, 7), (0, 1)])
def test_enumeration_matches_oracle(p, delta, max_count):
    got = check(p, delta, max_count)
    if delta == 0:  # the first optimal alignment is the single-alignment traceback's
        score, rows = msa.msa_align(p.seqs, p.alphabet, p.subst, p.gap)
        assert (got[0][0], got[0][2]) == (score, rows)


def test_larger_problems_and_caps():
    """Longer sequences: the walk's depth spans hundreds of columns; the cap stops
    it with alignments left."""
    for seed, lens in [(8200, [60, 55, 58]), (8201, [14, 12, 15, 13]), (8202, [300, 280])]:
        p = inputs.random_problem(seed, len(lens), lens, table=PAPER_TABLE, gap=-1)
        check(p, 2, 50)


def test_empty_and_degenerate_shapes():
    for lens in [(0, 0), (0, 5), (3, 0, 2), (1, 1, 1, 1)]:
        p = inputs.random_problem(8300 + sum(lens), len(lens), list(lens), table=PAPER_TABLE, gap=-1)
        check(p, 1, 100)


def test_bad_arguments():
    p = inputs.random_problem(8400, 3, [4, 4, 4])
    with pytest.raises(msa.MsaError) as ei:
        msadp.msa_near_optimal(p.seqs, p.alphabet, p.subst, p.gap, -1, 10)
    assert ei.value.code == msa.MSA_EINVAL
    with pytest.raises(msa.MsaError) as ei:
        msadp.msa_near_optimal(p.seqs, p.alphabet, p.subst, p.gap, 0, 0)
    assert ei.value.code == msa.MSA_EINVAL
