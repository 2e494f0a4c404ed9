"""The streamed line fill (k = 4..6; one warp per 32-line block over the whole last
axis, faces published as (value, epoch) entries) against the oracle, bit for
bit: shapes spanning several line blocks with ragged tails and several 8-step
blocks of the last axis, degenerate shapes, the ties-heavy scheme, other
topological column orders, a traceback buffer poisoned before the fill, a
withheld column, back-to-back executions of one plan on different inputs (the
previous launch's face entries carry an older epoch and must not be taken), and
serving, which runs the segmented line kernel instead."""
import numpy as np
import pytest

import inputs
import oracle
import paper_2311_17530_gb300 as msa
from paper_2311_17530_gb300 import msadp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# line blocks are 2x4x4 (k=4), 2x2x2x4 (k=5) and 2x2x2x2x2 (k=6), super-blocks
# 4x8x8, 4x4x2x4 and 4x4x2x2x2 lines; the last axis spans several 8-position
# chunks with a ragged tail
SHAPES = [
    (4, [9, 13, 10, 30]), (4, [9, 13, 10, 70]), (4, [3, 7, 9, 129]), (4, [17, 5, 6, 17]),
    (5, [5, 4, 5, 9, 40]), (5, [3, 4, 3, 9, 70]), (5, [4, 2, 5, 3, 23]),
    (6, [5, 4, 3, 3, 2, 20]), (6, [3, 5, 2, 4, 3, 9]), (6, [8, 4, 2, 2, 4, 33]),
]


@pytest.fixture(autouse=True)
def stream_kernel():
    msa.msa_config("fill_kernel", 5)
    yield
    msa.msa_config("fill_kernel", 0)
    msa.msa_config("test_shuffle_waves", 0)
    msa.msa_config("test_poison_tb", 0)


def run(p, plan=None):
    own = plan is None
    plan = plan or msa.Plan(p.k, p.lens, p.alphabet)
    try:
        d_res, d_sub = msadp.device_inputs(p)
        d_result, d_masks = msadp.device_outputs(sum(p.lens))
        plan.execute(d_res.data_ptr(), d_sub.data_ptr(), p.gap, d_result.data_ptr(), d_masks.data_ptr(),
                     torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        score, rows, status = msadp.decode_device_result(d_result, d_masks, p.seqs)
        return score, rows, status, (plan.read_tb() if status == 0 else None), plan.info()
    finally:
        if own:
            plan.close()


def check(p, plan=None):
    want = oracle.align(p.seqs, p.alphabet, p.subst, p.gap, want_tb=True)
    score, rows, status, tb, info = run(p, plan)
    assert info.fill_kernel == 5
    assert status == 0, (p.name, status)
    assert (score, rows) == (want.score, want.rows), p.name
    np.testing.assert_array_equal(tb, np.asarray(want.tb).reshape(tb.shape), err_msg=p.name)
    return info


@pytest.mark.parametrize("k,lens", SHAPES)
def test_shapes_match_oracle(k, lens):
    for rep, alphabet in enumerate((inputs.DNA, inputs.PROTEIN)):
        p = inputs.random_problem(7000 + 13 * k + sum(lens) + rep, k, lens, alphabet=alphabet, related=rep == 0)
        info = check(p)
        assert info.tile_extent[k - 1] == lens[-1] + 1  # one column spans the whole last axis
        assert info.tile_grid[k - 1] == 1


@pytest.mark.parametrize("k,lens", [
    (4, [0, 0, 0, 0]), (4, [1, 1, 1, 1]), (4, [0, 5, 3, 9]), (4, [6, 0, 0, 40]), (4, [2, 4, 4, 0]),
    (4, [1, 3, 3, 7]), (4, [2, 4, 4, 8]), (4, [3, 5, 5, 15]), (4, [12, 2, 1, 16]), (4, [1, 1, 1, 200]),
    (5, [0, 1, 0, 1, 0]), (5, [1, 1, 1, 3, 15]), (5, [2, 2, 2, 4, 31]), (5, [4, 3, 2, 1, 0]),
    (6, [0, 1, 0, 1, 0, 1]), (6, [1, 1, 1, 1, 1, 15]), (6, [3, 3, 1, 1, 1, 7]), (6, [4, 4, 2, 2, 2, 8]),
    (6, [2, 0, 3, 1, 2, 0]),
])
def test_degenerate_and_block_boundary_shapes(k, lens):
    check(inputs.random_problem(7100 + sum(lens) + 7 * k, k, lens, alphabet=inputs.PROTEIN))


def test_ties_heavy_scoring_scheme():
    """The paper's +1/0/-1/0 scheme (section 5.2): many equal candidates, so the
    lowest-mask rule decides most cells."""
    table = np.eye(4, dtype=np.int32)
    for k, lens in [(4, [9, 8, 10, 40]), (5, [4, 5, 3, 6, 20]), (6, [3, 4, 2, 3, 2, 17])]:
        check(inputs.random_problem(7200 + k, k, lens, table=table, gap=-1))


@pytest.mark.parametrize("seed", [1, 7, 12345])
def test_shuffled_column_orders(seed):
    """Tickets permuted inside every wave: another topological order of the same
    columns, so a missing dependency shows up as a different traceback byte."""
    msa.msa_config("test_shuffle_waves", seed)
    for k, lens in [(4, [9, 13, 10, 70]), (5, [5, 4, 5, 9, 40]), (6, [5, 4, 3, 3, 2, 20])]:
        check(inputs.random_problem(7300 + seed + k, k, lens, alphabet=inputs.PROTEIN, related=True))


def test_every_cell_written_over_a_poisoned_buffer():
    """The traceback tensor is filled with 0xFF before the fill; no cell of the
    tensor may keep it (0xFF is no valid move for k < 8) and all equal the oracle."""
    msa.msa_config("test_poison_tb", 1)
    for k, lens in [(4, [9, 13, 10, 70]), (5, [3, 4, 3, 9, 70]), (6, [3, 5, 2, 4, 3, 9])]:
        p = inputs.random_problem(7400 + k, k, lens, alphabet=inputs.DNA)
        score, rows, status, tb, info = run(p)
        assert status == 0
        assert not (tb == 0xFF).any()
        check(p)


@pytest.mark.parametrize("k,lens", [(4, [9, 13, 10, 70]), (6, [5, 4, 3, 3, 2, 20])])
def test_back_to_back_executions_take_only_this_launchs_entries(k, lens):
    """One plan executed on different inputs of the same shape, several times in a
    row: each launch's faces carry a new epoch (k = 4) or are read only after this
    launch's completion flags, zeroed at every launch (k = 6, whole-column form),
    so a consumer that took a face of the previous launch (a stale score) would
    disagree with the oracle."""
    probs = [inputs.random_problem(7500 + 10 * k + i, k, lens, alphabet=inputs.PROTEIN, related=i % 2 == 0)
             for i in range(4)]
    plan = msa.Plan(k, lens, inputs.PROTEIN)
    try:
        for p in probs + probs[:2]:
            check(p, plan)
    finally:
        plan.close()


@pytest.mark.parametrize("k,lens", [(4, [9, 13, 10, 70]), (6, [5, 4, 3, 3, 2, 20]), (6, [3, 4, 2, 3, 2, 30])])
def test_withheld_column_times_out_not_hangs(k, lens):
    """A withheld column publishes nothing valid (its faces carry tag 0, or its
    completion flag is never set), so its consumers give up after the wait limit
    and the plan reports a timeout; the next execution is whole again."""
    p = inputs.random_problem(7600 + k + lens[-1], k, lens)
    msa.msa_config("spin_timeout_ms", 200)
    msa.msa_config("test_withhold_tile", 0)
    try:
        assert run(p)[2] == msa.MSA_ETIMEOUT
    finally:
        msa.msa_config("test_withhold_tile", -1)
        msa.msa_config("spin_timeout_ms", 5000)
    check(p)


def test_automatic_choice_and_serving():
    """k = 4, 5 plans take the streamed kernel by default, k = 6 plans when the
    last axis fits the whole-column form; serving runs the segmented line kernel
    for the same shapes and matches the oracle."""
    msa.msa_config("fill_kernel", 0)
    for k in (4, 5, 6):
        msa.msa_set_line_segment(k, 0)  # default choices
    with msa.Plan(4, [9, 13, 10, 70], inputs.DNA) as plan:
        assert plan.info().fill_kernel == 5
    with msa.Plan(6, [3, 4, 3, 4, 3, 12], inputs.DNA) as plan:  # the whole-column form fits
        assert plan.info().fill_kernel == 5
    with msa.Plan(6, [3, 4, 3, 4, 3, 30], inputs.DNA) as plan:  # it does not: the line kernel
        assert plan.info().fill_kernel == 4
    for choice in (0, 5):
        msa.msa_config("fill_kernel", choice)
        probs = [inputs.random_problem(7700 + i, 4 + i % 2, [[9, 12, 10, 40], [4, 5, 3, 6, 20]][i % 2],
                                       related=True) for i in range(6)]
        handles = [msa.msa_submit(p.seqs, p.alphabet, p.subst, p.gap) for p in probs]
        msa.msa_drain()
        for h, p in zip(handles, probs):
            want = oracle.align(p.seqs, p.alphabet, p.subst, p.gap)
            assert msa.msa_poll(h, p.k, sum(p.lens)) == (want.score, want.rows)

