"""The line-sweep fill (k = 4..6) against the oracle, bit for bit: every compiled
segment length on shapes that span several line blocks and several segments
with ragged tails, degenerate shapes, other topological tile orders, a
traceback buffer poisoned before the fill, and a withheld tile."""
import numpy as np
import pytest

import inputs
import oracle
import paper_2311_17530_gb300 as msa
from paper_2311_17530_gb300 import msadp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SEGMENTS = {4: [8, 16, 32], 5: [16, 32], 6: [16, 25]}
# line blocks are 2x4x4 (k=4), 2x2x2x4 (k=5), 2^5 (k=6); every shape covers several
# blocks per line axis with a ragged tail and at least two segments of the last axis
SHAPES = {
    (4, 8): [9, 13, 10, 30], (4, 16): [9, 13, 10, 40], (4, 32): [9, 13, 10, 70],
    (5, 16): [5, 4, 5, 9, 40], (5, 32): [3, 4, 3, 9, 70],
    (6, 16): [4, 3, 4, 3, 4, 30], (6, 25): [3, 4, 3, 4, 3, 52],
}


@pytest.fixture(autouse=True)
def lines_kernel():
    msa.msa_config("fill_kernel", 4)
    yield
    msa.msa_config("fill_kernel", 0)
    msa.msa_config("test_shuffle_waves", 0)
    msa.msa_config("test_poison_tb", 0)
    for k in SEGMENTS:
        msa.msa_set_line_segment(k, 0)


def run(p):
    plan = msa.Plan(p.k, p.lens, p.alphabet)
    try:
        d_res, d_sub = msadp.device_inputs(p)
        d_result, d_masks = msadp.device_outputs(sum(p.lens))
        plan.execute(d_res.data_ptr(), d_sub.data_ptr(), p.gap, d_result.data_ptr(), d_masks.data_ptr(),
                     torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        score, rows, status = msadp.decode_device_result(d_result, d_masks, p.seqs)
        return score, rows, status, (plan.read_tb() if status == 0 else None), plan.info()
    finally:
        plan.close()


def check(p, z=None):
    want = oracle.align(p.seqs, p.alphabet, p.subst, p.gap, want_tb=True)
    score, rows, status, tb, info = run(p)
    assert info.fill_kernel == 4
    assert status == 0, (p.name, status)
    assert (score, rows) == (want.score, want.rows), p.name
    np.testing.assert_array_equal(tb, np.asarray(want.tb).reshape(tb.shape), err_msg=p.name)
    return info


@pytest.mark.parametrize("k,z", [(k, z) for k, zs in SEGMENTS.items() for z in zs])
def test_every_segment_length_matches_oracle(k, z):
    msa.msa_set_line_segment(k, z)
    lens = SHAPES[(k, z)]
    for rep, alphabet in enumerate((inputs.DNA, inputs.PROTEIN)):
        p = inputs.random_problem(4000 + 10 * k + z + rep, k, lens, alphabet=alphabet, related=rep == 0)
        info = check(p)
        rho = lens[-1] + 1
        nseg = -(-rho // z)
        assert info.tile_extent[k - 1] == -(-rho // nseg)
        assert info.tile_grid[k - 1] == nseg


@pytest.mark.parametrize("k,lens", [
    (4, [0, 0, 0, 0]), (4, [1, 1, 1, 1]), (4, [0, 5, 3, 9]), (4, [6, 0, 0, 40]), (4, [2, 4, 4, 0]),
    (4, [1, 3, 3, 31]), (4, [2, 4, 4, 32]), (4, [3, 5, 5, 33]), (4, [12, 2, 1, 7]),
    (5, [0, 1, 0, 1, 0]), (5, [1, 1, 1, 3, 15]), (5, [2, 2, 2, 4, 31]), (5, [4, 3, 2, 1, 0]),
    (6, [0, 0, 0, 0, 0, 0]), (6, [1, 1, 1, 1, 1, 24]), (6, [2, 2, 2, 2, 2, 25]), (6, [5, 1, 0, 2, 3, 4]),
])
def test_degenerate_and_block_boundary_shapes(k, lens):
    check(inputs.random_problem(4100 + sum(lens) + 7 * k, k, lens, alphabet=inputs.PROTEIN))


def test_ties_heavy_scoring_scheme():
    """The paper's +1/0/-1/0 scheme (section 5.2): many equal candidates, so the
    lowest-mask rule decides most cells."""
    table = np.eye(4, dtype=np.int32)
    for k, lens in [(4, [9, 8, 10, 40]), (5, [4, 5, 3, 6, 20]), (6, [3, 2, 3, 4, 3, 12])]:
        check(inputs.random_problem(4200 + k, k, lens, table=table, gap=-1))


@pytest.mark.parametrize("seed", [1, 7, 12345])
def test_shuffled_tile_orders(seed):
    """Tickets permuted inside every wave: another topological order of the same
    tiles, so a missing dependency shows up as a different traceback byte."""
    msa.msa_config("test_shuffle_waves", seed)
    for k, lens in [(4, [9, 13, 10, 70]), (5, [5, 4, 5, 9, 40]), (6, [4, 3, 4, 3, 4, 30])]:
        check(inputs.random_problem(4300 + seed + k, k, lens, alphabet=inputs.PROTEIN, related=True))


def test_every_cell_written_over_a_poisoned_buffer():
    """The traceback tensor is filled with 0xFF before the fill; no cell of the
    tensor may keep it (0xFF is no valid move for k < 8) and all equal the oracle."""
    msa.msa_config("test_poison_tb", 1)
    for k, lens in [(4, [9, 13, 10, 70]), (5, [3, 4, 3, 9, 70]), (6, [3, 4, 3, 4, 3, 52])]:
        p = inputs.random_problem(4400 + k, k, lens, alphabet=inputs.DNA)
        score, rows, status, tb, info = run(p)
        assert status == 0
        assert not (tb == 0xFF).any()
        check(p)


def test_withheld_tile_times_out_not_hangs():
    p = inputs.random_problem(4500, 4, [9, 13, 10, 70])
    msa.msa_config("spin_timeout_ms", 200)
    msa.msa_config("test_withhold_tile", 0)
    try:
        assert run(p)[2] == msa.MSA_ETIMEOUT
    finally:
        msa.msa_config("test_withhold_tile", -1)
        msa.msa_config("spin_timeout_ms", 5000)
    check(p)


def test_serving_batches_line_kernel_problems():
    """Continuous batching with several k = 4..6 requests in one persistent launch."""
    msa.msa_config("fill_kernel", 0)
    probs = [inputs.random_problem(4600 + i, 4 + i % 3, [[9, 12, 10, 40], [4, 5, 3, 6, 20], [3, 2, 3, 4, 3, 12]][i % 3],
                                   related=True) for i in range(9)]
    handles = [msa.msa_submit(p.seqs, p.alphabet, p.subst, p.gap) for p in probs]
    msa.msa_drain()
    for h, p in zip(handles, probs):
        want = oracle.align(p.seqs, p.alphabet, p.subst, p.gap)
        assert msa.msa_poll(h, p.k, sum(p.lens)) == (want.score, want.rows)
