"""GPU parity: libmsadp's CUDA path against the CPU oracle, bit for bit.

Integer arithmetic throughout, so the tolerance is zero: the same int32 score,
the same alignment under "lowest move mask wins", and (where the oracle can
afford the full tensor) the same traceback byte in every cell.
"""
import itertools
import json
import os

import numpy as np
import pytest

import inputs
import oracle
import paper_2311_17530_gb300 as msa
from paper_2311_17530_gb300 import msadp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _stream():
    return torch.cuda.current_stream().cuda_stream


def run_plan(p, plan=None, want_tb=False, residues=None, subst=None):
    own = plan is None
    plan = plan or msa.Plan(p.k, p.lens, p.alphabet)
    try:
        d_res, d_sub = msadp.device_inputs(p)
        if residues is not None:
            d_res = residues
        if subst is not None:
            d_sub = subst
        d_result, d_masks = msadp.device_outputs(sum(p.lens))
        plan.execute(d_res.data_ptr(), d_sub.data_ptr(), p.gap, d_result.data_ptr(), d_masks.data_ptr(),
                     _stream())
        torch.cuda.synchronize()
        score, rows, status = msadp.decode_device_result(d_result, d_masks, p.seqs)
        tb = plan.read_tb() if want_tb and status == 0 else None
        return score, rows, status, tb
    finally:
        if own:
            plan.close()


def check_problem(p, full_tb=True):
    o = oracle.align_problem(p, want_tb=full_tb)
    score, rows, status, tb = run_plan(p, want_tb=full_tb)
    assert status == 0, (p.name, status)
    assert score == o.score, (p.name, score, o.score)
    assert rows == o.rows, p.name
    if full_tb:
        np.testing.assert_array_equal(tb, o.tb, err_msg=p.name)


@pytest.mark.parametrize("k", [2, 3, 4, 5, 6])
def test_random_small_problems_full_tensor(k):
    hi = {2: 150, 3: 40, 4: 16, 5: 9, 6: 6}[k]
    rng = np.random.default_rng(100 + k)
    for rep in range(6):
        lens = [int(x) for x in rng.integers(0, hi + 1, size=k)]
        alphabet = inputs.PROTEIN if rep % 2 else inputs.DNA
        check_problem(inputs.random_problem(1000 * k + rep, k, lens, alphabet=alphabet, related=rep % 3 == 0))


@pytest.mark.parametrize("k,lens", [
    (2, [31, 63]), (2, [32, 64]), (2, [33, 65]), (2, [95, 1]), (2, [0, 200]), (2, [300, 0]),
    (3, [11, 11, 11]), (3, [12, 12, 12]), (3, [13, 24, 25]), (3, [0, 0, 0]), (3, [1, 1, 1]),
    (3, [0, 30, 7]), (4, [5, 6, 7, 12]), (4, [1, 0, 13, 2]), (5, [3, 4, 5, 7, 8]),
    (6, [2, 3, 4, 5, 3, 2]), (7, [2, 1, 3, 2, 1, 2, 3]), (8, [1, 2, 1, 2, 1, 2, 1, 2]),
])
def test_tile_boundaries_and_degenerate_shapes(k, lens):
    check_problem(inputs.random_problem(77 + sum(lens), k, lens))


def test_ties_heavy_scoring_scheme():
    """The paper's +1/0/-1/0 scheme (section 5.2) produces many equal scores."""
    table = np.eye(4, dtype=np.int32)
    for k, lens in [(2, [60, 50]), (3, [20, 25, 18]), (4, [9, 8, 10, 7])]:
        p = inputs.random_problem(5 + k, k, lens, table=table, gap=-1)
        check_problem(p)


def test_msa_align_c_abi_host_buffers():
    rng = np.random.default_rng(9)
    for rep in range(8):
        k = int(rng.integers(2, 6))
        hi = {2: 120, 3: 30, 4: 12, 5: 7}[k]
        p = inputs.random_problem(500 + rep, k, [int(x) for x in rng.integers(0, hi + 1, size=k)],
                                  alphabet=inputs.PROTEIN if rep % 2 else inputs.DNA)
        o = oracle.align_problem(p)
        score, rows = msa.msa_align(p.seqs, p.alphabet, p.subst, p.gap)
        assert (score, rows) == (o.score, o.rows), p.name
    p = inputs.pr1()
    g = json.load(open(os.path.join(GOLDEN, "pr1.json")))
    score, rows = msa.msa_align(p.seqs, p.alphabet, p.subst, p.gap)
    assert score == g["score"]
    assert rows == oracle.expand(p.seqs, bytes.fromhex(g["masks_hex"]))


def test_plan_reuse_is_deterministic():
    p = inputs.random_problem(3, 3, [37, 41, 29])
    with msa.Plan(p.k, p.lens, p.alphabet) as plan:
        a = run_plan(p, plan=plan, want_tb=True)
        b = run_plan(p, plan=plan, want_tb=True)
    assert a[:3] == b[:3]
    np.testing.assert_array_equal(a[3], b[3])


@pytest.mark.parametrize("name,kernel", [("pr1", 0), ("k2_protein", 0), ("k3_protein", 0), ("k4_dna", 4),
                                         ("k4_dna", 5), ("k6_protein", 4), ("k6_protein", 5)])
def test_full_size_workloads_against_stored_oracle_values(name, kernel):
    """Full-size workloads: score, alignment and sampled traceback bytes against
    values written by tests/golden/make_golden.py (oracle only); k = 4 DNA and
    k = 6 protein through both line kernels (segmented and streamed)."""
    path = os.path.join(GOLDEN, f"{name}.json")
    if not os.path.exists(path):
        pytest.skip(f"{path} not generated")
    g = json.load(open(path))
    p = inputs.WORKLOADS[name]()
    assert p.lens == g["lens"]
    msa.msa_config("fill_kernel", kernel)
    try:
        with msa.Plan(p.k, p.lens, p.alphabet) as plan:
            assert kernel == 0 or plan.info().fill_kernel == kernel
            score, rows, status, tb = run_plan(p, plan=plan, want_tb=True)
    finally:
        msa.msa_config("fill_kernel", 0)
    assert status == 0
    assert score == g["score"]
    assert rows == oracle.expand(p.seqs, bytes.fromhex(g["masks_hex"]))
    flat = tb.reshape(-1)
    idx = np.array([s[0] for s in g["tb_samples"]], dtype=np.int64)
    want = np.array([s[1] for s in g["tb_samples"]], dtype=np.uint8)
    np.testing.assert_array_equal(flat[idx], want)
    # properties that hold at any size: rescoring, de-gapping, column count
    from tests._independent import rescore_rows
    assert rescore_rows(rows, p.alphabet, p.subst, p.gap) == score
    assert [r.replace("-", "") for r in rows] == p.seqs


def test_device_side_input_errors():
    p = inputs.random_problem(4, 3, [10, 12, 9])
    bad = torch.tensor(list(b"ACGTXCGT" + b"A" * (sum(p.lens) - 8)), dtype=torch.uint8, device="cuda")
    assert run_plan(p, residues=bad)[2] == msa.MSA_EINVAL
    asym = p.subst.copy()
    asym[0, 1] = 2
    d_asym = torch.from_numpy(asym.reshape(-1).astype(np.int32)).cuda()
    assert run_plan(p, subst=d_asym)[2] == msa.MSA_EINVAL
    # x10^5 still fits the packed int32 keys for these short sequences: exact result
    scaled = inputs.Problem(p.name, p.seqs, p.alphabet, p.subst * 100000, p.gap * 100000)
    check_problem(scaled)
    # x10^7 does not: the device range check refuses it instead of overflowing
    huge = torch.from_numpy((p.subst * 10**7).reshape(-1).astype(np.int32)).cuda()
    assert run_plan(p, subst=huge)[2] == msa.MSA_ETOOBIG
    # the context is still usable and the same plan shape works again
    check_problem(p)


def test_dependency_wait_timeout_is_reported_not_hung():
    """A withheld tile release makes its dependants' bounded waits run out."""
    p = inputs.random_problem(6, 3, [40, 40, 40])
    msa.msa_config("spin_timeout_ms", 200)
    msa.msa_config("test_withhold_tile", 0)
    try:
        assert run_plan(p)[2] == msa.MSA_ETIMEOUT
        with pytest.raises(msa.MsaError) as ei:
            msa.msa_align(p.seqs, p.alphabet, p.subst, p.gap)
        assert ei.value.code == msa.MSA_ETIMEOUT
    finally:
        msa.msa_config("test_withhold_tile", -1)
        msa.msa_config("spin_timeout_ms", 5000)
    check_problem(p)


@pytest.mark.parametrize("kernel", [1, 2])
def test_k3_both_fill_kernels_block_boundaries(kernel):
    """k=3 through the generic tile kernel (1) and the column kernel (2): shapes
    straddling the column kernel's 32-row column blocks, 32-lane blocks and 8-step blocks."""
    msa.msa_config("fill_kernel", kernel)
    try:
        shapes = [(63, 31, 40), (64, 32, 100), (65, 33, 7), (130, 70, 50), (1, 1, 200),
                  (200, 1, 1), (0, 100, 100), (100, 0, 5), (3, 3, 0), (129, 97, 61)]
        for i, lens in enumerate(shapes):
            p = inputs.random_problem(900 + i, 3, list(lens),
                                      alphabet=inputs.PROTEIN if i % 2 else inputs.DNA, related=i % 3 == 0)
            with msa.Plan(3, p.lens, p.alphabet) as plan:
                assert plan.info().fill_kernel == kernel
            check_problem(p)
    finally:
        msa.msa_config("fill_kernel", 0)


@pytest.mark.parametrize("kernel", [1, 3])
def test_k2_tile_and_band_kernels_boundaries(kernel):
    """k=2 through the generic tile kernel (1) and the band kernel (3): shapes
    straddling the band kernel's 32-row bands and 32-column face blocks, empty
    and single-row or single-column problems."""
    msa.msa_config("fill_kernel", kernel)
    try:
        shapes = [(31, 31), (32, 32), (33, 33), (63, 95), (64, 1), (1, 64), (0, 50), (50, 0), (0, 0), (1, 1),
                  (97, 33), (200, 180), (31, 500), (500, 31), (95, 96)]
        for i, lens in enumerate(shapes):
            p = inputs.random_problem(1900 + i, 2, list(lens),
                                      alphabet=inputs.PROTEIN if i % 2 else inputs.DNA, related=i % 3 == 0)
            with msa.Plan(2, p.lens, p.alphabet) as plan:
                assert plan.info().fill_kernel == kernel
            check_problem(p)
    finally:
        msa.msa_config("fill_kernel", 0)


def test_k2_band_wait_timeout_is_reported_not_hung():
    """A withheld band never publishes its face, so the band below times out
    (three bands of 128 rows)."""
    p = inputs.random_problem(7, 2, [300, 80])
    with msa.Plan(2, p.lens, p.alphabet) as plan:
        assert plan.info().fill_kernel == 3
    msa.msa_config("spin_timeout_ms", 200)
    msa.msa_config("test_withhold_tile", 0)
    try:
        assert run_plan(p)[2] == msa.MSA_ETIMEOUT
    finally:
        msa.msa_config("test_withhold_tile", -1)
        msa.msa_config("spin_timeout_ms", 5000)
    check_problem(p)


def test_k3_auto_picks_column_kernel():
    p = inputs.k3_protein()
    with msa.Plan(3, [10, 10, 10], p.alphabet) as plan:
        assert plan.info().fill_kernel == 2


@pytest.mark.parametrize("kernel,k,lens", [(2, 3, [40, 37, 45]), (2, 3, [63, 95, 70]), (3, 2, [150, 170]),
                                           (3, 2, [33, 400]), (4, 4, [9, 13, 10, 40]), (1, 4, [9, 13, 10, 40]),
                                           (5, 4, [9, 13, 10, 40]), (5, 5, [5, 4, 5, 9, 40]),
                                           (5, 6, [5, 4, 3, 3, 2, 20])])
def test_every_fill_kernel_records_the_corner_key(kernel, k, lens):
    """Every fill kernel records the far corner's packed key; the traceback
    compares the rescored path with it. A consistent result (status 0, the
    oracle's score) shows the record and the check agree for each kernel."""
    msa.msa_config("fill_kernel", kernel)
    msa.msa_config("verify_corner", 1)  # the column kernel records it only when asked
    try:
        p = inputs.random_problem(6100 + sum(lens), k, lens, alphabet=inputs.PROTEIN, related=True)
        with msa.Plan(k, p.lens, p.alphabet) as plan:
            assert plan.info().fill_kernel == kernel
        o = oracle.align_problem(p)
        score, rows, status, _ = run_plan(p)
        assert status == 0 and (score, rows) == (o.score, o.rows)
    finally:
        msa.msa_config("verify_corner", 0)
        msa.msa_config("fill_kernel", 0)


@pytest.mark.parametrize("seed", [3, 99])
@pytest.mark.parametrize("kernel,k,lens", [(2, 3, [70, 65, 90]), (3, 2, [150, 170]), (1, 3, [30, 25, 28]),
                                           (1, 4, [9, 8, 10, 7]), (1, 5, [5, 4, 6, 5, 4]),
                                           (5, 4, [9, 13, 10, 70]), (5, 5, [5, 4, 5, 9, 40]),
                                           (5, 6, [5, 4, 3, 3, 2, 20])])
def test_shuffled_orders_over_a_poisoned_traceback(kernel, k, lens, seed):
    """Tickets permuted inside every wave (another topological order of the same
    tiles or columns) and the traceback tensor filled with 0xFF before the fill:
    every cell must still equal the oracle (a missed dependency or an unwritten
    cell would show), and no cell may keep 0xFF (no move for k < 8)."""
    msa.msa_config("fill_kernel", kernel)
    msa.msa_config("test_shuffle_waves", seed)
    msa.msa_config("test_poison_tb", 1)
    try:
        p = inputs.random_problem(6200 + seed + 10 * kernel + k, k, lens, alphabet=inputs.PROTEIN, related=True)
        with msa.Plan(k, p.lens, p.alphabet) as plan:
            assert plan.info().fill_kernel == kernel
        o = oracle.align_problem(p, want_tb=True)
        score, rows, status, tb = run_plan(p, want_tb=True)
        assert status == 0 and (score, rows) == (o.score, o.rows)
        assert not (tb == 0xFF).any()
        np.testing.assert_array_equal(tb, o.tb)
    finally:
        msa.msa_config("test_poison_tb", 0)
        msa.msa_config("test_shuffle_waves", 0)
        msa.msa_config("fill_kernel", 0)
