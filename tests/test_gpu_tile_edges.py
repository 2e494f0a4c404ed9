"""Every compiled tile edge of the generic kernel against the oracle (full
traceback tensor, score, alignment), and the autotuner's choice."""
import numpy as np
import pytest

import inputs
import oracle
import paper_2311_17530_gb300 as msa
from paper_2311_17530_gb300 import msadp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CANDIDATES = {2: [16, 32, 64], 3: [8, 12, 16], 4: [4, 5, 6], 5: [3, 4, 5], 6: [2, 3, 4], 7: [2, 3], 8: [2]}
# several tiles per axis for the largest edge, with ragged tails
SHAPES = {2: [150, 201], 3: [40, 35, 33], 4: [18, 14, 17, 12], 5: [11, 9, 10, 8, 7], 6: [8, 9, 7, 9, 8, 6],
          7: [5, 6, 4, 5, 6, 5, 4], 8: [3, 4, 3, 4, 3, 4, 3, 2]}


@pytest.fixture(autouse=True)
def restore():
    msa.msa_config("fill_kernel", 1)
    yield
    msa.msa_config("fill_kernel", 0)
    for k in CANDIDATES:
        msa.msa_set_tile_edge(k, 0)
    for k in (4, 5, 6):
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
        return score, rows, status, plan.read_tb(), plan.info()
    finally:
        plan.close()


@pytest.mark.parametrize("k,edge", [(k, e) for k, es in CANDIDATES.items() for e in es])
def test_every_tile_edge_matches_oracle(k, edge):
    msa.msa_set_tile_edge(k, edge)
    alphabet = inputs.PROTEIN if k % 2 else inputs.DNA
    p = inputs.random_problem(3000 + 10 * k + edge, k, SHAPES[k], alphabet=alphabet, related=True)
    want = oracle.align(p.seqs, p.alphabet, p.subst, p.gap, want_tb=True)
    score, rows, status, tb, info = run(p)
    assert status == 0
    assert info.tile_extent[:k] == [2 * edge if (k == 2 and i == 1) else edge for i in range(k)]
    assert (score, rows) == (want.score, want.rows)
    np.testing.assert_array_equal(tb, np.asarray(want.tb).reshape(tb.shape))


def test_autotune_picks_the_fastest_and_plans_follow():
    msa.msa_config("fill_kernel", 0)
    res = msa.msa_autotune([90, 100, 110], 20, repeats=2)
    kinds = {(c["kernel"], c["edge"]) for c in res["candidates"]}
    assert kinds == {("tiles", 8), ("tiles", 12), ("tiles", 16), ("column", 0)}
    best = min(res["candidates"], key=lambda c: c["ms"])
    assert res["best"] == best
    plan = msa.Plan(3, [90, 100, 110], inputs.PROTEIN)
    try:
        want_kernel = 2 if best["kernel"] == "column" else 1
        assert plan.info().fill_kernel == want_kernel
        if best["kernel"] == "tiles":
            assert msa.msa_get_tile_edge(3) == best["edge"]
    finally:
        plan.close()
    res4 = msa.msa_autotune([30, 32, 34, 36], 4, repeats=2)
    assert {(c["kernel"], c["edge"]) for c in res4["candidates"]} == {("tiles", 4), ("tiles", 5), ("tiles", 6),
                                                                      ("lines", 8), ("lines", 16), ("lines", 32),
                                                                      ("stream", 0)}
    best4 = res4["best"]
    if best4["kernel"] == "tiles":
        assert msa.msa_get_tile_edge(4) == best4["edge"]
    elif best4["kernel"] == "lines":
        assert msa.msa_get_line_segment(4) == best4["edge"]
    else:  # the streamed kernel: the best segment stays the choice where it cannot run
        lines = [c for c in res4["candidates"] if c["kernel"] == "lines"]
        assert msa.msa_get_line_segment(4) == min(lines, key=lambda c: c["ms"])["edge"]
    with msa.Plan(4, [30, 32, 34, 36], inputs.DNA) as plan4:
        assert plan4.info().fill_kernel == {"tiles": 1, "lines": 4, "stream": 5}[best4["kernel"]]
    # the tuned shape still gives the oracle's answer
    p = inputs.random_problem(3100, 4, [14, 17, 15, 13], related=True)
    want = oracle.align(p.seqs, p.alphabet, p.subst, p.gap)
    assert msa.msa_align(p.seqs, p.alphabet, p.subst, p.gap) == (want.score, want.rows)


def test_serving_with_non_default_edges():
    msa.msa_config("fill_kernel", 0)
    msa.msa_set_tile_edge(2, 64)
    msa.msa_set_tile_edge(4, 4)
    probs = [inputs.random_problem(3200 + i, (2, 4)[i % 2], [130, 170] if i % 2 == 0 else [9, 12, 10, 11],
                                   related=True) for i in range(8)]
    handles = [msa.msa_submit(p.seqs, p.alphabet, p.subst, p.gap) for p in probs]
    msa.msa_drain()
    for h, p in zip(handles, probs):
        want = oracle.align(p.seqs, p.alphabet, p.subst, p.gap)
        assert msa.msa_poll(h, p.k, sum(p.lens)) == (want.score, want.rows)
