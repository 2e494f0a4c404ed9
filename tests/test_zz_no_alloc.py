"""msa_align_noalloc: the entry point for callers that cannot allocate device
memory (another allocator owns the GPU, latency-critical loops, no recovery from
an allocation failure mid-request). It must give exactly what the allocating
entry point gives, call after call, although every call reuses -- and inherits
the leftovers of -- the same fixed scratch array inside the library.
"""
import pytest

import inputs
import oracle
import paper_2311_17530_gb300 as msa
from paper_2311_17530_gb300 import msadp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _noalloc(p):
    d_res, d_sub = msadp.device_inputs(p)
    d_result, d_masks = msadp.device_outputs(sum(p.lens))
    msadp.msa_align_noalloc(p.lens, p.alphabet, d_res.data_ptr(), d_sub.data_ptr(), p.gap,
                            d_result.data_ptr(), d_masks.data_ptr(), _stream())
    torch.cuda.synchronize()
    return msadp.decode_device_result(d_result, d_masks, p.seqs)


def _allocating(p):
    with msa.Plan(p.k, p.lens, p.alphabet) as plan:
        d_res, d_sub = msadp.device_inputs(p)
        d_result, d_masks = msadp.device_outputs(sum(p.lens))
        plan.execute(d_res.data_ptr(), d_sub.data_ptr(), p.gap, d_result.data_ptr(), d_masks.data_ptr(),
                     _stream())
        torch.cuda.synchronize()
        return msadp.decode_device_result(d_result, d_masks, p.seqs)


def test_noalloc_matches_allocating_entry_point_on_calls_in_a_row():
    # two different problems back to back, then the first again: each call must
    # be unaffected by what the previous one left in the shared scratch
    first = inputs.pr1()
    second = inputs.random_problem(42, 4, [30, 27, 33, 25], alphabet=inputs.PROTEIN, related=True)
    for p in (first, second, first):
        got = _noalloc(p)
        want = _allocating(p)
        assert got[2] == 0, (p.name, got[2])
        assert got == want, p.name


def test_noalloc_calls_queued_back_to_back_without_host_sync():
    """A, B and A again queued on one stream with no synchronisation in between,
    each with its own outputs: every call clears the launch state, flags and wave
    counters it needs on the stream, after the previous call's fill and traceback."""
    probs = [inputs.random_problem(43, 3, [60, 55, 70], alphabet=inputs.PROTEIN, related=True),
             inputs.random_problem(44, 4, [20, 18, 22, 17], alphabet=inputs.DNA, related=True)]
    probs.append(probs[0])
    outs = []
    for p in probs:
        d_res, d_sub = msadp.device_inputs(p)
        d_result, d_masks = msadp.device_outputs(sum(p.lens))
        msadp.msa_align_noalloc(p.lens, p.alphabet, d_res.data_ptr(), d_sub.data_ptr(), p.gap,
                                d_result.data_ptr(), d_masks.data_ptr(), _stream())
        outs.append((p, d_res, d_sub, d_result, d_masks))
    torch.cuda.synchronize()
    for p, _r, _s, d_result, d_masks in outs:
        score, rows, status = msadp.decode_device_result(d_result, d_masks, p.seqs)
        want = oracle.align_problem(p)
        assert status == 0, p.name
        assert (score, rows) == (want.score, want.rows), p.name  # the rows are the masks spelled out


def test_noalloc_largest_accepted_cube_is_exact():
    """The largest k = 3 cube whose working set fits the static array, against the oracle."""
    for n in range(200, 100, -1):
        p = inputs.random_problem(45, 3, [n, n, n], alphabet=inputs.DNA, related=True)
        d_res, d_sub = msadp.device_inputs(p)
        d_result, d_masks = msadp.device_outputs(sum(p.lens))
        try:
            msadp.msa_align_noalloc(p.lens, p.alphabet, d_res.data_ptr(), d_sub.data_ptr(), p.gap,
                                    d_result.data_ptr(), d_masks.data_ptr(), _stream())
        except msa.MsaError as e:
            assert e.code == msa.MSA_ETOOBIG
            continue
        torch.cuda.synchronize()
        score, rows, status = msadp.decode_device_result(d_result, d_masks, p.seqs)
        want = oracle.align_problem(p)
        assert status == 0 and (score, rows) == (want.score, want.rows)
        assert n < 200  # the first sizes tried were refused: this is the boundary
        return
    pytest.fail("no cube between 101 and 200 fits the static array")


def test_noalloc_rejects_problems_beyond_its_scratch():
    big = inputs.random_problem(1, 3, [400, 400, 400])
    d_res, d_sub = msadp.device_inputs(big)
    d_result, d_masks = msadp.device_outputs(sum(big.lens))
    with pytest.raises(msa.MsaError) as ei:
        msadp.msa_align_noalloc(big.lens, big.alphabet, d_res.data_ptr(), d_sub.data_ptr(), big.gap,
                                d_result.data_ptr(), d_masks.data_ptr(), _stream())
    assert ei.value.code == msa.MSA_ETOOBIG
    assert "scratch" in str(ei.value)
    # fewer cells than the array has bytes, but the working set (traceback bytes,
    # int32 score scratch, flags, order) is larger: refused by the second check
    mid = inputs.random_problem(2, 3, [200, 200, 200])
    d_res, d_sub = msadp.device_inputs(mid)
    d_result, d_masks = msadp.device_outputs(sum(mid.lens))
    with pytest.raises(msa.MsaError) as ei:
        msadp.msa_align_noalloc(mid.lens, mid.alphabet, d_res.data_ptr(), d_sub.data_ptr(), mid.gap,
                                d_result.data_ptr(), d_masks.data_ptr(), _stream())
    assert ei.value.code == msa.MSA_ETOOBIG
    assert "needs" in str(ei.value)
