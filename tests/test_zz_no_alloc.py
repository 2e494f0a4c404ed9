"""msa_align_noalloc: the entry point for callers that cannot allocate device
memory (another allocator owns the GPU, latency-critical loops, no recovery from
an allocation failure mid-request). It must give exactly what the allocating
entry point gives, call after call, although every call reuses -- and inherits
the leftovers of -- the same fixed scratch array inside the library.
"""
import pytest

import inputs
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


def test_noalloc_rejects_problems_beyond_its_scratch():
    big = inputs.random_problem(1, 3, [400, 400, 400])
    d_res, d_sub = msadp.device_inputs(big)
    d_result, d_masks = msadp.device_outputs(sum(big.lens))
    with pytest.raises(msa.MsaError) as ei:
        msadp.msa_align_noalloc(big.lens, big.alphabet, d_res.data_ptr(), d_sub.data_ptr(), big.gap,
                                d_result.data_ptr(), d_masks.data_ptr(), _stream())
    assert ei.value.code == msa.MSA_ETOOBIG
    assert "scratch" in str(ei.value)
