"""The paper's own scoring (+1 match, 0 mismatch, -1 residue/gap, 0 gap/gap;
section 5.2) at the largest k the library takes (7, 8), and a mix of k served
together: bit-exact against the oracle, full traceback tensor included."""
import numpy as np
import pytest

import inputs
import oracle
import paper_2311_17530_gb300 as msa
from paper_2311_17530_gb300 import msadp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("k,lens", [(7, [6, 5, 7, 6, 5, 6, 7]), (8, [4, 3, 4, 4, 3, 4, 3, 4]),
                                    (5, [13, 11, 12, 14, 10])])
def test_paper_scheme_high_k_full_tensor(k, lens):
    p = inputs.paper_problem(4000 + k, k, lens)
    want = oracle.align(p.seqs, p.alphabet, p.subst, p.gap, want_tb=True)
    plan = msa.Plan(k, p.lens, p.alphabet)
    try:
        d_res, d_sub = msadp.device_inputs(p)
        d_result, d_masks = msadp.device_outputs(sum(p.lens))
        plan.execute(d_res.data_ptr(), d_sub.data_ptr(), p.gap, d_result.data_ptr(), d_masks.data_ptr(),
                     torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        score, rows, status = msadp.decode_device_result(d_result, d_masks, p.seqs)
        assert status == 0
        assert (score, rows) == (want.score, want.rows)
        tb = plan.read_tb()
        np.testing.assert_array_equal(tb, np.asarray(want.tb).reshape(tb.shape))
    finally:
        plan.close()


def test_paper_scheme_mix_of_k_served():
    probs = [inputs.paper_problem(4100 + i, k, [int(x) for x in np.random.default_rng(i).integers(1, n, size=k)])
             for i, (k, n) in enumerate([(2, 90), (3, 25), (4, 9), (5, 7), (6, 5), (7, 4), (8, 3)] * 2)]
    handles = [msa.msa_submit(p.seqs, p.alphabet, p.subst, p.gap) for p in probs]
    msa.msa_drain()
    for h, p in zip(handles, probs):
        want = oracle.align(p.seqs, p.alphabet, p.subst, p.gap)
        assert msa.msa_poll(h, p.k, sum(p.lens)) == (want.score, want.rows), p.name
