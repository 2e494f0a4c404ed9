"""The library's limits, bit-exact against the oracle: the column kernel's
largest last axis (4096 positions) and largest alphabet (24 letters; 25 falls
back to the generic kernel), the largest alphabet the ABI takes (32 letters,
through the generic tile kernel and both line kernels),
and a long two-sequence problem over several tile waves."""
import numpy as np
import pytest

import inputs
import oracle
import paper_2311_17530_gb300 as msa
from paper_2311_17530_gb300 import msadp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LETTERS = "ABCDEFGHIJKLMNOPQRSTUVWXYZabcdef"


def run_full(p, want_kernel=None):
    want = oracle.align(p.seqs, p.alphabet, p.subst, p.gap, want_tb=True)
    plan = msa.Plan(p.k, p.lens, p.alphabet)
    try:
        if want_kernel is not None:
            assert plan.info().fill_kernel == want_kernel
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


def alphabet_problem(seed, k, lens, size):
    rng = np.random.default_rng(seed)
    table = inputs.protein_table(rng, size)
    return inputs.random_problem(seed, k, lens, alphabet=LETTERS[:size], table=table, gap=-6, related=True)


def test_column_kernel_longest_last_axis():
    p = inputs.random_problem(5000, 3, [20, 40, 4095], alphabet=inputs.PROTEIN, related=True)
    run_full(p, want_kernel=2)


@pytest.mark.parametrize("size,kernel", [(24, 2), (25, 1)])
def test_column_kernel_largest_alphabet(size, kernel):
    run_full(alphabet_problem(5100 + size, 3, [45, 37, 52], size), want_kernel=kernel)


@pytest.mark.parametrize("kernel,k,lens", [(1, 4, [13, 11, 14, 40]), (4, 4, [13, 11, 14, 40]),
                                           (5, 4, [13, 11, 14, 40]), (5, 6, [5, 4, 3, 4, 3, 24])])
def test_largest_alphabet_generic_and_line_kernels(kernel, k, lens):
    """32 letters through the generic tile kernel (1), the line kernel (4) and the
    streamed line kernel (5)."""
    msa.msa_config("fill_kernel", kernel)
    try:
        run_full(alphabet_problem(5200 if k == 4 else 5200 + k, k, lens, 32), want_kernel=kernel)
    finally:
        msa.msa_config("fill_kernel", 0)


def test_long_pair():
    run_full(inputs.random_problem(5300, 2, [3000, 2500], related=True))
