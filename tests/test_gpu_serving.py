"""Serving (continuous batching) through the C-ABI: every result must be the one
the request gets alone -- from the CPU oracle and from msa_align -- whatever it
was batched with, in every serving mode (batched with or without CUDA graphs,
one at a time)."""
import threading

import numpy as np
import pytest

import inputs
import oracle
import paper_2311_17530_gb300 as msa
from paper_2311_17530_gb300 import msadp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def mix(n, seed, scale=1):
    """Requests of mixed k, alphabet and shape (sizes the oracle finishes quickly)."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed + i)
        k = (2, 3, 4)[i % 3]
        hi = {2: 120, 3: 28, 4: 9}[k] * scale
        lens = [int(x) for x in rng.integers(0, hi + 1, size=k)]
        alphabet = inputs.DNA if i % 2 else inputs.PROTEIN
        out.append(inputs.random_problem(seed + i, k, lens, alphabet=alphabet, related=bool(i % 4)))
    return out


def serve(problems):
    handles = [msa.msa_submit(p.seqs, p.alphabet, p.subst, p.gap) for p in problems]
    msa.msa_drain()
    return [msa.msa_poll(h, p.k, sum(p.lens)) for h, p in zip(handles, problems)]


@pytest.fixture(autouse=True)
def default_settings():
    yield
    for key, value in (("batching", 1), ("use_graphs", 1), ("max_batch", 64)):
        msa.msa_config(key, value)


def test_served_results_equal_oracle_and_alone():
    probs = mix(36, 700)
    got = serve(probs)
    for p, res in zip(probs, got):
        want = oracle.align(p.seqs, p.alphabet, p.subst, p.gap)
        assert res == (want.score, want.rows), p.name
        assert msa.msa_align(p.seqs, p.alphabet, p.subst, p.gap) == res, p.name


@pytest.mark.parametrize("batching,graphs,max_batch", [(1, 1, 64), (1, 0, 64), (1, 1, 5), (0, 0, 1)])
def test_serving_modes_agree(batching, graphs, max_batch):
    msa.msa_config("batching", batching)
    msa.msa_config("use_graphs", graphs)
    msa.msa_config("max_batch", max_batch)
    # larger shapes: k=3 requests take the column kernel, k=2 several tile waves
    probs = mix(12, 900, scale=4) + [inputs.random_problem(950, 3, [100, 90, 80], alphabet=inputs.PROTEIN,
                                                           related=True)]
    got = serve(probs)
    for p, res in zip(probs, got):
        assert msa.msa_align(p.seqs, p.alphabet, p.subst, p.gap) == res, p.name
    small = [p for p in probs if p.cells <= 3_000_000]
    for p in small:
        want = oracle.align(p.seqs, p.alphabet, p.subst, p.gap)
        assert got[probs.index(p)] == (want.score, want.rows), p.name


def test_wait_any_reports_each_finished_request_once_and_cancel_releases():
    probs = mix(10, 1200)
    handles = [msa.msa_submit(p.seqs, p.alphabet, p.subst, p.gap) for p in probs]
    cancelled = {handles[3], handles[7]}
    for h in cancelled:
        msa.msa_cancel(h)
    seen = []
    while len(seen) < len(handles) - len(cancelled):
        h = msa.msa_wait_any(2_000_000)
        assert h is not None, "a request did not finish within 2 s"
        seen.append(h)
    assert len(set(seen)) == len(seen) and set(seen) == set(handles) - cancelled
    assert msa.msa_wait_any(1000) is None
    for h, p in zip(handles, probs):
        if h in cancelled:
            with pytest.raises(msa.MsaError) as ei:
                msa.msa_poll(h, p.k, sum(p.lens))
            assert ei.value.code == msa.MSA_EBADHANDLE
        else:
            want = oracle.align(p.seqs, p.alphabet, p.subst, p.gap)
            assert msa.msa_poll(h, p.k, sum(p.lens)) == (want.score, want.rows)
            with pytest.raises(msa.MsaError):  # the first completed poll released the handle
                msa.msa_poll(h, p.k, sum(p.lens))


def test_errors_stay_with_their_request():
    probs = mix(6, 1300)
    bad = inputs.random_problem(1310, 3, [10, 12, 9])
    huge = inputs.Problem(bad.name, bad.seqs, bad.alphabet, bad.subst * 10**7, bad.gap)
    handles = [msa.msa_submit(p.seqs, p.alphabet, p.subst, p.gap) for p in probs[:3]]
    h_huge = msa.msa_submit(huge.seqs, huge.alphabet, huge.subst, huge.gap)
    handles += [msa.msa_submit(p.seqs, p.alphabet, p.subst, p.gap) for p in probs[3:]]
    msa.msa_drain()
    with pytest.raises(msa.MsaError) as ei:
        msa.msa_poll(h_huge, huge.k, sum(huge.lens))
    assert ei.value.code == msa.MSA_ETOOBIG
    for h, p in zip(handles, probs):
        want = oracle.align(p.seqs, p.alphabet, p.subst, p.gap)
        assert msa.msa_poll(h, p.k, sum(p.lens)) == (want.score, want.rows)
    # host checks refuse at submit: a residue outside the alphabet, a request over the budget
    with pytest.raises(msa.MsaError) as ei:
        msa.msa_submit(["ACGX", "ACG"], inputs.DNA, inputs.dna_table(), -8)
    assert ei.value.code == msa.MSA_EINVAL
    with pytest.raises(msa.MsaError) as ei:
        msa.msa_submit(["A" * 3000] * 3, inputs.DNA, inputs.dna_table(), -8)
    assert ei.value.code == msa.MSA_ETOOBIG


def test_concurrent_submitters():
    probs = mix(24, 1400)
    results = [None] * len(probs)

    def worker(idx):
        for i in idx:
            p = probs[i]
            h = msa.msa_submit(p.seqs, p.alphabet, p.subst, p.gap)
            while True:
                r = msa.msa_poll(h, p.k, sum(p.lens))
                if r is not None:
                    results[i] = r
                    break

    threads = [threading.Thread(target=worker, args=(range(t, len(probs), 4),)) for t in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for p, res in zip(probs, results):
        want = oracle.align(p.seqs, p.alphabet, p.subst, p.gap)
        assert res == (want.score, want.rows), p.name


def test_served_large_k_batches_equal_oracle():
    # k = 5 and 6 requests of uneven shapes in one stream: the default tile edges for
    # these k fill each tile with two warps, batched with other problems of the group
    probs = []
    for i in range(8):
        rng = np.random.default_rng(1500 + i)
        k = 5 if i % 2 else 6
        hi = {5: 10, 6: 7}[k]
        lens = [int(x) for x in rng.integers(1, hi + 1, size=k)]
        probs.append(inputs.random_problem(1500 + i, k, lens, alphabet=inputs.DNA if i % 3 else inputs.PROTEIN,
                                           related=bool(i % 2)))
    got = serve(probs)
    for p, res in zip(probs, got):
        want = oracle.align(p.seqs, p.alphabet, p.subst, p.gap)
        assert res == (want.score, want.rows), p.name
