"""Write the stored expected values for the full-size workloads.

Calls only ``oracle/`` (plain full-tensor DP) on the seeded inputs of ``inputs/``;
nothing here comes from the CUDA path. For each workload it stores the optimal
SP score, the alignment as per-column move masks, and a seeded sample of traceback
bytes of the full tensor (row-major linear index over shape len_i + 1).

usage: python tests/golden/make_golden.py [workload ...]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import inputs  # noqa: E402
import oracle  # noqa: E402

N_SAMPLES = 4096


def sample_indices(shape, seed):
    n = int(np.prod(shape, dtype=np.int64))
    rng = np.random.default_rng(seed)
    idx = set(int(i) for i in rng.integers(0, n, size=N_SAMPLES))
    # the origin, the far corner and the last cell of every axis-aligned edge
    idx.add(0)
    idx.add(n - 1)
    strides = np.cumprod((1,) + tuple(shape[::-1]))[:-1][::-1]
    for i, s in enumerate(shape):
        idx.add(int((s - 1) * strides[i]))
    return sorted(idx)


def make(name):
    p = inputs.WORKLOADS[name]()
    t0 = time.time()
    r = oracle.align_problem(p, want_tb=True)
    dt = time.time() - t0
    shape = r.tb.shape
    flat = r.tb.reshape(-1)
    idx = sample_indices(shape, 12345)
    out = {
        "workload": name,
        "inputs": f"inputs.WORKLOADS['{name}']()",
        "made_by": "tests/golden/make_golden.py (oracle only)",
        "k": p.k,
        "lens": p.lens,
        "cells": p.cells,
        "score": r.score,
        "ncols": len(r.masks),
        "masks_hex": "".join(f"{m:02x}" for m in r.masks),
        "tb_samples": [[i, int(flat[i])] for i in idx],
        "oracle_seconds": round(dt, 2),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(f"{name}: score={r.score} ncols={len(r.masks)} oracle {dt:.1f}s -> {path}", flush=True)


if __name__ == "__main__":
    names = sys.argv[1:] or list(inputs.WORKLOADS)
    for n in names:
        make(n)
