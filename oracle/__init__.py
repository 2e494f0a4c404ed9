"""CPU oracle for optimal sum-of-pairs MSA by dynamic programming.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. It shares no code with the CUDA path (``libmsadp``).

``msa_oracle.c`` is the plain full-tensor definition of the method (section 2,
Eq. 1 generalised to 2^k-1 neighbours; section 4 per-cell scoring; section 5.2
sum-of-pairs columns with gap-gap 0; section 2 traceback). This wrapper only
marshals arguments and expands the returned move masks into gapped rows.

``oracle_pair_tables`` / ``oracle_msa_pruned`` (``pair_tables``, ``align_pruned``)
are the oracle of exact search-space pruning (section 6 proposes narrowing the
search to the partitions where an optimal alignment can lie) by the
Carrillo-Lipman bound: pairwise forward and backward tables and the same DP
restricted to the cells whose bound reaches a lower bound on the optimum;
``oracle_tile_bounds`` / ``oracle_msa_excluding`` (``tile_bounds``,
``align_excluding``) the per-tile bound a fill that skips whole tiles uses and
the DP with any set of cells left out; all pinned by
``tests/test_oracle_pruning.py``. ``oracle_msa_near_optimal``
(``align_near_optimal``) enumerates every alignment within a threshold of the
optimum (section 6: further optimal or near-optimal solutions), pinned by
``tests/test_oracle_near_optimal.py``.

``oracle_msa`` is pinned by ``tests/test_oracle_pins.py`` against brute
force enumeration, textbook Needleman-Wunsch, a closed form, permutation
invariance and the alignment invariants. The paper's own 6-sequence example
(section 5.2, optimal SP score -5) is parity unpinned: its sequences are not
published.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msa_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libmsa_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, single thread, portable flags)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


def load_library(path: str):
    """ctypes handle on a compiled oracle (the default one, or a planted mutant in tests)."""
    lib = ctypes.CDLL(path)
    lib.oracle_msa.restype = ctypes.c_int
    lib.oracle_msa.argtypes = [
        ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p, ctypes.c_int,
        ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]
    lib.oracle_pair_tables.restype = ctypes.c_int
    lib.oracle_pair_tables.argtypes = [
        ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int,
        ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    lib.oracle_msa_pruned.restype = ctypes.c_int
    lib.oracle_msa_pruned.argtypes = [
        ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p, ctypes.c_int,
        ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
        ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)]
    lib.oracle_tile_bounds.restype = ctypes.c_int
    lib.oracle_tile_bounds.argtypes = [
        ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p, ctypes.c_int,
        ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p]
    lib.oracle_msa_excluding.restype = ctypes.c_int
    lib.oracle_msa_excluding.argtypes = [
        ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p, ctypes.c_int,
        ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
        ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]
    lib.oracle_msa_near_optimal.restype = ctypes.c_int
    lib.oracle_msa_near_optimal.argtypes = [
        ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p, ctypes.c_int,
        ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
        ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = load_library(build())
    return _lib


@dataclasses.dataclass
class OracleResult:
    score: int
    masks: List[int]          # move mask per column, first column first
    rows: List[str]           # k gapped rows
    tb: Optional[np.ndarray]  # uint8 tensor, shape (len_i + 1), if requested
    H: Optional[np.ndarray]   # int64 tensor, if requested


def encode(seqs: Sequence[str], alphabet: str) -> np.ndarray:
    index = {c: i for i, c in enumerate(alphabet)}
    return np.array([index[c] for s in seqs for c in s], dtype=np.uint8)


def expand(seqs: Sequence[str], masks: Sequence[int], gap_char: str = "-") -> List[str]:
    """Gapped rows from column masks: row i takes its next residue when bit i is set."""
    pos = [0] * len(seqs)
    rows = [[] for _ in seqs]
    for m in masks:
        for i, s in enumerate(seqs):
            if (m >> i) & 1:
                rows[i].append(s[pos[i]])
                pos[i] += 1
            else:
                rows[i].append(gap_char)
    return ["".join(r) for r in rows]


def align_codes(lens: Sequence[int], codes: np.ndarray, A: int, subst: np.ndarray, gap: int,
                want_tb: bool = False, want_H: bool = False, lib=None):
    lib = lib or _load()
    k = len(lens)
    lens_arr = (ctypes.c_int32 * k)(*[int(n) for n in lens])
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    sub = np.ascontiguousarray(np.asarray(subst, dtype=np.int32).reshape(-1))
    shape = tuple(int(n) + 1 for n in lens)
    ncells = int(np.prod(shape, dtype=np.int64))
    tb = np.empty(shape, dtype=np.uint8) if want_tb else None
    H = np.empty(shape, dtype=np.int64) if want_H else None
    masks = np.zeros(max(1, int(sum(lens))), dtype=np.uint8)
    score = ctypes.c_int64(0)
    ncols = ctypes.c_int32(0)
    rc = lib.oracle_msa(
        k, lens_arr, codes.ctypes.data if codes.size else None, int(A),
        sub.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(gap), ctypes.byref(score),
        tb.ctypes.data if tb is not None else None, H.ctypes.data if H is not None else None,
        masks.ctypes.data, ctypes.byref(ncols))
    if rc != 0:
        raise ValueError(f"oracle_msa failed with {rc} (cells={ncells})")
    return int(score.value), [int(m) for m in masks[: ncols.value]], tb, H


def align(seqs: Sequence[str], alphabet: str, subst, gap: int, want_tb: bool = False,
          want_H: bool = False, lib=None) -> OracleResult:
    """Optimal global SP alignment of ``seqs`` (lowest move mask wins ties)."""
    codes = encode(seqs, alphabet)
    score, masks, tb, H = align_codes([len(s) for s in seqs], codes, len(alphabet),
                                      np.asarray(subst), gap, want_tb, want_H, lib)
    return OracleResult(score, masks, expand(seqs, masks), tb, H)


def align_problem(p, want_tb: bool = False, want_H: bool = False) -> OracleResult:
    return align(p.seqs, p.alphabet, p.subst, p.gap, want_tb, want_H)


# ---------------------------------------------------------------------------
# Exact search-space pruning (Carrillo-Lipman bound; the paper's future work,
# section 6): pairwise forward/backward tables and the DP over the cells whose
# bound reaches a lower bound on the optimum.

def pair_tables(a: str, b: str, alphabet: str, subst, gap: int, lib=None):
    """(fwd, bwd): int64 arrays of shape (len(a)+1, len(b)+1); fwd[p, q] is the
    optimal global score of a[:p] against b[:q], bwd[p, q] that of a[p:] against b[q:]."""
    lib = lib or _load()
    ca, cb = encode([a], alphabet), encode([b], alphabet)
    sub = np.ascontiguousarray(np.asarray(subst, dtype=np.int32).reshape(-1))
    fwd = np.empty((len(a) + 1, len(b) + 1), dtype=np.int64)
    bwd = np.empty_like(fwd)
    rc = lib.oracle_pair_tables(ca.ctypes.data if ca.size else None, len(a), cb.ctypes.data if cb.size else None,
                                len(b), len(alphabet), sub.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(gap),
                                fwd.ctypes.data, bwd.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle_pair_tables failed with {rc}")
    return fwd, bwd


class BoundAboveOptimum(ValueError):
    """The lower bound given to align_pruned exceeds the optimal score."""


def align_pruned(seqs: Sequence[str], alphabet: str, subst, gap: int, lower_bound: int, lib=None):
    """(OracleResult, cells left out): the DP restricted to cells whose
    Carrillo-Lipman bound reaches ``lower_bound``. Raises BoundAboveOptimum when
    no kept path reaches ``lower_bound``."""
    lib = lib or _load()
    k = len(seqs)
    lens = [len(s) for s in seqs]
    lens_arr = (ctypes.c_int32 * k)(*lens)
    codes = encode(seqs, alphabet)
    sub = np.ascontiguousarray(np.asarray(subst, dtype=np.int32).reshape(-1))
    masks = np.zeros(max(1, sum(lens)), dtype=np.uint8)
    score, ncols, excluded = ctypes.c_int64(0), ctypes.c_int32(0), ctypes.c_int64(0)
    rc = lib.oracle_msa_pruned(k, lens_arr, codes.ctypes.data if codes.size else None, len(alphabet),
                               sub.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(gap), int(lower_bound),
                               ctypes.byref(score), masks.ctypes.data, ctypes.byref(ncols), ctypes.byref(excluded))
    if rc == -3:
        raise BoundAboveOptimum(f"no kept path reaches {lower_bound}")
    if rc != 0:
        raise ValueError(f"oracle_msa_pruned failed with {rc}")
    ms = [int(m) for m in masks[: ncols.value]]
    return OracleResult(int(score.value), ms, expand(seqs, ms), None, None), int(excluded.value)



def tile_bounds(seqs: Sequence[str], alphabet: str, subst, gap: int, extents: Sequence[int], lib=None) -> np.ndarray:
    """Per-tile pruning bound (int64 array over the tile grid, tiles of ``extents``):
    the sum over pairs of the largest pairwise forward + backward score in the tile's
    rectangle, never below the largest cell bound inside the tile."""
    lib = lib or _load()
    k = len(seqs)
    lens = [len(s) for s in seqs]
    grid = tuple(-(-(n + 1) // int(e)) for n, e in zip(lens, extents))
    out = np.empty(grid, dtype=np.int64)
    codes = encode(seqs, alphabet)
    sub = np.ascontiguousarray(np.asarray(subst, dtype=np.int32).reshape(-1))
    rc = lib.oracle_tile_bounds(k, (ctypes.c_int32 * k)(*lens), codes.ctypes.data if codes.size else None,
                                len(alphabet), sub.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(gap),
                                (ctypes.c_int32 * k)(*[int(e) for e in extents]), out.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle_tile_bounds failed with {rc}")
    return out


def align_excluding(seqs: Sequence[str], alphabet: str, subst, gap: int, excluded: np.ndarray, lib=None):
    """The DP with the cells flagged in ``excluded`` (bool array of shape len_i + 1)
    left out; raises BoundAboveOptimum when no kept path reaches the corner."""
    lib = lib or _load()
    k = len(seqs)
    lens = [len(s) for s in seqs]
    ex = np.ascontiguousarray(np.asarray(excluded, dtype=np.uint8))
    assert ex.shape == tuple(n + 1 for n in lens)
    codes = encode(seqs, alphabet)
    sub = np.ascontiguousarray(np.asarray(subst, dtype=np.int32).reshape(-1))
    masks = np.zeros(max(1, sum(lens)), dtype=np.uint8)
    score, ncols = ctypes.c_int64(0), ctypes.c_int32(0)
    rc = lib.oracle_msa_excluding(k, (ctypes.c_int32 * k)(*lens), codes.ctypes.data if codes.size else None,
                                  len(alphabet), sub.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(gap),
                                  ex.ctypes.data, ctypes.byref(score), masks.ctypes.data, ctypes.byref(ncols))
    if rc == -3:
        raise BoundAboveOptimum("no kept path reaches the corner")
    if rc != 0:
        raise ValueError(f"oracle_msa_excluding failed with {rc}")
    ms = [int(m) for m in masks[: ncols.value]]
    return OracleResult(int(score.value), ms, expand(seqs, ms), None, None)


# ---------------------------------------------------------------------------
# Optimal and near-optimal alignments (section 6: forking at equally ranked
# paths, or within a user threshold).

def align_near_optimal(seqs: Sequence[str], alphabet: str, subst, gap: int, delta: int = 0,
                       max_count: int = 64, lib=None):
    """(alignments, more): every alignment scoring at least OPT - ``delta``, in
    increasing lexicographic order of the reversed column sequence (for
    ``delta`` = 0 the first is ``align``'s), at most ``max_count`` of them; ``more`` is True when the
    enumeration stopped at ``max_count``."""
    lib = lib or _load()
    k = len(seqs)
    lens = [len(s) for s in seqs]
    total = sum(lens)
    lens_arr = (ctypes.c_int32 * k)(*lens)
    codes = encode(seqs, alphabet)
    sub = np.ascontiguousarray(np.asarray(subst, dtype=np.int32).reshape(-1))
    masks = np.zeros((max_count, max(1, total)), dtype=np.uint8)
    ncols = np.zeros(max_count, dtype=np.int32)
    scores = np.zeros(max_count, dtype=np.int64)
    count, more = ctypes.c_int32(0), ctypes.c_int32(0)
    rc = lib.oracle_msa_near_optimal(k, lens_arr, codes.ctypes.data if codes.size else None, len(alphabet),
                                     sub.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(gap), int(delta),
                                     int(max_count), masks.ctypes.data, ncols.ctypes.data, scores.ctypes.data,
                                     ctypes.byref(count), ctypes.byref(more))
    if rc != 0:
        raise ValueError(f"oracle_msa_near_optimal failed with {rc}")
    out = []
    for a in range(count.value):
        ms = [int(m) for m in masks[a, : ncols[a]]]
        out.append(OracleResult(int(scores[a]), ms, expand(seqs, ms), None, None))
    return out, bool(more.value)
