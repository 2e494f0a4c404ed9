"""Thin ctypes binding of libmsadp (argument marshalling only).

Every step of the alignment runs inside libmsadp's CUDA kernels; this module only
converts Python values to the C-ABI declared in include/msadp.h and back. There
is no fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libmsadp.so")

MSA_OK = 0
MSA_PENDING = 1
MSA_EINVAL = -1
MSA_ETOOBIG = -2
MSA_ENOMEM = -3
MSA_ECUDA = -4
MSA_ETIMEOUT = -5
MSA_EBADHANDLE = -6
MAX_K = 8

_NAMES = {MSA_EINVAL: "MSA_EINVAL", MSA_ETOOBIG: "MSA_ETOOBIG", MSA_ENOMEM: "MSA_ENOMEM",
          MSA_ECUDA: "MSA_ECUDA", MSA_ETIMEOUT: "MSA_ETIMEOUT", MSA_EBADHANDLE: "MSA_EBADHANDLE"}

EXPORTED = ["msa_align", "msa_last_error", "msa_set_stream", "msa_config", "msa_plan_create",
            "msa_plan_execute", "msa_plan_get_info", "msa_plan_destroy", "msa_submit", "msa_poll",
            "msa_cancel", "msa_drain", "msa_wave_sizes", "msa_tile_shape", "msa_version",
            "msa_plan_read_tb", "msa_plan_timings", "msa_align_noalloc", "msa_wait_any",
            "msa_set_tile_edge", "msa_get_tile_edge", "msa_set_line_segment", "msa_get_line_segment",
            "msa_autotune", "msa_near_optimal", "msa_align_pruned", "msa_tile_bounds"]


class PruneStats(ctypes.Structure):
    _fields_ = [("lower_bound", ctypes.c_int64), ("tiles", ctypes.c_int64), ("tiles_skipped", ctypes.c_int64),
                ("cells_skipped", ctypes.c_int64), ("cells", ctypes.c_int64)]


class MsaError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{_NAMES.get(code, code)}: {message}")
        self.code = code


class PlanInfo(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("alphabet_size", ctypes.c_int32), ("cells", ctypes.c_int64),
                ("tb_strides", ctypes.c_int64 * MAX_K), ("tb_bytes", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_int64), ("tile_grid", ctypes.c_int32 * MAX_K),
                ("tile_extent", ctypes.c_int32 * MAX_K), ("tiles", ctypes.c_int64),
                ("waves", ctypes.c_int32), ("fill_kernel", ctypes.c_int32), ("d_tb", ctypes.c_void_p)]


MAX_TUNING_CANDIDATES = 8


class Tuning(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("ncand", ctypes.c_int32),
                ("cand_kernel", ctypes.c_int32 * MAX_TUNING_CANDIDATES),
                ("cand_edge", ctypes.c_int32 * MAX_TUNING_CANDIDATES),
                ("cand_ms", ctypes.c_float * MAX_TUNING_CANDIDATES), ("best", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("seqs", ctypes.POINTER(ctypes.c_char_p)),
                ("lens", ctypes.POINTER(ctypes.c_int32)), ("alphabet", ctypes.c_char_p),
                ("subst", ctypes.POINTER(ctypes.c_int32)), ("gap", ctypes.c_int32)]


DEVICE_RESULT_BYTES = 16  # msa_device_result: score, ncols, status, pad (int32 each)

_lib = None


def library() -> ctypes.CDLL:
    """The loaded libmsadp (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libmsadp is not built ({LIB_PATH} missing); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    i32p = ctypes.POINTER(ctypes.c_int32)
    L.msa_align.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_char_p), i32p, ctypes.c_char_p, i32p,
                            ctypes.c_int32, i32p, ctypes.c_char_p]
    L.msa_near_optimal.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_char_p), i32p, ctypes.c_char_p, i32p,
                                   ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, i32p, i32p]
    L.msa_align_pruned.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_char_p), i32p, ctypes.c_char_p, i32p,
                                   ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, i32p, ctypes.c_char_p,
                                   ctypes.POINTER(PruneStats)]
    L.msa_tile_bounds.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_char_p), i32p, ctypes.c_char_p, i32p,
                                  ctypes.c_int32, i32p, ctypes.c_void_p]
    L.msa_last_error.restype = ctypes.c_char_p
    L.msa_version.restype = ctypes.c_char_p
    L.msa_set_stream.argtypes = [ctypes.c_void_p]
    L.msa_config.argtypes = [ctypes.c_char_p, ctypes.c_int64]
    L.msa_plan_create.argtypes = [ctypes.c_int, i32p, ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]
    L.msa_plan_execute.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.msa_plan_get_info.argtypes = [ctypes.c_void_p, ctypes.POINTER(PlanInfo)]
    L.msa_plan_destroy.argtypes = [ctypes.c_void_p]
    L.msa_plan_read_tb.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
    L.msa_plan_timings.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]
    L.msa_align_noalloc.argtypes = [ctypes.c_int, i32p, ctypes.c_char_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.msa_submit.argtypes = [ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    L.msa_poll.argtypes = [ctypes.c_uint64, i32p, ctypes.c_char_p]
    L.msa_cancel.argtypes = [ctypes.c_uint64]
    L.msa_wait_any.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)]
    L.msa_set_tile_edge.argtypes = [ctypes.c_int, ctypes.c_int32]
    L.msa_get_tile_edge.argtypes = [ctypes.c_int, i32p]
    L.msa_set_line_segment.argtypes = [ctypes.c_int, ctypes.c_int32]
    L.msa_get_line_segment.argtypes = [ctypes.c_int, i32p]
    L.msa_autotune.argtypes = [ctypes.c_int, i32p, ctypes.c_int, ctypes.c_int32, ctypes.POINTER(Tuning)]
    L.msa_wave_sizes.argtypes = [ctypes.c_int, i32p, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32, i32p]
    L.msa_tile_shape.argtypes = [ctypes.c_int, i32p, i32p, i32p]
    _lib = L
    return L


def _check(rc: int) -> int:
    if rc < 0:
        raise MsaError(rc, library().msa_last_error().decode(errors="replace"))
    return rc


def last_error() -> str:
    return library().msa_last_error().decode(errors="replace")


def version() -> str:
    return library().msa_version().decode()


def _i32(values) -> ctypes.Array:
    vals = [int(v) for v in values]
    return (ctypes.c_int32 * max(1, len(vals)))(*vals)


def _table(subst) -> ctypes.Array:
    t = np.ascontiguousarray(np.asarray(subst, dtype=np.int64).reshape(-1))
    return _i32(t.tolist())


def _rows(buf: bytes, k: int, stride: int) -> List[str]:
    out = []
    for i in range(k):
        row = buf[i * stride:(i + 1) * stride]
        out.append(row.split(b"\0", 1)[0].decode())
    return out


def msa_align(seqs: Sequence[str], alphabet: str, subst, gap: int) -> Tuple[int, List[str]]:
    """Optimal SP alignment through the synchronous C-ABI call (host buffers)."""
    L = library()
    k = len(seqs)
    enc = [s.encode() for s in seqs]
    arr = (ctypes.c_char_p * max(1, k))(*enc)
    lens = _i32([len(s) for s in enc])
    stride = sum(len(s) for s in enc) + 1
    out = ctypes.create_string_buffer(k * stride)
    score = ctypes.c_int32(0)
    _check(L.msa_align(k, arr, lens, alphabet.encode(), _table(subst), int(gap), ctypes.byref(score), out))
    return int(score.value), _rows(out.raw, k, stride)


def msa_near_optimal(seqs: Sequence[str], alphabet: str, subst, gap: int, delta: int = 0,
                     max_count: int = 64) -> Tuple[List[Tuple[int, List[int], List[str]]], bool]:
    """Every alignment within ``delta`` of the optimum through the C-ABI call:
    ([(score, masks first column first, rows)], more)."""
    L = library()
    k = len(seqs)
    enc = [s.encode() for s in seqs]
    arr = (ctypes.c_char_p * max(1, k))(*enc)
    lens = _i32([len(s) for s in enc])
    total = sum(len(s) for s in enc)
    masks = np.zeros((max_count, max(1, total)), dtype=np.uint8)
    ncols = np.zeros(max_count, dtype=np.int32)
    scores = np.zeros(max_count, dtype=np.int64)
    count, more = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(L.msa_near_optimal(k, arr, lens, alphabet.encode(), _table(subst), int(gap), int(delta), int(max_count),
                              masks.ctypes.data, ncols.ctypes.data, scores.ctypes.data, ctypes.byref(count),
                              ctypes.byref(more)))
    out = []
    for a in range(count.value):
        ms = [int(m) for m in masks[a, : ncols[a]]]
        rows, pos = [[] for _ in range(k)], [0] * k
        for m in ms:
            for i in range(k):
                if (m >> i) & 1:
                    rows[i].append(seqs[i][pos[i]])
                    pos[i] += 1
                else:
                    rows[i].append("-")
        out.append((int(scores[a]), ms, ["".join(r) for r in rows]))
    return out, bool(more.value)


def msa_align_pruned(seqs: Sequence[str], alphabet: str, subst, gap: int,
                     lower_bound: Optional[int] = None) -> Tuple[int, List[str], dict]:
    """Optimal alignment with tiles below a lower bound left out (C-ABI call):
    (score, rows, stats); lower_bound None lets the device build one."""
    L = library()
    k = len(seqs)
    enc = [s.encode() for s in seqs]
    arr = (ctypes.c_char_p * max(1, k))(*enc)
    lens = _i32([len(s) for s in enc])
    stride = sum(len(s) for s in enc) + 1
    out = ctypes.create_string_buffer(k * stride)
    score = ctypes.c_int32(0)
    st = PruneStats()
    _check(L.msa_align_pruned(k, arr, lens, alphabet.encode(), _table(subst), int(gap),
                              0 if lower_bound is None else 1, int(lower_bound or 0), ctypes.byref(score), out,
                              ctypes.byref(st)))
    stats = {f: int(getattr(st, f)) for f, _ in PruneStats._fields_}
    return int(score.value), _rows(out.raw, k, stride), stats


def msa_tile_bounds(seqs: Sequence[str], alphabet: str, subst, gap: int, extents: Sequence[int]) -> np.ndarray:
    """Every tile's pruning bound for these tile extents, computed on the device."""
    L = library()
    k = len(seqs)
    enc = [s.encode() for s in seqs]
    arr = (ctypes.c_char_p * max(1, k))(*enc)
    lens = _i32([len(s) for s in enc])
    grid = [-(-(len(s) + 1) // e) for s, e in zip(enc, extents)]
    out = np.zeros(int(np.prod(grid)), dtype=np.int64)
    _check(L.msa_tile_bounds(k, arr, lens, alphabet.encode(), _table(subst), int(gap), _i32(list(extents)),
                             out.ctypes.data))
    return out


def msa_config(key: str, value: int) -> None:
    _check(library().msa_config(key.encode(), int(value)))


def msa_set_stream(stream_handle: Optional[int]) -> None:
    _check(library().msa_set_stream(ctypes.c_void_p(stream_handle or 0)))


def msa_wave_sizes(grid: Sequence[int]) -> List[int]:
    L = library()
    k = len(grid)
    total = sum(int(g) for g in grid) + 1
    out = (ctypes.c_int64 * total)()
    nw = ctypes.c_int32(0)
    _check(L.msa_wave_sizes(k, _i32(grid), out, total, ctypes.byref(nw)))
    return [int(out[i]) for i in range(nw.value)]


def msa_tile_shape(lens: Sequence[int]) -> Tuple[List[int], List[int]]:
    L = library()
    k = len(lens)
    ext = (ctypes.c_int32 * MAX_K)()
    grid = (ctypes.c_int32 * MAX_K)()
    _check(L.msa_tile_shape(k, _i32(lens), ext, grid))
    return list(ext[:k]), list(grid[:k])


class Plan:
    """A fixed problem shape with its device workspace (msa_plan_*)."""

    def __init__(self, k: int, lens: Sequence[int], alphabet: str):
        self._lib = library()
        self.k = k
        self.lens = [int(n) for n in lens]
        self.alphabet = alphabet
        h = ctypes.c_void_p()
        _check(self._lib.msa_plan_create(k, _i32(self.lens), alphabet.encode(), ctypes.byref(h)))
        self._h = h

    def execute(self, d_residues: int, d_subst: int, gap: int, d_result: int, d_masks: int,
                stream: Optional[int] = None) -> None:
        """Launch the hot path on device pointers (asynchronous on ``stream``)."""
        _check(self._lib.msa_plan_execute(self._h, ctypes.c_void_p(d_residues), ctypes.c_void_p(d_subst),
                                          int(gap), ctypes.c_void_p(d_result), ctypes.c_void_p(d_masks),
                                          ctypes.c_void_p(stream or 0)))

    def info(self) -> PlanInfo:
        inf = PlanInfo()
        _check(self._lib.msa_plan_get_info(self._h, ctypes.byref(inf)))
        return inf

    def read_tb(self) -> np.ndarray:
        """The traceback tensor of the last execution, unpadded, shape (len_i + 1)."""
        inf = self.info()
        raw = np.empty(int(inf.tb_bytes), dtype=np.uint8)
        _check(self._lib.msa_plan_read_tb(self._h, raw.ctypes.data, int(inf.tb_bytes)))
        shape = tuple(n + 1 for n in self.lens)
        strides = tuple(int(inf.tb_strides[i]) for i in range(self.k))
        return np.lib.stride_tricks.as_strided(raw, shape=shape, strides=strides).copy()

    def timings(self) -> Tuple[float, float, float]:
        """Mean (encode, fill, traceback) milliseconds over the executions timed since the previous call."""
        out = (ctypes.c_float * 3)()
        _check(self._lib.msa_plan_timings(self._h, out))
        return float(out[0]), float(out[1]), float(out[2])

    def close(self) -> None:
        if self._h:
            self._lib.msa_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def msa_align_noalloc(lens: Sequence[int], alphabet: str, d_residues: int, d_subst: int, gap: int,
                      d_result: int, d_masks: int, stream: Optional[int] = None) -> None:
    """One alignment on the library's fixed device scratch (no allocation).

    For callers that must not allocate device memory; pointers are device
    buffers as for Plan.execute. Asynchronous on ``stream``.
    """
    _check(library().msa_align_noalloc(len(lens), _i32(lens), alphabet.encode(), ctypes.c_void_p(d_residues),
                                       ctypes.c_void_p(d_subst), int(gap), ctypes.c_void_p(d_result),
                                       ctypes.c_void_p(d_masks), ctypes.c_void_p(stream or 0)))


def msa_submit(seqs: Sequence[str], alphabet: str, subst, gap: int) -> int:
    L = library()
    k = len(seqs)
    enc = [s.encode() for s in seqs]
    req = Request(k, (ctypes.c_char_p * max(1, k))(*enc), _i32([len(s) for s in enc]), alphabet.encode(),
                  _table(subst), int(gap))
    h = ctypes.c_uint64(0)
    _check(L.msa_submit(ctypes.byref(req), ctypes.byref(h)))
    return int(h.value)


def msa_poll(handle: int, k: int, total_len: int) -> Optional[Tuple[int, List[str]]]:
    """None while pending; (score, rows) when done; raises MsaError on failure."""
    L = library()
    stride = total_len + 1
    out = ctypes.create_string_buffer(k * stride)
    score = ctypes.c_int32(0)
    rc = L.msa_poll(ctypes.c_uint64(handle), ctypes.byref(score), out)
    if rc == MSA_PENDING:
        return None
    _check(rc)
    return int(score.value), _rows(out.raw, k, stride)


def msa_cancel(handle: int) -> None:
    _check(library().msa_cancel(ctypes.c_uint64(handle)))


def msa_drain() -> None:
    _check(library().msa_drain())


def msa_set_tile_edge(k: int, edge: int) -> None:
    _check(library().msa_set_tile_edge(int(k), int(edge)))


def msa_get_tile_edge(k: int) -> int:
    e = ctypes.c_int32(0)
    _check(library().msa_get_tile_edge(int(k), ctypes.byref(e)))
    return int(e.value)


def msa_set_line_segment(k: int, z: int) -> None:
    _check(library().msa_set_line_segment(int(k), int(z)))


def msa_get_line_segment(k: int) -> int:
    z = ctypes.c_int32(0)
    _check(library().msa_get_line_segment(int(k), ctypes.byref(z)))
    return int(z.value)


def msa_autotune(lens: Sequence[int], alphabet_size: int, repeats: int = 3) -> dict:
    """Time the compiled tile shapes (and the k=3 column, k=2 band or k=4..6 line kernel) for this
    shape; the fastest becomes the choice for k. Returns the candidates and the choice."""
    t = Tuning()
    _check(library().msa_autotune(len(lens), _i32(lens), int(alphabet_size), int(repeats), ctypes.byref(t)))
    names = {1: "tiles", 2: "column", 3: "band", 4: "lines", 5: "stream"}
    cands = [{"kernel": names[int(t.cand_kernel[i])], "edge": int(t.cand_edge[i]),
              "ms": float(t.cand_ms[i])} for i in range(t.ncand)]
    return {"k": int(t.k), "lens": list(lens), "candidates": cands, "best": cands[t.best]}


def msa_wait_any(timeout_us: int) -> Optional[int]:
    """Handle of the next finished request (completion order), or None after the timeout."""
    h = ctypes.c_uint64(0)
    rc = library().msa_wait_any(int(timeout_us), ctypes.byref(h))
    if rc == MSA_PENDING:
        return None
    _check(rc)
    return int(h.value)


# ---------------------------------------------------------------------------
# torch helpers: device tensors in, device tensors out (marshalling only).

def device_inputs(problem, device="cuda"):
    """Residues (uint8) and table (int32) of a problem as device tensors."""
    import torch
    res = np.frombuffer("".join(problem.seqs).encode(), dtype=np.uint8).copy()
    d_res = torch.from_numpy(res).to(device) if res.size else torch.zeros(1, dtype=torch.uint8, device=device)
    d_sub = torch.from_numpy(np.ascontiguousarray(problem.subst, dtype=np.int32).reshape(-1)).to(device)
    return d_res, d_sub


def device_outputs(total_len: int, device="cuda"):
    import torch
    d_result = torch.zeros(4, dtype=torch.int32, device=device)
    d_masks = torch.zeros(max(1, total_len), dtype=torch.uint8, device=device)
    return d_result, d_masks


def decode_device_result(d_result, d_masks, seqs: Sequence[str]) -> Tuple[int, List[str], int]:
    """(score, rows, status) from the device result block and reversed masks."""
    r = d_result.cpu().tolist()
    score, ncols, status = r[0], r[1], r[2]
    if status != 0:
        return score, [], status
    masks = d_masks[:ncols].cpu().numpy()[::-1]
    pos = [0] * len(seqs)
    rows = [[] for _ in seqs]
    for m in masks:
        for i, s in enumerate(seqs):
            if (int(m) >> i) & 1:
                rows[i].append(s[pos[i]])
                pos[i] += 1
            else:
                rows[i].append("-")
    return score, ["".join(r) for r in rows], status
