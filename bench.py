#!/usr/bin/env python
"""Benchmark: optimal DP-MSA fill + traceback on one GB300 (libmsadp).

One step = the whole hot path over one problem: encode residues + scale the pair
table, fill the k-dimensional tensor, trace back (hot-path steps a1-a5). The
default workload is k=3 protein 700/760/800 (427,302,261 cells). Its working set
(0.65 GB of traceback bytes and faces written per step) is far larger than the
129 MB L2, so no L2 flush is needed between steps; a workload whose traceback tensor fits in L2
(the k=2 pair, the 128^3 case) is timed one step at a time, with a write of
twice the L2 size before each step, outside the timed events.

value  : cells/s with inputs resident in HBM (plan execution on device buffers),
         CUDA events on the launching stream around exactly --steps steps.
e2e    : cells/s through msa_align() with host buffers (H2D of residues + table,
         D2H of the result block + masks inside the timed region).
roofline: the fill kernel against the integer-ALU bound: 2 (2^k - 1) integer
         operations per cell (a max and an add per predecessor) over 152 SMs x
         128 INT32 lanes x the SM clock.

--impl reference times the CPU oracle (plain full-tensor DP, one core) on a
bounded prefix sample of the same workload.

Multi-GPU: the problem does not shard; N ranks run independent replicas.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import inputs  # noqa: E402

METRIC = "DP cells/s"
UNIT = "cells/s"
SMS_GB300 = 152
# One 32-bit integer operation per issue slot: 4 SM sub-partitions x 32 lanes per clock.
# Integer adds issue at this rate; the max family (IMNMX, the three-input VIMNMX3 and the
# fused add-max VIADDMNMX) at half of it, each fused form doing two operations
# (tests/alu_peak_probe.cu under ncu).
INT32_LANES_PER_SM = 128
PEAK_BASIS = ("{sms} SMs x 4 issue slots x 32 lanes x {mhz:.0f} MHz: one 32-bit integer op per issue slot "
              "(adds full rate, maxes half rate but fused pairs count two)")
# the benchmark's workloads besides the headline one
PER_WORKLOADS = ("pr1", "k2_protein", "k3_protein", "k4_dna", "k6_protein")
SM_MAX_MHZ_FALLBACK = 2070.0


def alg_ops_per_cell(k: int) -> int:
    """Relaxations of one cell: 2^k - 1 predecessors, each an add and a max."""
    return 2 * ((1 << k) - 1)


def sm_max_mhz() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f).get("sm_max_mhz", SM_MAX_MHZ_FALLBACK))
    except Exception:
        return SM_MAX_MHZ_FALLBACK


def alu_peak_tiops(sms: int) -> float:
    return sms * INT32_LANES_PER_SM * sm_max_mhz() * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, v in zip(self.REASONS, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
            os.unlink(self.path)
        except Exception:
            return None
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def sample_prefix(p, target_cells: float):
    """Prefixes of the workload's sequences, all lengths scaled by one factor."""
    f = min(1.0, (target_cells / p.cells) ** (1.0 / p.k))
    lens = [max(1, int(round(n * f))) for n in p.lens]
    return p.prefix(lens)


def time_oracle(p, target_cells: float):
    import oracle
    q = sample_prefix(p, target_cells)
    t0 = time.perf_counter()
    oracle.align_problem(q)
    dt = time.perf_counter() - t0
    return q, dt


WIDE_Z = 25  # the longest last axis the streamed kernel's whole-column form (k = 6) holds

# Source files each fill kernel is compiled from (its own file and the headers it includes).
KERNEL_SOURCES = {
    "fill_col3": ["csrc/fill_col3.cu", "csrc/api_internal.h", "csrc/plan.h", "csrc/internal.h",
                  "csrc/device_common.cuh", "../include/msadp.h"],
    "fill_tiles": ["csrc/fill_tiles.cuh"] + [f"csrc/fill_tiles_k{k}.cu" for k in range(2, 9)] +
                  ["csrc/internal.h", "csrc/device_common.cuh", "../include/msadp.h"],
    "fill_band2": ["csrc/fill_band2.cu", "csrc/api_internal.h", "csrc/plan.h", "csrc/internal.h",
                   "csrc/device_common.cuh", "../include/msadp.h"],
    "fill_lines": ["csrc/fill_lines.cuh"] + [f"csrc/fill_lines_k{k}.cu" for k in range(4, 7)] +
                  ["csrc/internal.h", "csrc/device_common.cuh", "../include/msadp.h"],
    "fill_lines_wide": ["csrc/fill_lines_wide.cuh", "csrc/fill_stream_k6.cu", "csrc/internal.h",
                        "csrc/device_common.cuh", "../include/msadp.h"],
    "fill_lines_stream": ["csrc/fill_lines_stream.cuh", "csrc/fill_lines.cuh"] +
                         [f"csrc/fill_stream_k{k}.cu" for k in range(4, 7)] +
                         ["csrc/internal.h", "csrc/device_common.cuh", "../include/msadp.h"],
}


def kernel_source_digest(kernel: str) -> str:
    """Digest of the code (comments and blank lines removed) a fill kernel is built from."""
    import re
    h = hashlib.sha256()
    pkg = os.path.join(ROOT, "paper_2311_17530_gb300")
    for name in KERNEL_SOURCES[kernel]:
        src = open(os.path.normpath(os.path.join(pkg, name)), encoding="utf-8").read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        code = "\n".join(line.rstrip() for line in src.splitlines() if line.strip())
        h.update(code.encode())
    return h.hexdigest()[:16]


def measured_traffic(workload: str, kernel: str):
    """DRAM bytes per launch from a committed ncu summary, if taken on this kernel's source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(f"{kernel}:{workload}")
    except Exception:
        return None
    if not rec or rec.get("source_digest") != kernel_source_digest(kernel):
        return None
    return rec.get("dram_bytes_per_launch")


def serving_requests(n: int):
    """The seeded serving stream as ready-to-submit C-ABI request structs."""
    import ctypes

    from paper_2311_17530_gb300 import msadp
    out = []
    for i in range(n):
        p = inputs.serving_request(i)
        enc = [s.encode() for s in p.seqs]
        keep = (enc, (ctypes.c_char_p * p.k)(*enc), msadp._i32(p.lens), p.alphabet.encode(), msadp._table(p.subst))
        req = msadp.Request(p.k, keep[1], keep[2], keep[3], keep[4], int(p.gap))
        out.append((p, req, keep))
    return out


def serve_run(reqs, arrivals=None, collect=False, timeout_s=120.0):
    """Submit every request (at its Poisson arrival time, or all at once) through
    msa_submit; a second thread takes completions from msa_wait_any and releases
    them with msa_poll. Latency = completion seen - msa_submit returned."""
    import ctypes
    import threading

    from paper_2311_17530_gb300 import msadp
    L = msadp.library()
    n = len(reqs)
    submit_t = [0.0] * n
    done_t = [0.0] * n
    index = {}
    results = [None] * n if collect else None
    lock = threading.Lock()
    failure = []

    def completer():
        got = 0
        deadline = time.perf_counter() + timeout_s
        h = ctypes.c_uint64(0)
        score = ctypes.c_int32(0)
        while got < n:
            rc = L.msa_wait_any(100000, ctypes.byref(h))
            t = time.perf_counter()
            if rc == msadp.MSA_PENDING:
                if t > deadline:
                    failure.append("serving did not finish in time")
                    return
                continue
            with lock:
                i = index[h.value]
            done_t[i] = t
            p = reqs[i][0]
            stride = sum(p.lens) + 1
            buf = ctypes.create_string_buffer(p.k * stride)
            rc = L.msa_poll(h, ctypes.byref(score), buf)
            if rc != 0:
                failure.append(f"request {i}: status {rc} {msadp.last_error()}")
            elif collect:
                results[i] = (score.value, buf.raw)
            got += 1

    th = threading.Thread(target=completer)
    th.start()
    t0 = time.perf_counter()
    h = ctypes.c_uint64(0)
    for i, (p, req, _) in enumerate(reqs):
        if arrivals is not None:
            target = t0 + float(arrivals[i])
            while True:
                now = time.perf_counter()
                if now >= target:
                    break
                if target - now > 0.0006:
                    time.sleep(target - now - 0.0004)
        with lock:
            rc = L.msa_submit(ctypes.byref(req), ctypes.byref(h))
            submit_t[i] = time.perf_counter()
            if rc != 0:
                raise SystemExit(f"msa_submit: {msadp.last_error()}")
            index[h.value] = i
    th.join()
    if failure:
        raise SystemExit(failure[0])
    lat = np.array([done_t[i] - submit_t[i] for i in range(n)]) * 1e3
    span = max(done_t) - min(submit_t)
    cells = sum(r[0].cells for r in reqs)
    return {"alignments_per_s": n / span, "cells_per_s": cells / span, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean())}, results


def run_serving(n: int):
    """Served alignments/s and p50/p99 latency: plain one-at-a-time launches
    against continuous batching with graph-captured persistent launches, closed
    loop and under Poisson arrivals at multiples of the plain saturation rate."""
    from paper_2311_17530_gb300 import msadp
    reqs = serving_requests(n)

    def mode(batched):
        msadp.msa_config("batching", 1 if batched else 0)
        msadp.msa_config("use_graphs", 1)

    # tile shapes per k tuned on the stream's median shapes (protein alphabet)
    tuned = {k: msadp.msa_autotune(lens, 20, repeats=2)["best"]
             for k, lens in ((2, [1100, 1100]), (3, [170, 170, 170]), (4, [50, 50, 50, 50]))}
    mode(True)
    serve_run(reqs[:128])  # warm-up: arena, kernels, graphs
    mode(False)
    serve_run(reqs[:16])
    plain, res_plain = serve_run(reqs, collect=True)
    mode(True)
    batched, res_batched = serve_run(reqs, collect=True)
    if res_plain != res_batched:
        raise SystemExit("batched results differ from one-at-a-time results")
    rate = plain["alignments_per_s"]
    sweep = []
    for x in (0.25, 0.5, 1.0, 2.0, 4.0):
        arr = inputs.serving_arrivals(n, x * rate)
        for batched_mode in (True, False):
            mode(batched_mode)
            r, _ = serve_run(reqs, arrivals=arr)
            sweep.append({"mode": "batched+graphs" if batched_mode else "plain", "rate_x_plain_saturation": x,
                          "offered_per_s": x * rate, **r})
    mode(True)
    ks = [r[0].k for r in reqs]
    return {"requests": n, "stream": "seeded (request i: seed 5e6+i), k=2/3/4 at "
                                     f"{ks.count(2)}/{ks.count(3)}/{ks.count(4)}",
            "results_identical": True, "autotuned": tuned, "plain_closed_loop": plain, "batched_closed_loop": batched,
            "speedup_closed_loop": batched["alignments_per_s"] / plain["alignments_per_s"], "poisson_sweep": sweep}


def _oracle_warm(_: int) -> int:
    import oracle
    oracle.build()
    time.sleep(0.2)  # keep this worker busy so that every worker gets a warm-up task
    return os.getpid()


def _oracle_serving_request(i: int) -> int:
    import oracle
    p = inputs.serving_request(i)
    oracle.align_problem(p)
    return p.cells


def serving_cpu_baseline(n: int, procs: int = 0, timeout_s: float = 600.0):
    """The oracle on the first ``n`` requests of the serving stream, one request
    per task on ``procs`` spawned worker processes (default: every host core),
    timed after the workers have started and loaded the oracle. A worker that
    dies raises instead of leaving the run waiting."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    procs = procs or os.cpu_count() or 1
    ctx = mp.get_context("spawn")  # no fork of a process that holds a CUDA context
    with ProcessPoolExecutor(max_workers=procs, mp_context=ctx) as ex:
        list(ex.map(_oracle_warm, range(procs), timeout=timeout_s))
        t0 = time.perf_counter()
        cells = sum(ex.map(_oracle_serving_request, range(n), timeout=timeout_s))
        dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "alignments/s", "cores": procs, "kind": "oracle",
            "cells_per_s": cells / dt,
            "sample": f"oracle on requests 0..{n - 1} of the serving stream, one request per task, "
                      f"{procs} processes ({dt:.1f} s)"}


def max_over_ranks(x: float, dist, device) -> float:
    """The largest value of x over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units all ranks processed (weak scaling: every rank its own replica) over the max time."""
    return units_per_rank * world / seconds_max


def dist_setup():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    p = inputs.WORKLOADS[args.workload]()
    per_step = args.ref_cells
    for _ in range(args.warmup):
        time_oracle(p, per_step / 4)
    times, cells = [], 0
    q = None
    for _ in range(args.steps):
        q, dt = time_oracle(p, per_step)
        times.append(dt)
        cells = q.cells
    total = sum(times)
    value = cells * args.steps / total
    sample = f"oracle on prefixes {q.lens} of {p.name} ({cells} cells per step)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": {"workload": p.name, "k": p.k, "lens": p.lens, "cells": p.cells},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# CPU-baseline sample per workload (cells): about 1-10 s of the oracle on one core
PER_WORKLOAD_CPU_CELLS = {"pr1": 2.2e6, "k2_protein": 1.0e8, "k3_protein": 1.2e8, "k4_dna": 2.0e7,
                          "k6_protein": 5.0e6}


def measure_workload(name, steps, warmup, args, dist, dev, sms, world, rank, clocks=None, cpu_cells=None):
    """One workload's device-timed steps, fill-kernel roofline, end-to-end rate
    through msa_align and (rank 0, one GPU) the oracle's CPU sample."""
    import torch

    from paper_2311_17530_gb300 import msadp
    p = inputs.WORKLOADS[name]()
    total_len = sum(p.lens)
    # the autotuner picks the kernel and tile shape for this shape, unless a tile edge is given
    if args.tile_edge:
        msadp.msa_set_tile_edge(p.k, args.tile_edge)
        msadp.msa_config("fill_kernel", 1)
    tuning = None if (args.no_autotune or args.tile_edge) else msadp.msa_autotune(p.lens, len(p.alphabet), repeats=2)
    plan = msadp.Plan(p.k, p.lens, p.alphabet)
    info = plan.info()
    d_res, d_sub = msadp.device_inputs(p, dev)
    d_result, d_masks = msadp.device_outputs(total_len, dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.execute(d_res.data_ptr(), d_sub.data_ptr(), p.gap, d_result.data_ptr(), d_masks.data_ptr(),
                     stream.cuda_stream)

    # a traceback tensor (one byte per cell) smaller than L2 would stay cached
    # between steps: such workloads flush L2 before every step, outside the timing
    l2_bytes = getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 0) or 129 * 2**20
    flush = p.cells < l2_bytes
    scratch = torch.empty(2 * l2_bytes // 4, dtype=torch.int32, device=dev) if flush else None

    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    score, rows, status = msadp.decode_device_result(d_result, d_masks, p.seqs)
    if status != 0:
        raise SystemExit(f"{name}: device status {status}")
    golden = os.path.join(ROOT, "tests", "golden", f"{name}.json")
    checked = None
    if os.path.exists(golden):
        checked = json.load(open(golden))["score"] == score
        if not checked:
            raise SystemExit(f"{name}: score {score} differs from the stored oracle value")

    msadp.msa_config("timing", 1)
    try:
        plan.timings()
    except msadp.MsaError:
        pass
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    if clocks is not None:
        clocks.start()
    if flush:
        evs = []
        for _ in range(steps):
            scratch.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize(dev)
        ms_total = sum(a.elapsed_time(b) for a, b in evs)
    else:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        ms_total = ev0.elapsed_time(ev1)
    msadp.msa_config("timing", 0)
    enc_ms, fill_ms, tb_ms = plan.timings()
    # the fill kernel alone: median over 20 further executions, one at a time
    # (after the timed region, so its event reads do not touch `value`)
    fill_runs = []
    msadp.msa_config("timing", 1)
    for _ in range(20):
        if flush:
            scratch.fill_(1)
        step()
        fill_runs.append(plan.timings()[1])
    msadp.msa_config("timing", 0)
    ms_total = max_over_ranks(ms_total, dist, dev)
    if dist:
        dist.barrier()
    ms_step = ms_total / steps
    value = whole_job_rate(p.cells, world, ms_step / 1e3)

    # end to end through the public C-ABI with host buffers
    e2e = None
    if not args.no_e2e:
        for _ in range(max(1, warmup)):
            msadp.msa_align(p.seqs, p.alphabet, p.subst, p.gap)
        ts = []
        for _ in range(steps):
            if flush:
                scratch.fill_(1)
                torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            s2, _ = msadp.msa_align(p.seqs, p.alphabet, p.subst, p.gap)
            ts.append(time.perf_counter() - t0)
            assert s2 == score
        tot = max_over_ranks(sum(ts), dist, dev)
        e2e = {"value": whole_job_rate(p.cells * steps, world, tot), "unit": UNIT,
               "h2d_bytes_per_step": total_len + p.subst.size * 4,
               "d2h_bytes_per_step": 16 + total_len, "ms_per_step": 1e3 * tot / steps}

    kernel = {1: "fill_tiles", 2: "fill_col3", 3: "fill_band2", 4: "fill_lines",
              5: "fill_lines_stream"}[int(info.fill_kernel)]
    if kernel == "fill_lines_stream" and p.k == 6 and p.lens[-1] + 1 <= WIDE_Z:
        kernel = "fill_lines_wide"  # the streamed kernel's whole-column form
    ops = alg_ops_per_cell(p.k) * p.cells
    achieved = ops / (fill_ms / 1e3) / 1e12
    peak = alu_peak_tiops(sms)
    roofline = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TIOP/s",
                "frac": achieved / peak, "traffic": measured_traffic(name, kernel),
                "ops_per_cell": alg_ops_per_cell(p.k), "fill_ms": fill_ms,
                "fill_ms_median_of_20": statistics.median(fill_runs), "encode_ms": enc_ms,
                "traceback_ms": tb_ms, "peak_basis": PEAK_BASIS.format(sms=sms, mhz=sm_max_mhz())}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        q, dt = time_oracle(p, cpu_cells if cpu_cells is not None else PER_WORKLOAD_CPU_CELLS.get(name, 2e7))
        cpu = {"value": q.cells / dt, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
               "sample": f"oracle on prefixes {q.lens} of {p.name} ({q.cells} cells, {dt:.1f} s)"}
    out = {"value": value, "unit": UNIT, "steps": steps, "warmup": warmup, "ms_per_step": ms_step,
           "config": {"workload": p.name, "k": p.k, "lens": p.lens, "cells": p.cells, "tiles": int(info.tiles),
                      "tile_extent": list(info.tile_extent[:p.k]), "fill_kernel": kernel,
                      "l2": (f"L2 flushed before each step ({2 * l2_bytes >> 20} MiB write, untimed)" if flush
                             else "working set > L2 (no flush)"),
                      "score": score, "score_matches_oracle": checked, "autotune": tuning},
           "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 3 * steps}
    plan.close()
    if args.tile_edge:
        msadp.msa_config("fill_kernel", 0)
    return out


def measure_extensions(reps: int = 3):
    """The two extensions of the path the paper proposes (section 6), through their
    C-ABI calls with host buffers: exact pruning (k = 3 protein, k = 4 DNA: the
    lower bound used, tiles and cells left out, wall time, and cells/s counted over
    the whole tensor) and near-optimal enumeration (a related k = 3 protein
    problem: alignments within 0 and 3 of the optimum, wall time)."""
    from paper_2311_17530_gb300 import msadp
    out = {"pruning": {}, "near_optimal": {}}
    for name in ("k3_protein", "k4_dna"):
        p = inputs.WORKLOADS[name]()
        score, rows = msadp.msa_align(p.seqs, p.alphabet, p.subst, p.gap)
        msadp.msa_align_pruned(p.seqs, p.alphabet, p.subst, p.gap)  # warm-up
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            s2, r2, st = msadp.msa_align_pruned(p.seqs, p.alphabet, p.subst, p.gap)
            ts.append(time.perf_counter() - t0)
        t = statistics.median(ts)
        out["pruning"][name] = {
            "ms": 1e3 * t, "cells_per_s_whole_tensor": p.cells / t, "lower_bound": st["lower_bound"],
            "optimum": score, "same_result_as_msa_align": (s2, r2) == (score, rows),
            "tiles": st["tiles"], "tiles_skipped": st["tiles_skipped"], "cells_skipped": st["cells_skipped"],
            "cells": st["cells"], "fraction_skipped": st["cells_skipped"] / max(1, st["cells"]),
            "note": "host-buffer call: pairwise tables, bound, greedy feasible alignment, pruned generic-tile fill, "
                    "traceback, with per-call allocation and copies"}
    q = inputs.random_problem(17, 3, [120, 110, 130], alphabet=inputs.PROTEIN, related=True)
    for delta in (0, 3):
        msadp.msa_near_optimal(q.seqs, q.alphabet, q.subst, q.gap, delta, 256)
        t0 = time.perf_counter()
        al, more = msadp.msa_near_optimal(q.seqs, q.alphabet, q.subst, q.gap, delta, 256)
        out["near_optimal"][f"delta_{delta}"] = {"problem": q.name, "cells": q.cells, "ms": 1e3 * (time.perf_counter() - t0),
                                                 "alignments": len(al), "more_left": more,
                                                 "scores": sorted({a[0] for a in al}, reverse=True)}
    return out


def run_gb300(args, rank, world, local):
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clocks = ClockSampler(local)
    main = measure_workload(args.workload, args.steps, args.warmup, args, dist, dev, sms, world, rank, clocks=clocks,
                            cpu_cells=args.cpu_cells)
    # every other workload of the benchmark, one GPU: each its own value, roofline and
    # samples (the clock sampler keeps running through them, all of them GPU-busy)
    per_workload = None
    if world == 1 and not args.no_per_workload:
        per_workload = {}
        for name in PER_WORKLOADS:
            if name != args.workload:
                per_workload[name] = measure_workload(name, max(3, args.steps // 2), args.warmup, args, dist, dev,
                                                      sms, world, rank)
    clk = clocks.stop()
    clk_note = "sampled from the headline timed region through the per-workload measurements" \
        if per_workload else "sampled during the timed region"

    extensions = None
    if world == 1 and not args.no_extensions:
        try:
            extensions = measure_extensions()
        except Exception as exc:  # the headline figures stand without them
            extensions = {"error": f"{type(exc).__name__}: {exc}"}

    serving = None
    if world == 1 and not args.no_serving:
        serving = run_serving(args.serve_requests)
        if rank == 0 and not args.no_cpu_baseline:
            try:
                serving["cpu_baseline"] = serving_cpu_baseline(args.serve_cpu_requests)
            except Exception as exc:  # the GPU figures stand without it
                serving["cpu_baseline"] = {"error": f"{type(exc).__name__}: {exc}"}

    if rank == 0:
        cfg = dict(main["config"])
        cfg["parallelism"] = f"replicas{world}"
        line = {
            "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic", "config": cfg,
            "roofline": main["roofline"], "cpu_baseline": main["cpu_baseline"], "e2e": main["e2e"],
            "gpu_launches": main["gpu_launches"],
            "clocks": (dict(clk, window=clk_note) if clk else clk), "per_workload": per_workload, "serving": serving,
            "extensions": extensions,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="k3_protein", choices=sorted(inputs.WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-per-workload", action="store_true", help="time only the --workload line")
    ap.add_argument("--no-extensions", action="store_true", help="skip the pruning and enumeration measurements")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default tile shapes")
    ap.add_argument("--tile-edge", type=int, default=0, help="generic tile kernel with this tile edge")
    ap.add_argument("--serve-requests", type=int, default=2000, help="requests of the serving stream")
    ap.add_argument("--cpu-cells", type=float, default=1.2e8, help="cells of the cpu_baseline sample")
    ap.add_argument("--serve-cpu-requests", type=int, default=320,
                    help="serving-stream requests the oracle runs on every host core (serving cpu_baseline)")
    ap.add_argument("--ref-cells", type=float, default=5e7, help="cells per step of --impl reference")
    args = ap.parse_args()
    rank, world, local = dist_setup()
    if args.warmup < 3 and args.impl == "gb300":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_gb300(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
