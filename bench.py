#!/usr/bin/env python3
"""FastFCA-AS throughput on one GB300 (or N, one process per GPU).

Workload (one step): the long-duration mixture I = J = 3 mics/sources,
F = 513 bins, N = 20000 frames, complex64 storage, mixed precision (FP32
per-point arithmetic with compensated reductions, FP64 P(f) solves and
log-likelihood), 50 hybrid iterations with the L2 trace, then the Wiener
filter.  Metric: TF-point-iterations per second = N F iterations / time.
Inputs (y 246 MB, v 123 MB) exceed the 129 MB L2, so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank runs its own
independently seeded mixture (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1805_09498_gb300.synth import (CONFIGS, batch_lengths, make_batch_device,  # noqa: E402
                                          make_problem)

METRIC = "FastFCA-AS TF-point-iters/s (FP32+FP64 vs FP64 plain) and HBM roofline frac"
UNIT = "TF-point-iters/s"
WORKLOAD = "long_mixed"
CPU_SAMPLE_F = 16          # frequencies of the oracle's CPU sample


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# The sources the streaming passes are compiled from.
STREAM_SOURCES = ("paper_1805_09498_gb300/csrc/ffca_common.cuh", "paper_1805_09498_gb300/csrc/ffca_fastfca.cuh",
                  "paper_1805_09498_gb300/csrc/ffca_stream.cuh")


def sources_hash(files=STREAM_SOURCES) -> str:
    """Hash of the given source files (names and contents): the key under
    which figures measured by ncu are stored, so that figures taken on other
    kernel sources are not reported."""
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as fh:
            t = json.load(fh)
    except OSError:
        return None
    k = t.get("kernels", {}).get(kernel)
    if not k or t.get("csrc_sha") != sources_hash():
        return None
    return k.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock/throttle samples, kept for a [t0, t1] window."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index: int):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "100",
                                       "-i", str(index)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self, t0: float, t1: float):
        if self.p is None:
            return None
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        rows = []
        for line in out.splitlines():
            c = [x.strip() for x in line.split(",")]
            if len(c) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(c[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                ts += float("0." + c[0].split(".")[1]) if "." in c[0] else 0.0
                rows.append((ts, float(c[2]), float(c[3]), c[6:10]))
            except (ValueError, IndexError):
                continue
        win = [r for r in rows if t0 - 0.15 <= r[0] <= t1 + 0.15] or rows[-3:]
        if not win:
            return None
        reasons = sorted({self.NAMES[i] for r in win for i, s in enumerate(r[3]) if s == "Active"})
        return {"sm_mhz": statistics.median(r[1] for r in win), "sm_max_mhz": max(r[2] for r in win),
                "reasons": reasons, "samples": len(win)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws == 1:
        return 0, 1, 0, None
    import torch
    import torch.distributed as dist
    rank, local = int(os.environ["RANK"]), int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return rank, ws, local, dist


def _max_over_ranks(x: float, dist) -> float:
    """The largest x over the ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step: float, steps: int, ms_max: float, ws: int) -> float:
    """Weak scaling: every rank processes its own units; the job's rate is all
    ranks' units over the slowest rank's time."""
    return ws * units_per_rank_step * steps / (ms_max * 1e-3)


def rank_seed(rank: int) -> int:
    """Each rank draws its own mixture (independent problems, no exchange)."""
    return rank


def _sample_freqs(F: int, S: int) -> np.ndarray:
    return np.unique(np.linspace(0, F - 1, S).round().astype(int))


# ---------------------------------------------------------------- the oracle on the host cores
def _oracle_job(job):
    """One worker's share of an oracle run (a block of frequencies; the
    frequencies of the method are independent problems).  Returns the
    oracle's outputs and the worker's own seconds."""
    from oracle import fastfca_as as ffa
    from oracle import fca
    from oracle.fastfca_as import OpCounter
    kind, args = job
    t = time.perf_counter()
    if kind == "fastfca":
        y, v, lam, P, iters, p_update = args
        out = ffa.iterate(y, v, lam, P, iters, counter=OpCounter(), p_update=p_update)
    else:
        y, v, S, iters = args
        out = fca.iterate(y, v, S, iters, counter=OpCounter())
    return out, time.perf_counter() - t


class OraclePool:
    """Worker processes for the FP64 oracle on the host cores, one numpy
    thread each.  Started with `spawn` (the parent has a CUDA context, which a
    forked child must not inherit); jobs are blocks of frequencies."""

    def __init__(self, workers: int | None = None):
        import multiprocessing as mp
        self.workers = workers or os.cpu_count() or 1
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"  # inherited by the spawned workers
        try:
            self.pool = mp.get_context("spawn").Pool(self.workers)
            self.pool.map(_oracle_job, [("fastfca", (np.ones((1, 1, 4), complex), np.ones((1, 1, 4)),
                                                     np.ones((1, 1, 1)), np.ones((1, 1, 1), complex), 1, "fpi"))]
                          * self.workers)  # import the oracle in every worker before timing
        finally:
            for k, val in saved.items():
                if val is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = val

    def run(self, jobs):
        """Runs the jobs over the workers; returns (results, wall seconds)."""
        t = time.perf_counter()
        res = self.pool.map(_oracle_job, jobs, chunksize=1)
        return res, time.perf_counter() - t

    def close(self):
        self.pool.close()
        self.pool.join()


def _fastfca_jobs(y, v, lam, P, iters, blocks, p_update="fpi"):
    fb = np.array_split(np.arange(y.shape[1]), blocks)
    return [("fastfca", (y[:, b], v[:, b], lam[b], P[b], iters, p_update)) for b in fb if len(b)]


# ---------------------------------------------------------------- ours
def run_ours(args, cfg, rank, ws, local, dist):
    import torch

    from paper_1805_09498_gb300 import build as _build
    from paper_1805_09498_gb300 import ffca
    _build.build()
    I, J, F, N, iters = cfg["I"], cfg["J"], cfg["F"], cfg["N"], cfg["iters"]
    dev = torch.device("cuda", local)
    p = make_problem(I, J, F, N, seed=rank_seed(rank), alpha=cfg["alpha"], kappa=cfg["kappa"])
    yd, vd, lamd, Pd, _ = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="mixed", device=dev)
    v_init, lam_init, P_init = vd.clone(), lamd.clone(), Pd.clone()
    est = ffca.FastFCA(yd, vd, lamd, Pd, N=N)
    ld = yd.shape[2]
    out = torch.empty((J, I, F, ld), dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev)

    # accuracy leg input: the full estimation from the initial state
    tr_acc = est.iterate(iters)
    fs = _sample_freqs(F, CPU_SAMPLE_F)
    gpu_state = (vd[:, fs, :N].double().cpu().numpy(), lamd[fs].cpu().numpy(), Pd[fs].cpu().numpy())

    # the plain FP64 GPU form on the same mixture (a few iterations)
    fp64 = None
    if rank == 0:
        y64, v64, l64, P64, _ = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="fp64", device=dev)
        e64 = ffca.FastFCA(y64, v64, l64, P64, N=N)
        e64.iterate(1, trace=False)
        it64 = 5
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        e64.iterate(it64, trace=False)
        b.record(stream)
        torch.cuda.synchronize()
        ms64 = a.elapsed_time(b)
        fp64 = {"value": N * F * it64 / (ms64 * 1e-3), "unit": UNIT, "iters_timed": it64,
                "ms_per_iter": ms64 / it64}
        e64.close()
        del y64, v64, l64, P64
        torch.cuda.empty_cache()

    # the conventional FCA EM baseline (Sec. 3.3) on the same mixture and precision
    fca_line = None
    if rank == 0:
        Pinv = torch.linalg.inv(P_init.cpu()).to(dev)  # setup only (CPU LAPACK)
        S0 = (Pinv.conj().transpose(1, 2)[:, None] * lam_init[:, :, None, :].to(torch.complex128)
              ) @ Pinv[:, None]
        S0 = S0.contiguous()
        vf = v_init.clone()
        ef = ffca.FCA(yd, vf, S0, N=N)
        ef.iterate(1, trace=False)
        itf = 3
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        ef.iterate(itf, trace=False)
        b.record(stream)
        torch.cuda.synchronize()
        msf = a.elapsed_time(b)
        fca_line = {"value": N * F * itf / (msf * 1e-3), "unit": UNIT, "iters_timed": itf,
                    "ms_per_iter": msf / itf, "precision": "mixed (same as the main line)"}
        ef.close()
        del vf, S0, Pinv
        torch.cuda.empty_cache()

    vd.copy_(v_init); lamd.copy_(lam_init); Pd.copy_(P_init)

    def step():
        est.iterate(iters)      # trace copied back: the step's D2H result
        est.wiener(out)

    est.set_graph(True)  # the iteration loop replays from a CUDA graph (captured in the first warm-up step)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    time.sleep(0.3)
    ffca.ffca_timing_read(est.ctx)  # reset the launch counts
    ffca.ffca_timing_enable(est.ctx, False)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    if dist is not None:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    counts = ffca.ffca_timing_read(est.ctx)  # launches of the timed steps (no per-launch events there)
    # Per-kernel durations: the same number of steps again, continuing from
    # the same state, with a CUDA event pair around every launch on the
    # context's stream.  The event records serialise the launches (about 2 us
    # per launch, 7% of a step), so they stay out of the headline region.
    est.set_graph(False)  # events around every launch need the plain launches
    ffca.ffca_timing_enable(est.ctx, True)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    kt = ffca.ffca_timing_read(est.ctx)
    ffca.ffca_timing_enable(est.ctx, False)
    clk = clocks.stop(t0, t1)
    ms_max = _max_over_ranks(ms, dist)
    units_per_step = N * F * iters
    value = whole_job_rate(units_per_step, args.steps, ms_max, ws)

    # end to end through the C ABI with pinned host buffers
    y_h = torch.empty(yd.shape, dtype=yd.dtype, pin_memory=True); y_h.copy_(yd)
    v_h = torch.empty(vd.shape, dtype=vd.dtype, pin_memory=True); v_h.copy_(v_init)
    l_h = torch.empty(lamd.shape, dtype=lamd.dtype, pin_memory=True); l_h.copy_(lam_init)
    P_h = torch.empty(Pd.shape, dtype=Pd.dtype, pin_memory=True); P_h.copy_(P_init)
    o_h = torch.empty(out.shape, dtype=out.dtype, pin_memory=True)
    vo_h = torch.empty_like(v_h, pin_memory=True)
    lo_h = torch.empty_like(l_h, pin_memory=True)
    Po_h = torch.empty_like(P_h, pin_memory=True)

    # A second job slot (its own device arrays, context, stream and host
    # outputs), so that one job's host<->device copies overlap the other's
    # kernels: a user serving a stream of mixtures keeps two in flight.
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    est1 = ffca.FastFCA(yd, vd, lamd, Pd, N=N, stream=s1)
    yd2, vd2, lamd2, Pd2 = (torch.empty_like(t) for t in (yd, vd, lamd, Pd))
    est2 = ffca.FastFCA(yd2, vd2, lamd2, Pd2, N=N, stream=s2)
    out2 = torch.empty_like(out)
    for e in (est1, est2):
        e.set_graph(True)
    o_h2, vo_h2, lo_h2, Po_h2 = (torch.empty_like(t, pin_memory=True) for t in (o_h, vo_h, lo_h, Po_h))
    torch.cuda.synchronize()
    slots = [(est1, out, o_h, vo_h, lo_h, Po_h), (est2, out2, o_h2, vo_h2, lo_h2, Po_h2)]

    def e2e_job(e, o_dev, oh, voh, loh, Poh):
        """One job through the public C ABI: inputs up from pinned host memory,
        the iterations (with the trace), the Wiener output and the estimates
        back to host memory."""
        ffca.ffca_upload(e.ctx, y_h.data_ptr(), v_h.data_ptr(), l_h.data_ptr(), P_h.data_ptr())
        e.iterate(iters)
        ffca.ffca_wiener_host(e.ctx, o_dev.data_ptr(), oh.data_ptr())
        ffca.ffca_download(e.ctx, voh.data_ptr(), loh.data_ptr(), Poh.data_ptr())

    def run_jobs(n, in_flight):
        """n jobs, in_flight host threads each driving its own slot (the ctypes
        calls release the GIL while they wait on their stream)."""
        if in_flight == 1:
            for _ in range(n):
                e2e_job(*slots[0])
            return
        import threading
        share = [n // in_flight + (1 if k < n % in_flight else 0) for k in range(in_flight)]
        err = []

        def worker(k):
            try:
                for _ in range(share[k]):
                    e2e_job(*slots[k])
            except Exception as ex:  # surfaced after the join
                err.append(ex)
        th = [threading.Thread(target=worker, args=(k,)) for k in range(in_flight)]
        for t_ in th:
            t_.start()
        for t_ in th:
            t_.join()
        if err:
            raise err[0]

    def timed_jobs(n, in_flight):
        run_jobs(2 * in_flight, in_flight)  # warm-up
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        h0 = time.perf_counter()
        run_jobs(n, in_flight)
        torch.cuda.synchronize()
        return _max_over_ranks(time.perf_counter() - h0, dist)

    e2e_steps = max(4, min(args.steps, 20))
    e2e_s = timed_jobs(e2e_steps, 1)
    e2e_two = timed_jobs(e2e_steps, 2)
    # the pipelined jobs give the same estimates as the one-job run
    torch.cuda.synchronize()
    e2e_same = bool(torch.equal(vo_h2, vo_h) and torch.equal(Po_h2, Po_h))
    nbytes = lambda t: t.numel() * t.element_size()  # noqa: E731
    e2e = {"value": ws * units_per_step * e2e_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": nbytes(y_h) + nbytes(v_h) + nbytes(l_h) + nbytes(P_h),
           "d2h_bytes_per_step": nbytes(o_h) + nbytes(vo_h) + nbytes(lo_h) + nbytes(Po_h)
           + 8 * (iters + 1),
           "jobs": e2e_steps, "jobs_in_flight": 1,
           "how": "each step is one job through the C ABI from pinned host buffers (upload, 50 "
                  "iterations with the trace replayed from a CUDA graph, Wiener output and "
                  "estimates back to host), one after another on one stream",
           "two_jobs_in_flight": {"value": ws * units_per_step * e2e_steps / e2e_two,
                                  "how": "the same jobs from two slots on two streams driven by "
                                         "two host threads",
                                  "slots_agree": e2e_same}}
    est1.close()
    est2.close()
    del est1, est2, yd2, vd2, lamd2, Pd2, out2, o_h2, vo_h2, lo_h2, Po_h2, slots
    est.close()
    del est, yd, vd, lamd, Pd, out, y_h, v_h, l_h, P_h, o_h, vo_h, lo_h, Po_h
    torch.cuda.empty_cache()

    if rank != 0:
        return None
    pool = OraclePool()
    plain = run_plain_fp64(args, dev, pool)
    em = run_em(args, p, cfg, dev)
    batched = run_batched(args, dev)
    large = run_large_array(args, dev)
    adjoint = run_adjoint(dev)
    front = run_front_end(dev)

    # roofline of the dominant kernel: algorithmic bytes per launch / mean duration
    peaks, peak_src = _peaks()
    c, r = 8, 4
    bytes_per_tf = {"estep": I * c + 2 * J * r, "wcov": I * c + J * r}
    kernels = {}
    for k, bpt in bytes_per_tf.items():
        kms, kn = kt[k]
        if kn:
            avg = kms / kn
            kernels[k] = {"launches": kn, "avg_us": avg * 1e3, "bytes_per_launch": bpt * N * F,
                          "achieved_gbs": bpt * N * F / (avg * 1e-3) / 1e9}
    for k in ("psolve", "afinal", "loglik", "wiener", "prep"):
        kms, kn = kt[k]
        if kn:
            kernels[k] = {"launches": kn, "avg_us": kms / kn * 1e3}
    dom = max(("estep", "wcov"), key=lambda k: kt[k][0])
    kname = {"estep": "k_estep", "wcov": "k_wcov"}[dom]
    roof = {"bound": "hbm", "kernel": kname, "achieved": kernels[dom]["achieved_gbs"],
            "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": kernels[dom]["achieved_gbs"] / peaks["hbm_gbs"],
            "traffic": _ncu_traffic(kname), "peak_source": peak_src}

    cpu = None
    if ws == 1:
        cpu = cpu_baseline_and_error(p, cfg, fs, gpu_state, tr_acc, pool)
    pool.close()

    launches = int(sum(n for _, n in counts.values()))
    kernels["timing"] = ("CUDA events around every launch over a second run of the same steps "
                         "(the headline steps run without per-launch events)")
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: I={I} J={J} F={F} N={N}, c64 storage, mixed "
                               f"FP32/FP64, {iters} iterations + Wiener per step",
                   "iters_per_step": iters, "l2": "inputs 369 MB > 129 MB L2 (no flush)",
                   "state": "parameters carried from step to step",
                   "launches": "the iteration loop of a step replayed from a CUDA graph (trace slots "
                               "written on the device, copied back at the end of the step)",
                   "parallelism": f"replicas x{ws}"},
        "roofline": roof, "kernels": kernels,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "gpu_launches_per_step": launches / args.steps,
        "clocks": clk, "fp64_gpu": fp64,
        "speedup_mixed_vs_fp64_gpu": (value / ws / fp64["value"]) if fp64 else None,
        "fca_gpu": fca_line,
        "speedup_vs_fca_gpu": (value / ws / fca_line["value"]) if fca_line else None,
        "plain_fp64": plain,
        "em_update": em,
        "paper_context": ("the paper reports FastFCA-AS more than 420 times faster than conventional FCA "
                          "in parameter estimation (real-time factor; Sec. 5, MATLAB R2013a on an Intel "
                          "i7-2600 at 3.4 GHz, I = J = 3, 8 s mixtures at 16 kHz, 20 iterations): context "
                          "only, other hardware and software"),
        "host_cores": os.cpu_count(),
        "l2_per_point_after_fixed_point": float(tr_acc[-1] / (N * F)),
        "batched": batched,
        "large_array": large,
        "adjoint": adjoint,
        "stft_front_end": front,
    }


def _ncu_fp64(kernel: str):
    """FP64 operations per launch of `kernel` (2 per DFMA, 1 per DMUL / DADD,
    from ncu's executed-instruction counters) in the committed summary, if it
    was taken on the current kernel sources; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_fp64.json")) as fh:
            t = json.load(fh)
    except OSError:
        return None
    k = t.get("kernels", {}).get(kernel)
    if not k or t.get("csrc_sha") != sources_hash():
        return None
    return k


def run_plain_fp64(args, dev, pool):
    """The plain FP64 workload: I = J = 3, F = 257, N = 600, 20 iterations,
    every per-point operation in FP64; launch-bound at this size, so the
    timed runs replay the iteration loop from a CUDA graph (and, beside it,
    plain launches with the L2 trace).  The conventional FCA EM on the GPU on
    the same data and precision; the FP64 oracle (FastFCA-AS and FCA) on the
    whole workload on one host core and on all of them; the FP64-ALU fraction
    of the two streaming passes against the measured FP64 rate."""
    import torch
    from oracle import fastfca_as as ffa
    from oracle import fca
    from oracle.fastfca_as import OpCounter
    from paper_1805_09498_gb300 import ffca
    cfg = CONFIGS["plain_fp64"]
    I, J, F, N, iters = cfg["I"], cfg["J"], cfg["F"], cfg["N"], cfg["iters"]
    p = make_problem(I, J, F, N, seed=2, alpha=cfg["alpha"], kappa=cfg["kappa"])
    yd, vd, lamd, Pd, _ = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="fp64", device=dev)
    v0, l0, P0 = vd.clone(), lamd.clone(), Pd.clone()
    stream = torch.cuda.current_stream(dev)
    units = N * F * iters

    def timed(fn, reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def reset():
        vd.copy_(v0); lamd.copy_(l0); Pd.copy_(P0)

    est = ffca.FastFCA(yd, vd, lamd, Pd, N=N)
    tr = est.iterate(iters)
    vg, lg, Pg = vd[:, :, :N].cpu().numpy(), lamd.cpu().numpy(), Pd.cpu().numpy()
    t0 = time.perf_counter()
    rv, rl, rP, rt = ffa.iterate(p.y, p.v0, p.lam0, p.P0, iters, counter=OpCounter())
    one_core_s = time.perf_counter() - t0
    _, all_s = pool.run(_fastfca_jobs(p.y, p.v0, p.lam0, p.P0, iters, pool.workers))

    def relerr(a_, b_, ax):
        a_ = np.moveaxis(a_, ax, 0).reshape(F, -1)
        b_ = np.moveaxis(b_, ax, 0).reshape(F, -1)
        return float(np.max(np.linalg.norm(a_ - b_, axis=1) / np.linalg.norm(b_, axis=1)))
    err = {"v": relerr(vg, rv, 1), "lambda": relerr(lg, rl, 0), "P": relerr(Pg, rP, 0),
           "loglik_rel": float(np.max(np.abs(tr - rt) / np.abs(rt))),
           "measure": f"all {F} frequencies after {iters} iterations; normwise relative per frequency (max); "
                      "L2 trace relative (max over the trace)"}
    reps = 20
    est.set_graph(True)
    reset()
    for _ in range(3):
        est.iterate(iters, trace=False)
    ms_graph = timed(lambda: est.iterate(iters, trace=False), reps)
    est.set_graph(False)
    ms_trace = timed(lambda: est.iterate(iters), 5)
    ffca.ffca_timing_read(est.ctx)
    ffca.ffca_timing_enable(est.ctx, True)
    est.iterate(iters, trace=False)
    kt = ffca.ffca_timing_read(est.ctx)
    ffca.ffca_timing_enable(est.ctx, False)
    est.close()

    def resident_and_mixed():
        """The same workload with each problem resident on chip (one CTA per
        frequency, all 20 iterations in one launch), and both forms in the
        mixed precision at the same shape: rate and error against the oracle."""
        out = {}
        for prec in ("fp64", "mixed"):
            yq, vq, lq, Pq, _ = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec=prec, device=dev)
            v0q, l0q, P0q = vq.clone(), lq.clone(), Pq.clone()
            for form in ("resident", "streaming") if prec == "mixed" else ("resident",):
                vq.copy_(v0q); lq.copy_(l0q); Pq.copy_(P0q)
                e = ffca.FastFCA(yq, vq, lq, Pq, N=N)
                if form == "resident":
                    e.set_resident(True)
                trq = e.iterate(iters)
                errq = {"v": relerr(vq[:, :, :N].double().cpu().numpy(), rv, 1), "lambda": relerr(lq.cpu().numpy(), rl, 0),
                        "P": relerr(Pq.cpu().numpy(), rP, 0)}
                if prec == "fp64":
                    errq["loglik_rel"] = float(np.max(np.abs(trq - rt) / np.abs(rt)))
                else:
                    errq["loglik_per_point"] = float(np.max(np.abs(trq - rt)) / (N * F))
                e.set_graph(True)
                for _ in range(3):
                    e.iterate(iters, trace=False)
                msq = timed(lambda: e.iterate(iters, trace=False), reps)
                e.set_graph(False)
                msqt = timed(lambda: e.iterate(iters), 5)
                e.close()
                out[f"{form}_{prec}"] = {"value": units / (msq * 1e-3), "ms_per_run": msq,
                                         "with_trace": {"value": units / (msqt * 1e-3), "ms_per_run": msqt},
                                         "error_vs_oracle": errq}
            del yq, vq, lq, Pq, v0q, l0q, P0q
        out["how"] = ("graph replay of the 20 iterations, CUDA events, 20 runs (with_trace: plain launches, "
                      "L2 trace copied back); resident: ffca_set_resident, one launch per 20 iterations")
        return out

    forms = resident_and_mixed()
    peak64 = ffca.ffca_peak_fp64(stream)
    kernels = {}
    for k, kname, bpt in (("estep", "k_estep<double, 3, 3, 1, 0>", I * 16 + 2 * J * 8),
                          ("wcov", "k_wcov<double, 3, 3>", I * 16 + J * 8), ("psolve", None, 0)):
        kms, kn = kt[k]
        if not kn:
            continue
        us = kms / kn * 1e3
        kernels[k] = {"launches": kn, "avg_us": us}
        if bpt:
            kernels[k]["hbm_gbs"] = bpt * N * F / (us * 1e-6) / 1e9
            ops = _ncu_fp64(kname)
            if ops:
                ach = ops["fp64_flops_per_launch"] / (us * 1e-6) / 1e9
                kernels[k]["fp64"] = {"achieved_gflops": ach, "peak_gflops": peak64, "frac": ach / peak64,
                                      "flops_per_launch": ops["fp64_flops_per_launch"],
                                      "ncu_fp64_pipe_pct": ops.get("fp64_pipe_pct"),
                                      "peak": "measured by ffca_peak_fp64 in this run"}
    # the conventional FCA EM on the GPU, same data, FP64 (S_j = P^{-H} Lambda_j P^{-1} of the initial state)
    S0h = fca.spatial_from_joint(p.P0, p.lam0)
    S0 = torch.from_numpy(S0h).to(dev)
    vf = v0.clone()
    ef = ffca.FCA(yd, vf, S0, N=N)
    trf = ef.iterate(iters)
    fv, fS = vf[:, :, :N].cpu().numpy(), S0.cpu().numpy()
    t0 = time.perf_counter()
    frv, frS, frt = fca.iterate(p.y, p.v0, S0h, iters, counter=OpCounter())
    fca_one_s = time.perf_counter() - t0
    _, fca_all_s = pool.run([("fca", (p.y[:, b], p.v0[:, b], S0h[b], iters))
                             for b in np.array_split(np.arange(F), pool.workers) if len(b)])
    fca_err = {"v": relerr(fv, frv, 1), "S": relerr(fS, frS, 0),
               "loglik_rel": float(np.max(np.abs(trf - frt) / np.abs(frt)))}
    vf.copy_(v0); S0.copy_(torch.from_numpy(S0h).to(dev))
    ef.iterate(1, trace=False)
    ms_fca = timed(lambda: ef.iterate(iters, trace=False), 5)
    ef.close()
    del yd, vd, lamd, Pd, v0, l0, P0, vf, S0
    torch.cuda.empty_cache()
    return {"workload": f"plain_fp64: I={I} J={J} F={F} N={N}, c128, FP64 throughout, {iters} iterations",
            "value": units / (ms_graph * 1e-3), "unit": UNIT, "ms_per_run": ms_graph,
            "timing": "graph replay of the 20 iterations (launch-bound size), CUDA events, 20 runs",
            "with_trace": {"value": units / (ms_trace * 1e-3), "ms_per_run": ms_trace,
                           "how": "plain launches, L2 trace copied back"},
            "kernels": kernels, "fp64_peak_gflops_measured": peak64,
            "error_vs_oracle": err, "forms": forms,
            "oracle": {"one_core": {"value": units / one_core_s, "seconds": one_core_s, "cores": 1},
                       "all_cores": {"value": units / all_s, "seconds": all_s, "cores": pool.workers},
                       "sample": "the whole workload (every frequency, frame and iteration)"},
            "fca_gpu": {"value": units / (ms_fca * 1e-3), "ms_per_run": ms_fca, "error_vs_oracle": fca_err,
                        "precision": "fp64"},
            "fca_oracle": {"one_core": {"value": units / fca_one_s, "seconds": fca_one_s, "cores": 1},
                           "all_cores": {"value": units / fca_all_s, "seconds": fca_all_s,
                                         "cores": pool.workers}},
            "speedup_vs_fca_gpu": ms_fca / ms_graph,
            "speedup_vs_oracle_all_cores": (units / (ms_graph * 1e-3)) / (units / all_s),
            "speedup_oracle_fastfca_vs_fca": fca_one_s / one_core_s}


def run_em(args, p, cfg, dev):
    """The normal EM update of P (Sec. 4.6) on the long mixture: the same
    iterations per step with one streaming pass each (pass A with the EM
    sums, 48 B per point at I = J = 3) and the per-problem EM step instead
    of pass B and the fixed point; timed like the headline (trace copied
    back every step).  Beside it the error against the FP64 oracle's EM
    iterations on sampled frequencies and the L2 per point reached by both
    updates after the same iterations."""
    import torch
    from oracle import fastfca_as as ffa
    from oracle.fastfca_as import OpCounter
    from paper_1805_09498_gb300 import ffca
    I, J, F, N, iters = cfg["I"], cfg["J"], cfg["F"], cfg["N"], cfg["iters"]
    yd, vd, lamd, Pd, _ = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="mixed", device=dev)
    v0, l0, P0 = vd.clone(), lamd.clone(), Pd.clone()
    stream = torch.cuda.current_stream(dev)
    est = ffca.FastFCA(yd, vd, lamd, Pd, N=N)
    est.set_p_update("em")
    tr = est.iterate(iters)
    fs = _sample_freqs(F, 4)
    vg, lg, Pg = vd[:, fs, :N].double().cpu().numpy(), lamd[fs].cpu().numpy(), Pd[fs].cpu().numpy()
    t0 = time.perf_counter()
    rv, rl, rP, rt = ffa.iterate(p.y[:, fs], p.v0[:, fs], p.lam0[fs], p.P0[fs], iters, counter=OpCounter(),
                                 p_update="em")
    oracle_s = time.perf_counter() - t0

    def relerr(a_, b_, ax):
        a_ = np.moveaxis(a_, ax, 0).reshape(len(fs), -1)
        b_ = np.moveaxis(b_, ax, 0).reshape(len(fs), -1)
        return float(np.max(np.linalg.norm(a_ - b_, axis=1) / np.linalg.norm(b_, axis=1)))
    err = {"v": relerr(vg, rv, 1), "lambda": relerr(lg, rl, 0), "P": relerr(Pg, rP, 0),
           "loglik_per_point": abs(ffa.loglik(p.y[:, fs], vg, lg, Pg) - rt[-1]) / (len(fs) * N),
           "measure": f"after {iters} EM iterations from the same initial state, on {len(fs)} sampled "
                      "frequencies; normwise relative error per frequency (max)"}
    vd.copy_(v0); lamd.copy_(l0); Pd.copy_(P0)
    est.set_graph(True)  # traced iterations replayed from a CUDA graph (captured in the warm-up)
    for _ in range(max(args.warmup, 3)):
        est.iterate(iters)
    reps = max(3, min(args.steps, 20))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        est.iterate(iters)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    est.set_graph(False)  # events around every launch need the plain launches
    ffca.ffca_timing_read(est.ctx)
    ffca.ffca_timing_enable(est.ctx, True)
    est.iterate(iters)
    kt = ffca.ffca_timing_read(est.ctx)
    ffca.ffca_timing_enable(est.ctx, False)
    est.close()
    peaks, _ = _peaks()
    bpt = I * 8 + 2 * J * 4
    kms, kn = kt["estep"]
    em_us = kms / kn * 1e3
    gbs = bpt * N * F / (em_us * 1e-6) / 1e9
    out = {"workload": f"long mixture with the normal EM update of P: I={I} J={J} F={F} N={N}, c64, "
                       f"{iters} iterations with the L2 trace, replayed from a CUDA graph",
           "value": N * F * iters / (ms * 1e-3), "unit": UNIT, "ms_per_run": ms, "runs_timed": reps,
           "kernels": {"em_pass": {"avg_us": em_us, "bytes_per_launch": bpt * N * F, "achieved_gbs": gbs,
                                   "frac_of_measured_hbm": gbs / peaks["hbm_gbs"]},
                       "em_step": {"avg_us": kt["psolve"][0] / kt["psolve"][1] * 1e3}},
           "l2_per_point_after": tr[-1] / (N * F),
           "error_vs_oracle": err, "oracle_em_seconds": oracle_s}
    del yd, vd, lamd, Pd, v0, l0, P0
    torch.cuda.empty_cache()
    return out


def run_adjoint(dev):
    """The adjoint workload: gradients of NLL = -L2 and of the Wiener
    estimate's squared error against the known source images with respect to
    (v, Lambda, P), I = J = 4, F = 257, N = 2000, FP32 per point (c64), the
    posteriors recomputed in one streaming pass; error against the FP64
    gradient oracle on sampled frequencies."""
    import torch
    from oracle import adjoint as adj
    from paper_1805_09498_gb300 import ffca
    cfg = CONFIGS["adjoint"]
    I, J, F, N = cfg["I"], cfg["J"], cfg["F"], cfg["N"]
    p = make_problem(I, J, F, N, seed=5, alpha=cfg["alpha"], kappa=cfg["kappa"], keep_images=True)
    yd, vd, lamd, Pd, _ = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="mixed", device=dev)
    s = torch.zeros((J, I, F, yd.shape[2]), dtype=torch.complex64)
    s[..., :N] = torch.from_numpy(p.x).to(torch.complex64)
    s = s.to(dev)
    est = ffca.FastFCA(yd, vd, lamd, Pd, N=N)
    dv, dl, dP = torch.zeros_like(vd), torch.empty_like(lamd), torch.empty_like(Pd)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": f"adjoint: I={I} J={J} F={F} N={N}, c64 per point, FP64 per frequency"}
    fs = _sample_freqs(F, 8)
    for name, call, ref in (
            ("nll", lambda: ffca.ffca_nll_grad(est.ctx, dv.data_ptr(), dl.data_ptr(), dP.data_ptr()),
             lambda: adj.nll_grad(p.y[:, fs], p.v0[:, fs], p.lam0[fs], p.P0[fs])),
            ("wiener_se", lambda: ffca.ffca_wiener_se_grad(est.ctx, s.data_ptr(), dv.data_ptr(),
                                                           dl.data_ptr(), dP.data_ptr()),
             lambda: adj.wiener_se_grad(p.y[:, fs], p.x[:, :, fs], p.v0[:, fs], p.lam0[fs], p.P0[fs]))):
        for _ in range(3):
            call()
        reps = 20
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            call()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        rv, rl, rP = ref()

        def relerr(g, r, ax):
            g = np.moveaxis(g, ax, 0).reshape(len(fs), -1)
            r = np.moveaxis(r, ax, 0).reshape(len(fs), -1)
            return float(np.max(np.linalg.norm(g - r, axis=1) / np.linalg.norm(r, axis=1)))
        out[name] = {"value": N * F / (ms * 1e-3), "unit": "TF-points/s (loss + all gradients)",
                     "ms_per_call": ms,
                     "error_vs_oracle": {
                         "v": relerr(dv[:, fs, :N].double().cpu().numpy(), rv, 1),
                         "lambda": relerr(dl[fs].cpu().numpy(), rl, 0),
                         "P": relerr(dP[fs].cpu().numpy(), rP, 0),
                         "measure": f"{len(fs)} sampled frequencies, normwise relative per frequency (max)"}}
    est.close()
    return out


def run_large_array(args, dev):
    """The large-array workload: I = 8 mics, J = 6 sources, F = 513, N = 4000,
    complex64, mixed precision, 30 iterations per run; beside it the plain
    FP64 GPU form and the conventional FCA EM on the GPU (same data, same
    precision as the main run, its comparison in the paper), and the error
    against the FP64 oracle on sampled frequencies."""
    import torch
    from oracle import fastfca_as as ffa
    from oracle.fastfca_as import OpCounter
    from paper_1805_09498_gb300 import ffca
    cfg = CONFIGS["large_array"]
    I, J, F, N, iters = cfg["I"], cfg["J"], cfg["F"], cfg["N"], cfg["iters"]
    p = make_problem(I, J, F, N, seed=1, alpha=cfg["alpha"], kappa=cfg["kappa"])
    yd, vd, lamd, Pd, _ = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="mixed", device=dev)
    v_init, lam_init, P_init = vd.clone(), lamd.clone(), Pd.clone()
    stream = torch.cuda.current_stream(dev)
    est = ffca.FastFCA(yd, vd, lamd, Pd, N=N)

    def timed(fn, reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    # accuracy: one full run from the initial state against the oracle
    tr = est.iterate(iters)
    fs = _sample_freqs(F, 3)
    vg, lg, Pg = vd[:, fs, :N].double().cpu().numpy(), lamd[fs].cpu().numpy(), Pd[fs].cpu().numpy()
    rv, rl, rP, rt = ffa.iterate(p.y[:, fs], p.v0[:, fs], p.lam0[fs], p.P0[fs], iters,
                                 counter=OpCounter())

    def relerr(a_, b_, ax):
        a_ = np.moveaxis(a_, ax, 0).reshape(len(fs), -1)
        b_ = np.moveaxis(b_, ax, 0).reshape(len(fs), -1)
        return float(np.max(np.linalg.norm(a_ - b_, axis=1) / np.linalg.norm(b_, axis=1)))
    err = {"v": relerr(vg, rv, 1), "lambda": relerr(lg, rl, 0), "P": relerr(Pg, rP, 0),
           "loglik_per_point": abs(ffa.loglik(p.y[:, fs], vg, lg, Pg) - rt[-1]) / (len(fs) * N),
           "measure": f"after {iters} iterations from the same initial state, on {len(fs)} sampled "
                      "frequencies; normwise relative error per frequency (max)"}

    est.set_graph(True)  # traced iterations replayed from a CUDA graph (captured in the warm-up)
    for _ in range(max(args.warmup, 3)):
        est.iterate(iters)
    reps = 5
    ffca.ffca_timing_read(est.ctx)
    ms = timed(lambda: est.iterate(iters), reps)
    est.set_graph(False)  # events around every launch need the plain launches
    ffca.ffca_timing_read(est.ctx)  # drop the counts of the untimed runs
    ffca.ffca_timing_enable(est.ctx, True)
    est.iterate(iters)
    kt = ffca.ffca_timing_read(est.ctx)
    ffca.ffca_timing_enable(est.ctx, False)
    est.close()
    kernels = {}
    for k, bpt in (("estep", I * 8 + 2 * J * 4), ("wcov", I * 8 + J * 4), ("psolve", 0),
                   ("afinal", 0), ("loglik", 0)):
        kms, kn = kt[k]
        if kn:
            kernels[k] = {"launches": kn, "avg_us": kms / kn * 1e3}
            if bpt:
                kernels[k]["achieved_gbs"] = bpt * N * F / (kms / kn * 1e-3) / 1e9
    units = N * F * iters
    out = {"workload": f"large_array: I={I} J={J} F={F} N={N}, c64 storage, mixed FP32/FP64, "
                       f"{iters} iterations with the L2 trace, replayed from a CUDA graph",
           "value": units / (ms * 1e-3), "unit": UNIT, "ms_per_run": ms, "runs_timed": reps,
           "kernels": kernels, "error_vs_oracle": err}

    # the normal EM update of P (Sec. 4.6) on the same mixture: one pass per iteration
    vd.copy_(v_init); lamd.copy_(lam_init); Pd.copy_(P_init)
    eem = ffca.FastFCA(yd, vd, lamd, Pd, N=N)
    eem.set_p_update("em")
    trm = eem.iterate(iters)
    vg, lg, Pg = vd[:, fs, :N].double().cpu().numpy(), lamd[fs].cpu().numpy(), Pd[fs].cpu().numpy()
    mv, ml, mP, mt = ffa.iterate(p.y[:, fs], p.v0[:, fs], p.lam0[fs], p.P0[fs], iters, counter=OpCounter(),
                                 p_update="em")
    eem.set_graph(True)
    for _ in range(3):
        eem.iterate(iters)
    ms_em = timed(lambda: eem.iterate(iters), reps)
    eem.set_graph(False)
    ffca.ffca_timing_read(eem.ctx)
    ffca.ffca_timing_enable(eem.ctx, True)
    eem.iterate(iters)
    ktm = ffca.ffca_timing_read(eem.ctx)
    ffca.ffca_timing_enable(eem.ctx, False)
    eem.close()
    out["em_update"] = {
        "value": units / (ms_em * 1e-3), "unit": UNIT, "ms_per_run": ms_em, "runs_timed": reps,
        "kernels": {"em_pass": {"avg_us": ktm["estep"][0] / ktm["estep"][1] * 1e3,
                                "achieved_gbs": (I * 8 + 2 * J * 4) * N * F / (ktm["estep"][0] / ktm["estep"][1] * 1e-3) / 1e9},
                    "em_step": {"avg_us": ktm["psolve"][0] / ktm["psolve"][1] * 1e3}},
        "l2_per_point_after": float(trm[-1]) / (N * F),
        "error_vs_oracle": {"v": relerr(vg, mv, 1), "lambda": relerr(lg, ml, 0), "P": relerr(Pg, mP, 0),
                            "measure": f"after {iters} EM iterations from the same initial state, on {len(fs)} "
                                       "sampled frequencies; normwise relative error per frequency (max)"}}

    # the plain FP64 GPU form on the same mixture
    y64, v64, l64, P64, _ = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec="fp64", device=dev)
    e64 = ffca.FastFCA(y64, v64, l64, P64, N=N)
    e64.iterate(1, trace=False)
    it64 = 3
    ms64 = timed(lambda: e64.iterate(it64, trace=False), 1)
    e64.close()
    del y64, v64, l64, P64
    out["fp64_gpu"] = {"value": N * F * it64 / (ms64 * 1e-3), "unit": UNIT, "iters_timed": it64,
                       "ms_per_iter": ms64 / it64}
    out["speedup_mixed_vs_fp64_gpu"] = out["value"] / out["fp64_gpu"]["value"]

    # conventional FCA EM on the GPU, same data and precision, from the same model
    Pinv = torch.linalg.inv(P_init.cpu()).to(dev)  # setup only (CPU LAPACK)
    S0 = ((Pinv.conj().transpose(1, 2)[:, None] * lam_init[:, :, None, :].to(torch.complex128))
          @ Pinv[:, None]).contiguous()
    vf = v_init.clone()
    ef = ffca.FCA(yd, vf, S0, N=N)
    ef.iterate(1, trace=False)
    itf = 3
    msf = timed(lambda: ef.iterate(itf, trace=False), 1)
    ef.close()
    out["fca_gpu"] = {"value": N * F * itf / (msf * 1e-3), "unit": UNIT, "iters_timed": itf,
                      "ms_per_iter": msf / itf, "precision": "mixed (same as the FastFCA-AS run)"}
    out["speedup_vs_fca_gpu"] = out["value"] / out["fca_gpu"]["value"]
    del est, yd, vd, lamd, Pd, v_init, lam_init, P_init, vf, S0, Pinv
    torch.cuda.empty_cache()
    return out


def run_front_end(dev):
    """The STFT front end and overlap-add back end (Table 1 conditions) at the
    long mixture's size: the STFT of I = 3 channels of (N - 1) 512 + 1024
    samples (N = 20000 frames) and the inverse of the Wiener output's J I = 9
    spectra; algorithmic bytes = samples read + spectra written (or back);
    error against numpy's FFT on sampled frames."""
    import torch
    from paper_1805_09498_gb300 import ffca
    N, L, H = 20000, ffca.STFT_L, ffca.STFT_H
    S = (N - 1) * H + L
    g = torch.Generator(device=dev)
    g.manual_seed(31)
    x = torch.randn((3, S), generator=g, device=dev, dtype=torch.float32)
    X, n = ffca.stft(x)
    Xw = torch.randn((9, ffca.STFT_F, X.shape[2]), generator=g, device=dev, dtype=torch.complex64)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": f"STFT of 3 channels x {S} samples (N = {N} frames, F = 513) and inverse of 9 "
                       "spectra of the same size, c64 / float32"}
    for name, fn, byt in (("stft", lambda: ffca.stft(x), 3 * S * 4 + 3 * ffca.STFT_F * N * 8),
                          ("istft", lambda: ffca.istft(Xw, n), 9 * ffca.STFT_F * N * 8 + 9 * (N + 1) * H * 4)):
        for _ in range(3):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(10):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / 10
        out[name] = {"ms": ms, "bytes": byt, "achieved_gbs": byt / (ms * 1e-3) / 1e9}
    fr = [0, 1, 9999, N - 1]
    xs = x.cpu().double().numpy()
    w = np.sin(np.pi * np.arange(L) / L)
    ref = np.stack([np.fft.rfft(xs[:, k * H: k * H + L] * w, axis=-1) for k in fr], axis=-1)
    got = X[:, :, fr].cpu().numpy()
    out["stft"]["error_vs_numpy_fft"] = float(np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)))
    del x, X, Xw
    torch.cuda.empty_cache()
    return out


def run_batched(args, dev):
    """The batched workload: 256 mixtures of uneven length (I = 4, J = 3,
    F = 257, N uniform in [200, 4000]), complex64, 20 iterations, run as one
    batch (one launch per pass, the iteration loop replayed from a CUDA
    graph) and, as the comparison, as 256 sequential plain-FP64 runs of the
    single-mixture API on the same data.  Both timed with CUDA events."""
    import torch
    from paper_1805_09498_gb300 import ffca
    cfg = CONFIGS["batched"]
    I, J, F, M, iters = cfg["I"], cfg["J"], cfg["F"], cfg["M"], cfg["iters"]
    Ns = batch_lengths(M, cfg["N_min"], cfg["N_max"], seed=17)
    y, v, lam, P, Ns, off = make_batch_device(I, J, F, Ns, seed=23, device=dev, alpha=cfg["alpha"],
                                              kappa=cfg["kappa"])
    v_init, lam_init, P_init = v.clone(), lam.clone(), P.clone()
    units = int(np.sum(Ns)) * F * iters
    stream = torch.cuda.current_stream(dev)
    est = ffca.FastFCABatch(y, v, lam, P, Ns, graph=True)
    # partition autotuning on real iterations (setup, not timed), then back to the initial state
    cand_a, cand_b, ms_a, ms_b = est.autotune(rounds=2)
    v.copy_(v_init); lam.copy_(lam_init); P.copy_(P_init)

    def reset():
        v.copy_(v_init); lam.copy_(lam_init); P.copy_(P_init)

    def timed(fn, reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    for _ in range(max(args.warmup, 3)):
        est.iterate(iters, trace=False)
    reps = 5
    ffca.ffca_timing_read(est.ctx)
    ms = timed(lambda: est.iterate(iters, trace=False), reps)
    launches = int(sum(n for _, n in ffca.ffca_timing_read(est.ctx).values())) // reps
    # per-kernel times from one plain (non-graph) run with event timing
    ffca.ffca_set_graph(est.ctx, False)
    ffca.ffca_timing_enable(est.ctx, True)
    est.iterate(iters, trace=False)
    kt = ffca.ffca_timing_read(est.ctx)
    ffca.ffca_timing_enable(est.ctx, False)
    tf = int(np.sum(Ns)) * F
    kernels = {}
    for k, bpt in (("estep", I * 8 + 2 * J * 4), ("wcov", I * 8 + J * 4), ("psolve", 0), ("prep", 0)):
        kms, kn = kt[k]
        if kn:
            kernels[k] = {"launches": kn, "avg_us": kms / kn * 1e3}
            if bpt:
                kernels[k]["achieved_gbs"] = bpt * tf / (kms / kn * 1e-3) / 1e9
    reset()
    est.iterate(iters, trace=False)
    ll_b = est.loglik()
    torch.cuda.synchronize()
    vb, lb, Pb = v.clone(), lam.clone(), P.clone()
    est.close()

    # 256 sequential plain-FP64 runs on the same data (FP64 copies of each mixture)
    runs = []
    yv, vv0 = ffca.batch_views(y, I, F, off), ffca.batch_views(v_init, J, F, off)
    for m in range(M):
        n = int(Ns[m])
        ym = yv[m].to(torch.complex128).contiguous()
        vm = vv0[m].to(torch.float64).contiguous()
        lm, Pm = lam_init[m].clone(), P_init[m].clone()
        runs.append((ffca.FastFCA(ym, vm, lm, Pm, N=n), ym, vm, lm, Pm, vm.clone()))

    def seq():
        for r in runs:
            r[0].iterate(iters, trace=False)

    seq()  # warm-up, then back to the initial state
    for m, r in enumerate(runs):
        r[2].copy_(r[5]); r[3].copy_(lam_init[m]); r[4].copy_(P_init[m])
    ms_seq = timed(seq, 1)
    # accuracy of the batched mixed-precision result against the FP64 runs
    e = {"v": 0.0, "lambda": 0.0, "P": 0.0, "loglik_per_point": 0.0}
    vbv = ffca.batch_views(vb, J, F, off)
    for m, r in enumerate(runs):
        n = int(Ns[m])
        def rel(a_, b_):
            a_ = a_.reshape(F, -1) if a_.dim() > 1 else a_
            nrm = lambda t: t.abs().pow(2).sum(-1).sqrt()  # noqa: E731
            return float((nrm(a_ - b_.reshape(a_.shape)) / nrm(b_.reshape(a_.shape))).max())
        e["v"] = max(e["v"], rel(vbv[m][:, :, :n].double().permute(1, 0, 2).contiguous(),
                                 r[2][:, :, :n].permute(1, 0, 2).contiguous()))
        e["lambda"] = max(e["lambda"], rel(lb[m], r[3]))
        e["P"] = max(e["P"], rel(Pb[m], r[4]))
        e["loglik_per_point"] = max(e["loglik_per_point"], abs(ll_b[m] - r[0].loglik()) / (n * F))
    e["measure"] = ("batched mixed precision vs the sequential FP64 runs, after 20 iterations from "
                    "the same state; normwise relative error per frequency, max over mixtures")
    for r in runs:
        r[0].close()
    del runs, yv, vv0, vbv, y, v, lam, P, v_init, lam_init, P_init, vb, lb, Pb
    torch.cuda.empty_cache()
    return {"workload": f"batched: M={M} mixtures, I={I} J={J} F={F}, N uniform in "
                        f"[{cfg['N_min']}, {cfg['N_max']}] (total {int(np.sum(Ns))} frames), "
                        f"c64, {iters} iterations",
            "value": units / (ms * 1e-3), "unit": UNIT, "ms_per_run": ms, "runs_timed": reps,
            "graph": True, "gpu_launches_per_run": launches, "kernels": kernels,
            "autotune": {"chosen": {"pass_a": cand_a, "pass_b": cand_b},
                         "ms_per_candidate": {"pass_a": [round(x, 4) for x in ms_a],
                                              "pass_b": [round(x, 4) for x in ms_b]},
                         "candidates": "per-segment cost (frames) x grid waves; 0 = default"},
            "sequential_fp64": {"value": units / (ms_seq * 1e-3), "unit": UNIT, "ms_total": ms_seq,
                                "runs": M},
            "speedup_vs_sequential_fp64": ms_seq / ms, "error_vs_fp64": e}


def cpu_baseline_and_error(p, cfg, fs, gpu_state, tr_gpu, pool):
    """The FP64 oracle on bounded samples of the workload (all frames, all
    iterations), timed on the host: on one core over CPU_SAMPLE_F
    frequencies, and on all cores (one worker process per core, a block of
    frequencies each) over CPU_SAMPLE_F frequencies per worker; and the GPU
    result's error against the one-core run on its frequencies."""
    from oracle import fastfca_as as ffa
    from oracle.fastfca_as import OpCounter
    iters, N, F = cfg["iters"], cfg["N"], cfg["F"]
    t = time.perf_counter()
    v, lam, P, tr = ffa.iterate(p.y[:, fs], p.v0[:, fs], p.lam0[fs], p.P0[fs], iters,
                                counter=OpCounter())
    dt = time.perf_counter() - t
    fa = _sample_freqs(F, min(F, CPU_SAMPLE_F * pool.workers))
    _, dt_all = pool.run(_fastfca_jobs(p.y[:, fa], p.v0[:, fa], p.lam0[fa], p.P0[fa], iters, pool.workers))

    def relerr(a, b, ax):
        a = np.moveaxis(a, ax, 0).reshape(len(fs), -1)
        b = np.moveaxis(b, ax, 0).reshape(len(fs), -1)
        return float(np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)))

    vg, lg, Pg = gpu_state
    err = {"v": relerr(vg, v, 1), "lambda": relerr(lg, lam, 0), "P": relerr(Pg, P, 0),
           "loglik_per_point": abs(ffa.loglik(p.y[:, fs], vg, lg, Pg) - tr[-1]) / (len(fs) * N),
           "measure": f"after {iters} iterations from the same initial state, on the sampled "
                      "frequencies; normwise relative error per frequency (max)"}
    return {"value": len(fa) * N * iters / dt_all, "unit": UNIT, "cores": pool.workers, "kind": "oracle",
            "sample": f"{len(fa)} of {F} frequencies x {N} frames x {iters} iterations, numpy FP64, "
                      f"{pool.workers} worker processes of one thread (a block of frequencies each)",
            "seconds": dt_all,
            "one_core": {"value": len(fs) * N * iters / dt, "cores": 1, "seconds": dt,
                         "sample": f"{len(fs)} of {F} frequencies x {N} frames x {iters} iterations"},
            "error_vs_oracle": err}


# ---------------------------------------------------------------- profiling case
def run_case(a):
    """One fixed, small run for kernel profiling (e.g. under ncu), not timed:
    `iters` hybrid iterations and one Wiener pass of a seeded mixture of the
    given shape (P drawn with alpha = 0.3, cond < 10, or alpha = 0.2,
    cond < 50 for I = 8), or with --case-batch M, a batch of M mixtures with
    lengths uniform in [200, 4000] through the batch API, or with --case-stft,
    `iters` rounds of the STFT of I channels of N frames and its inverse."""
    import torch
    from paper_1805_09498_gb300 import build as _build
    from paper_1805_09498_gb300 import ffca
    _build.build()
    alpha, kappa = (0.2, 50.0) if a.case_I == 8 else (0.3, 10.0)
    if a.case_stft:
        S = (a.case_N - 1) * ffca.STFT_H + ffca.STFT_L
        g = torch.Generator(device="cuda")
        g.manual_seed(31)
        x = torch.randn((a.case_I, S), generator=g, device="cuda", dtype=torch.float32)
        for _ in range(a.case_iters):
            X, n = ffca.stft(x)
            xr = ffca.istft(X, n)
        torch.cuda.synchronize()
        err = float((xr[:, ffca.STFT_L:S - ffca.STFT_L] - x[:, ffca.STFT_L:S - ffca.STFT_L]).abs().max())
        print("case done; STFT round trip max error:", err)
        return
    if a.case_batch:
        cdt = torch.complex64 if a.case_prec == "mixed" else torch.complex128
        Ns = batch_lengths(a.case_batch, 200, 4000, seed=17)
        y, v, lam, P, Ns, _ = make_batch_device(a.case_I, a.case_J, a.case_F, Ns, seed=23, device="cuda",
                                                alpha=alpha, kappa=kappa, complex_dtype=cdt)
        est = ffca.FastFCABatch(y, v, lam, P, Ns)
        if a.case_p_update != "fixed_point":
            est.set_p_update(a.case_p_update, a.case_mu)
        tr = est.iterate(a.case_iters)
        torch.cuda.synchronize()
        est.close()
    else:
        p = make_problem(a.case_I, a.case_J, a.case_F, a.case_N, seed=0, alpha=alpha, kappa=kappa)
        yd, vd, lamd, Pd, N = ffca.to_device(p.y, p.v0, p.lam0, p.P0, prec=a.case_prec)
        est = ffca.FastFCA(yd, vd, lamd, Pd, N=N)
        if a.case_p_update != "fixed_point":
            est.set_p_update(a.case_p_update, a.case_mu)
        if a.case_resident:
            est.set_resident(True)
        tr = est.iterate(a.case_iters)
        est.wiener()
        torch.cuda.synchronize()
        est.close()
    print("case done; L2 trace:", tr[0], "->", tr[-1])


# ---------------------------------------------------------------- reference arm
def _reference_worker(conn, y, v, lam, P):
    """One host core of the reference arm: holds its block of frequencies and
    runs one hybrid iteration with its L2 per message."""
    from oracle import fastfca_as as ffa
    from oracle.fastfca_as import OpCounter
    cnt = OpCounter()
    conn.send("ready")
    while conn.recv() is not None:
        ffa.loglik(y, v, lam, P)
        v, lam, P = ffa.hybrid_iteration(y, v, lam, P, 1, cnt)
        conn.send("done")


def run_reference(args, cfg, rank, ws):
    """The FP64 oracle on the host cores as the reference arm: one worker
    process per core (one numpy thread each, started with spawn), each
    holding a block of CPU_SAMPLE_F of the workload's frequencies; a step is
    one hybrid iteration with its L2 on every block, the workers in
    parallel."""
    if rank != 0:
        return None
    import multiprocessing as mp
    I, J, F, N = cfg["I"], cfg["J"], cfg["F"], cfg["N"]
    workers = os.cpu_count() or 1
    p = make_problem(I, J, F, N, seed=0, alpha=cfg["alpha"], kappa=cfg["kappa"])
    fs = _sample_freqs(F, min(F, CPU_SAMPLE_F * workers))
    blocks = [b for b in np.array_split(fs, workers) if len(b)]
    ctx = mp.get_context("spawn")
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    procs, conns = [], []
    for b in blocks:
        a, c = ctx.Pipe()
        pr = ctx.Process(target=_reference_worker, args=(c, p.y[:, b], p.v0[:, b], p.lam0[b], p.P0[b]),
                         daemon=True)
        pr.start()
        procs.append(pr)
        conns.append(a)
    for c in conns:
        c.recv()

    def step():
        for c in conns:
            c.send(1)
        for c in conns:
            c.recv()

    for _ in range(args.warmup):
        step()
    t = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t
    for c in conns:
        c.send(None)
    for pr in procs:
        pr.join(timeout=30)
    value = len(fs) * N * args.steps / dt
    sample = (f"{len(fs)} of {F} frequencies x {N} frames, one hybrid iteration + L2 per step, numpy FP64, "
              f"{len(blocks)} worker processes of one thread (a block of frequencies each)")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{WORKLOAD}: I={I} J={J} F={F} N={N}", "parallelism": "cpu"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": len(blocks), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--case", action="store_true",
                    help="run one small untimed case for profiling (the --case-* options) and exit")
    ap.add_argument("--case-I", type=int, default=3)
    ap.add_argument("--case-J", type=int, default=3)
    ap.add_argument("--case-F", type=int, default=513)
    ap.add_argument("--case-N", type=int, default=8000)
    ap.add_argument("--case-iters", type=int, default=2)
    ap.add_argument("--case-prec", choices=("mixed", "fp64"), default="mixed")
    ap.add_argument("--case-batch", type=int, default=0, help="mixtures of a batch (0: one mixture)")
    ap.add_argument("--case-p-update", default="fixed_point")
    ap.add_argument("--case-mu", type=float, default=0.0)
    ap.add_argument("--case-resident", action="store_true",
                    help="iterate with each problem resident on chip (ffca_set_resident)")
    ap.add_argument("--case-stft", action="store_true",
                    help="the STFT of I channels of N frames and the inverse of I spectra instead")
    args = ap.parse_args()
    if args.case:
        run_case(args)
        return
    cfg = CONFIGS[WORKLOAD]
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        ws = int(os.environ.get("WORLD_SIZE", "1"))
        res = run_reference(args, cfg, rank, ws)
    else:
        rank, ws, local, dist = _dist()
        res = run_ours(args, cfg, rank, ws, local, dist)
        if dist is not None:
            dist.destroy_process_group()
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
