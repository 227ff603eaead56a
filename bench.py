"""Benchmark of the fictitious-wave FDTD forward solve on B300.

One benchmark step = one complete forward solve (every leapfrog step of the
time loop, CPML, source injection, receiver DTFT, Green's functions) of the
marine 1-D VTI workload on its 128 x 128 x 96-node non-uniform grid
(162 x 162 x 130 padded samples, 4th order, 3 frequencies, 64 receivers).
The metric is padded cell-steps per second (Gcell-steps/s).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank solves its own
transmitter position (sources are independent problems, weak scaling); the
only collective is the max over ranks of the timed duration.

``--impl reference`` times the FP64 CPU oracle (the reference arm) on the
host cores, each step a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2304_00233_b300 import workloads as W  # noqa: E402

WORKLOAD = "marine_1d_128x128x96"


def _slab_cells(wl):
    np1, np2, np3 = wl.npad
    nb2 = 2 * wl.nb
    return nb2 * np2 * np3 + np1 * nb2 * np3 + np1 * np2 * nb2


def algorithmic_bytes(wl):
    """Bytes per leapfrog step the method must move at minimum (FP32):
    6 fields read + written and 3 dt/eps read = 60 B per padded cell, plus
    4 CPML memory arrays read + written (32 B) per cell and per axis whose
    slab it lies in, plus 32 B per compensated volume-DTFT accumulator."""
    cells = int(np.prod(wl.npad))
    b = 60 * cells + 32 * _slab_cells(wl)
    if wl.volume:
        b += 32 * 6 * len(wl.freqs) * int(np.prod(wl.shape))
    return b


def per_kernel_bytes(wl):
    """Minimal bytes of each half-step launch of the two-launch step:
    E launch reads H, E, dt/eps and writes E (48 B/cell); H launch reads E, H
    and writes H (36 B/cell); each has 2 CPML arrays per slab axis."""
    cells = int(np.prod(wl.npad))
    vol = 32 * 3 * len(wl.freqs) * int(np.prod(wl.shape)) if wl.volume else 0
    return 48 * cells + 16 * _slab_cells(wl) + vol, 36 * cells + 16 * _slab_cells(wl) + vol


def kernel_fingerprint():
    """Short sha256 of the stencil kernels' source with comments and spacing
    removed: a DRAM traffic figure recorded by ncu is only reported while the
    kernels it was taken from are unchanged."""
    h = hashlib.sha256()
    for f in ("emm_kernels.cu", "emm_internal.h"):
        with open(os.path.join(ROOT, "paper_2304_00233_b300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", re.sub(r"//[^\n]*", "", src), flags=re.S)
        h.update(re.sub(r"\s+", " ", src).strip().encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload):
    """DRAM bytes (read + write) of one leapfrog step (E + H launch) from the
    ncu summary of this workload, or None if there is none for the current
    kernels."""
    p = os.path.join(ROOT, "profiles", f"k_update_{workload}.md")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        m = re.search(r"traffic-record: fingerprint=(\w+) bytes_per_step=(\d+)", fh.read())
    if not m or m.group(1) != kernel_fingerprint():
        return None
    return int(m.group(2))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # the raw samples go to BENCH_LOG_DIR (default: the system's temporary
        # directory); the JSON line carries their summary
        log_dir = os.environ.get("BENCH_LOG_DIR") or tempfile.gettempdir()
        self.path = os.path.join(log_dir, f"emm_bench_clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(wl, nt):
    """Wall time of `nt` oracle steps (setup subtracted)."""
    import oracle
    t0 = time.perf_counter()
    oracle.forward_workload(wl, nt=0)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.forward_workload(wl, nt=nt)
    return max(time.perf_counter() - t0 - t_setup, 1e-9)


def cpu_baseline(wl, budget_s=15.0):
    import oracle
    threads = oracle.threads()
    probe_nt = 4
    t = oracle_sample(wl, probe_nt)
    nt = int(min(400, max(8, budget_s / (t / probe_nt))))
    t = oracle_sample(wl, nt)
    cells = int(np.prod(wl.npad))
    return {"value": cells * nt / t / 1e9, "unit": "Gcell-steps/s", "cores": threads, "kind": "oracle",
            "sample": f"{nt} leapfrog steps of {wl.name} (FP64 oracle, {threads} OpenMP threads), "
                      f"{t:.1f} s"}


# ---- multi-GPU (one process per GPU): sharding over transmitters ----
TOW_SPACING = 200.0  # m between the transmitters of consecutive ranks


def rank_source(src, rank):
    """Transmitter of rank `rank`: the workload's, shifted along the tow line
    (x) by rank * 200 m.  Sources are independent problems, so ranks share
    nothing but the timing (weak scaling)."""
    return np.asarray(src, dtype=np.float64) + np.array([TOW_SPACING * rank, 0.0, 0.0])


def max_over_ranks(v, dist=None, device="cpu"):
    """The slowest rank's value (the job's time): all-reduce MAX, or v itself
    in a single process."""
    if dist is None:
        return float(v)
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world, cells, nt, steps, seconds):
    """Whole-job throughput in Gcell-steps/s: every rank advances `cells`
    padded cells `nt` steps per solve, `steps` solves, in `seconds`."""
    return world * cells * nt * steps / seconds / 1e9


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle on the host cores, each step a
    bounded sample (a fixed number of leapfrog steps) of the same workload."""
    if rank != 0:
        return 0
    import oracle
    wl = W.WORKLOADS[args.workload]()
    threads = oracle.threads()
    cells = int(np.prod(wl.npad))
    probe = oracle_sample(wl, 2) / 2
    # each step: enough leapfrog steps for ~90 s over the whole run
    nt = int(min(400, max(2, 90.0 / max(1, args.steps + args.warmup) / probe)))
    for _ in range(args.warmup):
        oracle_sample(wl, nt)
    times = [oracle_sample(wl, nt) for _ in range(args.steps)]
    tot = sum(times)
    value = cells * nt * args.steps / tot / 1e9
    line = {"metric": "FDTD forward Gcell-steps/s", "value": value, "unit": "Gcell-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": wl.name, "padded_cells": cells, "timesteps_per_step": nt,
                       "note": "each step is a bounded sample of the solve's leapfrog steps"},
            "cpu_baseline": {"value": value, "unit": "Gcell-steps/s", "cores": threads, "kind": "oracle",
                             "sample": f"{nt} leapfrog steps of {wl.name} per step"},
            "e2e": {"value": value, "unit": "Gcell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def gradient_survey_line(emm, torch, stream, job_max):
    """Least-squares misfit gradient of the 8-transmitter gradient survey
    (192 x 192 x 128 NU grid): observed data from the model with the
    resistor plus 2 % noise (not timed), then the misfit and its gradient
    with respect to the cell sigma_h, sigma_v at the model without it, with
    the E snapshots of as many final steps as the free device memory holds;
    against one forward solve per transmitter on the same grid."""
    import dataclasses
    # release the allocator's cached blocks first: a tensor allocated inside
    # a large cached block (the earlier gradient's workspace) would pin it
    gc.collect()
    torch.cuda.empty_cache()
    wl = W.gradient_survey(with_resistor=False)
    obs = W.gradient_survey(with_resistor=True)
    grid = emm.grid_for(wl)
    smin = float(obs.sigma.min())
    dt, _, _ = grid.time_step(smin, wl.omega0)
    nt = int(np.ceil(wl.t_max / dt))
    survey = emm.survey_for(wl, nt=nt, sigma_min=smin)
    pos = W.GRADIENT_SOURCES
    sig_obs = torch.from_numpy(obs.sigma.astype(np.float32)).cuda()
    G_obs, bwork = emm.forward_batch(grid, survey, sig_obs, pos)
    d = G_obs.cpu().numpy() * W.observed_noise(G_obs.shape)
    del bwork, sig_obs, G_obs
    sh = torch.from_numpy(wl.sigma_h).cuda()
    sv = torch.from_numpy(wl.sigma_v).cuda()
    sigma = emm.stagger_sigma(grid, sh, sv)
    work = emm.Workspace(grid, survey)
    emm.forward_async(grid, survey, sigma, work)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    emm.forward_async(grid, survey, sigma, work)
    f1.record(stream)
    torch.cuda.synchronize()
    assert emm.status(work) == emm.EMM_OK
    fwd_ms = job_max(f0.elapsed_time(f1) / 1e3) * 1e3
    del work
    ck = max(1, int(round(nt ** 0.5)))
    gc.collect()
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    print(f"gradient survey: {free / 1e9:.1f} GB free, {torch.cuda.memory_allocated() / 1e9:.1f} GB allocated, "
          f"{torch.cuda.memory_reserved() / 1e9:.1f} GB reserved by torch", file=sys.stderr)
    room = free - (6 << 30)
    snap = emm.snapshot_bytes(grid, survey, ck)
    stored = min(nt, int(max(0, room) // snap)) // ck * ck
    while stored > 0 and emm.gradient_workspace_size(grid, survey, ck, stored) > room:
        stored -= ck
    # warm-up on a short run of the same problem
    emm.survey_misfit_gradient(grid, dataclasses.replace(survey, nt=2 * ck), sh, sv, pos[:1], d[:1],
                               ckpt_every=ck)
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    misfit, gh, gv, _ = emm.survey_misfit_gradient(grid, survey, sh, sv, pos, d, ckpt_every=ck,
                                                   stored_steps=stored)
    g1.record(stream)
    torch.cuda.synchronize()
    ms = job_max(g0.elapsed_time(g1) / 1e3) * 1e3
    ok = bool(torch.isfinite(gh).all().item() and torch.isfinite(gv).all().item())
    return {"workload": "gradient_survey_192x192x128", "nsrc": len(pos), "timesteps_per_solve": nt,
            "cells": grid.cells, "ms": ms, "forward_ms": fwd_ms, "ratio_to_forward": ms / (len(pos) * fwd_ms),
            "ckpt_every": ck, "stored_steps": stored, "snapshot_gb": stored * snap / 1e9,
            "free_gb_before": free / 1e9, "misfit": misfit.item(), "finite": ok,
            "what": "emm_stagger_sigma, then per transmitter emm_misfit_gradient (forward sweep, residual "
                    "of the noisy resistor-model data, adjoint sweep) and emm_stagger_sigma_adjoint into "
                    "the sigma_h, sigma_v gradients; ratio against one forward solve per transmitter"}


def graph_line(emm, torch, stream, job_max, grid, survey, sigma, work, steps, rate, value):
    """The benchmark solve replayed `steps` times from a CUDA graph of its
    time loop (emm_plan_create once, emm_plan_run per solve)."""
    t0 = time.perf_counter()
    plan = emm.Plan(grid, survey, sigma, work)
    torch.cuda.synchronize()
    capture_ms = 1e3 * (time.perf_counter() - t0)
    plan.run_async(sigma)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(steps):
        plan.run_async(sigma)
    p1.record(stream)
    torch.cuda.synchronize()
    assert emm.status(work) == emm.EMM_OK
    gval = rate(job_max(p0.elapsed_time(p1) / 1e3))
    del plan
    return {"value": gval, "unit": "Gcell-steps/s", "vs_stream_launches": gval / value,
            "capture_and_instantiate_ms": capture_ms,
            "what": "emm_plan_run: the solve's time loop captured once as a CUDA graph and replayed"}


def jobs_line(emm, torch, stream, job_max):
    """The uneven-grid work list (3 x 96^3, 3 x 160 x 160 x 120, 2 x 200 x
    200 x 140 nodes, each with its own transmitter): the eight forward solves
    one after the other (emm_forward each), against emm_forward_jobs with the
    work-list launches and with the strategy emm_jobs_tune picks."""
    import dataclasses
    wls = W.uneven_jobs()
    probs, sig, works, cells, steps = [], [], [], 0, 0
    for wl in wls:
        g = emm.grid_for(wl)
        nt = emm.steps_for(wl, g)
        probs.append((g, emm.survey_for(wl, nt=nt)))
        sig.append(torch.from_numpy(wl.sigma.astype(np.float32)).cuda())
        works.append(emm.Workspace(g, probs[-1][1]))
        cells += g.cells * nt
        steps = max(steps, nt)
    short = [(g, dataclasses.replace(s, nt=30)) for g, s in probs]
    for (g, s), sg, w in zip(short, sig, works):
        emm.forward_async(g, s, sg, w)
    emm.forward_jobs(short, sig, strategy=emm.JOBS_LIST)
    jw = emm.JobsWork(probs)
    best, tune_ms = emm.jobs_tune(probs, sig, jw, steps=40)
    torch.cuda.synchronize()

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        return job_max(a.elapsed_time(b) / 1e3)

    def one_at_a_time():
        for (g, s), sg, w in zip(probs, sig, works):
            emm.forward_async(g, s, sg, w)

    seq = timed(one_at_a_time)
    for (g, s), w in zip(probs, works):
        assert emm.status(w) == emm.EMM_OK
    rates = {}
    for k in sorted({emm.JOBS_LIST, best}):
        t = timed(lambda: emm.forward_jobs(probs, sig, work=jw, check=False, strategy=k))
        assert all(st == emm.EMM_OK for st in jw.status())
        same = all(torch.equal(torch.view_as_complex(r)[: s.nrec], torch.view_as_complex(w.rec)[: s.nrec])
                   for r, w, (_, s) in zip(jw.rec, works, probs))
        rates[emm.JOBS_STRATEGIES[k]] = {"value": cells / t / 1e9, "ms": 1e3 * t, "bitwise_equal": same}
    return {"problems": [w.name for w in wls], "cell_steps": cells, "max_timesteps": steps,
            "value": rates[emm.JOBS_STRATEGIES[best]]["value"], "unit": "Gcell-steps/s",
            "strategy": emm.JOBS_STRATEGIES[best], "one_at_a_time": cells / seq / 1e9,
            "speedup": seq / (rates[emm.JOBS_STRATEGIES[best]]["ms"] / 1e3), "ms_one_at_a_time": 1e3 * seq,
            "strategies": rates, "tune_ms_40_steps": tune_ms,
            "what": "emm_forward_jobs by the strategy emm_jobs_tune picks (and by work-list launches: one E "
                    "and one H launch per step over the tiles of all eight grids) against emm_forward of each "
                    "problem in turn, device-resident inputs"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(W.WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-gradient", action="store_true",
                    help="skip the gradient / forward time ratio (one emm_gradient call after the timed region)")
    ap.add_argument("--graph", action="store_true",
                    help="add the CUDA-graph line (the solve replayed from a captured time loop)")
    ap.add_argument("--no-jobs", action="store_true",
                    help="skip the uneven-grid work-list line (eight grids, one launch per half-step)")
    ap.add_argument("--no-gradient-survey", action="store_true",
                    help="skip the 8-transmitter misfit-gradient line on the 192 x 192 x 128 grid (about a minute)")
    ap.add_argument("--no-airwave", action="store_true",
                    help="skip the air-boundary line (uniform-xy marine model with and without air on top)")
    ap.add_argument("--batch", type=int, default=32,
                    help="transmitters of the batched-survey line (emm_forward_batch; 0 = skip)")
    ap.add_argument("--timesteps", type=int, default=0,
                    help="override the leapfrog steps per solve (short profiling runs only)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import paper_2304_00233_b300 as emm
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    wl = W.WORKLOADS[args.workload]()
    # weak scaling: rank r solves the transmitter shifted 200 m along the tow line
    wl.src = rank_source(wl.src, rank)
    grid = emm.grid_for(wl)
    nt = args.timesteps if args.timesteps > 0 else emm.steps_for(wl, grid)
    survey = emm.survey_for(wl, nt=nt)
    cells = grid.cells
    sigma_host = torch.from_numpy(wl.sigma.astype(np.float32)).pin_memory()
    sigma = sigma_host.cuda()
    work = emm.Workspace(grid, survey)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        emm.forward_async(grid, survey, sigma, work)
    torch.cuda.synchronize()
    assert emm.status(work) == emm.EMM_OK

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def job_max(v):
        return max_over_ranks(v, dist, "cuda")

    # ---- timed region: K device-resident solves ----
    e_ms, h_ms, loop_ms = [], [], []
    with ClockSampler(local) as clk:
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            t = emm.forward_timed(grid, survey, sigma, work, every=64)
            e_ms.append(t["e_ms"])
            h_ms.append(t["h_ms"])
            loop_ms.append(t["loop_ms"])
        ev1.record(stream)
        barrier()
    elapsed = job_max(ev0.elapsed_time(ev1) / 1e3)
    clocks = clk.summary()
    value = aggregate_rate(world, cells, nt, args.steps, elapsed)

    # ---- e2e: pinned host sigma in, receiver Green's functions out ----
    rec_host = torch.empty(work.rec.shape, dtype=work.rec.dtype).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sig_dev = sigma_host.to("cuda", non_blocking=True)
        emm.forward_async(grid, survey, sig_dev, work)
        rec_host.copy_(work.rec, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = job_max(time.perf_counter() - t0)
    barrier()
    e2e_value = aggregate_rate(world, cells, nt, args.steps, e2e_s)

    peak, peak_kind = measured_peaks()
    e_mean, h_mean = float(np.mean(e_ms)), float(np.mean(h_ms))
    alg = algorithmic_bytes(wl)
    be, bh = per_kernel_bytes(wl)
    # one leapfrog step as the time loop runs it: E and H back to back, each
    # launch a programmatic dependent of the one before
    step_s = float(np.mean(loop_ms)) / nt / 1e3
    achieved = alg / step_s / 1e9
    kernel_launches = args.steps * (1 + 2 * nt + (1 if survey.nrec else 0) + (1 if survey.volume else 0))
    line = {
        "metric": "FDTD forward Gcell-steps/s", "value": value, "unit": "Gcell-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "grid_nodes": list(wl.shape), "padded": list(grid.npad),
                   "padded_cells": cells, "rd": wl.rd, "timesteps_per_solve": nt,
                   "nfreq": len(wl.freqs), "nrec": survey.nrec, "volume_dtft": bool(wl.volume),
                   "parallelism": f"{world} independent transmitters" if world > 1 else "single GPU",
                   "l2": "no flush: per-solve working set (fields, 1/eps, CPML) exceeds the 126 MB L2"},
        "roofline": {"bound": "hbm", "kernel": "leapfrog step = k_update_E + k_update_H",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": ("of measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
                                   if peak_kind == "measured" else "of fallback 6.4 TB/s"),
                     "algorithmic_bytes_per_step": alg, "step_ms": 1e3 * step_s,
                     "step_ms_from": "CUDA events around the whole time loop / leapfrog steps",
                     "isolated_step_ms": e_mean + h_mean,
                     "traffic": recorded_traffic(wl.name),
                     "kernels": {"k_update_E": {"ms": e_mean, "min_bytes": be, "gbs": be / e_mean / 1e6},
                                 "k_update_H": {"ms": h_mean, "min_bytes": bh, "gbs": bh / h_mean / 1e6}}},
        "e2e": {"value": e2e_value, "unit": "Gcell-steps/s",
                "h2d_bytes_per_step": int(sigma_host.numel() * 4),
                "d2h_bytes_per_step": int(rec_host.numel() * 8)},
        "gpu_launches": kernel_launches,
        "clocks": clocks,
    }
    # the same solve replayed from a CUDA graph of its time loop (emm_plan);
    # opt-in (--graph): a default run that included it did not finish
    if args.graph:
        line["graph"] = graph_line(emm, torch, stream, job_max, grid, survey, sigma, work, args.steps,
                                   lambda sec: aggregate_rate(world, cells, nt, args.steps, sec), value)
    if args.batch > 0:
        # batched survey: transmitters every 200 m along the tow line
        # (x = -3100 + 200 k, 50 m above the seabed), advanced together;
        # a short warm-up run, one timed solve (CUDA events)
        import dataclasses
        pos = np.array([[-3100.0 + TOW_SPACING * (k + args.batch * rank), 0.0, float(wl.src[2])]
                        for k in range(args.batch)])
        emm.forward_batch(grid, dataclasses.replace(survey, nt=30), sigma, pos)
        bwork = torch.empty(emm.batch_workspace_size(grid, survey, len(pos)) + 256, dtype=torch.uint8,
                            device=sigma.device)
        torch.cuda.synchronize()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        emm.forward_batch(grid, survey, sigma, pos, work=bwork)  # (checks the device status)
        b1.record(stream)
        torch.cuda.synchronize()
        bsec = job_max(b0.elapsed_time(b1) / 1e3)
        bval = aggregate_rate(world, cells * args.batch, nt, 1, bsec)
        del bwork
        # the same with the first 8 transmitters only
        few = pos[: min(8, len(pos))]
        _, fwork = emm.forward_batch(grid, dataclasses.replace(survey, nt=30), sigma, few)
        fwork = torch.empty(emm.batch_workspace_size(grid, survey, len(few)) + 256, dtype=torch.uint8,
                            device=sigma.device)
        torch.cuda.synchronize()
        b0.record(stream)
        emm.forward_batch(grid, survey, sigma, few, work=fwork)
        b1.record(stream)
        torch.cuda.synchronize()
        fval = aggregate_rate(world, cells * len(few), nt, 1, job_max(b0.elapsed_time(b1) / 1e3))
        del fwork
        line["batch"] = {"nsrc": args.batch, "value": bval, "unit": "Gcell-steps/s", "ms_per_solve": 1e3 * bsec,
                         "vs_one_at_a_time": bval / value,
                         "nsrc_8": {"value": fval, "vs_one_at_a_time": fval / value},
                         "what": "emm_forward_batch: transmitters sharing grid, sigma and receivers in the same "
                                 "launches, against the device-resident single-transmitter value"}
    if not args.no_airwave and wl.name.startswith("marine"):
        # top boundary with air (Sec. 3.3): the marine model on a grid uniform
        # in x and y, one warm-up and one timed solve with and without air
        awl = W.marine_1d_air()
        agrid = emm.grid_for(awl)
        ant = emm.steps_for(awl, agrid)
        asig = torch.from_numpy(awl.sigma.astype(np.float32)).cuda()
        acells = agrid.cells
        rates = {}
        for air in (False, True):
            asurvey = emm.survey_for(awl, nt=ant, airwave=air)
            awork = emm.Workspace(agrid, asurvey)
            emm.forward_async(agrid, asurvey, asig, awork)
            torch.cuda.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            emm.forward_async(agrid, asurvey, asig, awork)
            a1.record(stream)
            torch.cuda.synchronize()
            assert emm.status(awork) == emm.EMM_OK
            rates[air] = aggregate_rate(world, acells, ant, 1, job_max(a0.elapsed_time(a1) / 1e3))
            del awork
        line["airwave"] = {"workload": awl.name, "value": rates[True], "unit": "Gcell-steps/s",
                           "without_air": rates[False], "overhead": rates[False] / rates[True],
                           "timesteps_per_solve": ant,
                           "what": "forward solve with air above the sea surface (plane DFTs after every "
                                   "half step) against the same model with CPML on the top face"}
    if not args.no_gradient:
        # gradient of Re(sum conj(v) G) for a seeded cotangent v: one warm-up
        # call, one timed call (CUDA events), against one forward solve
        rng = np.random.default_rng(230400237)
        v = rng.standard_normal((survey.nrec, 6, len(wl.freqs))) + 1j * rng.standard_normal(
            (survey.nrec, 6, len(wl.freqs)))
        vt = torch.from_numpy(v).cuda()
        ck = max(1, int(round(nt ** 0.5)))
        emm.vjp(grid, survey, sigma, vt, ckpt_every=ck)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        emm.vjp(grid, survey, sigma, vt, ckpt_every=ck, check=False)
        g1.record(stream)
        torch.cuda.synchronize()
        grad_ms = job_max(g0.elapsed_time(g1) / 1e3) * 1e3
        fwd_ms = 1e3 * elapsed / args.steps
        # the same with the E snapshots of as many final steps as the free
        # device memory holds (less 6 GB for the outputs and the allocator),
        # which the reverse sweep then does not recompute
        gc.collect()
        torch.cuda.empty_cache()
        free, _ = torch.cuda.mem_get_info()
        snap = emm.snapshot_bytes(grid, survey, ck)
        room = free - (6 << 30)
        stored = min(nt, int(max(0, room) // snap)) // ck * ck
        while stored > 0 and emm.gradient_workspace_size(grid, survey, ck, stored) > room:
            stored -= ck
        emm.vjp(grid, survey, sigma, vt, ckpt_every=ck, stored_steps=stored, check=False)
        torch.cuda.synchronize()
        g0.record(stream)
        emm.vjp(grid, survey, sigma, vt, ckpt_every=ck, stored_steps=stored, check=False)
        g1.record(stream)
        torch.cuda.synchronize()
        st_ms = job_max(g0.elapsed_time(g1) / 1e3) * 1e3
        line["gradient"] = {"ms": st_ms, "forward_ms": fwd_ms, "ratio_to_forward": st_ms / fwd_ms,
                            "ckpt_every": ck, "stored_steps": stored,
                            "snapshot_gb": stored * snap / 1e9,
                            "recompute_only_ms": grad_ms, "ratio_recompute_only": grad_ms / fwd_ms,
                            "what": "emm_gradient_stored: forward sweep keeping checkpoints and the E snapshots "
                                    "of the last stored_steps steps in device memory, recomputation of the "
                                    "earlier segments and the adjoint sweep, one cotangent of all receiver "
                                    "data; recompute_only: every segment recomputed (emm_gradient)"}
    if not args.no_jobs:
        line["jobs"] = jobs_line(emm, torch, stream, job_max)
    if not args.no_gradient_survey:
        line["gradient_survey"] = gradient_survey_line(emm, torch, stream, job_max)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(W.WORKLOADS[args.workload]())
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
