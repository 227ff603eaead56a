"""Benchmark of the fictitious-wave FDTD forward solve on B300.

One benchmark step = one complete forward solve (every leapfrog step of the
time loop, CPML, source injection, receiver and volume DTFT, Green's
functions) of the 3-D anomaly workload: 256 x 256 x 160 non-uniform nodes
(294 x 294 x 198 padded samples), 8th order, 3 frequencies, 201 receivers
and the volume DTFT of all six components over the 10.5 M interior samples.
The metric is padded cell-steps per second (Gcell-steps/s).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank solves its own
transmitter position (sources are independent problems, weak scaling); the
collectives are the max over ranks of the timed duration, one gather of the
receiver Green's functions to rank 0 after the timed region, and, in the
gradient-survey line, the sum of the per-transmitter gradients.

``--impl reference`` times the FP64 CPU oracle (the reference arm) on the
host cores, each step a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import platform
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

WORKLOAD = "anomaly_3d_256x256x160"
MARINE = "marine_1d_128x128x96"
E2E_SOLVES = 3          # end-to-end solves timed (each reads back the volume)
GOLDEN_DIR = os.path.join(ROOT, "tests", "golden")


def log(msg):
    """A progress line on stderr (the JSON result line goes to stdout)."""
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def _slab_cells(wl):
    np1, np2, np3 = wl.npad
    nb2 = 2 * wl.nb
    return nb2 * np2 * np3 + np1 * nb2 * np3 + np1 * np2 * nb2


def algorithmic_bytes(wl, ring):
    """Bytes per leapfrog step the method must move at minimum (FP32):
    6 fields read + written and 3 dt/eps read = 60 B per padded cell, plus
    4 CPML memory arrays read + written (32 B) per cell and per axis whose
    slab it lies in, plus, with the volume DTFT, 32 B per compensated
    accumulator (read + written) once per `ring` steps: the DTFT of `ring`
    steps is added to each accumulator in one pass."""
    cells = int(np.prod(wl.npad))
    b = 60 * cells + 32 * _slab_cells(wl)
    if wl.volume:
        b += 32 * 6 * len(wl.freqs) * int(np.prod(wl.shape)) // ring
    return b


def per_kernel_bytes(wl, ring):
    """Minimal bytes of each launch, per leapfrog step: the E launch reads H,
    E, dt/eps and writes E (48 B/cell), the H launch reads E, H and writes H
    (36 B/cell), each with 2 CPML arrays read + written per slab axis; a
    volume-DTFT launch reads the six fields of each of its `ring` steps (24 B
    per interior sample and step) and reads + writes its 6 x nfreq
    compensated accumulators (32 B each) once."""
    cells = int(np.prod(wl.npad))
    nint = int(np.prod(wl.shape))
    vol = (24 * ring + 32 * 6 * len(wl.freqs)) * nint / ring if wl.volume else 0
    return {"k_update_E": 48 * cells + 16 * _slab_cells(wl), "k_update_H": 36 * cells + 16 * _slab_cells(wl),
            "k_volume_dft": vol}


def bench_config(wl, nt, world):
    """The `config` object of both arms (same keys and values)."""
    return {"workload": wl.name, "grid_nodes": list(wl.shape), "padded": list(wl.npad),
            "padded_cells": int(np.prod(wl.npad)), "rd": wl.rd, "timesteps_per_solve": int(nt),
            "nfreq": len(wl.freqs), "nrec": len(wl.rec), "volume_dtft": bool(wl.volume),
            "parallelism": f"{world} independent transmitters" if world > 1 else "single GPU",
            "l2": "no flush: per-solve working set (fields, dt/eps, CPML, volume accumulators) "
                  "exceeds the 126 MB L2"}


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
    """DRAM bytes (read + write) of one leapfrog step (every launch of the
    step) from the ncu summary of this workload, or None if there is none for
    the current kernels."""
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


def cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or "unknown"


# ---- error against the FP64 oracle's stored results ----
def _rel_l2_masked(got, ref, floor=1e-6):
    got, ref = np.asarray(got).ravel(), np.asarray(ref).ravel()
    keep = np.abs(ref) > floor * np.abs(ref).max()
    if not keep.any():
        return 0.0
    return float(np.linalg.norm(got[keep] - ref[keep]) / np.linalg.norm(ref[keep]))


def _max_rel_masked(got, ref, floor=1e-6):
    got, ref = np.asarray(got).ravel(), np.asarray(ref).ravel()
    keep = np.abs(ref) > floor * np.abs(ref).max()
    return float(np.max(np.abs(got[keep] - ref[keep]) / np.abs(ref[keep]))) if keep.any() else 0.0


def golden_error(wl, nt, G, vol=None):
    """Error of the solve's Green's functions against the FP64 oracle's
    stored result of the same workload and step count (tests/golden/, written
    by the oracle alone): relative L2 over the entries above 1e-6 of the
    largest, per field kind, and the largest pointwise relative error there;
    volume at the golden's seeded samples.  None when there is no golden of
    this step count."""
    p = os.path.join(GOLDEN_DIR, f"{wl.name}.npz")
    if not os.path.exists(p):
        return {"available": False, "why": "no stored oracle result"}
    g = np.load(p)
    if int(g["nt"]) != int(nt):
        return {"available": False, "why": f"stored oracle result has nt={int(g['nt'])}, solve nt={nt}"}
    G = np.asarray(G)
    out = {"available": True, "oracle_nt": int(g["nt"]),
           "rec_rel_l2_E": _rel_l2_masked(G[:, :3], g["G"][:, :3]),
           "rec_rel_l2_H": _rel_l2_masked(G[:, 3:], g["G"][:, 3:]),
           "rec_max_rel_E": _max_rel_masked(G[:, :3], g["G"][:, :3]),
           "rec_max_rel_H": _max_rel_masked(G[:, 3:], g["G"][:, 3:])}
    if vol is not None and "vol_idx" in g.files:
        flat = np.asarray(vol).transpose(0, 2, 3, 4, 1).reshape(-1, vol.shape[1])
        got, ref = flat[g["vol_idx"]], g["vol_G"]
        isE = g["vol_idx"] < 3 * int(np.prod(wl.shape))
        out.update({"vol_samples": int(len(g["vol_idx"])),
                    "vol_rel_l2_E": _rel_l2_masked(got[isE], ref[isE]),
                    "vol_rel_l2_H": _rel_l2_masked(got[~isE], ref[~isE])})
    out["bound"] = "2e-4 relative L2 (FP32 fields against the FP64 oracle)"
    return out


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


# ---- the FP64 oracle on the host cores ----
def oracle_setup(wl):
    """Wall time of an oracle run of zero steps (tables, allocations)."""
    import oracle
    t0 = time.perf_counter()
    oracle.forward_workload(wl, nt=0)
    return time.perf_counter() - t0


def oracle_sample(wl, nt, t_setup=None):
    """Wall time of `nt` oracle steps (the set-up of a zero-step run
    subtracted; measured here unless given)."""
    import oracle
    if t_setup is None:
        t_setup = oracle_setup(wl)
    t0 = time.perf_counter()
    oracle.forward_workload(wl, nt=nt)
    return max(time.perf_counter() - t0 - t_setup, 1e-9)


def _one_thread_rate(name, nt, timeout=240):
    """Oracle cell-steps/s on one thread (a child process with
    OMP_NUM_THREADS=1), or None if it does not finish in time."""
    code = ("import sys, json; sys.path.insert(0, %r)\n"
            "import bench, numpy as np\n"
            "from paper_2304_00233_b300 import workloads as W\n"
            "wl = W.WORKLOADS[%r](); t = bench.oracle_sample(wl, %d)\n"
            "print(json.dumps({'t': t, 'cells': int(np.prod(wl.npad))}))" % (ROOT, name, nt))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           timeout=timeout)
        d = json.loads(r.stdout.strip().splitlines()[-1])
        return d["cells"] * nt / d["t"] / 1e9, d["t"]
    except (subprocess.TimeoutExpired, ValueError, IndexError, KeyError):
        return None, None


def cpu_baseline(wl, budget_s=15.0):
    """The oracle as it stands, on all host cores, on a bounded sample of the
    workload's leapfrog steps; beside it the same on one thread."""
    import oracle
    threads = oracle.threads()
    probe_nt = 2
    t_setup = oracle_setup(wl)
    t = oracle_sample(wl, probe_nt, t_setup)
    nt = int(min(400, max(2, budget_s / (t / probe_nt))))
    t = oracle_sample(wl, nt, t_setup)
    cells = int(np.prod(wl.npad))
    one_nt = 1 if cells > 5_000_000 else 4
    one, one_t = _one_thread_rate(wl.name, one_nt)
    return {"value": cells * nt / t / 1e9, "unit": "Gcell-steps/s", "cores": threads, "kind": "oracle",
            "sample": f"{nt} leapfrog steps of {wl.name} (FP64 oracle, {threads} OpenMP threads), {t:.1f} s",
            "one_thread": {"value": one, "unit": "Gcell-steps/s",
                           "sample": f"{one_nt} leapfrog steps on 1 thread"
                                     + (f", {one_t:.1f} s" if one_t else ": did not finish")},
            "cpu_model": cpu_model(), "nproc": os.cpu_count()}


# ---- multi-GPU (one process per GPU): sharding over transmitters ----
TOW_SPACING = 200.0  # m between the transmitters of consecutive ranks


def rank_source(src, rank):
    """Transmitter of rank `rank`: the workload's, shifted along the tow line
    (x) by rank * 200 m.  Sources are independent problems, so ranks share
    nothing during the solve (weak scaling)."""
    return np.asarray(src, dtype=np.float64) + np.array([TOW_SPACING * rank, 0.0, 0.0])


def shard(items, rank, world):
    """The items (transmitters) rank `rank` of `world` handles: every
    world-th one from its rank on."""
    return items[rank::world]


def max_over_ranks(v, dist=None, device="cpu"):
    """The slowest rank's value (the job's time): all-reduce MAX, or v itself
    in a single process."""
    if dist is None:
        return float(v)
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(t, dist=None):
    """In-place sum of a tensor over the ranks (the per-transmitter gradient
    volumes of a sharded survey); t itself in a single process."""
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def gather_to_rank0(t, dist=None, world=1):
    """Every rank's tensor (same shape) stacked on rank 0 ([world, ...]);
    None on the other ranks.  A single process gets t[None]."""
    if dist is None:
        return t[None]
    import torch
    # complex values travel as their real and imaginary parts
    src = torch.view_as_real(t).contiguous() if t.is_complex() else t.contiguous()
    parts = [torch.empty_like(src) for _ in range(world)]
    dist.all_gather(parts, src)
    if dist.get_rank() != 0:
        return None
    out = torch.stack(parts)
    return torch.view_as_complex(out) if t.is_complex() else out


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
    probe_dt = oracle.forward_workload(wl, nt=0)["dt"]
    nt_full = wl.nt if wl.nt is not None else int(np.ceil(wl.t_max / probe_dt))
    t_setup = oracle_setup(wl)
    probe = oracle_sample(wl, 1, t_setup)
    # each step: enough leapfrog steps for ~90 s of stepping over the whole run
    nt = int(min(400, max(1, 90.0 / max(1, args.steps + args.warmup) / probe)))
    for _ in range(args.warmup):
        oracle_sample(wl, nt, t_setup)
    times = [oracle_sample(wl, nt, t_setup) for _ in range(args.steps)]
    tot = sum(times)
    value = cells * nt * args.steps / tot / 1e9
    line = {"metric": "FDTD forward Gcell-steps/s", "value": value, "unit": "Gcell-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": bench_config(wl, nt_full, world),
            "cpu_baseline": {"value": value, "unit": "Gcell-steps/s", "cores": threads, "kind": "oracle",
                             "sample": f"each step {nt} leapfrog steps of {wl.name} (of {nt_full} per solve), "
                                       f"setup excluded", "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "Gcell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def timed_events(stream, fn):
    """Device seconds of fn() between two CUDA events on `stream`."""
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3


def marine_line(emm, torch, stream, job_max, world, rank, solves=3):
    """The marine 1-D VTI workload (128 x 128 x 96 nodes, 4th order, no
    volume DTFT): `solves` device-resident solves after a warm-up, the
    leapfrog-step roofline, and the error against the oracle's stored result."""
    wl = W.WORKLOADS[MARINE]()
    wl.src = rank_source(wl.src, rank)
    grid = emm.grid_for(wl)
    nt = emm.steps_for(wl, grid)
    survey = emm.survey_for(wl, nt=nt)
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    work = emm.Workspace(grid, survey)
    emm.forward_async(grid, survey, sigma, work)
    torch.cuda.synchronize()
    loops, es, hs = [], [], []

    def run():
        for _ in range(solves):
            t = emm.forward_timed(grid, survey, sigma, work, every=64)
            loops.append(t["loop_ms"])
            es.append(t["e_ms"])
            hs.append(t["h_ms"])

    sec = job_max(timed_events(stream, run))
    assert emm.status(work) == emm.EMM_OK
    peak, _ = measured_peaks()
    step_s = float(np.mean(loops)) / nt / 1e3
    alg = algorithmic_bytes(wl, emm.VOLUME_RING)
    G = torch.view_as_complex(work.rec)[: survey.nrec].cpu().numpy()
    return {"ctx": (wl, grid, survey, sigma, work, nt),
            "line": {"workload": wl.name, "value": aggregate_rate(world, grid.cells, nt, solves, sec),
                     "unit": "Gcell-steps/s", "timesteps_per_solve": nt, "padded_cells": grid.cells,
                     "solves": solves, "ms_per_solve": 1e3 * sec / solves,
                     "roofline": {"achieved": alg / step_s / 1e9, "peak": peak, "frac": alg / step_s / 1e9 / peak,
                                  "unit": "GB/s", "algorithmic_bytes_per_step": alg, "step_ms": 1e3 * step_s,
                                  "traffic": recorded_traffic(wl.name),
                                  "k_update_E_ms": float(np.mean(es)), "k_update_H_ms": float(np.mean(hs))},
                     "error_vs_oracle": golden_error(wl, nt, G) if rank == 0 else None}}


def gradient_survey_line(emm, torch, stream, job_max, dist, rank, world):
    """Least-squares misfit gradient of the 8-transmitter gradient survey
    (192 x 192 x 128 NU grid): observed data from the model with the
    resistor plus 2 % noise (not timed), then the misfit and its gradient
    with respect to the cell sigma_h, sigma_v at the model without it, with
    the forward fields recomputed from checkpoints every 200 steps: once
    recomputing every segment, once with the E snapshots of as many final
    steps as the free device memory holds (less 6 GB); against one forward
    solve per transmitter on the same grid.  Under torchrun the transmitters
    are shared out over the ranks and the gradients summed."""
    import dataclasses
    # release the allocator's cached blocks first: a tensor allocated inside
    # a large cached block (an earlier gradient's workspace) would pin it
    gc.collect()
    torch.cuda.empty_cache()
    wl = W.gradient_survey(with_resistor=False)
    obs = W.gradient_survey(with_resistor=True)
    grid = emm.grid_for(wl)
    smin = float(obs.sigma.min())
    dt, _, _ = grid.time_step(smin, wl.omega0)
    nt = int(np.ceil(wl.t_max / dt))
    survey = emm.survey_for(wl, nt=nt, sigma_min=smin)
    pos_all = W.GRADIENT_SOURCES
    sig_obs = torch.from_numpy(obs.sigma.astype(np.float32)).cuda()
    G_obs, bwork = emm.forward_batch(grid, survey, sig_obs, pos_all)
    d_all = G_obs.cpu().numpy() * W.observed_noise(G_obs.shape)
    del bwork, sig_obs, G_obs
    pos, d = shard(pos_all, rank, world), shard(d_all, rank, world)
    sh = torch.from_numpy(wl.sigma_h).cuda()
    sv = torch.from_numpy(wl.sigma_v).cuda()
    sigma = emm.stagger_sigma(grid, sh, sv)
    work = emm.Workspace(grid, survey)
    emm.forward_async(grid, survey, sigma, work)
    torch.cuda.synchronize()
    fwd_ms = job_max(timed_events(stream, lambda: emm.forward_async(grid, survey, sigma, work))) * 1e3
    assert emm.status(work) == emm.EMM_OK
    del work
    ck = 200
    # warm-up on a short run of the same problem
    emm.survey_misfit_gradient(grid, dataclasses.replace(survey, nt=2 * ck), sh, sv, pos[:1], d[:1],
                               ckpt_every=ck)
    torch.cuda.synchronize()
    out = {"workload": "gradient_survey_192x192x128", "nsrc": len(pos_all), "timesteps_per_solve": nt,
           "cells": grid.cells, "forward_ms": fwd_ms, "ckpt_every": ck}

    def run(stored):
        res = {}

        def go():
            res["r"] = emm.survey_misfit_gradient(grid, survey, sh, sv, pos, d, ckpt_every=ck, stored_steps=stored)

        ms = job_max(timed_events(stream, go)) * 1e3
        misfit, gh, gv, _ = res["r"]
        sum_over_ranks(misfit, dist)
        sum_over_ranks(gh, dist)
        sum_over_ranks(gv, dist)
        ok = bool(torch.isfinite(gh).all().item() and torch.isfinite(gv).all().item())
        return ms, misfit.item(), ok

    ms0, misfit0, ok0 = run(0)
    out["recompute_only"] = {"ms": ms0, "ratio_to_forward": ms0 / (len(pos_all) * fwd_ms / world),
                             "snapshot_gb": 0.0, "misfit": misfit0, "finite": ok0}
    gc.collect()
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    print(f"gradient survey: {free / 1e9:.1f} GB free, {torch.cuda.memory_allocated() / 1e9:.1f} GB allocated, "
          f"{torch.cuda.memory_reserved() / 1e9:.1f} GB reserved by torch", file=sys.stderr, flush=True)
    room = free - (6 << 30)
    snap = emm.snapshot_bytes(grid, survey, ck)
    stored = min(nt, int(max(0, room) // snap)) // ck * ck
    while stored > 0 and emm.gradient_workspace_size(grid, survey, ck, stored) > room:
        stored -= ck
    ms1, misfit1, ok1 = run(stored)
    out["stored"] = {"ms": ms1, "ratio_to_forward": ms1 / (len(pos_all) * fwd_ms / world),
                     "stored_steps": stored, "snapshot_gb": stored * snap / 1e9, "free_gb_before": free / 1e9,
                     "misfit": misfit1, "finite": ok1}
    out["ratio_to_forward"] = min(out["recompute_only"]["ratio_to_forward"], out["stored"]["ratio_to_forward"])
    out["what"] = ("emm_stagger_sigma, then per transmitter emm_misfit_gradient (forward sweep with "
                   "checkpoints every 200 steps, residual of the noisy resistor-model data, reverse sweep "
                   "recomputing the segments whose E snapshots are not kept, adjoint) and "
                   "emm_stagger_sigma_adjoint into the sigma_h, sigma_v gradients; ratio against one forward "
                   "solve per transmitter")
    return out


def graph_line(emm, torch, stream, job_max, grid, survey, sigma, work, steps, rate, value):
    """The solve replayed `steps` times from a CUDA graph of its time loop
    (emm_plan_create once, emm_plan_run per solve)."""
    t0 = time.perf_counter()
    plan = emm.Plan(grid, survey, sigma, work, stream=stream)
    torch.cuda.synchronize()
    capture_ms = 1e3 * (time.perf_counter() - t0)
    log(f"graph: captured and instantiated in {capture_ms:.0f} ms")
    plan.run_async(sigma, stream=stream)
    torch.cuda.synchronize()
    log("graph: first replay done")

    def run():
        for _ in range(steps):
            plan.run_async(sigma, stream=stream)

    gval = rate(job_max(timed_events(stream, run)))
    log("graph: timed replays done")
    assert emm.status(work) == emm.EMM_OK
    plan.close()
    log("graph: plan destroyed")
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
    torch.cuda.synchronize()
    log("jobs: short single solves done")
    emm.forward_jobs(short, sig, strategy=emm.JOBS_LIST)
    log("jobs: short work-list solve done")
    jw = emm.JobsWork(probs)
    best, tune_ms = emm.jobs_tune(probs, sig, jw, steps=40)
    torch.cuda.synchronize()
    log(f"jobs: tuned ({emm.JOBS_STRATEGIES[best]})")

    def one_at_a_time():
        for (g, s), sg, w in zip(probs, sig, works):
            emm.forward_async(g, s, sg, w)

    seq = job_max(timed_events(stream, one_at_a_time))
    log("jobs: one at a time done")
    for (g, s), w in zip(probs, works):
        assert emm.status(w) == emm.EMM_OK
    rates = {}
    for k in sorted({emm.JOBS_LIST, best}):
        t = job_max(timed_events(stream, lambda: emm.forward_jobs(probs, sig, work=jw, check=False, strategy=k)))
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


def survey_line(emm, torch, stream, job_max, world, rank, nsrc=32):
    """The batched survey: `nsrc` transmitters along the tow line over the
    marine model (x = -3100 + 200 k, 50 m above the seabed) plus the eight
    uneven grids (each with its own transmitter), all advanced in ONE
    persistent cooperative launch (emm_forward_persistent), its tile shape and
    resident-CTA count picked by emm_persist_tune, the whole solve replayed from a CUDA
    graph (emm_persist_plan_run); against the same problems one at a time
    (emm_forward of each transmitter and grid in turn)."""
    wl = W.marine_1d()
    grid = emm.grid_for(wl)
    nt = emm.steps_for(wl, grid)
    survey = emm.survey_for(wl, nt=nt)
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    pos = np.array([[-3100.0 + TOW_SPACING * (k + nsrc * rank), 0.0, 950.0] for k in range(nsrc)])
    tasks, sigmas, cells = [(grid, survey, pos)], [sigma], grid.cells * nt * nsrc
    for u in W.uneven_jobs():
        gu = emm.grid_for(u)
        ntu = emm.steps_for(u, gu)
        tasks.append((gu, emm.survey_for(u, nt=ntu), None))
        sigmas.append(torch.from_numpy(u.sigma.astype(np.float32)).cuda())
        cells += gu.cells * ntu
    work = emm.PersistWork(tasks)
    best, tune_ms = emm.persist_tune(work, sigmas, steps=40)
    plan = emm.PersistPlan(work, sigmas, opts=best, stream=stream)
    plan.run_async(stream)
    torch.cuda.synchronize()
    sec = job_max(timed_events(stream, lambda: plan.run_async(stream)))
    top, each = work.status(stream)
    assert top == emm.EMM_OK and all(v == emm.EMM_OK for v in each)
    G_plan = [g.clone() for g in work.G()]
    plan.close()
    # one at a time: each transmitter of the tow line, then each grid
    works = [emm.Workspace(g, s) for g, s, _ in tasks]
    tow = [dataclasses_replace(survey, src=tuple(float(v) for v in p)) for p in pos]

    def one_at_a_time():
        for s_k in tow:
            emm.forward_async(grid, s_k, sigma, works[0])
        for (g, s, _), sg, w in zip(tasks[1:], sigmas[1:], works[1:]):
            emm.forward_async(g, s, sg, w)

    one_at_a_time()
    torch.cuda.synchronize()
    sec1 = job_max(timed_events(stream, one_at_a_time))
    # the last transmitter and every grid: bitwise equal to their own solves
    same = torch.equal(torch.view_as_complex(works[0].rec)[: survey.nrec], G_plan[0][-1]) and all(
        torch.equal(torch.view_as_complex(w.rec)[: s.nrec], G[0]) for (_, s, _), w, G in zip(tasks[1:], works[1:],
                                                                                             G_plan[1:]))
    value = world * cells / sec / 1e9
    return {"problems": f"{nsrc} tow-line transmitters on {wl.name} + {len(tasks) - 1} uneven grids",
            "cell_steps": cells, "value": value, "unit": "Gcell-steps/s", "ms": 1e3 * sec,
            "one_at_a_time": world * cells / sec1 / 1e9, "ms_one_at_a_time": 1e3 * sec1,
            "speedup": sec1 / sec, "tile_shape": ["32x8x2", "32x4x4"][best.tile_shape],
            "ctas_per_sm": best.ctas_per_sm,
            "tune_ms_40_steps": {f"{['32x8x2', '32x4x4'][k[0]]}/{k[1]}": v for k, v in tune_ms.items()},
            "bitwise_equal": bool(same),
            "what": "emm_persist_plan_run: the whole survey (set-up, one persistent cooperative launch with "
                    "bounded grid barriers between half-steps, normalisation) replayed from a CUDA graph, "
                    "against emm_forward of every transmitter and grid in turn; device-resident inputs"}


def dataclasses_replace(obj, **kw):
    import dataclasses
    return dataclasses.replace(obj, **kw)


def batch_line(emm, torch, stream, job_max, world, rank, grid, survey, sigma, single_value, nsrc):
    """Batched survey on the marine model: transmitters every 200 m along
    the tow line (x = -3100 + 200 k, 50 m above the seabed) advanced
    together; a short warm-up run, one timed solve; then the first 8."""
    import dataclasses
    cells, nt = grid.cells, survey.nt
    pos = np.array([[-3100.0 + TOW_SPACING * (k + nsrc * rank), 0.0, float(survey.src[2])]
                    for k in range(nsrc)])
    out = {}
    for name, p in (("all", pos), ("nsrc_8", pos[: min(8, len(pos))])):
        emm.forward_batch(grid, dataclasses.replace(survey, nt=30), sigma, p)
        bwork = torch.empty(emm.batch_workspace_size(grid, survey, len(p)) + 256, dtype=torch.uint8,
                            device=sigma.device)
        torch.cuda.synchronize()
        bsec = job_max(timed_events(stream, lambda: emm.forward_batch(grid, survey, sigma, p, work=bwork)))
        out[name] = (aggregate_rate(world, cells * len(p), nt, 1, bsec), bsec)
        del bwork
    return {"nsrc": nsrc, "value": out["all"][0], "unit": "Gcell-steps/s", "ms_per_solve": 1e3 * out["all"][1],
            "vs_one_at_a_time": out["all"][0] / single_value,
            "nsrc_8": {"value": out["nsrc_8"][0], "vs_one_at_a_time": out["nsrc_8"][0] / single_value},
            "what": "emm_forward_batch on the marine model: transmitters sharing grid, sigma and receivers in "
                    "the same launches, against the device-resident single-transmitter marine value"}


def airwave_line(emm, torch, stream, job_max, world):
    """Top boundary with air (Sec. 3.3): the marine model on a grid uniform
    in x and y, one warm-up and one timed solve with and without air."""
    awl = W.marine_1d_air()
    agrid = emm.grid_for(awl)
    ant = emm.steps_for(awl, agrid)
    asig = torch.from_numpy(awl.sigma.astype(np.float32)).cuda()
    rates = {}
    for air in (False, True):
        asurvey = emm.survey_for(awl, nt=ant, airwave=air)
        awork = emm.Workspace(agrid, asurvey)
        emm.forward_async(agrid, asurvey, asig, awork)
        torch.cuda.synchronize()
        sec = job_max(timed_events(stream, lambda: emm.forward_async(agrid, asurvey, asig, awork)))
        assert emm.status(awork) == emm.EMM_OK
        rates[air] = aggregate_rate(world, agrid.cells, ant, 1, sec)
        del awork
    return {"workload": awl.name, "value": rates[True], "unit": "Gcell-steps/s", "without_air": rates[False],
            "overhead": rates[False] / rates[True], "timesteps_per_solve": ant,
            "what": "forward solve with air above the sea surface (plane FFTs after every half step) against "
                    "the same model with CPML on the top face"}


def gradient_line(emm, torch, stream, job_max, grid, survey, sigma, fwd_ms):
    """Gradient of Re(sum conj(v) G) on the marine model for a seeded
    cotangent v: one warm-up call and one timed call recomputing every
    segment, then the same with the E snapshots of as many final steps as
    the free device memory holds (less 6 GB), against one forward solve."""
    nt = survey.nt
    rng = np.random.default_rng(230400237)
    v = rng.standard_normal((survey.nrec, 6, len(survey.freqs))) + 1j * rng.standard_normal(
        (survey.nrec, 6, len(survey.freqs)))
    vt = torch.from_numpy(v).cuda()
    ck = max(1, int(round(nt ** 0.5)))
    emm.vjp(grid, survey, sigma, vt, ckpt_every=ck)
    torch.cuda.synchronize()
    grad_ms = job_max(timed_events(stream, lambda: emm.vjp(grid, survey, sigma, vt, ckpt_every=ck,
                                                           check=False))) * 1e3
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
    st_ms = job_max(timed_events(stream, lambda: emm.vjp(grid, survey, sigma, vt, ckpt_every=ck,
                                                         stored_steps=stored, check=False))) * 1e3
    return {"workload": MARINE, "ms": st_ms, "forward_ms": fwd_ms, "ratio_to_forward": st_ms / fwd_ms,
            "ckpt_every": ck, "stored_steps": stored, "snapshot_gb": stored * snap / 1e9,
            "recompute_only_ms": grad_ms, "ratio_recompute_only": grad_ms / fwd_ms,
            "what": "emm_gradient_stored: forward sweep keeping checkpoints and the E snapshots of the last "
                    "stored_steps steps in device memory, recomputation of the earlier segments and the adjoint "
                    "sweep, one cotangent of all receiver data; recompute_only: every segment recomputed "
                    "(emm_gradient)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(W.WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the headline line (no marine, batch, airwave, gradient, jobs or survey lines)")
    ap.add_argument("--no-marine", action="store_true", help="skip the marine-model line")
    ap.add_argument("--no-gradient", action="store_true",
                    help="skip the gradient / forward time ratio on the marine model")
    ap.add_argument("--graph", action="store_true",
                    help="add the CUDA-graph line (the marine solve replayed from a captured time loop)")
    ap.add_argument("--no-jobs", action="store_true",
                    help="skip the uneven-grid work-list line (eight grids, one launch per half-step)")
    ap.add_argument("--no-survey", action="store_true",
                    help="skip the batched-survey line (32 transmitters + 8 uneven grids in one persistent launch)")
    ap.add_argument("--no-gradient-survey", action="store_true",
                    help="skip the 8-transmitter misfit-gradient line on the 192 x 192 x 128 grid")
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
    if os.environ.get("BENCH_STACKS_AFTER_S"):
        # diagnostics: every thread's Python stack on stderr if the run is
        # still going after this many seconds
        import faulthandler
        faulthandler.dump_traceback_later(float(os.environ["BENCH_STACKS_AFTER_S"]), exit=False)
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
    tims = []
    with ClockSampler(local) as clk:
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            tims.append(emm.forward_timed(grid, survey, sigma, work, every=64))
        ev1.record(stream)
        barrier()
    elapsed = job_max(ev0.elapsed_time(ev1) / 1e3)
    clocks = clk.summary()
    value = aggregate_rate(world, cells, nt, args.steps, elapsed)
    assert emm.status(work) == emm.EMM_OK
    G_dev = torch.view_as_complex(work.rec)[: survey.nrec].clone()
    err = None
    if rank == 0:
        err = golden_error(wl, nt, G_dev.cpu().numpy(),
                           None if work.vol is None else torch.view_as_complex(work.vol).cpu().numpy())
    # the one gather of the survey's results: every rank's receiver G on rank 0
    gathered = gather_to_rank0(G_dev, dist, world)

    # ---- e2e: pinned host sigma in, receiver and volume Green's functions out ----
    e2e_solves = max(1, min(args.steps, E2E_SOLVES))
    rec_host = torch.empty(work.rec.shape, dtype=work.rec.dtype).pin_memory()
    vol_host = None if work.vol is None else torch.empty(work.vol.shape, dtype=work.vol.dtype).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_solves):
        sig_dev = sigma_host.to("cuda", non_blocking=True)
        emm.forward_async(grid, survey, sig_dev, work)
        rec_host.copy_(work.rec, non_blocking=True)
        if vol_host is not None:
            vol_host.copy_(work.vol, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = job_max(time.perf_counter() - t0)
    barrier()
    e2e_value = aggregate_rate(world, cells, nt, e2e_solves, e2e_s)
    d2h = int(rec_host.numel() * 8) + (0 if vol_host is None else int(vol_host.numel() * 8))
    del vol_host

    peak, peak_kind = measured_peaks()
    e_mean = float(np.mean([t["e_ms"] for t in tims]))
    h_mean = float(np.mean([t["h_ms"] for t in tims]))
    v_mean = float(np.mean([t["v_ms"] for t in tims]))
    alg = algorithmic_bytes(wl, emm.VOLUME_RING)
    kb = per_kernel_bytes(wl, emm.VOLUME_RING)
    # one leapfrog step as the time loop runs it: E, volume DTFT and H back to
    # back, each launch a programmatic dependent of the one before
    step_s = float(np.mean([t["loop_ms"] for t in tims])) / nt / 1e3
    achieved = alg / step_s / 1e9
    # k_prepare, E and H per step, one volume DTFT per VOLUME_RING steps,
    # the normalisations
    per_solve = (1 + 2 * nt + (-(-nt // emm.VOLUME_RING) if survey.volume else 0) + (1 if survey.nrec else 0)
                 + (1 if survey.volume else 0))
    kernels = {"k_update_E": e_mean, "k_update_H": h_mean}
    if survey.volume:
        kernels["k_volume_dft"] = v_mean
    line = {
        "metric": "FDTD forward Gcell-steps/s", "value": value, "unit": "Gcell-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(wl, nt, world),
        "roofline": {"bound": "hbm", "kernel": "leapfrog step = k_update_E + k_volume_dft + k_update_H"
                                               if survey.volume else "leapfrog step = k_update_E + k_update_H",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": ("of measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
                                   if peak_kind == "measured" else "of fallback 6.4 TB/s"),
                     "algorithmic_bytes_per_step": alg, "step_ms": 1e3 * step_s,
                     "step_ms_from": "CUDA events around the whole time loop / leapfrog steps",
                     "isolated_step_ms": e_mean + h_mean + (v_mean if survey.volume else 0.0),
                     "traffic": recorded_traffic(wl.name),
                     "kernels": {k: {"ms": ms, "min_bytes": kb[k], "gbs": kb[k] / ms / 1e6,
                                     "frac": kb[k] / ms / 1e6 / peak} for k, ms in kernels.items()}},
        "error_vs_oracle": err,
        "e2e": {"value": e2e_value, "unit": "Gcell-steps/s", "solves": e2e_solves,
                "h2d_bytes_per_step": int(sigma_host.numel() * 4), "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps * per_solve,
        "clocks": clocks,
        "gathered_transmitters": None if gathered is None else int(gathered.shape[0]),
    }
    del work
    gc.collect()
    torch.cuda.empty_cache()
    log(f"headline done: {value:.2f} Gcell-steps/s")
    extras = not args.no_extras
    if extras and not args.no_marine:
        m = marine_line(emm, torch, stream, job_max, world, rank)
        line["marine"] = m["line"]
        log("marine line done")
        mwl, mgrid, msurvey, msigma, mwork, mnt = m["ctx"]
        mvalue = m["line"]["value"]
        # the marine solve replayed from a CUDA graph of its time loop
        # (emm_plan), opt-in (--graph) so that the default run stays within
        # its time; the work-list lines after it then run in a process that
        # has created, run and destroyed a plan
        if args.graph:
            line["graph"] = graph_line(emm, torch, stream, job_max, mgrid, msurvey, msigma, mwork, 3,
                                       lambda sec: aggregate_rate(world, mgrid.cells, mnt, 3, sec), mvalue)
            log("graph line done")
        if args.batch > 0:
            line["batch"] = batch_line(emm, torch, stream, job_max, world, rank, mgrid, msurvey, msigma,
                                       mvalue, args.batch)
            log("batch line done")
        if not args.no_airwave:
            line["airwave"] = airwave_line(emm, torch, stream, job_max, world)
            log("airwave line done")
        if not args.no_gradient:
            line["gradient"] = gradient_line(emm, torch, stream, job_max, mgrid, msurvey, msigma,
                                             m["line"]["ms_per_solve"])
            log("gradient line done")
    if extras and not args.no_jobs:
        line["jobs"] = jobs_line(emm, torch, stream, job_max)
        log("jobs line done")
    if extras and not args.no_survey:
        line["survey"] = survey_line(emm, torch, stream, job_max, world, rank)
        log("survey line done")
    if extras and not args.no_gradient_survey:
        line["gradient_survey"] = gradient_survey_line(emm, torch, stream, job_max, dist, rank, world)
        log("gradient survey line done")
    if extras and not args.no_marine:
        del mwork, m
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(W.WORKLOADS[args.workload]())
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
