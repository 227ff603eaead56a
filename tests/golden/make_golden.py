"""Write the stored oracle results the GPU parity tests compare against.

Only the FP64 oracle (``oracle/``) computes these values; the seeded inputs
come from ``paper_2304_00233_b300.workloads``.  Nothing here touches the CUDA
library.  Usage:  python tests/golden/make_golden.py [name ...]

  whole_space_64          full step count, 32 receivers
  marine_1d_128x128x96    full step count, 64 receivers, 3 frequencies
  anomaly_3d_256x256x160  first 2000 steps (the full grid, rd=4), 201
                          receivers and 4096 seeded samples of the volume DTFT
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2304_00233_b300 import workloads as W  # noqa: E402

ANOMALY_NT = 2000
VOL_SAMPLES = 4096


def volume_sample_indices(w, count=VOL_SAMPLES, seed=230400236):
    n1, n2, n3 = w.shape
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(6 * n1 * n2 * n3, size=count, replace=False)).astype(np.int64)


def make(name):
    w = W.WORKLOADS[name]()
    kw = {}
    if name.startswith("anomaly_3d"):
        kw = dict(nt=ANOMALY_NT, volume=False, vol_samples=volume_sample_indices(w))
    t0 = time.time()
    r = oracle.forward_workload(w, **kw)
    secs = time.time() - t0
    out = dict(G=r["G"], jhat=r["jhat"], dt=r["dt"], nt=r["nt"], vmax=r["vmax"],
               seconds=secs, threads=oracle.threads())
    if "vol_samples_G" in r:
        out["vol_idx"] = kw["vol_samples"]
        out["vol_G"] = r["vol_samples_G"]
    path = os.path.join(HERE, f"{name}.npz")
    np.savez_compressed(path, **out)
    print(f"{name}: nt={r['nt']} dt={r['dt']:.6e} {secs:.1f}s -> {path}", flush=True)


if __name__ == "__main__":
    for name in (sys.argv[1:] or list(W.WORKLOADS)):
        make(name)
