"""Write the stored oracle results the GPU parity tests compare against.

Only the FP64 oracle (``oracle/``) computes these values; the seeded inputs
come from ``paper_2304_00233_b300.workloads``.  Nothing here touches the CUDA
library.  Every step count and time step below is the oracle's own (its dt
from the CFL rule of Sec. 3.2, nt = ceil(t_max / dt)).

Usage:  python tests/golden/make_golden.py [name ...]

  whole_space_64          full step count, 32 receivers
  marine_1d_128x128x96    full step count, 64 receivers, 3 frequencies
  anomaly_3d_256x256x160  full step count (the full grid, rd=4), 201
                          receivers and 4096 seeded samples of the volume DTFT
  gradient_survey_48      the 48^3 copy of the gradient survey at its full
                          step count: observed data of the model with the
                          resistor times the seeded 2 % noise, then the
                          least-squares misfit and its gradient with respect
                          to the cell sigma_h, sigma_v at the model without
                          it, summed over both transmitters
  gradient_fd_48          central differences of the same misfit (first
                          transmitter, FD_NT steps) at 20 cells drawn with
                          default_rng(230400235), for sigma_h and sigma_v,
                          beside the oracle's adjoint gradient at those cells
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2304_00233_b300 import workloads as W  # noqa: E402

VOL_SAMPLES = 4096
FD_NT = 2000          # steps of the finite-difference golden (1.76 s of fictitious time)
FD_CELLS = 20
FD_SEED = 230400235
FD_STEP = 1e-3        # relative perturbation of one cell value


def volume_sample_indices(w, count=VOL_SAMPLES, seed=230400236):
    n1, n2, n3 = w.shape
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(6 * n1 * n2 * n3, size=count, replace=False)).astype(np.int64)


def fd_cells(wl, count=FD_CELLS, seed=FD_SEED):
    """Flat indices into the [n3-1][n2-1][n1-1] cell array, drawn uniformly
    without replacement."""
    ncell = (len(wl.z) - 1) * (len(wl.y) - 1) * (len(wl.x) - 1)
    return np.sort(np.random.default_rng(seed).choice(ncell, size=count, replace=False)).astype(np.int64)


def make(name):
    w = W.WORKLOADS[name]()
    kw = {}
    if name.startswith("anomaly_3d"):
        kw = dict(volume=False, vol_samples=volume_sample_indices(w))
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


def _survey48(nt=None):
    """Oracle keyword arguments of the 48^3 gradient copy: sigma_min of the
    observed (resistor) model fixes dt and the CPML for both models; nt is
    ceil(t_max / dt) with the oracle's own dt unless given."""
    obs = W.gradient_survey_48(with_resistor=True)
    wl = W.gradient_survey_48(with_resistor=False)
    smin = float(obs.sigma.min())
    kw = dict(rd=wl.rd, nb=wl.nb, ne=wl.ne, omega0=wl.omega0, fmax=wl.fmax, sigma_min=smin,
              moment=wl.moment, rec=wl.rec, freqs=wl.freqs)
    dt = oracle.forward(wl.x, wl.y, wl.z, wl.sigma, nt=0, **kw)["dt"]
    kw["nt"] = int(np.ceil(wl.t_max / dt)) if nt is None else int(nt)
    return obs, wl, kw, dt


def _observed48(obs, kw):
    sig = oracle.stagger(obs.x, obs.y, obs.z, obs.sigma_h, obs.sigma_v)
    d = np.stack([oracle.forward(obs.x, obs.y, obs.z, sig, src=tuple(s), **kw)["G"]
                  for s in W.GRADIENT_SOURCES_48])
    return d * W.observed_noise(d.shape)


def make_gradient48():
    t0 = time.time()
    obs, wl, kw, dt = _survey48()
    d = _observed48(obs, kw)
    misfit, gh, gv, G = [], 0.0, 0.0, []
    for k, s in enumerate(W.GRADIENT_SOURCES_48):
        r = oracle.misfit_gradient(wl.x, wl.y, wl.z, wl.sigma_h, wl.sigma_v, d[k], src=tuple(s),
                                   ckpt_every=100, **kw)
        misfit.append(r["misfit"])
        gh = gh + r["grad_h"]
        gv = gv + r["grad_v"]
        G.append(r["G"])
    secs = time.time() - t0
    path = os.path.join(HERE, "gradient_survey_48.npz")
    np.savez_compressed(path, d_obs=d, G=np.stack(G), misfit=np.array(misfit), grad_h=gh, grad_v=gv,
                        dt=dt, nt=kw["nt"], sigma_min=kw["sigma_min"], seconds=secs,
                        threads=oracle.threads())
    print(f"gradient_survey_48: nt={kw['nt']} dt={dt:.6e} misfit={sum(misfit):.6e} {secs:.1f}s -> {path}",
          flush=True)


def make_fd48():
    t0 = time.time()
    obs, wl, kw, dt = _survey48(nt=FD_NT)
    s0 = tuple(W.GRADIENT_SOURCES_48[0])
    d = _observed48(obs, kw)[0]
    ref = oracle.misfit_gradient(wl.x, wl.y, wl.z, wl.sigma_h, wl.sigma_v, d, src=s0, ckpt_every=50, **kw)
    cells = fd_cells(wl, FD_CELLS)

    def misfit(sh, sv):
        G = oracle.forward(wl.x, wl.y, wl.z, oracle.stagger(wl.x, wl.y, wl.z, sh, sv), src=s0, **kw)["G"]
        r = G - d
        return 0.5 * float(np.sum(r.real ** 2 + r.imag ** 2))

    fd = np.zeros((2, FD_CELLS))
    for p, name in enumerate(("sigma_h", "sigma_v")):
        base = getattr(wl, name)
        for k, c in enumerate(cells):
            h = FD_STEP * base.flat[c]
            up, dn = base.copy(), base.copy()
            up.flat[c] += h
            dn.flat[c] -= h
            args_up = (up, wl.sigma_v) if p == 0 else (wl.sigma_h, up)
            args_dn = (dn, wl.sigma_v) if p == 0 else (wl.sigma_h, dn)
            fd[p, k] = (misfit(*args_up) - misfit(*args_dn)) / (2.0 * h)
            print(f"  fd {name} cell {c}: {fd[p, k]:.6e} adjoint "
                  f"{(ref['grad_h'] if p == 0 else ref['grad_v']).flat[c]:.6e}", flush=True)
    adj = np.stack([ref["grad_h"].ravel()[cells], ref["grad_v"].ravel()[cells]])
    secs = time.time() - t0
    path = os.path.join(HERE, "gradient_fd_48.npz")
    np.savez_compressed(path, cells=cells, fd=fd, adjoint=adj, d_obs=d, misfit=ref["misfit"], nt=FD_NT,
                        dt=dt, sigma_min=kw["sigma_min"], step=FD_STEP, seconds=secs,
                        threads=oracle.threads())
    print(f"gradient_fd_48: max |fd - adjoint| / max |adjoint| = "
          f"{np.abs(fd - adj).max() / np.abs(adj).max():.3e} {secs:.1f}s -> {path}", flush=True)


SPECIAL = {"gradient_survey_48": make_gradient48, "gradient_fd_48": make_fd48}

if __name__ == "__main__":
    for name in (sys.argv[1:] or list(W.WORKLOADS) + list(SPECIAL)):
        SPECIAL.get(name, lambda n=name: make(n))()
