"""The conductivity gradient of the least-squares survey misfit (the
gradient survey's checks), GPU against the FP64 oracle and against finite
differences.

* The 48^3 copy of the gradient survey at its full step count (the oracle's
  own dt and nt = ceil(t_max / dt)), both transmitters: misfit, sigma_h and
  sigma_v gradients and G against the oracle's stored results
  (tests/golden/gradient_survey_48.npz, written by the oracle alone).  The
  residual G - d is mostly the 2 % noise, so an FP32 error of G relative to
  |G| is |G| / |G - d| times larger relative to the residual; the bounds
  scale by that ratio (from the oracle's own G and d).
* The 20 cells drawn with default_rng(230400235) on the same copy
  (FD_NT steps, first transmitter): the GPU gradient against the oracle's
  FP64 central differences of the misfit and against the oracle's adjoint
  gradient at those cells (tests/golden/gradient_fd_48.npz).
* The full 192 x 192 x 128 survey grid (a shorter step count, stated
  below): the GPU gradient at 20 cells drawn with default_rng(230400235)
  from the cells within 200 m of the first transmitter against
  Richardson-combined central differences of the GPU's own misfit, the
  derivative the adjoint must give of the forward map it transposes."""
import os

import numpy as np
import pytest

import paper_2304_00233_b300 as emm
from paper_2304_00233_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

GOLD = os.path.join(os.path.dirname(__file__), "golden")
GRAD_TOL = 1e-5      # relative L2 of the gradient, FP32 fields against FP64 (as tests/test_gpu_misfit.py)
MISFIT_TOL = 1e-5


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def _copy48(nt, sigma_min):
    wl = W.gradient_survey_48(with_resistor=False, nt=nt)
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, nt=nt, sigma_min=sigma_min)
    return wl, grid, survey


@pytest.mark.skipif(not os.path.exists(os.path.join(GOLD, "gradient_survey_48.npz")),
                    reason="golden file not generated")
def test_gradient_survey_copy_full_steps_against_oracle():
    g = np.load(os.path.join(GOLD, "gradient_survey_48.npz"))
    wl, grid, survey = _copy48(int(g["nt"]), float(g["sigma_min"]))
    dt, _, _ = grid.time_step(survey.sigma_min, survey.omega0)
    assert dt == pytest.approx(float(g["dt"]), rel=1e-13)      # the oracle's own dt
    misfit, gh, gv, G = emm.survey_misfit_gradient(
        grid, survey, torch.from_numpy(wl.sigma_h).cuda(), torch.from_numpy(wl.sigma_v).cuda(),
        W.GRADIENT_SOURCES_48, g["d_obs"], ckpt_every=200)
    amp = max(1.0, float(np.linalg.norm(g["G"]) / np.linalg.norm(g["G"] - g["d_obs"])))
    assert misfit.item() == pytest.approx(float(np.sum(g["misfit"])), rel=MISFIT_TOL * amp)
    assert _rel(G.cpu().numpy(), g["G"]) < 2e-4
    eh, ev = _rel(gh.cpu().numpy(), g["grad_h"]), _rel(gv.cpu().numpy(), g["grad_v"])
    assert eh < GRAD_TOL * amp and ev < GRAD_TOL * amp, (eh, ev, amp)


@pytest.mark.skipif(not os.path.exists(os.path.join(GOLD, "gradient_fd_48.npz")),
                    reason="golden file not generated")
def test_gradient_at_20_cells_against_oracle_finite_differences():
    g = np.load(os.path.join(GOLD, "gradient_fd_48.npz"))
    wl, grid, survey = _copy48(int(g["nt"]), float(g["sigma_min"]))
    _, gh, gv, _ = emm.survey_misfit_gradient(
        grid, survey, torch.from_numpy(wl.sigma_h).cuda(), torch.from_numpy(wl.sigma_v).cuda(),
        W.GRADIENT_SOURCES_48[:1], g["d_obs"][None], ckpt_every=200)
    cells = g["cells"]
    got = np.stack([gh.cpu().numpy().ravel()[cells], gv.cpu().numpy().ravel()[cells]])
    for p in range(2):
        scale = np.abs(g["fd"][p]).max()
        assert scale > 0
        # the oracle's own adjoint and its central differences agree first
        assert np.abs(g["adjoint"][p] - g["fd"][p]).max() < 1e-4 * scale
        assert np.abs(got[p] - g["fd"][p]).max() < 1e-3 * scale, (p, got[p], g["fd"][p])


# the full survey grid: a shorter run (2000 steps, 1.75 s of the 6.4 s of
# fictitious time), its first transmitter, data of the resistor model with noise
FD_NT_FULL = 2000


def _source_cells(wl, src, count=20, seed=230400235):
    """Cells (flat indices into [n3-1][n2-1][n1-1]) drawn uniformly from those
    whose centre lies within 200 m of the transmitter along each axis.  FP32
    differences of the misfit resolve the derivative only where a cell's
    change moves the data by far more than the FP32 rounding of G (about
    1e-7 of |G|): near the transmitter a 5 % change of one cell does; a cell
    far from it changes the data by less than that rounding."""
    xc, yc, zc = (0.5 * (a[:-1] + a[1:]) for a in (wl.x, wl.y, wl.z))
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    near = (np.abs(X - src[0]) <= 200.0) & (np.abs(Y - src[1]) <= 200.0) & (np.abs(Z - src[2]) <= 200.0)
    keep = np.flatnonzero(near.ravel())
    return np.sort(np.random.default_rng(seed).choice(keep, size=count, replace=False))


def test_full_grid_gradient_at_20_cells_against_gpu_finite_differences():
    obs = W.gradient_survey(with_resistor=True)
    wl = W.gradient_survey(with_resistor=False)
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, nt=FD_NT_FULL, sigma_min=float(obs.sigma.min()))
    src = W.GRADIENT_SOURCES[:1]
    G_obs, _ = emm.forward_batch(grid, survey, torch.from_numpy(obs.sigma.astype(np.float32)).cuda(), src)
    d = G_obs.cpu().numpy() * W.observed_noise(G_obs.shape)
    sh0, sv0 = torch.from_numpy(wl.sigma_h).cuda(), torch.from_numpy(wl.sigma_v).cuda()
    _, gh, gv, _ = emm.survey_misfit_gradient(grid, survey, sh0, sv0, src, d, ckpt_every=200)
    work = emm.Workspace(grid, survey)
    dt = torch.from_numpy(d[0]).cuda()

    def misfit(sh, sv):
        sigma = emm.stagger_sigma(grid, sh, sv)
        G, _ = emm.forward(grid, survey, sigma, work)
        r = G - dt
        return 0.5 * float(torch.sum(r.real ** 2 + r.imag ** 2).item())

    cells = _source_cells(wl, src[0])
    grads = (gh.cpu().numpy().ravel(), gv.cpu().numpy().ravel())
    for p, base in enumerate((sh0, sv0)):
        fd = np.zeros(len(cells))
        for k, c in enumerate(cells):
            v0 = float(base.view(-1)[c].item())

            def diff(h):
                up, dn = base.clone(), base.clone()
                up.view(-1)[c] = v0 + h
                dn.view(-1)[c] = v0 - h
                args = ((up, sv0), (dn, sv0)) if p == 0 else ((sh0, up), (sh0, dn))
                return (misfit(*args[0]) - misfit(*args[1])) / (2.0 * h)

            h = 0.05 * v0
            fd[k] = (4.0 * diff(0.5 * h) - diff(h)) / 3.0     # Richardson: O(h^4)
        got = grads[p][cells]
        scale = np.abs(fd).max()
        assert scale > 0
        err = np.abs(got - fd) / scale
        assert err.max() < 2e-2, (p, err, got, fd)
        assert _rel(got, fd) < 1e-2
