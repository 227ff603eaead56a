"""GPU conductivity model map and least-squares misfit gradient against the
oracle.

* ``emm_stagger_sigma`` (FP64 means rounded once to FP32) against the
  oracle's FP64 map rounded to FP32: equal up to one FP32 ulp (the two sum
  the same four terms in different orders before the rounding);
* ``emm_stagger_sigma_adjoint`` against the oracle's transpose (FP64,
  1e-13) and its accumulation into the outputs;
* ``emm_misfit_gradient`` + the transpose (``survey_misfit_gradient``)
  against ``oracle.misfit_gradient`` on small NU cases and on the 48^3 copy
  of the gradient survey: misfit within 1e-5 relative, gradients with
  respect to sigma_h and sigma_v within the relative L2 bound of the
  staggered gradient (FP32 fields against FP64), both scaled by |G| / |G - d|
  where the residual is mostly noise (its relative FP32 error is that much
  larger than G's);
* a survey of two transmitters gives the sum of its single-transmitter
  calls (the misfit bit for bit; the gradients up to the order of the
  atomic receiver additions of the adjoint), and the autograd function
  returns the same gradients."""
import numpy as np
import pytest

import oracle
import paper_2304_00233_b300 as emm
from paper_2304_00233_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

GRAD_TOL = 1e-5
MISFIT_TOL = 1e-5


def _cells(wl):
    return (len(wl.z) - 1, len(wl.y) - 1, len(wl.x) - 1)


def _random_cells(wl, seed):
    rng = np.random.default_rng(seed)
    sh = np.exp(rng.uniform(np.log(0.3), np.log(3.0), _cells(wl)))
    sv = np.exp(rng.uniform(np.log(0.3), np.log(3.0), _cells(wl)))
    return sh, sv


@pytest.mark.parametrize("n", [(23, 19, 17), (40, 36, 30)])
def test_stagger_against_oracle(n):
    wl = W.small_case(n=n, rd=2, seed=4, nt=10, volume=False)
    sh, sv = _random_cells(wl, 5)
    grid = emm.grid_for(wl)
    got = emm.stagger_sigma(grid, torch.from_numpy(sh).cuda(), torch.from_numpy(sv).cuda()).cpu().numpy()
    ref = oracle.stagger(wl.x, wl.y, wl.z, sh, sv).astype(np.float32)
    ulp = np.spacing(np.abs(ref))
    assert np.all(np.abs(got - ref) <= ulp), np.max(np.abs(got - ref) / ulp)


def test_stagger_adjoint_against_oracle_and_accumulates():
    wl = W.small_case(n=(31, 27, 22), rd=2, seed=6, nt=10, volume=False)
    grid = emm.grid_for(wl)
    rng = np.random.default_rng(7)
    g = rng.standard_normal((3, len(wl.z), len(wl.y), len(wl.x)))
    gt = torch.from_numpy(g).cuda()
    gh, gv = emm.stagger_sigma_adjoint(grid, gt)
    rh, rv = oracle.stagger_T(wl.x, wl.y, wl.z, g)
    np.testing.assert_allclose(gh.cpu().numpy(), rh, rtol=1e-13, atol=1e-13 * np.abs(rh).max())
    np.testing.assert_allclose(gv.cpu().numpy(), rv, rtol=1e-13, atol=1e-13 * np.abs(rv).max())
    gh2, gv2 = emm.stagger_sigma_adjoint(grid, gt, gh.clone(), gv.clone())
    assert torch.equal(gh2, gh + gh) and torch.equal(gv2, gv + gv)


def _oracle_kw(wl, survey, grid):
    """Oracle arguments of a survey.  The oracle takes its own dt from
    sigma_min (Sec. 3.2); the library's dt is checked against it here, apart
    from the comparisons of the results."""
    kw = dict(rd=wl.rd, nb=wl.nb, ne=wl.ne, omega0=wl.omega0, nt=survey.nt, fmax=wl.fmax,
              sigma_min=survey.sigma_min, src=tuple(survey.src), az=wl.src_az, dip=wl.src_dip,
              moment=wl.moment, rec=wl.rec, freqs=wl.freqs)
    odt = oracle.forward(wl.x, wl.y, wl.z, wl.sigma, **{**kw, "nt": 0, "rec": None})["dt"]
    dt, _, _ = grid.time_step(survey.sigma_min, survey.omega0)
    assert dt == pytest.approx(odt, rel=1e-13)
    return kw


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("rd", [2, 4])
def test_misfit_gradient_against_oracle(rd):
    wl = W.small_case(n=(26, 22, 20), rd=rd, seed=30 + rd, nt=120, volume=False, nb=5, nfreq=2)
    sh, sv = _random_cells(wl, 31)
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, sigma_min=0.2)
    kw = _oracle_kw(wl, survey, grid)
    # observed data: the oracle's response of another model, with noise; weights drop one channel
    d = oracle.forward(wl.x, wl.y, wl.z, oracle.stagger(wl.x, wl.y, wl.z, 1.4 * sh, 0.7 * sv), **kw)["G"]
    d = d * W.observed_noise(d.shape, seed=32)
    w = np.random.default_rng(33).uniform(0.5, 2.0, d.shape)
    w[:, 4, :] = 0.0
    ref = oracle.misfit_gradient(wl.x, wl.y, wl.z, sh, sv, d, w, ckpt_every=30, **kw)
    misfit, gh, gv, G = emm.survey_misfit_gradient(
        grid, survey, torch.from_numpy(sh).cuda(), torch.from_numpy(sv).cuda(), [survey.src], d[None],
        weight=w, ckpt_every=17)
    assert misfit.item() == pytest.approx(ref["misfit"], rel=MISFIT_TOL)
    assert _rel(gh.cpu().numpy(), ref["grad_h"]) < GRAD_TOL
    assert _rel(gv.cpu().numpy(), ref["grad_v"]) < GRAD_TOL
    assert _rel(G[0].cpu().numpy(), ref["G"]) < 2e-4


def test_gradient_survey_copy_against_oracle():
    """The 48^3 copy of the gradient survey (marine layering, data of the
    model with the resistor, gradient at the model without it), one
    transmitter, a short fixed step count."""
    obs = W.gradient_survey_48(with_resistor=True, nt=150)
    wl = W.gradient_survey_48(with_resistor=False, nt=150)
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, sigma_min=float(obs.sigma.min()))
    kw = _oracle_kw(wl, survey, grid)
    d = oracle.forward(obs.x, obs.y, obs.z, oracle.stagger(obs.x, obs.y, obs.z, obs.sigma_h, obs.sigma_v), **kw)["G"]
    d = d * W.observed_noise(d.shape)
    ref = oracle.misfit_gradient(wl.x, wl.y, wl.z, wl.sigma_h, wl.sigma_v, d, ckpt_every=25, **kw)
    misfit, gh, gv, _ = emm.survey_misfit_gradient(
        grid, survey, torch.from_numpy(wl.sigma_h).cuda(), torch.from_numpy(wl.sigma_v).cuda(), [survey.src],
        d[None], ckpt_every=12)
    # Here the residual G - d is mostly the 2 % noise, so an FP32 error of G
    # relative to |G| is |G| / |G - d| (about 70) times larger relative to
    # the residual, which the misfit and the gradient inherit: the bounds
    # scale by that ratio (from the oracle's own G and d).
    amp = max(1.0, float(np.linalg.norm(ref["G"]) / np.linalg.norm(ref["G"] - d)))
    assert misfit.item() == pytest.approx(ref["misfit"], rel=MISFIT_TOL * amp)
    assert _rel(gh.cpu().numpy(), ref["grad_h"]) < GRAD_TOL * amp
    assert _rel(gv.cpu().numpy(), ref["grad_v"]) < GRAD_TOL * amp


def test_survey_sum_stored_steps_and_autograd():
    wl = W.small_case(n=(21, 19, 17), rd=2, seed=40, nt=90, volume=False, nb=5, nfreq=2)
    sh, sv = _random_cells(wl, 41)
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, sigma_min=0.25)
    c = np.array(survey.src)
    pos = np.array([c, c + np.array([35.0, -20.0, 10.0])])
    rng = np.random.default_rng(42)
    d = rng.standard_normal((2, len(wl.rec), 6, 2)) * 1e-9 + 1j * rng.standard_normal((2, len(wl.rec), 6, 2)) * 1e-9
    sht, svt = torch.from_numpy(sh).cuda(), torch.from_numpy(sv).cuda()
    m2, gh2, gv2, G2 = emm.survey_misfit_gradient(grid, survey, sht, svt, pos, d, ckpt_every=30)
    parts = [emm.survey_misfit_gradient(grid, survey, sht, svt, pos[k:k + 1], d[k:k + 1], ckpt_every=30)
             for k in range(2)]
    def rel(a, b):
        return (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item()

    assert torch.equal(m2, parts[0][0] + parts[1][0])
    assert rel(gh2, parts[0][1] + parts[1][1]) < 1e-6 and rel(gv2, parts[0][2] + parts[1][2]) < 1e-6
    assert torch.equal(G2[1], parts[1][3][0])
    # keeping the E snapshots of the last segments changes nothing but the
    # order of the atomic receiver additions
    m3, gh3, gv3, _ = emm.survey_misfit_gradient(grid, survey, sht, svt, pos, d, ckpt_every=30, stored_steps=60)
    assert torch.equal(m3, m2)
    assert rel(gh3, gh2) < 1e-6 and rel(gv3, gv2) < 1e-6
    # autograd
    a, b = sht.clone().requires_grad_(True), svt.clone().requires_grad_(True)
    loss = emm.cell_misfit(a, b, grid, survey, pos, d, ckpt_every=30)
    (2.0 * loss).backward()
    assert torch.equal(loss.detach(), m2[0])
    assert rel(a.grad, 2.0 * gh2) < 1e-6 and rel(b.grad, 2.0 * gv2) < 1e-6
