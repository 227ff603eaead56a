"""GPU gradient (emm_gradient) against the oracle's exact discrete adjoint.

Small non-uniform cases for rd = 1..4 with CPML, a tilted source and several
receivers and frequencies: the conductivity gradient of Re(sum conj(v) G)
from the CUDA path (FP32 fields, FP64 gradient accumulation) is compared with
the FP64 oracle's, as a relative L2 error over all samples.  The autograd
wrapper is checked against the direct call."""
import numpy as np
import pytest

import oracle
import paper_2304_00233_b300 as emm
from paper_2304_00233_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

# FP32 forward and adjoint fields against FP64: relative L2 of the gradient
# (measured on B300: 0.9e-7 .. 2.1e-7 for these cases)
GRAD_TOL = 1e-5

CASES = [dict(rd=1, n=(22, 20, 18)), dict(rd=2, n=(23, 19, 17)), dict(rd=3, n=(26, 22, 20)),
         dict(rd=4, n=(28, 26, 24))]


def _same_time_step(wl, grid, survey):
    """The oracle takes its own dt (Sec. 3.2, from the same sigma_min); the
    library's dt must agree with it, checked apart from the gradient."""
    ref = oracle.forward(wl.x, wl.y, wl.z, wl.sigma, rd=wl.rd, nb=wl.nb, ne=wl.ne, omega0=wl.omega0,
                         nt=0, fmax=wl.fmax, sigma_min=survey.sigma_min)["dt"]
    dt, _, _ = grid.time_step(survey.sigma_min, survey.omega0)
    assert dt == pytest.approx(ref, rel=1e-13)


def _problem(rd, n, nt=140, seed=21):
    wl = W.small_case(n=n, rd=rd, seed=seed, nt=nt, volume=False, nb=5, nfreq=2)
    rng = np.random.default_rng(seed + 1)
    v = rng.standard_normal((len(wl.rec), 6, 2)) + 1j * rng.standard_normal((len(wl.rec), 6, 2))
    return wl, v


@pytest.mark.parametrize("case", CASES, ids=[f"rd{c['rd']}" for c in CASES])
def test_gradient_against_oracle(case):
    wl, v = _problem(case["rd"], case["n"])
    grid, survey = emm.grid_for(wl), emm.survey_for(wl, nt=wl.nt)
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    grad, G = emm.vjp(grid, survey, sigma, torch.from_numpy(v).cuda(), ckpt_every=17)
    torch.cuda.synchronize()
    _same_time_step(wl, grid, survey)
    ref = oracle.vjp(wl.x, wl.y, wl.z, wl.sigma, v, rd=wl.rd, nb=wl.nb, ne=wl.ne, omega0=wl.omega0,
                     nt=wl.nt, fmax=wl.fmax, sigma_min=survey.sigma_min, src=wl.src, az=wl.src_az,
                     dip=wl.src_dip, moment=wl.moment, rec=wl.rec, freqs=wl.freqs, ckpt_every=20)
    g = grad.cpu().numpy()
    err = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert err < GRAD_TOL, err
    # the forward sweep's G is the forward solver's
    G_ref, _ = emm.forward(grid, survey, sigma)
    assert torch.allclose(G, G_ref, rtol=0, atol=0)


def test_checkpoint_spacing_and_autograd():
    wl, v = _problem(2, (21, 18, 16), nt=90)
    grid, survey = emm.grid_for(wl), emm.survey_for(wl, nt=wl.nt)
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    vt = torch.from_numpy(v).cuda()
    g1, _ = emm.vjp(grid, survey, sigma, vt, ckpt_every=1)
    g2, _ = emm.vjp(grid, survey, sigma, vt, ckpt_every=90)
    rel = (torch.linalg.norm(g1 - g2) / torch.linalg.norm(g1)).item()
    assert rel < 1e-5, rel        # same arithmetic up to the order of atomic receiver adds
    s = sigma.clone().double().requires_grad_(True)
    G = emm.green_functions(s, grid, survey, ckpt_every=30)
    loss = torch.real(torch.sum(torch.conj(vt) * G))
    loss.backward()
    rel = (torch.linalg.norm(s.grad - g1) / torch.linalg.norm(g1)).item()
    assert rel < 1e-5, rel


def test_gradient_interior_blocks_against_oracle():
    # wide enough in x for 32 x 8 blocks whose cells and taps all lie outside
    # the CPML shell (the vectorised interior path of the adjoint)
    wl, v = _problem(2, (54, 26, 22), nt=90, seed=31)
    grid, survey = emm.grid_for(wl), emm.survey_for(wl, nt=wl.nt)
    np0 = len(wl.x) + 2 * (wl.nb + wl.ne)
    lo = wl.nb + wl.rd
    assert any(i0 >= lo and i0 + 31 <= np0 - 2 - lo for i0 in range(0, np0, 32))
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    grad, _ = emm.vjp(grid, survey, sigma, torch.from_numpy(v).cuda(), ckpt_every=23)
    _same_time_step(wl, grid, survey)
    ref = oracle.vjp(wl.x, wl.y, wl.z, wl.sigma, v, rd=wl.rd, nb=wl.nb, ne=wl.ne, omega0=wl.omega0,
                     nt=wl.nt, fmax=wl.fmax, sigma_min=survey.sigma_min, src=wl.src, az=wl.src_az,
                     dip=wl.src_dip, moment=wl.moment, rec=wl.rec, freqs=wl.freqs, ckpt_every=30)
    g = grad.cpu().numpy()
    err = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert err < GRAD_TOL, err


@pytest.mark.parametrize("stored", [25, 40, 1000])
def test_stored_snapshots_match_recomputation(stored):
    # the forward sweep keeps the E snapshots of the last segments (25 steps:
    # two segments of 10, 40: all but the first few, 1000: all of them); the
    # reverse sweep then skips their recomputation
    wl, v = _problem(2, (21, 18, 16), nt=90)
    grid, survey = emm.grid_for(wl), emm.survey_for(wl, nt=wl.nt)
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    vt = torch.from_numpy(v).cuda()
    g0, G0 = emm.vjp(grid, survey, sigma, vt, ckpt_every=10)
    g1, G1 = emm.vjp(grid, survey, sigma, vt, ckpt_every=10, stored_steps=stored)
    assert torch.equal(G0, G1)
    rel = (torch.linalg.norm(g1 - g0) / torch.linalg.norm(g0)).item()
    assert rel < 1e-5, rel        # same arithmetic up to the order of atomic receiver adds
    assert emm.gradient_workspace_size(grid, survey, 10, stored) > emm.gradient_workspace_size(grid, survey, 10)
