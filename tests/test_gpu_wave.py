"""Wavefront solve (emm_forward_wave): one persistent launch advancing
z-layers of tiles through several time steps per sweep, each tile waiting
on per-layer completion counts for the layers it reads.

Every tile runs the per-CTA code of the plain launches on the same inputs
and the receiver DTFT adds the same terms in the same step order, so G must
equal emm_forward's bit for bit: for rd = 1..4, several sweep depths,
receivers spread over many z-layers, the marine workload at its full step
count, and the degenerate step counts 0, 1 and 2."""
import dataclasses

import numpy as np
import pytest

import paper_2304_00233_b300 as emm
from paper_2304_00233_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def _sig(wl):
    return torch.from_numpy(wl.sigma.astype(np.float32)).cuda()


@pytest.mark.parametrize("rd", [1, 2, 3, 4])
def test_wave_equals_forward_bitwise(rd):
    wl = W.small_case(n=(40, 36, 44), rd=rd, seed=20 + rd, nt=70, volume=False, nfreq=2)
    grid, survey = emm.grid_for(wl), emm.survey_for(wl)
    sigma = _sig(wl)
    ref, _ = emm.forward(grid, survey, sigma)
    for depth in (1, 2, 3):
        G, _ = emm.forward_wave(grid, survey, sigma, depth=depth)
        assert torch.equal(G, ref), depth


def test_wave_degenerate_step_counts_and_no_receivers():
    wl = W.small_case(n=(30, 28, 26), rd=2, seed=9, nt=2, volume=False)
    grid, sigma = emm.grid_for(wl), _sig(wl)
    for nt in (0, 1, 2):
        survey = emm.survey_for(wl, nt=nt)
        ref, _ = emm.forward(grid, survey, sigma)
        G, _ = emm.forward_wave(grid, survey, sigma, depth=2)
        assert torch.equal(G, ref), nt
    quiet = dataclasses.replace(emm.survey_for(wl, nt=40), rec=np.zeros((0, 3)))
    emm.forward_wave(grid, quiet, sigma, depth=3)   # checks the device status


def test_wave_marine_full_steps():
    wl = W.marine_1d()
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, nt=emm.steps_for(wl, grid))
    sigma = _sig(wl)
    ref, _ = emm.forward(grid, survey, sigma)
    G, _ = emm.forward_wave(grid, survey, sigma, depth=2)
    assert torch.equal(G, ref)
