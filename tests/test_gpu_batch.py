"""Batched transmitters (emm_forward_batch) against one-at-a-time solves.

Several transmitters on one grid and conductivity advance in the same
launches; each must give exactly (bitwise) what emm_forward gives for it
alone, and the FP64 oracle's Green's functions within the parity bound."""
import numpy as np
import pytest

import oracle
import paper_2304_00233_b300 as emm
from paper_2304_00233_b300 import workloads as W

from _parity import REL_L2_TOL, compare_G

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def _positions(wl, k):
    rng = np.random.default_rng(99)
    c = np.array([0.5 * (wl.x[0] + wl.x[-1]), 0.5 * (wl.y[0] + wl.y[-1]), 0.5 * (wl.z[0] + wl.z[-1])])
    span = np.array([wl.x[-1] - wl.x[0], wl.y[-1] - wl.y[0], wl.z[-1] - wl.z[0]])
    return c + rng.uniform(-0.2, 0.2, (k, 3)) * span


@pytest.mark.parametrize("rd,n", [(2, (37, 29, 23)), (4, (41, 38, 31))], ids=["rd2", "rd4"])
def test_batch_equals_single_solves(rd, n):
    wl = W.small_case(rd=rd, n=n, nt=120, volume=False, nfreq=2)
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, nt=wl.nt)
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    pos = _positions(wl, 3)
    Gb, _ = emm.forward_batch(grid, survey, sigma, pos)
    torch.cuda.synchronize()
    for k in range(3):
        sk = emm.survey_for(wl, nt=wl.nt, src=tuple(pos[k]))
        Gk, _ = emm.forward(grid, sk, sigma)
        assert torch.equal(Gb[k], Gk), k


def test_batch_against_oracle():
    wl = W.small_case(rd=3, n=(45, 33, 26), nt=140, volume=False, nfreq=3)
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, nt=wl.nt)
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    pos = _positions(wl, 2)
    Gb, _ = emm.forward_batch(grid, survey, sigma, pos)
    Gb = Gb.cpu().numpy()
    for k in range(2):
        ref = oracle.forward_workload(wl, src=tuple(pos[k]))
        eE, eH = compare_G(Gb[k], ref["G"])
        assert eE < REL_L2_TOL and eH < REL_L2_TOL, (k, eE, eH)
