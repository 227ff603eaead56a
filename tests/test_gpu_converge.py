"""Device-side convergence termination (the corner test of Sec. 4.1) against
the FP64 oracle's own corner test.

The stop step is an integer both paths decide from their corner DTFTs (FP32
fields accumulated in FP64 here, FP64 fields in the oracle); the cases below
converge well inside the step range, and the test asserts the same stop step.
The Green's functions then meet the usual 2e-4 bound, and equal bit for bit a
plain emm_forward of that many steps (the same arithmetic, stopped)."""
import numpy as np
import pytest

import oracle
import paper_2304_00233_b300 as emm
from paper_2304_00233_b300 import workloads as W

from _parity import REL_L2_TOL, compare_G

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

NT_MAX = 4000


def _converge(wl, nt_max):
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, nt=nt_max)
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    work = emm.Workspace(grid, survey)
    n = emm.forward_converge(grid, survey, sigma, work)
    assert emm.status(work) == emm.EMM_OK
    G = torch.view_as_complex(work.rec)[: survey.nrec].cpu().numpy()
    return n, G, grid, sigma


def _plain(wl, grid, sigma, nt):
    survey = emm.survey_for(wl, nt=nt)
    G, _ = emm.forward(grid, survey, sigma)
    return G.cpu().numpy()


@pytest.mark.parametrize("rd", [1, 2, 4])
def test_stop_step_and_green_functions_match_oracle(rd):
    wl = W.small_case(rd=rd, nt=NT_MAX, volume=False, nfreq=2)
    ref = oracle.forward_workload(wl, convergence=True)
    assert ref["nt"] < NT_MAX  # the case converges inside the range
    n, G, grid, sigma = _converge(wl, NT_MAX)
    assert n == ref["nt"]
    eE, eH = compare_G(G, ref["G"])
    assert eE < REL_L2_TOL and eH < REL_L2_TOL, (eE, eH)
    assert np.array_equal(G, _plain(wl, grid, sigma, n))


def test_step_limit_before_convergence():
    wl = W.small_case(rd=2, nt=NT_MAX, volume=False, nfreq=2)
    n, G, grid, sigma = _converge(wl, 350)  # checks after steps 0, 100, 200, 300
    assert n == 350
    assert np.array_equal(G, _plain(wl, grid, sigma, 350))


def test_fewer_steps_than_the_first_check():
    wl = W.small_case(rd=2, nt=NT_MAX, volume=False, nfreq=2)
    n, G, grid, sigma = _converge(wl, 60)
    assert n == 60
    assert np.array_equal(G, _plain(wl, grid, sigma, 60))
