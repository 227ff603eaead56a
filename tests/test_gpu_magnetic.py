"""Magnetic dipole sources (survey.src_kind = 1) on the GPU against the FP64
oracle, which is pinned to the analytic whole-space magnetic dipole
(tests/test_oracle_physics.py, P8M).

M sits on the H samples and enters the H update at t_{n+1}; the outputs are
G^EH and G^HH (the correspondence of Eq. 5).  Same bound as the electric
parity tests: relative L2 2e-4 over entries above 1e-6 of the maximum, for
the receivers and the volume DTFT."""
import numpy as np
import pytest

import oracle
import paper_2304_00233_b300 as emm
from paper_2304_00233_b300 import workloads as W

from _parity import REL_L2_TOL, compare_G

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

SMALL = [dict(rd=1, n=(40, 36, 30)), dict(rd=2, n=(37, 29, 23)), dict(rd=3, n=(45, 33, 26)),
         dict(rd=4, n=(41, 38, 31))]


@pytest.mark.parametrize("case", SMALL, ids=[f"rd{c['rd']}" for c in SMALL])
def test_magnetic_source_against_oracle(case):
    wl = W.small_case(rd=case["rd"], n=case["n"], nt=160, volume=True, nfreq=3)
    ref = oracle.forward_workload(wl, magnetic=True)
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, nt=160, src_kind=1)
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    G, vol = emm.forward(grid, survey, sigma)
    eE, eH = compare_G(G.cpu().numpy(), ref["G"])
    assert eE < REL_L2_TOL and eH < REL_L2_TOL, (eE, eH)
    vE, vH = compare_G(vol.cpu().numpy(), ref["vol"])
    assert vE < REL_L2_TOL and vH < REL_L2_TOL, (vE, vH)


def test_magnetic_source_differs_from_electric():
    # the same dipole as J and as M gives different fields (the switch is live)
    wl = W.small_case(rd=2, nt=80, volume=False, nfreq=2)
    grid = emm.grid_for(wl)
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    ge, _ = emm.forward(grid, emm.survey_for(wl, nt=80), sigma)
    gm, _ = emm.forward(grid, emm.survey_for(wl, nt=80, src_kind=1), sigma)
    ge, gm = ge.cpu().numpy(), gm.cpu().numpy()
    assert np.abs(ge - gm).max() > 0.1 * np.abs(ge).max()


def test_magnetic_batch_bitwise_equal_to_single_solves():
    wl = W.small_case(rd=2, nt=60, volume=False, nfreq=2)
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, nt=60, src_kind=1)
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    pos = np.array([wl.src, wl.src + np.array([40.0, -25.0, 10.0])])
    Gb, _ = emm.forward_batch(grid, survey, sigma, pos)
    Gb = Gb.cpu().numpy()
    for k in range(len(pos)):
        single = emm.survey_for(wl, nt=60, src_kind=1, src=tuple(pos[k]))
        G1, _ = emm.forward(grid, single, sigma)
        assert np.array_equal(Gb[k], G1.cpu().numpy())


def test_gradient_rejects_magnetic_source():
    wl = W.small_case(rd=2, nt=20, volume=False, nfreq=2)
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, nt=20, src_kind=1)
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    dG = torch.zeros((survey.nrec, 6, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(emm.EmmError):
        emm.vjp(grid, survey, sigma, dG)
