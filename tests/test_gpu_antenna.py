"""Antennas of finite length (survey.src_length > 0) on the GPU against the
FP64 oracle, whose antenna is pinned by superposition
(tests/test_oracle_physics.py::test_extended_antenna_is_the_mean_of_its_sub_dipoles).

The current is spread over src_points sub-dipoles at the midpoints of equal
segments; the GPU sums their stencils on the union box of each component and
injects it in a separate launch after the E (electric) or H (magnetic) step.
Bound as for the point dipoles: relative L2 2e-4 over entries above 1e-6 of
the maximum."""
import numpy as np
import pytest

import oracle
import paper_2304_00233_b300 as emm
from paper_2304_00233_b300 import workloads as W

from _parity import REL_L2_TOL, compare_G

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

CASES = [dict(rd=2, n=(37, 29, 23), kind=0), dict(rd=3, n=(45, 33, 26), kind=1),
         dict(rd=4, n=(41, 38, 31), kind=0)]


@pytest.mark.parametrize("case", CASES, ids=[f"rd{c['rd']}_kind{c['kind']}" for c in CASES])
def test_antenna_against_oracle(case):
    wl = W.small_case(rd=case["rd"], n=case["n"], nt=160, volume=True, nfreq=3)
    ref = oracle.forward_workload(wl, src_length=150.0, src_points=4, magnetic=bool(case["kind"]))
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, nt=160, src_kind=case["kind"], src_length=150.0, src_points=4)
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    G, vol = emm.forward(grid, survey, sigma)
    eE, eH = compare_G(G.cpu().numpy(), ref["G"])
    assert eE < REL_L2_TOL and eH < REL_L2_TOL, (eE, eH)
    vE, vH = compare_G(vol.cpu().numpy(), ref["vol"])
    assert vE < REL_L2_TOL and vH < REL_L2_TOL, (vE, vH)


def test_one_point_antenna_matches_the_point_dipole():
    # one sub-dipole sits at the centre: the separate injection launch gives the
    # fused point-dipole result up to the rounding of the split update
    wl = W.small_case(rd=2, nt=120, volume=False, nfreq=2)
    grid = emm.grid_for(wl)
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    gp, _ = emm.forward(grid, emm.survey_for(wl, nt=120), sigma)
    ga, _ = emm.forward(grid, emm.survey_for(wl, nt=120, src_length=80.0, src_points=1), sigma)
    gp, ga = gp.cpu().numpy(), ga.cpu().numpy()
    assert np.abs(ga - gp).max() <= 1e-5 * np.abs(gp).max()


def test_antenna_batch_bitwise_equal_to_single_solves():
    wl = W.small_case(rd=2, nt=60, volume=False, nfreq=2)
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, nt=60, src_length=120.0, src_points=3)
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    pos = np.array([wl.src, wl.src + np.array([-30.0, 20.0, 5.0])])
    Gb, _ = emm.forward_batch(grid, survey, sigma, pos)
    Gb = Gb.cpu().numpy()
    for k in range(len(pos)):
        single = emm.survey_for(wl, nt=60, src_length=120.0, src_points=3, src=tuple(pos[k]))
        G1, _ = emm.forward(grid, single, sigma)
        assert np.array_equal(Gb[k], G1.cpu().numpy())
