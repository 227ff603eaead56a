"""Air above the model (Sec. 3.3) on the GPU against the FP64 oracle, whose
air continuation is pinned on Fourier modes (tests/test_oracle_airwave.py).

Uniform x and y (the DFT of the interface plane needs it), a stretched z
axis, a sea of 1 S/m over a resistive layer, a tilted dipole and receivers
below the interface.  The GPU runs the plane DFTs in FP32 (direct sums with
FP64-tabulated twiddles); the bound is the usual relative L2 of 2e-4 over
entries above 1e-6 of the maximum."""
import math

import numpy as np
import pytest

import oracle
import paper_2304_00233_b300 as emm
from paper_2304_00233_b300 import workloads as W

from _parity import REL_L2_TOL, compare_G

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def _air_workload(rd, nt=200):
    x = np.arange(28) * 60.0 - 810.0
    y = np.arange(24) * 70.0 - 805.0
    z = np.concatenate([[0.0], np.cumsum(40.0 * 1.04 ** np.arange(21))])
    cell = np.ones((len(z) - 1, len(y) - 1, len(x) - 1))
    cell[12:14] = 0.05
    sig = W.staggered_conductivity(cell, 0.8 * cell, x, y, z).astype(np.float32).astype(np.float64)
    rec = np.array([[-300.0, 40.0, 60.0], [250.0, -100.0, 100.0], [420.0, 210.0, 45.0],
                    [-90.0, -330.0, 150.0]])
    return W.Workload(f"air_rd{rd}", x, y, z, sig, rd, 8, rd + 3, np.array([35.0, -20.0, 160.0]),
                      0.4, 0.3, 1.0, rec, np.array([0.5, 1.5]), 2 * math.pi, 2.0, 0.0,
                      volume=True, nt=nt)


@pytest.mark.parametrize("rd", [1, 2, 3, 4])
def test_airwave_against_oracle(rd):
    wl = _air_workload(rd)
    ref = oracle.forward_workload(wl, airwave=True)
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, airwave=True)
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    G, vol = emm.forward(grid, survey, sigma)
    eE, eH = compare_G(G.cpu().numpy(), ref["G"])
    assert eE < REL_L2_TOL and eH < REL_L2_TOL, (eE, eH)
    vE, vH = compare_G(vol.cpu().numpy(), ref["vol"])
    assert vE < REL_L2_TOL and vH < REL_L2_TOL, (vE, vH)
    # the air changes the fields (the boundary is live)
    G0, _ = emm.forward(grid, emm.survey_for(wl), sigma)
    assert np.abs(G0.cpu().numpy() - G.cpu().numpy()).max() > 1e-3 * np.abs(G0.cpu().numpy()).max()


@pytest.mark.parametrize("rd", [1, 2, 3, 4])
def test_split_air_solve_equals_the_sequential_one(rd):
    # without the volume DTFT an electric-dipole air solve launches each
    # half-step in two parts on two streams (the tile layers next to the
    # interface, with the air transforms, beside the rest); with it, one
    # sequence on one stream.  The same cells by the same arithmetic: the
    # receivers get the same bits.
    wl = _air_workload(rd, nt=150)
    grid = emm.grid_for(wl)
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    G_seq, _ = emm.forward(grid, emm.survey_for(wl, airwave=True), sigma)
    wl.volume = False
    G_split, vol = emm.forward(grid, emm.survey_for(wl, airwave=True), sigma)
    assert vol is None
    assert torch.equal(G_split, G_seq)


def test_airwave_batch_bitwise_equal_to_single_solves():
    wl = _air_workload(2, nt=60)
    wl.volume = False
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, airwave=True)
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    pos = np.array([wl.src, wl.src + np.array([-60.0, 30.0, 20.0])])
    Gb, _ = emm.forward_batch(grid, survey, sigma, pos)
    Gb = Gb.cpu().numpy()
    for k in range(len(pos)):
        G1, _ = emm.forward(grid, emm.survey_for(wl, airwave=True, src=tuple(pos[k])), sigma)
        assert np.array_equal(Gb[k], G1.cpu().numpy())


def test_airwave_rejects_non_uniform_xy_and_shallow_sources():
    wl = W.small_case(rd=2, nt=5, volume=False)
    grid = emm.grid_for(wl)
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    with pytest.raises(emm.EmmError) as e:
        emm.forward(grid, emm.survey_for(wl, airwave=True), sigma)
    assert e.value.code == emm.EMM_EINVAL
    aw = _air_workload(2, nt=5)
    aw.volume = False
    g2 = emm.grid_for(aw)
    s2 = torch.from_numpy(aw.sigma.astype(np.float32)).cuda()
    with pytest.raises(emm.EmmError) as e:
        emm.forward(g2, emm.survey_for(aw, airwave=True, src=(35.0, -20.0, 10.0)), s2)
    assert e.value.code == emm.EMM_EOUTSIDE
