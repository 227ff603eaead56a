"""emm_forward_static (the entry point that allocates no device memory)
against emm_forward, through the C-ABI.

Two calls in a row on different problems (the second finds the first one's
contents in the shared static scratch) must each match emm_forward on the same
inputs within the parity bound; a problem beyond the scratch size is refused
with EMM_EWORKSPACE before anything is enqueued; a second call leaves the
device's free memory unchanged.  This file is collected last
so that it runs both alone in a fresh process and after every other test."""
import numpy as np
import pytest

import paper_2304_00233_b300 as emm
from paper_2304_00233_b300 import workloads as W

from _parity import REL_L2_TOL, compare_G

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

EMM_OK, EMM_EWORKSPACE = 0, 6


def _problem(rd, n, volume, seed):
    wl = W.small_case(rd=rd, n=n, nt=150, volume=volume, nfreq=2, seed=seed)
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, nt=150)
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    return grid, survey, sigma


def _outputs(grid, survey):
    nf = len(survey.freqs)
    rec = torch.full((max(survey.nrec, 1), 6, nf, 2), float("nan"), dtype=torch.float64, device="cuda")
    vol = None
    if survey.volume:
        n1, n2, n3 = grid.n
        vol = torch.full((6, nf, n3, n2, n1, 2), float("nan"), dtype=torch.float64, device="cuda")
    return rec, vol


def _as_complex(a):
    a = a.cpu().numpy()
    return a[..., 0] + 1j * a[..., 1]


def test_static_scratch_matches_workspace_entry_point_twice():
    cases = [dict(rd=2, n=(37, 29, 23), volume=True, seed=11),
             dict(rd=3, n=(33, 41, 27), volume=False, seed=12)]
    for case in cases:
        grid, survey, sigma = _problem(**case)
        assert emm.workspace_size(grid, survey) <= (64 << 20)
        rec, vol = _outputs(grid, survey)
        st = emm.forward_static(grid, survey, sigma, rec, vol)
        assert st == EMM_OK
        G_ref, vol_ref = emm.forward(grid, survey, sigma)
        torch.cuda.synchronize()
        eE, eH = compare_G(_as_complex(rec)[: survey.nrec], G_ref.cpu().numpy())
        assert eE < REL_L2_TOL and eH < REL_L2_TOL, (case, eE, eH)
        if survey.volume:
            vE, vH = compare_G(_as_complex(vol), vol_ref.cpu().numpy())
            assert vE < REL_L2_TOL and vH < REL_L2_TOL, (case, vE, vH)


def test_second_static_call_changes_no_device_memory():
    # the first call may load the library's device code (and with it the
    # static array); the second must leave the device's free memory as it was
    grid, survey, sigma = _problem(rd=2, n=(31, 27, 25), volume=True, seed=13)
    rec, vol = _outputs(grid, survey)
    assert emm.forward_static(grid, survey, sigma, rec, vol) == EMM_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert emm.forward_static(grid, survey, sigma, rec, vol) == EMM_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_scratch_refuses_oversized_problem():
    wl = W.marine_1d()
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, nt=4)
    assert emm.workspace_size(grid, survey) > (64 << 20)
    sigma = torch.ones((3,) + tuple(reversed(grid.n)), dtype=torch.float32, device="cuda")
    rec, vol = _outputs(grid, survey)
    with pytest.raises(emm.EmmError) as err:
        emm.forward_static(grid, survey, sigma, rec, vol)
    assert err.value.code == EMM_EWORKSPACE
    torch.cuda.synchronize()
    assert torch.isnan(rec).all()  # nothing was enqueued
