"""Forward-solve plans (emm_plan_create / emm_plan_run): the time loop
captured once as a CUDA graph and replayed.  Every run must give exactly
what emm_forward gives for the same conductivity (the same launches, with
the same parameters, in the same order), for a second conductivity on the
same plan, with the launches a magnetic source adds, and with the air
boundary's plane transforms in the captured loop."""
import numpy as np
import pytest

import paper_2304_00233_b300 as emm
from paper_2304_00233_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def _sig(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("kind", [0, 1])
def test_plan_runs_equal_forward(kind):
    wl = W.small_case(rd=2, n=(33, 29, 25), nt=90, volume=True, nfreq=2)
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, src_kind=kind)
    s1 = _sig(wl.sigma)
    # a second model, no conductivity below the survey's sigma_min
    s2 = _sig(wl.sigma * (1.2 + 0.2 * np.sin(np.arange(wl.sigma.size) * 0.37)).reshape(wl.sigma.shape))
    plan = emm.Plan(grid, survey, s1)
    for sg in (s1, s2, s1):
        G, vol = plan.run(sg)
        G_ref, vol_ref = emm.forward(grid, survey, sg)
        assert torch.equal(G, G_ref)
        assert torch.equal(vol, vol_ref)


def test_plan_with_air_boundary_equals_forward_and_closes():
    # the air boundary adds the plane-transform launches after every half
    # step to the captured loop; the plan is closed explicitly and the
    # workspace then serves a plain solve
    from test_gpu_airwave import _air_workload
    wl = _air_workload(2, nt=80)
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, airwave=True)
    s1 = _sig(wl.sigma)
    work = emm.Workspace(grid, survey)
    plan = emm.Plan(grid, survey, s1, work)
    G, vol = plan.run(s1)
    G = G.clone()
    vol = vol.clone()
    plan.close()
    G_ref, vol_ref = emm.forward(grid, survey, s1)
    assert torch.equal(G, G_ref) and torch.equal(vol, vol_ref)
    G2, _ = emm.forward(grid, survey, s1, work)
    assert torch.equal(G2, G_ref)
