"""Forward-solve plans (emm_plan_create / emm_plan_run): the time loop
captured once as a CUDA graph and replayed.  Every run must give exactly
what emm_forward gives for the same conductivity (the same launches, with
the same parameters, in the same order), for a second conductivity on the
same plan, and with the launches a magnetic source adds."""
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
