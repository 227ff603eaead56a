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


def test_plan_of_a_split_air_solve_equals_forward():
    # without the volume DTFT the air solve runs on two streams; the plan
    # captures both (forked from and joined back to its stream)
    from test_gpu_airwave import _air_workload
    wl = _air_workload(3, nt=70)
    wl.volume = False
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, airwave=True)
    s1 = _sig(wl.sigma)
    plan = emm.Plan(grid, survey, s1)
    for _ in range(2):
        G, _ = plan.run(s1)
        G_ref, _ = emm.forward(grid, survey, s1)
        assert torch.equal(G, G_ref)
    plan.close()


_PLAN_THEN_JOBS = r"""
import dataclasses, sys
import numpy as np, torch
import paper_2304_00233_b300 as emm
from paper_2304_00233_b300 import workloads as W
wl = W.marine_1d()
g = emm.grid_for(wl)
s = emm.survey_for(wl, nt=emm.steps_for(wl, g))
sg = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
plan = emm.Plan(g, s, sg, emm.Workspace(g, s))
for _ in range(4):
    plan.run_async(sg)
torch.cuda.synchronize()
plan.close()
probs, sig = [], []
for w in W.uneven_jobs():
    gj = emm.grid_for(w)
    probs.append((gj, emm.survey_for(w, nt=30)))
    sig.append(torch.from_numpy(w.sigma.astype(np.float32)).cuda())
ref, _ = emm.forward_jobs(probs, sig, strategy=emm.JOBS_SEQUENTIAL)
ref = [r.clone() for r in ref]
for k in (emm.JOBS_STREAMS, emm.JOBS_LIST):
    out, _ = emm.forward_jobs(probs, sig, strategy=k)
    assert all(torch.equal(a, b) for a, b in zip(out, ref)), emm.JOBS_STRATEGIES[k]
torch.cuda.synchronize()
print("plan-then-jobs ok")
"""


def test_jobs_after_plan_complete_and_agree():
    # a full-length marine plan replayed four times, then the eight uneven
    # grids as work lists in one process: every strategy completes and
    # gives the sequential strategy's bits.  (With programmatic dependent
    # launches on the stream-per-problem strategy's own streams this
    # sequence once never completed; those launches are now plain ones.)
    # A child process with a time limit turns a recurrence into a failure.
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _PLAN_THEN_JOBS], cwd=root, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "plan-then-jobs ok" in r.stdout
