"""Work-list solves (emm_forward_jobs): several problems of uneven grid
sizes, step counts and receiver sets advanced together, by each strategy
(work-list launches, one after the other, one stream each) and by the one
the autotuner picks.

Each problem's Green's functions must equal a plain emm_forward of that
problem bit for bit (every CTA runs the same code on the same data as in
the problem's own launch), and one of them is checked against the FP64
oracle directly, for rd = 2 and 4."""
import numpy as np
import pytest

import oracle
import paper_2304_00233_b300 as emm
from paper_2304_00233_b300 import workloads as W

from _parity import REL_L2_TOL, compare_G

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


@pytest.mark.parametrize("rd", [2, 4])
def test_uneven_problems_equal_single_solves(rd):
    wls = [W.small_case(n=(24, 21, 18), rd=rd, seed=1, nt=90, volume=False, nfreq=2),
           W.small_case(n=(41, 35, 29), rd=rd, seed=2, nt=130, volume=False, nfreq=3),
           W.small_case(n=(30, 44, 26), rd=rd, seed=3, nt=60, volume=False, nfreq=1)]
    probs = [(emm.grid_for(w), emm.survey_for(w)) for w in wls]
    sig = [torch.from_numpy(w.sigma.astype(np.float32)).cuda() for w in wls]
    singles = [emm.forward(g, s, sg)[0] for (g, s), sg in zip(probs, sig)]
    work = None
    for strategy in (emm.JOBS_LIST, emm.JOBS_SEQUENTIAL, emm.JOBS_STREAMS):
        Gs, work = emm.forward_jobs(probs, sig, work=work, strategy=strategy)
        for G, G1 in zip(Gs, singles):
            assert torch.equal(G, G1), strategy
    # the autotuner picks one of them; the solve after it is the same again
    best, ms = emm.jobs_tune(probs, sig, work, steps=20)
    assert best in (emm.JOBS_LIST, emm.JOBS_SEQUENTIAL, emm.JOBS_STREAMS)
    assert all(t > 0 for t in ms.values())
    Gs, _ = emm.forward_jobs(probs, sig, work=work)
    assert work.strategy is not None and all(torch.equal(a, b) for a, b in zip(Gs, singles))
    ref = oracle.forward_workload(wls[1])
    eE, eH = compare_G(Gs[1].cpu().numpy(), ref["G"])
    assert eE < REL_L2_TOL and eH < REL_L2_TOL, (eE, eH)


def test_one_problem_and_the_full_list():
    wl = W.small_case(n=(22, 20, 18), rd=2, seed=5, nt=70, volume=False)
    g, s = emm.grid_for(wl), emm.survey_for(wl)
    sg = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    (G,), _ = emm.forward_jobs([(g, s)], [sg], strategy=emm.JOBS_LIST)
    G1, _ = emm.forward(g, s, sg)
    assert torch.equal(G, G1)
    # sixteen problems (the most one list takes), alternating two sizes
    wl2 = W.small_case(n=(19, 17, 15), rd=2, seed=6, nt=40, volume=False)
    g2, s2 = emm.grid_for(wl2), emm.survey_for(wl2)
    sg2 = torch.from_numpy(wl2.sigma.astype(np.float32)).cuda()
    probs = [(g, s), (g2, s2)] * 8
    Gs, _ = emm.forward_jobs(probs, [sg, sg2] * 8, strategy=emm.JOBS_LIST)
    G2, _ = emm.forward(g2, s2, sg2)
    for k, Gk in enumerate(Gs):
        assert torch.equal(Gk, G1 if k % 2 == 0 else G2)
