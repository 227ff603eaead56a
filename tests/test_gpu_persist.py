"""Persistent work list (emm_forward_persistent): several problems -- grids
of uneven sizes, one of them a batch of transmitters -- advanced in one
cooperative launch with grid barriers between the half-steps.

* Every problem's receiver Green's functions equal its own emm_forward (or
  emm_forward_batch) result bit for bit: the same per-CTA code runs on the
  same inputs, only the launch differs.
* One problem against the FP64 oracle within the parity bound.
* The CUDA-graph plan of the whole solve replays to the same bits, and
  follows new conductivity values written into the bound buffers.
* The autotuner times both tile shapes (32 x 8 x 2 and 32 x 4 x 4 cells)
  with every resident-CTA count and returns the fastest; both shapes give
  the same bits.
* Bounded waits: a two-CTA launch whose second CTA withholds its arrival at
  the first grid barrier (a host-set test option; no fault, trap or endless
  loop) ends with EMM_ETIMEOUT after the short wait bound, and the next
  clean run on the same workspace gives EMM_OK and the right bits.  The
  host's convergence poll likewise gives EMM_ETIMEOUT under a tiny bound
  and drains the stream."""
import dataclasses

import numpy as np
import pytest

import oracle
import paper_2304_00233_b300 as emm
from paper_2304_00233_b300 import workloads as W

from _parity import REL_L2_TOL, compare_G

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def _tasks(rd, nt=60):
    """Three problems of one order: two single transmitters on different
    small grids and a batch of three transmitters on a third grid."""
    cases = [W.small_case(n=(40, 36, 30), rd=rd, seed=3, nt=nt, volume=False, nfreq=2),
             W.small_case(n=(29, 33, 27), rd=rd, seed=4, nt=nt - 17, volume=False, nfreq=2),
             W.small_case(n=(45, 31, 25), rd=rd, seed=5, nt=nt, volume=False, nfreq=2)]
    tasks, sigmas = [], []
    for k, wl in enumerate(cases):
        grid = emm.grid_for(wl)
        survey = emm.survey_for(wl)
        pos = None
        if k == 2:
            c = np.array(survey.src)
            pos = np.array([c, c + [40.0, -25.0, 10.0], c + [-35.0, 20.0, -15.0]])
        tasks.append((grid, survey, pos))
        sigmas.append(torch.from_numpy(wl.sigma.astype(np.float32)).cuda())
    return cases, tasks, sigmas


def _singles(tasks, sigmas):
    out = []
    for (grid, survey, pos), sg in zip(tasks, sigmas):
        if pos is None:
            G, _ = emm.forward(grid, survey, sg)
            out.append(G[None])
        else:
            G, _ = emm.forward_batch(grid, survey, sg, pos)
            out.append(G)
    return out


@pytest.mark.parametrize("rd", [2, 4])
def test_persistent_equals_single_solves_bitwise(rd):
    _, tasks, sigmas = _tasks(rd)
    work = emm.PersistWork(tasks)
    got = emm.forward_persistent(work, sigmas, opts=emm.PersistOpts())
    ref = _singles(tasks, sigmas)
    for g, r in zip(got, ref):
        assert torch.equal(g, r)
    # fewer resident CTAs per SM, and the other tile shape: other walks and
    # other tiles over the same cells, the same arithmetic per cell
    for opts in (emm.PersistOpts(ctas_per_sm=1), emm.PersistOpts(tile_shape=1), emm.PersistOpts(2, tile_shape=1)):
        got1 = emm.forward_persistent(work, sigmas, opts=opts)
        for g, r in zip(got1, ref):
            assert torch.equal(g, r), opts


def test_persistent_against_oracle():
    cases, tasks, sigmas = _tasks(3, nt=80)
    work = emm.PersistWork(tasks[:2])
    got = emm.forward_persistent(work, sigmas[:2], opts=emm.PersistOpts())
    ref = oracle.forward_workload(cases[1], nt=tasks[1][1].nt)
    eE, eH = compare_G(got[1][0].cpu().numpy(), ref["G"])
    assert eE < REL_L2_TOL and eH < REL_L2_TOL, (eE, eH)


def test_persistent_graph_plan_and_tuner():
    _, tasks, sigmas = _tasks(2)
    work = emm.PersistWork(tasks)
    best, ms = emm.persist_tune(work, sigmas, steps=10)
    # every tile shape with every resident-CTA count up to its occupancy limit
    assert {k[0] for k in ms} == {0, 1} and best.key() in ms and all(v > 0 for v in ms.values())
    assert min(ms, key=ms.get) == best.key()
    ref = [g.clone() for g in emm.forward_persistent(work, sigmas, opts=best)]
    plan = emm.PersistPlan(work, sigmas, opts=best)
    plan.run_async()
    top, each = work.status()
    assert top == emm.EMM_OK and all(v == emm.EMM_OK for v in each)
    for g, r in zip(work.G(), ref):
        assert torch.equal(g, r)
    # new values in the bound conductivity buffers: the replay follows them
    for sg in sigmas:
        sg.mul_(1.5)
    new = [g.clone() for g in emm.forward_persistent(work, sigmas, opts=best)]
    for g in work.rec:
        g.zero_()
    plan.run_async()
    work.status()
    for g, r, old in zip(work.G(), new, ref):
        assert torch.equal(g, r) and not torch.equal(r, old)
    plan.close()


def test_grid_barrier_wait_runs_out_then_clean_run():
    _, tasks, sigmas = _tasks(2, nt=20)
    work = emm.PersistWork(tasks)
    ref = [g.clone() for g in emm.forward_persistent(work, sigmas, opts=emm.PersistOpts())]
    # two resident CTAs; CTA 1 leaves without arriving at the first barrier
    bad = emm.PersistOpts(max_ctas=2, wait_s=0.02, skip_arrival=1)
    emm.forward_persistent(work, sigmas, opts=bad, check=False)
    top, _ = work.status()
    assert top == emm.EMM_ETIMEOUT
    got = emm.forward_persistent(work, sigmas, opts=emm.PersistOpts())
    top, each = work.status()
    assert top == emm.EMM_OK and all(v == emm.EMM_OK for v in each)
    for g, r in zip(got, ref):
        assert torch.equal(g, r)


def test_convergence_poll_timeout_drains_stream(monkeypatch):
    wl = W.marine_1d()
    grid = emm.grid_for(wl)
    survey = emm.survey_for(wl, nt=400)
    sigma = torch.from_numpy(wl.sigma.astype(np.float32)).cuda()
    work = emm.Workspace(grid, survey)
    monkeypatch.setenv("EMM_POLL_TIMEOUT_S", "1e-9")
    with pytest.raises(emm.EmmError) as err:
        emm.forward_converge(grid, survey, sigma, work)
    assert err.value.code == emm.EMM_ETIMEOUT
    monkeypatch.delenv("EMM_POLL_TIMEOUT_S")
    # the stream was drained: the next run proceeds normally
    short = dataclasses.replace(survey, nt=150)
    n = emm.forward_converge(grid, short, sigma, work)
    assert n == 150 and emm.status(work) == emm.EMM_OK
