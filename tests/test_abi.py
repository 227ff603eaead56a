"""The C-ABI library loads (no GPU needed) and exports every function that
include/emm.h declares; host-side error paths return the documented codes."""
import os
import re

import numpy as np
import pytest

import paper_2304_00233_b300 as emm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(emm_\w+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    lib = emm.load_library()
    declared = _declared()
    assert declared, "no declarations parsed"
    assert declared == set(emm.EXPORTED), declared ^ set(emm.EXPORTED)
    for name in declared:
        assert hasattr(lib, name), name


def test_strerror_codes():
    for code in range(9):
        assert emm.strerror(code)
    assert emm.strerror(99) == "unknown error"


def test_grid_errors():
    x = np.arange(10.0)
    with pytest.raises(emm.EmmError) as e:
        emm.make_grid(x, x, x, rd=5)
    assert e.value.code == emm.EMM_EINVAL
    with pytest.raises(emm.EmmError):
        emm.make_grid(x[::-1], x, x, rd=2)           # not ascending
    with pytest.raises(emm.EmmError):
        emm.make_grid(x, x, x, rd=3, nb=2)          # nb < rd
    g = emm.make_grid(x, x, x, rd=2, nb=4, ne=3)
    assert g.npad == (24, 24, 24) and g.cells == 24 ** 3
    with pytest.raises(emm.EmmError) as e:
        g.locate(0, (-100.0, 4.0, 4.0))             # left of the grid
    assert e.value.code == emm.EMM_EOUTSIDE
    with pytest.raises(emm.EmmError) as e:
        g.locate(0, (-4.5, 4.0, 4.0))               # inside the pads but in the CPML
    assert e.value.code == emm.EMM_EOUTSIDE
    g.locate(0, (4.2, 4.0, 4.0))


def test_survey_errors_before_any_device_call():
    x = np.arange(12.0) * 10
    g = emm.make_grid(x, x, x, rd=2, nb=4, ne=3)
    good = emm.Survey(omega0=1.0, fmax=1.0, sigma_min=1.0, nt=10, src=(55, 55, 55),
                      rec=np.array([[40.0, 50.0, 60.0]]), freqs=[1.0])
    assert emm.workspace_size(g, good) > 0
    for bad in (dict(omega0=0.0), dict(fmax=-1.0), dict(sigma_min=0.0), dict(nt=-1), dict(freqs=[]),
                dict(src_kind=2), dict(src_length=-1.0), dict(src_length=100.0, src_points=0),
                dict(src_length=100.0, src_points=257)):
        s = emm.Survey(**{**good.__dict__, **bad})
        with pytest.raises(emm.EmmError) as e:
            emm.workspace_size(g, s)
        assert e.value.code == emm.EMM_EINVAL


def test_antenna_workspace_holds_the_union_boxes():
    # an antenna's weights need more room than a point dipole's (2rd)^3 boxes
    x = np.arange(40.0) * 10
    g = emm.make_grid(x, x, x, rd=2, nb=4, ne=3)
    point = emm.Survey(omega0=1.0, fmax=1.0, sigma_min=1.0, nt=10, src=(195, 195, 195),
                       rec=np.array([[150.0, 150.0, 150.0]]), freqs=[1.0])
    ant = emm.Survey(**{**point.__dict__, "src_length": 60.0, "src_points": 6})
    assert emm.workspace_size(g, ant) > emm.workspace_size(g, point)



def test_volume_ring_depth_matches_the_header_and_the_workspace():
    # EMM_VOLUME_RING in the header, the binding's constant and the field
    # ring the workspace holds for a solve with the volume DTFT agree
    hdr = open(os.path.join(ROOT, "include", "emm.h")).read()
    assert int(re.search(r"#define EMM_VOLUME_RING (\d+)", hdr).group(1)) == emm.VOLUME_RING
    x = np.arange(1000.0) * 10
    y = np.arange(6.0) * 10
    g = emm.make_grid(x, y, y, rd=2, nb=4, ne=3)
    s0 = emm.Survey(omega0=1.0, fmax=1.0, sigma_min=1.0, nt=10, src=(4995, 25, 25),
                    rec=np.array([[4000.0, 25.0, 25.0]]), freqs=[1.0, 2.0])
    s1 = emm.Survey(**{**s0.__dict__, "volume": True})
    nint = 1000 * 6 * 6
    acc = 6 * 2 * nint * 16                 # compensated accumulators
    cells = int(np.prod(g.npad)) * 4        # bytes of one field component (rows unpadded)
    ring = emm.workspace_size(g, s1) - emm.workspace_size(g, s0) - acc
    k = emm.VOLUME_RING - 1                 # slots beside the state's own
    assert k * 6 * cells <= ring <= k * 6 * (cells * 1.07 + 256) + 256


def test_work_list_layout_and_errors():
    from paper_2304_00233_b300 import workloads as W
    wls = [W.small_case(n=(20, 18, 16), rd=2, nt=10, volume=False), W.small_case(n=(26, 22, 19), rd=2, nt=12,
                                                                                  volume=False)]
    probs = [(emm.grid_for(w), emm.survey_for(w)) for w in wls]
    sizes = [emm.workspace_size(g, s) for g, s in probs]
    jobs, keep = emm._jobs_c(probs, [None, None], [None, None])
    n = emm.C.c_size_t(0)
    offs = (emm.C.c_size_t * 2)()
    assert emm.load_library().emm_jobs_workspace_size(2, jobs, emm.C.byref(n), offs) == emm.EMM_OK
    assert offs[0] == 0 and offs[1] >= sizes[0] and offs[1] % 256 == 0
    assert n.value >= offs[1] + sizes[1]
    lib = emm.load_library()
    assert lib.emm_jobs_workspace_size(0, jobs, emm.C.byref(n), None) == emm.EMM_EINVAL
    assert lib.emm_jobs_workspace_size(17, jobs, emm.C.byref(n), None) == emm.EMM_EINVAL
    # differing FD orders, or a volume DTFT, are refused
    w4 = W.small_case(n=(24, 22, 20), rd=4, nt=10, volume=False)
    bad, keep2 = emm._jobs_c([probs[0], (emm.grid_for(w4), emm.survey_for(w4))], [None, None], [None, None])
    assert lib.emm_jobs_workspace_size(2, bad, emm.C.byref(n), None) == emm.EMM_EINVAL
    wv = W.small_case(n=(20, 18, 16), rd=2, nt=10, volume=True)
    bad, keep3 = emm._jobs_c([probs[0], (emm.grid_for(wv), emm.survey_for(wv))], [None, None], [None, None])
    assert lib.emm_jobs_workspace_size(2, bad, emm.C.byref(n), None) == emm.EMM_EINVAL
    # a workspace that is too small is refused before anything is enqueued
    assert lib.emm_forward_jobs(2, jobs, emm.JOBS_LIST, None, 0, None) == emm.EMM_EWORKSPACE
    assert lib.emm_forward_jobs(2, jobs, 3, None, 0, None) == emm.EMM_EINVAL


def test_persistent_work_list_layout_and_errors():
    from paper_2304_00233_b300 import workloads as W
    C = emm.C
    wls = [W.small_case(n=(20, 18, 16), rd=2, nt=10, volume=False),
           W.small_case(n=(26, 22, 19), rd=2, nt=12, volume=False)]
    probs = [(emm.grid_for(w), emm.survey_for(w)) for w in wls]
    pos = np.array([probs[1][1].src, np.array(probs[1][1].src) + [30.0, 0.0, 0.0]])
    keep = []

    def tasks(items):
        arr = (emm._Task * len(items))()
        for j, (g, s, p) in enumerate(items):
            sc, k = s._c()
            keep.extend([sc, k, p])
            arr[j].grid, arr[j].survey = g.handle, C.pointer(sc)
            arr[j].nsrc = 1 if p is None else len(p)
            arr[j].src_pos = emm._dp(p) if p is not None else None
        return arr

    lib = emm.load_library()
    good = tasks([(probs[0][0], probs[0][1], None), (probs[1][0], probs[1][1], pos)])
    n = C.c_size_t(0)
    offs = (C.c_size_t * 2)()
    assert lib.emm_persist_workspace_size(2, good, C.byref(n), offs) == emm.EMM_OK
    # a 256-byte header, then each task's forward workspace (the second a batch of two)
    assert offs[0] == 256 and offs[1] >= 256 + emm.workspace_size(*probs[0]) and offs[1] % 256 == 0
    assert n.value >= offs[1] + emm.batch_workspace_size(probs[1][0], probs[1][1], 2)
    assert lib.emm_persist_workspace_size(0, good, C.byref(n), None) == emm.EMM_EINVAL
    assert lib.emm_persist_workspace_size(17, good, C.byref(n), None) == emm.EMM_EINVAL
    # a batch without positions, a volume DTFT, or differing FD orders are refused
    assert lib.emm_persist_workspace_size(
        1, tasks([(probs[1][0], probs[1][1], None)]), C.byref(n), None) == emm.EMM_OK
    nopos = tasks([(probs[1][0], probs[1][1], None)])
    nopos[0].nsrc = 2
    assert lib.emm_persist_workspace_size(1, nopos, C.byref(n), None) == emm.EMM_EINVAL
    wv = W.small_case(n=(20, 18, 16), rd=2, nt=10, volume=True)
    assert lib.emm_persist_workspace_size(
        1, tasks([(emm.grid_for(wv), emm.survey_for(wv), None)]), C.byref(n), None) == emm.EMM_EINVAL
    w4 = W.small_case(n=(24, 22, 20), rd=4, nt=10, volume=False)
    mixed = tasks([(probs[0][0], probs[0][1], None), (emm.grid_for(w4), emm.survey_for(w4), None)])
    assert lib.emm_persist_workspace_size(2, mixed, C.byref(n), None) == emm.EMM_EINVAL
    # no workspace, or negative options: refused before anything is enqueued
    assert lib.emm_forward_persistent(2, good, None, None, 0, None) == emm.EMM_EWORKSPACE
    bad = emm.PersistOpts(ctas_per_sm=-1)
    assert lib.emm_forward_persistent(2, good, C.byref(bad), None, 0, None) == emm.EMM_EINVAL
    assert lib.emm_persist_plan_run(None, None) == emm.EMM_EINVAL


def test_wave_workspace_and_refusals():
    from paper_2304_00233_b300 import workloads as W
    C = emm.C
    lib = emm.load_library()
    wl = W.small_case(n=(24, 22, 20), rd=2, nt=30, volume=False)
    g, s = emm.grid_for(wl), emm.survey_for(wl)
    n1, n2 = C.c_size_t(0), C.c_size_t(0)
    sc, k = s._c()
    assert lib.emm_wave_workspace_size(g.handle, C.byref(sc), 1, C.byref(n1)) == emm.EMM_OK
    assert lib.emm_wave_workspace_size(g.handle, C.byref(sc), 4, C.byref(n2)) == emm.EMM_OK
    # the forward workspace, then the tile order and the counters
    assert n1.value == n2.value > emm.workspace_size(g, s)
    for depth in (0, 65):
        assert lib.emm_wave_workspace_size(g.handle, C.byref(sc), depth, C.byref(n1)) == emm.EMM_EINVAL
    wv = W.small_case(n=(24, 22, 20), rd=2, nt=30, volume=True)
    sv, kv = emm.survey_for(wv)._c()
    assert lib.emm_wave_workspace_size(g.handle, C.byref(sv), 2, C.byref(n1)) == emm.EMM_EINVAL
    # no workspace: refused before anything is enqueued
    assert lib.emm_forward_wave(g.handle, C.byref(sc), None, 2, None, 0, None, None) in (emm.EMM_EWORKSPACE,
                                                                                          emm.EMM_EINVAL)


def test_new_entry_points_refuse_bad_arguments_on_the_host():
    C = emm.C
    lib = emm.load_library()
    x = np.arange(12.0) * 10
    g = emm.make_grid(x, x, x, rd=2, nb=4, ne=3)
    good = emm.Survey(omega0=1.0, fmax=1.0, sigma_min=1.0, nt=10, src=(55, 55, 55),
                      rec=np.array([[40.0, 50.0, 60.0]]), freqs=[1.0])
    bad = emm.Survey(**{**good.__dict__, "nt": -1})
    sb, keep = bad._c()
    sg, keep2 = good._c()
    h = C.c_void_p()
    # plans: invalid survey, missing output handle; run and destroy of no plan
    assert lib.emm_plan_create(g.handle, C.byref(sb), None, None, 0, None, None, None, C.byref(h)) == emm.EMM_EINVAL
    assert lib.emm_plan_create(g.handle, C.byref(sg), None, None, 0, None, None, None, None) == emm.EMM_EINVAL
    assert lib.emm_plan_run(None, None, None) == emm.EMM_EINVAL
    lib.emm_plan_destroy(None)
    # misfit gradient: no observed data or no misfit scalar
    dummy = C.c_void_p(16)
    assert lib.emm_misfit_gradient(g.handle, C.byref(sg), dummy, None, None, 4, 0, dummy, 1 << 30, dummy, dummy,
                                   dummy, None) == emm.EMM_EINVAL
    assert lib.emm_misfit_gradient(g.handle, C.byref(sg), dummy, dummy, None, 4, 0, dummy, 1 << 30, dummy, None,
                                   dummy, None) == emm.EMM_EINVAL
    # staggering: missing arrays, a workspace too small for the cell widths
    n = C.c_size_t(0)
    assert lib.emm_stagger_workspace_size(g.handle, C.byref(n)) == emm.EMM_OK and n.value == 3 * 11 * 8
    assert lib.emm_stagger_sigma(g.handle, None, dummy, dummy, n.value, dummy, None) == emm.EMM_EINVAL
    assert lib.emm_stagger_sigma(g.handle, dummy, dummy, dummy, n.value - 8, dummy, None) == emm.EMM_EWORKSPACE
    assert lib.emm_stagger_sigma_adjoint(g.handle, dummy, dummy, n.value - 8, dummy, dummy, None) == \
        emm.EMM_EWORKSPACE
