"""Host setup of the CUDA library against the FP64 oracle (CPU only).

Integer index maps (stencil starts, valid rows, CPML slab maps, source and
receiver cells) must agree bit-exactly; node coordinates too (same defining
expressions); FD rows, CPML coefficients, interpolation weights and the time
step to 1e-12 relative.  The library evaluates the rows of [V^T]^{-1} from the
Lagrange closed form, the oracle by the Newton/Bjorck-Pereyra route, so the
two share no arithmetic."""
import numpy as np
import pytest

import oracle
import paper_2304_00233_b300 as emm
from paper_2304_00233_b300 import workloads as W


def _cases():
    yield W.small_case(rd=1)
    yield W.small_case(rd=2, n=(31, 29, 23))
    yield W.small_case(rd=3, n=(26, 30, 27))
    yield W.small_case(rd=4, n=(33, 28, 25))
    yield W.whole_space()
    yield W.marine_1d()


CASES = list(_cases())


@pytest.mark.parametrize("wl", CASES, ids=[w.name for w in CASES])
def test_axis_tables_match_oracle(wl):
    g = emm.grid_for(wl)
    r = wl.rd
    for a, x in enumerate((wl.x, wl.y, wl.z)):
        o = oracle.axis_tables(x, wl.rd, wl.nb, wl.ne)
        X, _ = g.table(a, emm.TAB_NODES)
        Xh, _ = g.table(a, emm.TAB_HALF)
        np.testing.assert_array_equal(X, o["X"])
        np.testing.assert_array_equal(Xh, o["Xh"])
        cp, sp = g.table(a, emm.TAB_DPLUS)
        cm, sm = g.table(a, emm.TAB_DMINUS)
        npad = len(Xh)
        lo_p, hi_p, lo_m, hi_m = o["ranges"]
        want_sp = np.array([i - r + 1 if lo_p <= i <= hi_p else -1 for i in range(npad)])
        want_sm = np.array([i - r if lo_m <= i <= hi_m else -1 for i in range(npad)])
        np.testing.assert_array_equal(sp, want_sp)
        np.testing.assert_array_equal(sm, want_sm)
        for mine, ref in ((cp, o["cp"]), (cm, o["cm"])):
            scale = np.abs(ref).max(axis=1, keepdims=True) + 1e-300
            assert np.max(np.abs(mine - ref) / scale) < 1e-12
        _, si = g.table(a, emm.TAB_SLAB_INT)
        _, sh = g.table(a, emm.TAB_SLAB_HALF)
        np.testing.assert_array_equal(si, o["slab"])
        np.testing.assert_array_equal(sh, o["slabh"])


@pytest.mark.parametrize("wl", CASES, ids=[w.name for w in CASES])
def test_time_step_and_cpml_match_oracle(wl):
    g = emm.grid_for(wl)
    smin = float(np.min(wl.sigma))
    dt, eta, vmax = g.time_step(smin, wl.omega0)
    probe = oracle.forward(wl.x, wl.y, wl.z, wl.sigma, rd=wl.rd, nb=wl.nb, ne=wl.ne,
                           omega0=wl.omega0, nt=0, fmax=wl.fmax, src=wl.src, az=wl.src_az,
                           dip=wl.src_dip)
    assert dt == pytest.approx(probe["dt"], rel=1e-13)
    assert eta == pytest.approx(probe["eta"], rel=1e-13)
    assert vmax == pytest.approx(probe["vmax"], rel=1e-14)
    for a, x in enumerate((wl.x, wl.y, wl.z)):
        # each side with its own vmax and dt (equal to 1e-13 above)
        o = oracle.axis_tables(x, wl.rd, wl.nb, wl.ne, vmax=probe["vmax"], fmax=wl.fmax, dt=probe["dt"])
        ab = g.cpml_tables(a, vmax, wl.fmax, dt)
        np.testing.assert_allclose(ab, o["pml"], rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("wl", CASES, ids=[w.name for w in CASES])
def test_source_receiver_stencils_match_oracle(wl):
    g = emm.grid_for(wl)
    pts = np.concatenate([wl.src[None], wl.rec])
    for p in pts:
        for comp in range(6):
            s_lib, w_lib = g.locate(comp, p)
            s_orc, w_orc = oracle.locate(wl.x, wl.y, wl.z, wl.rd, wl.nb, wl.ne, comp, p)
            np.testing.assert_array_equal(s_lib, s_orc)
            np.testing.assert_allclose(w_lib, w_orc, rtol=1e-12, atol=1e-13)
            np.testing.assert_allclose(w_lib.sum(axis=1), 1.0, rtol=1e-12)


def test_locate_ties_and_cpml_edges():
    """A point exactly on a node picks that node (max{i: P_i <= p}); the last
    position whose stencil stays out of the CPML is accepted, the next one is
    rejected, identically on both sides."""
    x = np.arange(20) * 25.0
    g = emm.make_grid(x, x, x, rd=2, nb=5, ne=3)
    for comp in range(6):
        for p in (x[7], x[7] + 12.5, x[0], x[0] - 50.0, x[-1], x[-1] + 50.0, x[-1] + 75.0, x[0] - 75.0):
            pos = np.array([p, x[9], x[10] + 3.0])
            try:
                mine = g.locate(comp, pos)
            except emm.EmmError as e:
                assert e.code == emm.EMM_EOUTSIDE
                mine = None
            try:
                ref = oracle.locate(x, x, x, 2, 5, 3, comp, pos)
            except oracle.OracleError:
                ref = None
            assert (mine is None) == (ref is None), (comp, p)
            if mine is not None:
                np.testing.assert_array_equal(mine[0], ref[0])
