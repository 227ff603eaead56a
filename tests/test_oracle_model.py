"""Pins of the oracle's conductivity model map and its misfit gradient.

The staggered conductivity of Sec. 3.6 (face-area weighted mean of the cells
around each E edge) is pinned by what the definition fixes in closed form:

M1  constant cell fields give the same constants (sigma_h on xx, yy; sigma_v
    on zz);
M2  a cell field linear along an axis across the edge gives, at interior
    nodes, the field at (x_{i-1} + x_{i+1}) / 2 (the width-weighted centroid
    of the two cells), and along the edge's own axis the cell's own value;
M3  a layered model (sigma_h a function of depth only) gives the
    thickness-weighted arithmetic mean of the two layers at each node on
    the tangential components (Eq. 26) and the own cell on sigma_zz;
M4  samples on the model's faces take the one cell they touch;
M5  stagger_T is the transpose (dot-product test, 1e-13);

and the least-squares misfit gradient with respect to the cell values by
central differences of the misfit through ``oracle.forward`` (FP64,
Richardson-combined): single cells of sigma_h and sigma_v and a random
direction, plus zero weights dropping data."""
import numpy as np
import pytest

import oracle
from paper_2304_00233_b300 import workloads as W


def _axes(seed=5, n=(9, 8, 7)):
    rng = np.random.default_rng(seed)
    return [np.cumsum(rng.uniform(10.0, 30.0, m)) for m in n]


def _cells(x, y, z):
    return (len(z) - 1, len(y) - 1, len(x) - 1)


def test_m1_constants():
    x, y, z = _axes()
    s = oracle.stagger(x, y, z, np.full(_cells(x, y, z), 2.5), np.full(_cells(x, y, z), 0.75))
    # the normalised weights sum to one up to rounding
    np.testing.assert_allclose(s[0], 2.5, rtol=4e-16)
    np.testing.assert_allclose(s[1], 2.5, rtol=4e-16)
    np.testing.assert_allclose(s[2], 0.75, rtol=4e-16)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_m2_linear_field(axis):
    xs = _axes(seed=11 + axis)
    x, y, z = xs
    a, b = 1.7, 0.013
    centre = 0.5 * (xs[axis][:-1] + xs[axis][1:])
    shape = _cells(x, y, z)
    f = a + b * centre
    field = np.broadcast_to(f.reshape([-1 if d == 2 - axis else 1 for d in range(3)]), shape).copy()
    s = oracle.stagger(x, y, z, field, field)
    node = xs[axis]
    for c in range(3):
        comp = np.moveaxis(s[c], 2 - axis, 0)      # sample index along `axis` first
        if c == axis:
            # along its own axis a sample takes its own cell, the last one the last cell
            want = np.concatenate([f, f[-1:]])
        else:
            mid = a + b * 0.5 * (node[:-2] + node[2:])
            want = np.concatenate([f[:1], mid, f[-1:]])
        got = comp.reshape(len(node), -1)
        np.testing.assert_allclose(got, np.broadcast_to(want[:, None], got.shape), rtol=1e-14, atol=0)


def test_m3_layered_thickness_average():
    x, y, z = _axes(seed=21)
    rng = np.random.default_rng(3)
    lay_h = rng.uniform(0.1, 3.0, len(z) - 1)
    lay_v = rng.uniform(0.1, 3.0, len(z) - 1)
    shape = _cells(x, y, z)
    sh = np.broadcast_to(lay_h[:, None, None], shape).copy()
    sv = np.broadcast_to(lay_v[:, None, None], shape).copy()
    s = oracle.stagger(x, y, z, sh, sv)
    dz = np.diff(z)
    for k in range(1, len(z) - 1):
        want = (dz[k - 1] * lay_h[k - 1] + dz[k] * lay_h[k]) / (dz[k - 1] + dz[k])
        np.testing.assert_allclose(s[0][k], want, rtol=1e-14)
        np.testing.assert_allclose(s[1][k], want, rtol=1e-14)
        np.testing.assert_allclose(s[2][k], lay_v[k], rtol=1e-14)


def test_m4_faces_take_their_cell():
    x, y, z = _axes(seed=31)
    rng = np.random.default_rng(4)
    sh = rng.uniform(0.1, 3.0, _cells(x, y, z))
    sv = rng.uniform(0.1, 3.0, _cells(x, y, z))
    s = oracle.stagger(x, y, z, sh, sv)
    # E_x on the edge y = y_0, z = z_0 touches only the cells j = 0, k = 0
    np.testing.assert_allclose(s[0][0, 0, :-1], sh[0, 0, :], rtol=4e-16)
    np.testing.assert_allclose(s[0][0, 0, -1], sh[0, 0, -1], rtol=4e-16)
    # E_z on the corner edge x = x_last, y = y_last
    np.testing.assert_allclose(s[2][:-1, -1, -1], sv[:, -1, -1], rtol=4e-16)


def test_m5_transpose():
    x, y, z = _axes(seed=41, n=(10, 9, 8))
    rng = np.random.default_rng(6)
    sh = rng.standard_normal(_cells(x, y, z))
    sv = rng.standard_normal(_cells(x, y, z))
    g = rng.standard_normal((3, len(z), len(y), len(x)))
    gh, gv = oracle.stagger_T(x, y, z, g)
    lhs = float(np.sum(oracle.stagger(x, y, z, sh, sv) * g))
    rhs = float(np.sum(sh * gh) + np.sum(sv * gv))
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + 1.0)


# --- misfit gradient with respect to the cell conductivities ----------------

def _misfit_case(seed=8, n=(13, 12, 11), nt=60):
    wl = W.small_case(n=n, rd=2, seed=seed, nt=nt, volume=False, nb=4, nfreq=2)
    rng = np.random.default_rng(seed + 1)
    shape = _cells(wl.x, wl.y, wl.z)
    sh = np.exp(rng.uniform(np.log(0.4), np.log(2.5), shape))
    sv = np.exp(rng.uniform(np.log(0.4), np.log(2.5), shape))
    smin = 0.3
    probe = oracle.forward(wl.x, wl.y, wl.z, oracle.stagger(wl.x, wl.y, wl.z, sh, sv), rd=wl.rd, nb=wl.nb,
                           ne=wl.ne, omega0=wl.omega0, nt=0, fmax=wl.fmax, sigma_min=smin)
    kw = dict(rd=wl.rd, nb=wl.nb, ne=wl.ne, omega0=wl.omega0, nt=nt, fmax=wl.fmax, sigma_min=smin,
              dt=probe["dt"], src=wl.src, az=wl.src_az, dip=wl.src_dip, moment=wl.moment, rec=wl.rec,
              freqs=wl.freqs)
    # observed data: the response of a perturbed model
    G1 = oracle.forward(wl.x, wl.y, wl.z, oracle.stagger(wl.x, wl.y, wl.z, 1.3 * sh, 0.8 * sv), **kw)["G"]
    d = G1 * W.observed_noise(G1.shape, seed=seed + 2)
    w = rng.uniform(0.5, 2.0, G1.shape)
    return wl, sh, sv, d, w, kw


def _misfit(wl, sh, sv, d, w, kw):
    G = oracle.forward(wl.x, wl.y, wl.z, oracle.stagger(wl.x, wl.y, wl.z, sh, sv), **kw)["G"]
    r = G - d
    return 0.5 * float(np.sum(w * (r.real ** 2 + r.imag ** 2)))


def _central(f, eps):
    # central differences at eps and eps/2, Richardson-combined (error O(eps^4))
    def cd(e):
        return (f(e) - f(-e)) / (2 * e)
    return (4.0 * cd(eps / 2) - cd(eps)) / 3.0


def test_misfit_value_and_cell_gradients():
    wl, sh, sv, d, w, kw = _misfit_case()
    res = oracle.misfit_gradient(wl.x, wl.y, wl.z, sh, sv, d, w, ckpt_every=13, **kw)
    assert res["misfit"] == pytest.approx(_misfit(wl, sh, sv, d, w, kw), rel=1e-14)
    rng = np.random.default_rng(9)
    cells = [tuple(rng.integers(0, m) for m in sh.shape) for _ in range(3)]
    # the cell under the source and one on the model's face
    cells += [(sh.shape[0] // 2, sh.shape[1] // 2, sh.shape[2] // 2), (0, sh.shape[1] - 1, 0)]
    for c in cells:
        for which, g in (("h", res["grad_h"]), ("v", res["grad_v"])):
            def f(e, c=c, which=which):
                a, b = sh.copy(), sv.copy()
                (a if which == "h" else b)[c] *= 1.0 + e
                return _misfit(wl, a, b, d, w, kw)
            fd = _central(f, 2e-4) / (sh if which == "h" else sv)[c]
            assert g[c] == pytest.approx(fd, rel=2e-6, abs=1e-9 * np.abs(g).max()), (c, which)


def test_misfit_directional_derivative():
    wl, sh, sv, d, w, kw = _misfit_case(seed=18)
    res = oracle.misfit_gradient(wl.x, wl.y, wl.z, sh, sv, d, w, ckpt_every=20, **kw)
    rng = np.random.default_rng(19)
    dh, dv = rng.standard_normal(sh.shape) * sh, rng.standard_normal(sv.shape) * sv
    fd = _central(lambda e: _misfit(wl, sh + e * dh, sv + e * dv, d, w, kw), 1e-4)
    an = float(np.sum(res["grad_h"] * dh) + np.sum(res["grad_v"] * dv))
    assert an == pytest.approx(fd, rel=1e-7)


def test_zero_weights_drop_data():
    wl, sh, sv, d, w, kw = _misfit_case(seed=28, nt=40)
    w0 = w.copy()
    w0[:, 3:, :] = 0.0                      # drop the H channels
    d0 = d.copy()
    d0[:, 3:, :] = 1e3                      # whatever they hold
    a = oracle.misfit_gradient(wl.x, wl.y, wl.z, sh, sv, d, w0, **kw)
    b = oracle.misfit_gradient(wl.x, wl.y, wl.z, sh, sv, d0, w0, **kw)
    assert a["misfit"] == b["misfit"]
    assert np.array_equal(a["grad_h"], b["grad_h"]) and np.array_equal(a["grad_v"], b["grad_v"])
