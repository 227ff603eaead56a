"""Pins of the oracle's time stepping, CPML, source, receivers and DTFT.

P7  A discrete plane-wave eigenmode of the staggered leapfrog advances with the
    frequency of the Appendix A dispersion relation (Eq. A8), every component,
    to rounding.  Pins curl signs, staggering, D+/D- pairing, the leapfrog
    order and eps = sigma / (2 omega0) (Sec. 2.2).
P14 Constant fields: the DTFT (Eq. 25, with the dt of Eq. 6) equals the
    closed-form geometric series, which pins the time labels of E (n+1) and
    H (n+1/2).
P8  Homogeneous whole space: Green's functions (Eq. 7) against the analytic
    field of an electric dipole in a conductor, inline E_x and broadside H_z.
P8M The same for a magnetic dipole M injected in the H update (Eq. 1 and the
    correspondence of Eq. 5): E = m x grad g, g = e^{ikr}/(4 pi r), so a
    z-directed m gives E_y = -m (1 - ikr) e^{ikr} / (4 pi r^2) inline and
    E_x = +m (1 - ikr) e^{ikr} / (4 pi r^2) broadside, and
    H_z = m (1 - ikr - k^2 r^2) e^{ikr} / (4 pi i w mu r^3) on both lines.
P12 Mirror symmetries of an x-directed dipole at the centre of a symmetric
    non-uniform grid, all six components of the volume DTFT.
P9  Wavelet independence: G = E'/J' (Eq. 7) with two source wavelets of
    different bandwidth agree to the truncation level, which pins the
    consistency of the injected source (sampled at t_{n+1/2}) with the J'
    of the normalisation.
P10 Invariance of G under omega0 -> 4 omega0 with fmax -> 2 fmax.
P11 Reciprocity G_xx(r; s) = G_xx(s; r) on a heterogeneous model.
P6  dt = 0.99/eta stays bounded; dt = 1.02/eta grows without bound.
A10 Samples whose stencils leave the array stay exactly zero.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2304_00233_b300 import workloads as W

MU0 = 4e-7 * math.pi
HALF = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (0, 1, 1), (1, 0, 1), (1, 1, 0)]


def _fornberg(rd):
    return {1: [1.0], 2: [9 / 8, -1 / 24], 3: [75 / 64, -25 / 384, 3 / 640],
            4: [1225 / 1024, -245 / 3072, 49 / 5120, -5 / 7168]}[rd]


def _positions(x, nbe, npad):
    """Padded integer and half node positions for a uniform axis (edge spacing
    repeated, as the oracle pads)."""
    d = x[1] - x[0]
    X = x[0] + (np.arange(npad + 1) - nbe) * d
    return X, 0.5 * (X[:-1] + X[1:])


@pytest.mark.parametrize("rd", [1, 2, 3, 4])
def test_p7_plane_wave_eigenmode(rd):
    nt = 4
    n, nb, ne = 4 * rd * nt + 20, rd, 0
    d = np.array([40.0, 55.0, 47.0])
    axes = [np.arange(n) * d[a] for a in range(3)]
    npad = n + 2 * (nb + ne)
    sigma, omega0 = 0.7, 2 * math.pi
    v = math.sqrt(2 * omega0 / (MU0 * sigma))
    kvec = np.array([2 * math.pi / (9.0 * d[0]), 2 * math.pi / (13.0 * d[1]),
                     -2 * math.pi / (11.0 * d[2])])
    c = _fornberg(rd)
    K = np.array([2.0 / d[a] * sum(ci * math.sin((i + 0.5) * kvec[a] * d[a])
                                   for i, ci in enumerate(c)) for a in range(3)])
    A = np.cross(K, [0.3, -1.0, 0.8])          # A . K = 0
    probe = oracle.forward(*axes, np.full((3, n, n, n), sigma), rd=rd, nb=nb, ne=ne,
                           omega0=omega0, nt=0, fmax=1.0, inject=False, pml=False)
    dt = probe["dt"]
    s = 0.5 * v * dt * np.linalg.norm(K)       # sin(omega dt / 2), Eq. A8
    assert 0 < s < 1
    w = 2 * math.asin(s) / dt
    B = dt / (2 * MU0 * s) * np.cross(K, A)
    amp = np.concatenate([A, B])
    pos = [_positions(axes[a], nb + ne, npad) for a in range(3)]

    def field(t_e, t_h):
        out = np.zeros((6, npad, npad, npad))
        for comp in range(6):
            P = [pos[a][HALF[comp][a]][:npad] for a in range(3)]
            ph = (kvec[0] * P[0][None, None, :] + kvec[1] * P[1][None, :, None]
                  + kvec[2] * P[2][:, None, None])
            t = t_e if comp < 3 else t_h
            out[comp] = amp[comp] * np.cos(ph - w * t)
        return out

    res = oracle.forward(*axes, np.full((3, n, n, n), sigma), rd=rd, nb=nb, ne=ne,
                         omega0=omega0, nt=nt, fmax=1.0, inject=False, pml=False,
                         init_fields=field(0.0, 0.5 * dt), want_fields=True)
    want = field(nt * dt, (nt + 0.5) * dt)
    m = 2 * rd * nt + 2
    sl = (slice(None), slice(m, npad - m), slice(m, npad - m), slice(m, npad - m))
    for comp in range(6):
        got, ref = res["fields"][sl][comp], want[sl][comp]
        err = np.abs(got - ref).max() / np.abs(amp[comp])
        assert err < 1e-10, (comp, err)
    # sanity: the numerical frequency differs from the continuum one
    assert abs(w - v * np.linalg.norm(kvec)) > 1e-6 * w


def test_p14_dtft_geometric_series():
    wl = W.small_case(rd=2, nt=57, volume=False)
    npad = wl.npad
    E0, H0 = 1.7, -0.45
    init = np.zeros((6, npad[2], npad[1], npad[0]))
    init[0] = E0        # Ex constant: every D+ of it vanishes
    init[5] = H0        # Hz constant: every D- of it vanishes
    res = oracle.forward(wl.x, wl.y, wl.z, wl.sigma, rd=wl.rd, nb=wl.nb, ne=wl.ne,
                         omega0=wl.omega0, nt=57, fmax=wl.fmax, rec=wl.rec,
                         freqs=wl.freqs, inject=False, init_fields=init)
    dt, N = res["dt"], 57
    for f, fr in enumerate(wl.freqs):
        wp = (1 + 1j) * math.sqrt(2 * math.pi * fr * wl.omega0)
        z = np.exp(1j * wp * dt)
        geo = (1 - z ** N) / (1 - z)
        accE = E0 * dt * z * geo                 # E^{n+1} at (n+1) dt
        accH = H0 * dt * np.exp(0.5j * wp * dt) * geo   # H^{n+1/2} at (n+1/2) dt
        np.testing.assert_allclose(res["acc"][:, 0, f], accE, rtol=1e-10)
        np.testing.assert_allclose(res["acc"][:, 5, f], accH, rtol=1e-10)
        for comp in (1, 2, 3, 4):
            assert np.abs(res["acc"][:, comp, f]).max() < 1e-12 * abs(accE)
        # source spectrum: sum_n p s(t_{n+1/2}) e^{i w' t_{n+1/2}} dt
        t = (np.arange(N) + 0.5) * dt
        s = wl.moment * np.exp(-(math.pi * wl.fmax * (t - 1.5 / wl.fmax)) ** 2)
        np.testing.assert_allclose(res["jhat"][f], np.sum(s * np.exp(1j * wp * t)) * dt,
                                   rtol=1e-12)


def _dipole_whole_space(r, f, sigma):
    om = 2 * math.pi * f
    k = np.sqrt(1j * om * MU0 * sigma)
    ex_inline = np.exp(1j * k * r) * (1 - 1j * k * r) / (2 * math.pi * sigma * r ** 3)
    hz_broad = (1 - 1j * k * r) * np.exp(1j * k * r) / (4 * math.pi * r ** 2)
    ex_broad = -np.exp(1j * k * r) * (1 - 1j * k * r - (k * r) ** 2) / (4 * math.pi * sigma * r ** 3)
    return ex_inline, hz_broad, ex_broad


def test_p8_whole_space_dipole():
    wl = W.whole_space()
    off = np.arange(400.0, 1601.0, 200.0)
    broad = np.stack([np.zeros_like(off), off, np.zeros_like(off)], 1)
    inline = np.stack([off, np.zeros_like(off), np.zeros_like(off)], 1)
    wl.rec = np.concatenate([inline, broad])
    res = oracle.forward_workload(wl)
    G = res["G"][:, :, 0]
    ex_in, hz_b, ex_b = _dipole_whole_space(off, 0.5, 1.0)
    k = len(off)
    for got, ref in ((G[:k, 0], ex_in), (G[k:, 5], hz_b), (G[k:, 0], ex_b)):
        amp = np.abs(got) / np.abs(ref) - 1
        ph = np.degrees(np.angle(got / ref))
        # the paper's accuracy class is 1.5 % / 1 degree; this grid does better
        assert np.abs(amp).max() < 5e-3, amp
        assert np.abs(ph).max() < 0.25, ph
    # fields that vanish by symmetry on these lines
    assert np.abs(G[:k, 1:]).max() < 1e-6 * np.abs(G[:k, 0]).max()


def _magnetic_dipole_whole_space(r, f, sigma):
    """Fields of a unit z-directed magnetic dipole at distance r in the plane
    z = 0: the E factor of m x r_hat, and H_z (Eq. 1, e^{-i w t})."""
    om = 2 * math.pi * f
    k = np.sqrt(1j * om * MU0 * sigma)
    e_fac = -(1 - 1j * k * r) * np.exp(1j * k * r) / (4 * math.pi * r ** 2)
    hz = (1 - 1j * k * r - (k * r) ** 2) * np.exp(1j * k * r) / (4 * math.pi * 1j * om * MU0 * r ** 3)
    return e_fac, hz


def test_p8m_whole_space_magnetic_dipole():
    wl = W.whole_space()
    off = np.arange(400.0, 1601.0, 200.0)
    broad = np.stack([np.zeros_like(off), off, np.zeros_like(off)], 1)
    inline = np.stack([off, np.zeros_like(off), np.zeros_like(off)], 1)
    wl.rec = np.concatenate([inline, broad])
    res = oracle.forward_workload(wl, magnetic=True, az=0.0, dip=math.pi / 2)
    G = res["G"][:, :, 0]
    e_fac, hz = _magnetic_dipole_whole_space(off, 0.5, 1.0)
    k = len(off)
    # m x r_hat: z x x = +y inline, z x y = -x broadside
    for got, ref in ((G[:k, 1], e_fac), (G[k:, 0], -e_fac), (G[:k, 5], hz), (G[k:, 5], hz)):
        amp = np.abs(got) / np.abs(ref) - 1
        ph = np.degrees(np.angle(got / ref))
        assert np.abs(amp).max() < 5e-3, amp
        assert np.abs(ph).max() < 0.25, ph
    # E along m and the radial E vanish on these lines
    assert np.abs(G[:k, [0, 2]]).max() < 1e-6 * np.abs(G[:k, 1]).max()


def _ranges(comp, axis, npa, r):
    """Samples of `comp` updated along `axis` (grid: integer samples 0..np-1,
    half samples 0..np-2; an update needs every stencil on the grid)."""
    if comp < 3:
        return (0, npa - 2) if axis == comp else (r, npa - 1 - r)
    return (0, npa - 1) if axis == comp - 3 else (r - 1, npa - 1 - r)


def _dynamic_mask(comp, npad, r):
    m = np.zeros(npad[::-1], bool)
    sl = []
    for axis in (2, 1, 0):
        lo, hi = _ranges(comp, axis, npad[axis], r)
        sl.append(slice(lo, hi + 1))
    m[tuple(sl)] = True
    return m


def _mirror_index(n, half):
    i = np.arange(n)
    return (n - 2 - i) if half else (n - 1 - i)


def test_p12_symmetry():
    x = W.symmetric_axis(26, 700.0, 40.0)
    y = W.symmetric_axis(24, 650.0, 45.0)
    z = W.symmetric_axis(22, 600.0, 50.0)
    n = (len(x), len(y), len(z))
    sig = np.ones((3, n[2], n[1], n[0])) * np.array([1.0, 1.0, 0.4])[:, None, None, None]
    res = oracle.forward(x, y, z, sig, rd=2, nb=6, ne=4, omega0=2 * math.pi, nt=150,
                         fmax=2.0, freqs=[1.0], volume=True)
    vol = res["vol"][:, 0]            # [6][n3][n2][n1]
    # parity of (Ex,Ey,Ez,Hx,Hy,Hz) under x->-x, y->-y, z->-z for p = x-hat
    # (E is a polar vector, H a pseudo-vector; x-reflection also flips p)
    parity = {0: (1, -1, -1, -1, 1, 1), 1: (1, -1, 1, -1, 1, -1), 2: (1, 1, -1, -1, -1, 1)}
    scaleE, scaleH = np.abs(vol[:3]).max(), np.abs(vol[3:]).max()
    for axis, par in parity.items():
        for comp in range(6):
            h = HALF[comp][axis]
            nn = n[axis]
            idx = np.arange(nn - 1) if h else np.arange(nn)
            mir = _mirror_index(nn, h)[idx]
            a = np.take(vol[comp], idx, axis=2 - axis)
            b = np.take(vol[comp], mir, axis=2 - axis)
            err = np.abs(a - par[comp] * b).max() / (scaleE if comp < 3 else scaleH)
            assert err < 1e-9, (axis, comp, err)


def test_p10_omega0_invariance():
    wl = W.small_case(rd=2, nt=150, volume=False)
    kw = dict(rd=wl.rd, nb=wl.nb, ne=wl.ne, nt=150, src=wl.src, az=wl.src_az,
              dip=wl.src_dip, rec=wl.rec, freqs=wl.freqs)
    a = oracle.forward(wl.x, wl.y, wl.z, wl.sigma, omega0=2 * math.pi, fmax=2.0, **kw)
    b = oracle.forward(wl.x, wl.y, wl.z, wl.sigma, omega0=8 * math.pi, fmax=4.0, **kw)
    assert b["dt"] == a["dt"] / 2
    np.testing.assert_allclose(b["G"], a["G"], rtol=1e-9, atol=1e-9 * np.abs(a["G"]).max())


def test_p9_wavelet_independence():
    x = W.uniform_axis(32, 50.0)
    sig = np.ones((3, 32, 32, 32))
    rec = np.array([[200.0, 0.0, 0.0], [400.0, 0.0, 0.0], [0.0, 300.0, 0.0], [250.0, 150.0, 100.0]])
    kw = dict(rd=2, nb=8, ne=7, omega0=2 * math.pi, nt=500, src=(0.0, 0.0, 0.0), rec=rec, freqs=[0.5, 1.0],
              sigma_min=0.9)
    a = oracle.forward(x, x, x, sig, fmax=1.0, **kw)["G"]
    b = oracle.forward(x, x, x, sig, fmax=1.6, **kw)["G"]
    # the wavelets' spectra differ by a factor of several at 1 Hz; G agrees
    # to about 2e-6 (truncation, and the CPML's fmax-dependent alpha)
    assert np.abs(a - b)[:, 0].max() < 1e-4 * np.abs(a[:, 0]).max()


def test_p11_reciprocity():
    x = np.arange(34) * 50.0 - 825.0
    rng = np.random.default_rng(11)
    cell = np.exp(rng.uniform(-0.5, 0.5, (33, 33, 33)))
    sig = W.staggered_conductivity(cell, cell, x, x, x)
    s = np.array([-210.0, 35.0, -40.0])
    r = np.array([230.0, -60.0, 45.0])
    kw = dict(rd=2, nb=8, ne=4, omega0=2 * math.pi, nt=400, fmax=1.0, freqs=[0.5, 1.0])
    a = oracle.forward(x, x, x, sig, src=s, rec=r[None], **kw)["G"][0, 0]
    b = oracle.forward(x, x, x, sig, src=r, rec=s[None], **kw)["G"][0, 0]
    assert np.abs(a - b).max() < 1e-3 * np.abs(a).max(), np.abs(a - b) / np.abs(a)


@pytest.mark.parametrize("factor,bounded", [(0.99, True), (1.02, False)])
def test_p6_cfl(factor, bounded):
    n = 14
    x = np.arange(n) * 50.0
    rng = np.random.default_rng(5)
    probe = oracle.forward(x, x, x, np.ones((3, n, n, n)), rd=2, nb=2, ne=0,
                           omega0=2 * math.pi, nt=0, fmax=1.0, inject=False, pml=False)
    dt = factor * 0.99 ** -1 * probe["dt"]
    npad = n + 4
    init = rng.standard_normal((6, npad, npad, npad))
    init[3:] *= 1.0 / (MU0 * probe["vmax"])   # H scaled like E / impedance
    for comp in range(6):                     # only samples the scheme updates
        init[comp][~_dynamic_mask(comp, (npad,) * 3, 2)] = 0.0
    res = oracle.forward(x, x, x, np.ones((3, n, n, n)), rd=2, nb=2, ne=0,
                         omega0=2 * math.pi, nt=1500, dt=dt, fmax=1.0, inject=False,
                         pml=False, init_fields=init, want_fields=True)
    growth = np.abs(res["fields"][:3]).max() / np.abs(init[:3]).max()
    if bounded:
        assert growth < 20.0, growth
    else:
        assert growth > 1e6, growth


def test_a10_edge_samples_stay_zero():
    wl = W.small_case(rd=3, nt=40, volume=False)
    res = oracle.forward_workload(wl, want_fields=True)
    F = res["fields"]
    r = wl.rd
    np3, np2, np1 = F.shape[1:]
    for comp in range(6):
        for axis in range(3):
            npa = (np1, np2, np3)[axis]
            lo, hi = _ranges(comp, axis, npa, r)
            a = np.moveaxis(F[comp], 2 - axis, 0)
            assert np.all(a[:lo] == 0) and np.all(a[hi + 1:] == 0), (comp, axis)
            assert np.abs(a[lo:hi + 1]).max() > 0
    assert np.abs(F).max() > 0


def test_extended_antenna_is_the_mean_of_its_sub_dipoles():
    """An antenna of length L as N sub-dipoles (the current spread uniformly
    over its length): by linearity its G equals the mean of the N point-dipole
    G at the segment midpoints, each run alone (same wavelet and moment, so
    the same normalisation)."""
    wl = W.small_case(rd=2, nt=120, volume=False, nfreq=2)
    L, N = 150.0, 3
    d = np.array([math.cos(wl.src_dip) * math.cos(wl.src_az), math.cos(wl.src_dip) * math.sin(wl.src_az),
                  math.sin(wl.src_dip)])
    for magnetic in (False, True):
        ext = oracle.forward_workload(wl, src_length=L, src_points=N, magnetic=magnetic)["G"]
        pts = [wl.src + (-0.5 + (k + 0.5) / N) * L * d for k in range(N)]
        mean = sum(oracle.forward_workload(wl, src=tuple(p), magnetic=magnetic)["G"] for p in pts) / N
        np.testing.assert_allclose(ext, mean, rtol=0, atol=1e-12 * np.abs(mean).max())
        # and the antenna is not the point dipole at its centre
        point = oracle.forward_workload(wl, magnetic=magnetic)["G"]
        assert np.abs(ext - point).max() > 1e-6 * np.abs(point).max()
