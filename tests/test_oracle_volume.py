"""Pins of the oracle's volume DTFT (Sec. 3.5, Eq. 19 and 25) and of its
corner stopping rule (Sec. 4.1, reading A18), each against something other
than the oracle's own volume code.

* Constant fields: with E_x and H_z constant and no source, every curl
  vanishes, so each interior volume sample accumulates a closed-form
  geometric series: E at the labels (n+1) dt, H at (n+1/2) dt, each term
  times dt (reading A4), normalised as Eq. 7 normalises receivers.  A swapped
  E/H label, a dropped dt or a wrong normalisation fails it.
* A receiver placed exactly on a staggered sample of its component has
  Kronecker interpolation weights (row 0 of [V^T]^{-1} at a knot, Eq. 12),
  so its Green's function must equal the volume Green's function of that
  sample.  The receiver path is pinned on its own (P8, P14), so an offset
  error in the volume's interior index (the nb + ne shift) or a component
  mix-up fails it.
* The sampled volume (``vol_samples``, flat [6][n3][n2][n1] indices) equals
  the full volume at those indices (to the rounding of the normalisation).
* The corner rule: the stop step N of a run with ``convergence`` is the first
  check (steps 1 + 100 m) at which, for each of the 8 interior corners, the
  lowest-frequency DTFT of the six components changed by at most 1e-5 of
  its size since the check 100 steps earlier.  Plain runs of N, N - 100 and
  N - 200 steps read the corner accumulators through ``vol_samples``; the
  rule holds between N - 100 and N and fails between N - 200 and N - 100."""
import math

import numpy as np
import pytest

import oracle
from paper_2304_00233_b300 import workloads as W

# staggering of each component along x, y, z (1 = half node)
HALF = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (0, 1, 1), (1, 0, 1), (1, 1, 0)]


def _norm(comp, f_hz, omega0):
    # Eq. 7 for an electric source: sqrt(-i w / (2 w0)) on E, 1 on H
    if comp >= 3:
        return 1.0
    return math.sqrt(2 * math.pi * f_hz / (2 * omega0)) * np.exp(-0.25j * math.pi)


def test_volume_dtft_of_constant_fields():
    wl = W.small_case(n=(22, 20, 18), rd=2, nt=43, volume=True)
    npad = wl.npad
    E0, H0 = -0.8, 2.3
    init = np.zeros((6, npad[2], npad[1], npad[0]))
    init[0] = E0
    init[5] = H0
    res = oracle.forward(wl.x, wl.y, wl.z, wl.sigma, rd=wl.rd, nb=wl.nb, ne=wl.ne,
                         omega0=wl.omega0, nt=43, fmax=wl.fmax, freqs=wl.freqs,
                         inject=False, init_fields=init, volume=True)
    dt, N = res["dt"], 43
    vol = res["vol"]                    # [6][nf][n3][n2][n1]
    for f, fr in enumerate(wl.freqs):
        wp = (1 + 1j) * math.sqrt(2 * math.pi * fr * wl.omega0)
        z = np.exp(1j * wp * dt)
        geo = (1 - z ** N) / (1 - z)
        accE = E0 * dt * z * geo                       # E^{n+1} at (n+1) dt
        accH = H0 * dt * np.exp(0.5j * wp * dt) * geo  # H^{n+1/2} at (n+1/2) dt
        jh = res["jhat"][f]
        np.testing.assert_allclose(vol[0, f], _norm(0, fr, wl.omega0) * accE / jh, rtol=1e-10)
        np.testing.assert_allclose(vol[5, f], _norm(5, fr, wl.omega0) * accH / jh, rtol=1e-10)
        for comp in (1, 2, 3, 4):
            assert np.abs(vol[comp, f]).max() < 1e-12 * abs(accE / jh)


def _sample_position(wl, comp, ijk):
    axes = (wl.x, wl.y, wl.z)
    pos = []
    for a in range(3):
        i = ijk[a]
        pos.append(0.5 * (axes[a][i] + axes[a][i + 1]) if HALF[comp][a] else axes[a][i])
    return np.array(pos)


@pytest.mark.parametrize("rd", [2, 4])
def test_receiver_on_a_sample_equals_the_volume_sample(rd):
    wl = W.small_case(n=(30, 28, 26), rd=rd, nt=90, volume=True, seed=12)
    n = wl.shape
    rng = np.random.default_rng(2304)
    mid = [n[a] // 2 for a in range(3)]
    recs, want = [], []
    for comp in range(6):
        for _ in range(3):
            # within a few samples of the source, where the fields are large
            ijk = [mid[a] + int(rng.integers(-6, 7)) for a in range(3)]
            recs.append(_sample_position(wl, comp, ijk))
            want.append((comp, ijk))
    res = oracle.forward(wl.x, wl.y, wl.z, wl.sigma, rd=wl.rd, nb=wl.nb, ne=wl.ne,
                         omega0=wl.omega0, nt=wl.nt, fmax=wl.fmax, src=wl.src, az=wl.src_az,
                         dip=wl.src_dip, rec=np.array(recs), freqs=wl.freqs, volume=True)
    vol, G = res["vol"], res["G"]
    for r, (comp, (i, j, k)) in enumerate(want):
        got = G[r, comp]
        ref = vol[comp, :, k, j, i]
        scale = np.abs(vol[comp]).max()
        assert np.abs(got - ref).max() < 1e-11 * scale, (comp, i, j, k, got, ref)
        # a neighbouring sample is a different value: the test can see an offset
        assert np.abs(vol[comp, :, k, j, i + 1] - ref).max() > 1e-6 * scale


def test_sampled_volume_equals_full_volume():
    wl = W.small_case(n=(21, 19, 17), rd=3, nt=60, volume=True, seed=5)
    nint = int(np.prod(wl.shape))
    idx = np.sort(np.random.default_rng(9).choice(6 * nint, 300, replace=False))
    kw = dict(rd=wl.rd, nb=wl.nb, ne=wl.ne, omega0=wl.omega0, nt=wl.nt, fmax=wl.fmax, src=wl.src,
              az=wl.src_az, dip=wl.src_dip, freqs=wl.freqs)
    full = oracle.forward(wl.x, wl.y, wl.z, wl.sigma, volume=True, **kw)["vol"]
    part = oracle.forward(wl.x, wl.y, wl.z, wl.sigma, vol_samples=idx, **kw)["vol_samples_G"]
    flat = full.transpose(0, 2, 3, 4, 1).reshape(6 * nint, -1)
    # the same accumulators; the normalisation rounds in another order
    np.testing.assert_allclose(part, flat[idx], rtol=1e-14, atol=0)


def _corner_indices(wl):
    n1, n2, n3 = wl.shape
    nint = n1 * n2 * n3
    out = []
    for c in range(6):
        for q in range(8):
            i = n1 - 1 if q & 1 else 0
            j = n2 - 1 if q & 2 else 0
            k = n3 - 1 if q & 4 else 0
            out.append(c * nint + (k * n2 + j) * n1 + i)
    return np.array(out, dtype=np.int64)


def _corner_acc(wl, nt, idx, flo):
    res = oracle.forward_workload(wl, nt=nt, volume=False, vol_samples=idx)
    g = res["vol_samples_G"][:, flo].reshape(6, 8)
    fr = wl.freqs[flo]
    # undo Eq. 7's normalisation: the raw accumulators of the corner test
    norm = np.array([_norm(c, fr, wl.omega0) for c in range(6)])[:, None]
    return g * res["jhat"][flo] / norm


def _converged(new, old, tol=1e-5):
    dn = np.sqrt(np.sum(np.abs(new - old) ** 2, axis=0))
    un = np.sqrt(np.sum(np.abs(new) ** 2, axis=0))
    return bool(np.all(un > 0) and np.all(dn <= tol * un))


@pytest.mark.parametrize("rd", [1, 2])
def test_corner_stopping_rule(rd):
    wl = W.small_case(n=(26, 24, 20), rd=rd, nt=4000, volume=False, nfreq=2)
    N = oracle.forward_workload(wl, convergence=True)["nt"]
    assert N < 4000 and (N - 1) % 100 == 0 and N > 201
    flo = int(np.argmin(wl.freqs))
    idx = _corner_indices(wl)
    a, b, c = (_corner_acc(wl, n, idx, flo) for n in (N, N - 100, N - 200))
    assert _converged(a, b)
    assert not _converged(b, c)
