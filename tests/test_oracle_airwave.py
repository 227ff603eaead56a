"""Pins of the oracle's top boundary with air (Sec. 3.3).

Above the interface the air field is harmonic and vanishes far away: a mode
e^{i k.x} of the interface plane decays as e^{-|k| h} at the height h, and H
is the gradient of a harmonic potential.  Both are checked on single discrete
Fourier modes of a padded plane, against closed forms derived from the
potential (not from the implementation's wavenumber formula):
  E:  cos(k.x + t) -> cos(k.x + t) e^{-|k| h} at the same x-y positions;
  H:  H_z = sin(k.x + t) on the interface gives H = -grad phi with
      phi = sin(k.x + t) e^{-|k| h} / |k|, i.e.
      H_x = kx / |k| cos(k.x + t) e^{-|k| h} at H_x's positions (x_i, y_{j+1/2}),
      H_y = ky / |k| cos(k.x + t) e^{-|k| h} at H_y's positions (x_{i+1/2}, y_j).
The whole solver with air on top stays bounded and keeps source-receiver
reciprocity to the level of the all-CPML case."""
import math

import numpy as np
import pytest

import oracle
from paper_2304_00233_b300 import workloads as W

NX, NY, DX, DY = 24, 18, 40.0, 55.0


def _mode(p, q):
    return 2 * math.pi * p / (NX * DX), 2 * math.pi * q / (NY * DY)


@pytest.mark.parametrize("p,q", [(1, 0), (0, 2), (3, -2), (5, 4)])
def test_e_mode_decays_as_exp_minus_k_h(p, q):
    kx, ky = _mode(p, q)
    x = np.arange(NX) * DX
    y = np.arange(NY) * DY
    ph = kx * x[None, :] + ky * y[:, None] + 0.3
    h = np.array([40.0, 80.0, 120.0])
    out = oracle.air_extrapolate(np.cos(ph), DX, DY, h, kind=0)
    k = math.hypot(kx, ky)
    for r in range(len(h)):
        np.testing.assert_allclose(out[r], np.cos(ph) * math.exp(-k * h[r]), atol=1e-11)


@pytest.mark.parametrize("p,q", [(1, 0), (0, 2), (3, -2), (5, 4)])
def test_h_is_the_gradient_of_a_harmonic_potential(p, q):
    kx, ky = _mode(p, q)
    k = math.hypot(kx, ky)
    xi, xh = np.arange(NX) * DX, (np.arange(NX) + 0.5) * DX
    yi, yh = np.arange(NY) * DY, (np.arange(NY) + 0.5) * DY
    hz = np.sin(kx * xh[None, :] + ky * yh[:, None] + 0.7)        # H_z at (x_{i+1/2}, y_{j+1/2})
    h = np.array([20.0, 60.0])
    out = oracle.air_extrapolate(hz, DX, DY, h, kind=1)
    for r in range(len(h)):
        d = math.exp(-k * h[r])
        hx = kx / k * np.cos(kx * xi[None, :] + ky * yh[:, None] + 0.7) * d   # at (x_i, y_{j+1/2})
        hy = ky / k * np.cos(kx * xh[None, :] + ky * yi[:, None] + 0.7) * d   # at (x_{i+1/2}, y_j)
        np.testing.assert_allclose(out[r, 0], hx, atol=1e-11)
        np.testing.assert_allclose(out[r, 1], hy, atol=1e-11)


def test_uniform_field_has_no_horizontal_h():
    out = oracle.air_extrapolate(np.full((NY, NX), 2.5), DX, DY, [30.0], kind=1)
    assert np.abs(out).max() < 1e-12
    e = oracle.air_extrapolate(np.full((NY, NX), 2.5), DX, DY, [30.0], kind=0)
    np.testing.assert_allclose(e, 2.5, atol=1e-12)


def _air_case():
    """Uniform x, y (the FFT needs it), stretched z; sea of 1 S/m with a
    buried resistor; source and receivers below the interface."""
    x = np.arange(30) * 60.0 - 870.0
    z = np.concatenate([[0.0], np.cumsum(40.0 * 1.04 ** np.arange(25))])
    cell = np.ones((len(z) - 1, len(x) - 1, len(x) - 1))
    cell[14:17] = 0.05
    sig = W.staggered_conductivity(cell, cell, x, x, z)
    return x, z, sig


def test_bounded_and_reciprocal_with_air():
    x, z, sig = _air_case()
    kw = dict(rd=2, nb=8, ne=4, omega0=2 * math.pi, fmax=1.0, freqs=[0.5, 1.0], airwave=True)
    s = np.array([-200.0, 30.0, 120.0])
    r = np.array([240.0, -60.0, 80.0])
    # bounded: the field energy after the pulse has left decays, it does not grow
    f1 = oracle.forward(x, x, z, sig, src=s, rec=r[None], nt=800, want_fields=True, **kw)["fields"]
    f2 = oracle.forward(x, x, z, sig, src=s, rec=r[None], nt=1600, want_fields=True, **kw)["fields"]
    assert np.isfinite(f2).all() and np.abs(f2).max() <= np.abs(f1).max()
    a = oracle.forward(x, x, z, sig, src=s, rec=r[None], nt=500, **kw)["G"][0, 0]
    b = oracle.forward(x, x, z, sig, src=r, rec=s[None], nt=500, **kw)["G"][0, 0]
    assert np.abs(a - b).max() < 1e-3 * np.abs(a).max(), np.abs(a - b) / np.abs(a)
    # the air changes the field (the boundary is live)
    c = oracle.forward(x, x, z, sig, src=s, rec=r[None], nt=500, **{**kw, "airwave": False})["G"][0, 0]
    assert np.abs(a - c).max() > 1e-2 * np.abs(c).max()


def test_airwave_needs_uniform_xy():
    wl = W.small_case(rd=2, nt=5, volume=False)
    with pytest.raises(Exception):
        oracle.forward_workload(wl, airwave=True)
