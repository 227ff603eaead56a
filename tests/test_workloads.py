"""Input generators: the grid generator of Sec. 3.7 (P5) and the medium
homogenisation of Sec. 3.6 that builds the staggered conductivities."""
import math

import numpy as np
import pytest

from paper_2304_00233_b300 import workloads as W


@pytest.mark.parametrize("n,L,dx", [(64, 6400.0, 40.0), (16, 1000.0, 40.0),
                                    (143, 14300.0, 40.0), (10, 30.0, 1.0)])
def test_p5_nugrid_identity(n, L, dx):
    x = W.create_nugrid(n, L, dx)
    assert len(x) == n + 1 and x[0] == 0.0
    assert x[1] == pytest.approx(dx, rel=1e-12)
    assert x[-1] == pytest.approx(L, rel=1e-12)       # L = dx (q^n - 1)/(q - 1), Eq. 21
    q = (x[2] - x[1]) / (x[1] - x[0])
    np.testing.assert_allclose(np.diff(x)[1:] / np.diff(x)[:-1], q, rtol=1e-9)
    assert q > 1


def test_p5_uniform_branch_and_errors():
    np.testing.assert_array_equal(W.create_nugrid(8, 80.0, 10.0), np.arange(9) * 10.0)
    with pytest.raises(ValueError):
        W.create_nugrid(10, 50.0, 10.0)   # L < n dx: no q > 1


def test_axes_shapes_and_symmetry():
    x = W.symmetric_axis(128, 6400.0, 40.0)
    assert len(x) == 128 and np.all(np.diff(x) > 0)
    np.testing.assert_array_equal(x, -x[::-1])
    assert x[64] - x[63] == pytest.approx(40.0)
    assert x[-1] == pytest.approx(6400.0)
    z = W.seabed_axis(1000.0, 16, 1000.0, 79, 8000.0, 40.0)
    assert len(z) == 96 and z[0] == pytest.approx(0.0, abs=1e-9) and z[16] == 1000.0
    w = W.marine_1d()
    assert w.shape == (128, 128, 96) and w.npad == (162, 162, 130)
    w = W.whole_space()
    assert w.shape == (64, 64, 64) and w.npad == (98, 98, 98)


def test_homogenisation_layers():
    """A cell cut by a layer boundary: sigma_h is the thickness-weighted
    arithmetic mean, sigma_v the harmonic mean (Eq. 20)."""
    model = W.LayeredModel([-1e30, 100.0], [2.0, 0.5], [4.0, 0.25])
    x = np.array([0.0, 10.0])
    z = np.array([80.0, 130.0])          # 20 m of layer 0, 30 m of layer 1
    sh, sv = W.cell_conductivity(model, x, x, z)
    assert sh[0, 0, 0] == pytest.approx((20 * 2.0 + 30 * 0.5) / 50)
    assert sv[0, 0, 0] == pytest.approx(50 / (20 / 4.0 + 30 / 0.25))


def test_staggered_uniform_and_block():
    x = np.linspace(0, 100, 6)
    sh = np.full((5, 5, 5), 0.7)
    sig = W.staggered_conductivity(sh, sh * 0.5, x, x, x)
    np.testing.assert_allclose(sig[:2], 0.7)
    np.testing.assert_allclose(sig[2], 0.35)
    model = W.LayeredModel([-1e30], [1.0], [1.0], [W.Box((-5, -5, 20), (5, 5, 40), 0.1)])
    g = np.array([-10.0, 0.0, 10.0])
    zz = np.array([0.0, 20.0, 40.0, 60.0])
    sh, sv = W.cell_conductivity(model, g, g, zz)
    # box covers half of each x/y cell face over the middle z cell
    np.testing.assert_allclose(sh[1], 0.25 * 0.1 + 0.75 * 1.0)
    np.testing.assert_allclose(sh[0], 1.0)


def test_workloads_deterministic():
    a, b = W.small_case(seed=3), W.small_case(seed=3)
    np.testing.assert_array_equal(a.sigma, b.sigma)
    assert np.all(a.sigma == a.sigma.astype(np.float32).astype(np.float64))


def test_gradient_survey_and_uneven_grids():
    g = W.gradient_survey()
    assert g.shape == (192, 192, 128) and g.sigma_h.shape == (127, 191, 191)
    assert np.diff(g.x).min() == pytest.approx(40.0, rel=1e-9)
    assert np.diff(g.x).max() < 210.0 and np.diff(g.z).max() < 210.0
    # the resistor lies 1000-1100 m below the seabed in the observed-data model only
    r = W.gradient_survey(with_resistor=True)
    assert r.sigma_h.min() == pytest.approx(0.02) and g.sigma_h.min() == pytest.approx(1.0)
    assert g.sigma_v.min() == pytest.approx(0.5)
    assert np.all(np.abs(W.GRADIENT_SOURCES[:, 0]) < g.x[-1])
    c = W.gradient_survey_48()
    assert c.shape == (48, 48, 48) and np.all(np.abs(c.rec[:, 0]) < c.x[-1])
    for (n1, n3), wl in zip(W.UNEVEN_GRIDS, W.uneven_jobs()):
        assert wl.shape == (n1, n1, n3)
        assert np.all(np.abs(wl.rec[:, 0]) <= 0.8 * wl.x[-1])
        assert np.diff(wl.x).max() == pytest.approx(200.0, rel=0.05)


def test_observed_noise_is_seeded_and_two_percent():
    a = W.observed_noise((200, 6, 3))
    b = W.observed_noise((200, 6, 3))
    assert np.array_equal(a, b)
    d = a - 1.0
    assert abs(d.mean()) < 2e-3
    # each of the real and imaginary parts has standard deviation 0.02 / sqrt(2)
    assert d.real.std() == pytest.approx(0.02 / math.sqrt(2.0), rel=0.05)
    assert d.imag.std() == pytest.approx(0.02 / math.sqrt(2.0), rel=0.05)
