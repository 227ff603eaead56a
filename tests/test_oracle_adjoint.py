"""Pins of the oracle's exact discrete adjoint (the gradient reference).

The paper computes no gradient, so the adjoint is pinned to the forward map
itself, through the independent forward code path ``oracle.forward``:

G1  directional derivative: <grad, d> equals the central difference of
    L(sigma) = Re(sum conj(v) G(sigma)) along random directions d, to the
    finite-difference truncation level (FP64, relative 1e-7);
G2  single samples, including a sample on the model edge whose value the pads
    replicate (the gradient folds the pads back onto it);
G3  the same with the CPML switched off, and for rd = 1, 3 and 4;
G4  the result does not depend on the checkpoint spacing (bitwise).

dt and sigma_min are held fixed, as the gradient defines them."""
import numpy as np
import pytest

import oracle
from paper_2304_00233_b300 import workloads as W


def _case(rd=2, seed=3, n=(14, 12, 11), nt=70):
    wl = W.small_case(n=n, rd=rd, seed=seed, nt=nt, volume=False, nb=4, nfreq=2)
    rng = np.random.default_rng(seed + 100)
    nrec = len(wl.rec)
    v = rng.standard_normal((nrec, 6, 2)) + 1j * rng.standard_normal((nrec, 6, 2))
    smin = 0.9 * float(wl.sigma.min())
    probe = oracle.forward(wl.x, wl.y, wl.z, wl.sigma, rd=wl.rd, nb=wl.nb, ne=wl.ne,
                           omega0=wl.omega0, nt=0, fmax=wl.fmax, sigma_min=smin)
    kw = dict(rd=wl.rd, nb=wl.nb, ne=wl.ne, omega0=wl.omega0, nt=nt, fmax=wl.fmax,
              sigma_min=smin, dt=probe["dt"], src=wl.src, az=wl.src_az, dip=wl.src_dip,
              moment=wl.moment, rec=wl.rec, freqs=wl.freqs)
    return wl, v, kw


def _loss(wl, sigma, v, kw, **over):
    G = oracle.forward(wl.x, wl.y, wl.z, sigma, **{**kw, **over})["G"]
    return float(np.real(np.sum(np.conj(v) * G)))


def _directional(wl, v, kw, grad, seed, **over):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal(wl.sigma.shape) * wl.sigma
    # central differences at eps and eps/2, Richardson-combined (error O(eps^4))
    def cd(eps):
        return (_loss(wl, wl.sigma + eps * d, v, kw, **over) - _loss(wl, wl.sigma - eps * d, v, kw, **over)) / (2 * eps)
    fd = (4.0 * cd(5e-5) - cd(1e-4)) / 3.0
    return fd, float(np.sum(grad * d))


@pytest.mark.parametrize("seed", [11, 12])
def test_g1_directional_derivative(seed):
    wl, v, kw = _case()
    grad = oracle.vjp(wl.x, wl.y, wl.z, wl.sigma, v, **kw, ckpt_every=9)
    fd, an = _directional(wl, v, kw, grad, seed)
    assert abs(fd - an) <= 1e-7 * abs(fd), (fd, an)


def test_g2_single_samples_and_edge_fold():
    wl, v, kw = _case()
    grad = oracle.vjp(wl.x, wl.y, wl.z, wl.sigma, v, **kw, ckpt_every=13)
    n1, n2, n3 = len(wl.x), len(wl.y), len(wl.z)
    picks = [(0, n3 // 2, n2 // 2, n1 // 2), (1, 3, 4, 5), (2, n3 // 2, 2, n1 - 3),
             (0, 0, 0, 0), (2, n3 - 1, n2 - 1, n1 - 1)]     # the last two are edge samples
    for c, k, j, i in picks:
        h = 1e-5 * wl.sigma[c, k, j, i]
        sp, sm = wl.sigma.copy(), wl.sigma.copy()
        sp[c, k, j, i] += h
        sm[c, k, j, i] -= h
        fd = (_loss(wl, sp, v, kw) - _loss(wl, sm, v, kw)) / (2 * h)
        an = grad[c, k, j, i]
        scale = np.abs(grad).max()
        assert abs(fd - an) <= 1e-6 * scale + 1e-7 * abs(fd), ((c, k, j, i), fd, an, scale)


@pytest.mark.parametrize("rd,over", [(2, dict(pml=False)), (1, {}), (3, {}), (4, {})],
                         ids=["no-cpml", "rd1", "rd3", "rd4"])
def test_g3_parts_and_orders(rd, over):
    wl, v, kw = _case(rd=rd, n=(15, 13, 12) if rd < 4 else (18, 17, 16), nt=60)
    grad = oracle.vjp(wl.x, wl.y, wl.z, wl.sigma, v, **kw, **over, ckpt_every=8)
    fd, an = _directional(wl, v, kw, grad, 5, **over)
    assert abs(fd - an) <= 1e-7 * abs(fd), (fd, an)


def test_g4_checkpoint_spacing_is_irrelevant():
    wl, v, kw = _case(nt=40)
    g1 = oracle.vjp(wl.x, wl.y, wl.z, wl.sigma, v, **kw, ckpt_every=1)
    g2 = oracle.vjp(wl.x, wl.y, wl.z, wl.sigma, v, **kw, ckpt_every=7)
    g3 = oracle.vjp(wl.x, wl.y, wl.z, wl.sigma, v, **kw, ckpt_every=40)
    assert np.array_equal(g1, g2) and np.array_equal(g1, g3)
