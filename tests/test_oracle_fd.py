"""Pins of the oracle's finite-difference machinery (Sec. 3.1-3.2).

P1  D+/D- and interpolation rows are exact on polynomials of degree <= 2r-1
    (the defining property of row 0/1 of [V^T]^{-1}, Eq. 9-11).
P2  uniform limit equals the textbook staggered coefficients (Appendix A),
    read from a golden fixture and re-derived here in exact rational arithmetic.
P3  derivative error on a smooth stretched grid falls as h^(2r).
P4  [V^T]^{-1} from unit vectors (Eq. 12) agrees with a dense LU inverse.
P6  eta of Sec. 3.2 equals the von Neumann bound of Appendix A (Eq. A8 at the
    Nyquist corner) on a uniform grid.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "staggered_fd_coefficients.txt")


def _golden():
    out = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        tok = line.split()
        rd = int(tok[0])
        out[rd] = ([Fraction(t) for t in tok[1:1 + rd]], Fraction(tok[1 + rd]))
    return out


def _rng_knots(rng, m, span=100.0):
    d = rng.uniform(0.3, 1.7, m - 1) * span / m
    return np.concatenate([[0.0], np.cumsum(d)]) + rng.uniform(-500, 500)


@pytest.mark.parametrize("rd", [1, 2, 3, 4])
def test_p1_polynomial_exactness(rd):
    rng = np.random.default_rng(100 + rd)
    m = 2 * rd
    for trial in range(20):
        knots = _rng_knots(rng, m)
        x = rng.uniform(knots[0], knots[-1])
        w0 = oracle.row_weights(knots, x, 0)
        w1 = oracle.row_weights(knots, x, 1)
        for deg in range(m):
            # p(s) = ((s - c)/h)^deg with c, h local so values stay O(1)
            c, h = knots.mean(), knots[-1] - knots[0]
            f = ((knots - c) / h) ** deg
            p = ((x - c) / h) ** deg
            dp = deg * ((x - c) / h) ** (deg - 1) / h if deg else 0.0
            assert abs(w0 @ f - p) <= 1e-10 * max(1.0, abs(p))
            assert abs(w1 @ f - dp) <= 1e-10 / h * max(1.0, abs(dp) * h)
        # degree 2r is NOT reproduced in general (the order is exactly 2r)
        f = ((knots - knots.mean()) / (knots[-1] - knots[0])) ** m
        p = ((x - knots.mean()) / (knots[-1] - knots[0])) ** m
        if trial == 0:
            assert abs(w0 @ f - p) > 1e-8


def _exact_staggered(rd):
    """Exact c_1..c_rd: row 1 of [V^T]^{-1} for knots at half-integers
    -r+1/2 .. r-1/2 about x=0, solved in rational arithmetic."""
    m = 2 * rd
    t = [Fraction(2 * k - m + 1, 2) for k in range(m)]
    # solve V^T a = e_j for each j via Gauss-Jordan on Fractions; want row 1
    A = [[tk ** p for p in range(m)] for tk in t]
    inv = [[Fraction(int(i == j)) for j in range(m)] for i in range(m)]
    A = [row[:] for row in A]
    for col in range(m):
        piv = next(r for r in range(col, m) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        inv[col], inv[piv] = inv[piv], inv[col]
        pv = A[col][col]
        A[col] = [v / pv for v in A[col]]
        inv[col] = [v / pv for v in inv[col]]
        for r in range(m):
            if r != col and A[r][col] != 0:
                fac = A[r][col]
                A[r] = [a - fac * b for a, b in zip(A[r], A[col])]
                inv[r] = [a - fac * b for a, b in zip(inv[r], inv[col])]
    row1 = inv[1]  # weights of f(t_0..t_{m-1}) for f'(0)
    return [row1[rd - 1 + i] for i in range(1, rd + 1)], sum(abs(v) for v in row1)


@pytest.mark.parametrize("rd", [1, 2, 3, 4])
def test_p2_uniform_limit(rd):
    gold_c, gold_sum = _golden()[rd]
    ex_c, ex_sum = _exact_staggered(rd)
    assert ex_c == gold_c and ex_sum == gold_sum  # fixture vs exact derivation
    dx = 37.5
    x = np.arange(30) * dx - 400.0
    t = oracle.axis_tables(x, rd, nb=5, ne=3)
    c = np.array([float(v) for v in gold_c])
    # D+ at a half node, taps F[i-r+1..i+r]: -c_r..-c_1, c_1..c_r over dx
    want = np.concatenate([-c[::-1], c]) / dx
    for i in range(rd - 1, len(t["Xh"]) - rd):
        np.testing.assert_allclose(t["cp"][i], want, rtol=1e-12, atol=1e-14 / dx)
    for i in range(rd, len(t["Xh"]) - rd):
        np.testing.assert_allclose(t["cm"][i], want, rtol=1e-12, atol=1e-14 / dx)
    assert t["dmax"] == pytest.approx(float(gold_sum) / dx, rel=1e-12)


@pytest.mark.parametrize("rd", [1, 2, 3, 4])
def test_p3_order_of_accuracy(rd):
    """Max error of D+/D- applied to sin(k x) on the smooth map
    x(s) = s + 0.3 sin(s) (s uniform, spacing h) over the interior rows."""
    errs = []
    hs = [0.2, 0.1, 0.05]
    for h in hs:
        s = np.arange(0.0, 6.0 + 1e-9, h)
        x = s + 0.3 * np.sin(s)
        t = oracle.axis_tables(x, rd, nb=rd, ne=0)
        X, Xh = t["X"], t["Xh"]
        f = lambda u: np.sin(1.3 * u)
        df = lambda u: 1.3 * np.cos(1.3 * u)
        e = 0.0
        m = 2 * rd
        nbe = rd
        for i in range(nbe + rd, nbe + len(x) - rd - 1):
            e = max(e, abs(t["cp"][i] @ f(X[i - rd + 1:i + rd + 1]) - df(Xh[i])))
            e = max(e, abs(t["cm"][i] @ f(Xh[i - rd:i + rd]) - df(X[i])))
        errs.append(e)
    orders = [math.log(errs[k] / errs[k + 1], 2) for k in range(2)]
    assert min(orders) > 2 * rd - 0.6, (errs, orders)


@pytest.mark.parametrize("m", [2, 3, 4, 5, 6, 7, 8])
def test_p4_vandermonde_vs_lu(m):
    rng = np.random.default_rng(m)
    t = np.sort(rng.uniform(-3.0, 3.0, m))
    W = oracle.vander_inverse(t)
    VT = np.vander(t, m, increasing=True)  # rows t_i^p
    Winv = np.linalg.inv(VT)
    np.testing.assert_allclose(W, Winv, rtol=1e-9, atol=1e-9 * np.abs(Winv).max())
    np.testing.assert_allclose(VT @ W, np.eye(m), atol=1e-11)


@pytest.mark.parametrize("rd", [1, 2, 3, 4])
def test_p6_eta_is_von_neumann_bound(rd):
    """On a uniform grid, eta = (1/2) v sqrt(sum D_max^2) equals the largest
    sin(omega dt/2)/dt allowed by Eq. A8, i.e. max_k of
    v sqrt(sum_a (sum_i c_i sin((i-1/2) k_a d_a)/d_a)^2)."""
    gold_c, _ = _golden()[rd]
    c = np.array([float(v) for v in gold_c])
    d = (40.0, 55.0, 70.0)
    v = 2500.0
    kk = np.linspace(0, math.pi, 2001)
    per_axis = []
    for da in d:
        s = np.abs(sum(ci * np.sin((i + 0.5) * kk) for i, ci in enumerate(c))) / da
        per_axis.append(s.max())
    bound = v * math.sqrt(sum(p * p for p in per_axis))
    dm = [oracle.axis_tables(np.arange(12) * da, rd, nb=rd, ne=1)["dmax"] for da in d]
    eta = 0.5 * v * math.sqrt(sum(q * q for q in dm))
    assert eta == pytest.approx(bound, rel=1e-9)
