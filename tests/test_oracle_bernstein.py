"""Pins for the oracle's Bernstein machinery against facts that do not come
from the oracle itself: exact rational arithmetic (sympy), scipy's Bernstein
polynomials, evaluation identities of the Bernstein form (Sec. II-D, Eq. (BF)),
range enclosure (Thm. 1), subdivision (Sec. II-E) and the quadratic
convergence of the bounds (Thm. 2, Cor. 1)."""
import itertools

import numpy as np
import pytest
import sympy as sp
from numpy.polynomial import polynomial as npoly
from scipy.interpolate import BPoly, PPoly
from scipy.special import comb

import oracle


# --------------------------------------------------------------------------
# test-side helpers written from the definitions (independent of the oracle)
# --------------------------------------------------------------------------

def bernstein_basis(n, t):
    j = np.arange(n + 1)
    return comb(n, j) * np.power.outer(t, j) * np.power.outer(1.0 - t, n - j)


def eval_bernstein_form(b, lo, hi, x):
    """sum_J b_J prod_r C(n_r, j_r) t_r^j_r (1-t_r)^(n_r-j_r) at points x (m, l)."""
    x = np.atleast_2d(x)
    out = np.empty(x.shape[0])
    for m, pt in enumerate(x):
        val = b
        for r in range(b.ndim):
            t = (pt[r] - lo[r]) / (hi[r] - lo[r])
            val = np.tensordot(bernstein_basis(b.shape[r] - 1, t), val, axes=([0], [0]))
        out[m] = val
    return out


def eval_monomial(a, x):
    x = np.atleast_2d(x)
    if a.ndim == 1:
        return npoly.polyval(x[:, 0], a)
    if a.ndim == 2:
        return npoly.polyval2d(x[:, 0], x[:, 1], a)
    if a.ndim == 3:
        return npoly.polyval3d(x[:, 0], x[:, 1], x[:, 2], a)
    out = np.empty(x.shape[0])
    for m, pt in enumerate(x):
        val = a
        for r in range(a.ndim):
            val = np.tensordot(pt[r] ** np.arange(a.shape[r]), val, axes=([0], [0]))
        out[m] = val
    return out


def exact_bernstein_sympy(a_int, lo, hi):
    """Bernstein coefficients in exact rationals: substitute x = lo + (hi-lo) t,
    then solve the linear system that matches the Bernstein expansion with the
    power-basis coefficients (the definition, not the closed form)."""
    l = a_int.ndim
    N = [s - 1 for s in a_int.shape]
    t = sp.symbols("t0:%d" % l)
    lo_r = [sp.Rational(v) for v in lo]
    hi_r = [sp.Rational(v) for v in hi]
    p = 0
    for J in itertools.product(*[range(n + 1) for n in N]):
        term = sp.Integer(int(a_int[J]))
        for r in range(l):
            term *= (lo_r[r] + (hi_r[r] - lo_r[r]) * t[r]) ** J[r]
        p += term
    p = sp.Poly(sp.expand(p), *t)
    idx = list(itertools.product(*[range(n + 1) for n in N]))
    bs = sp.symbols("b0:%d" % len(idx))
    expansion = 0
    for bsym, J in zip(bs, idx):
        basis = 1
        for r in range(l):
            basis *= sp.binomial(N[r], J[r]) * t[r] ** J[r] * (1 - t[r]) ** (N[r] - J[r])
        expansion += bsym * basis
    diff = sp.Poly(sp.expand(expansion), *t) - p
    sol = sp.solve(diff.coeffs(), bs, dict=True)[0]
    out = np.empty(a_int.shape)
    for bsym, J in zip(bs, idx):
        out[J] = float(sol[bsym])
    return out


# --------------------------------------------------------------------------
# monomial -> Bernstein (Sec. II-D)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed,shape,lo,hi", [
    (1, (3, 4), ["-1", "-1/2"], ["1", "3/2"]),
    (2, (4,), ["1/3"], ["2"]),
    (3, (2, 2, 3), ["-1", "0", "-2"], ["1", "1", "1/4"]),
])
def test_conversion_matches_exact_rationals(seed, shape, lo, hi):
    rng = np.random.default_rng(seed)
    a = rng.integers(-5, 6, size=shape).astype(float)
    lo_f = [float(sp.Rational(v)) for v in lo]
    hi_f = [float(sp.Rational(v)) for v in hi]
    exact = exact_bernstein_sympy(a, lo, hi)
    got = oracle.bernstein_from_monomial(a, lo_f, hi_f)
    scale = max(1.0, np.abs(exact).max())
    assert np.abs(got - exact).max() <= 1e-14 * scale


@pytest.mark.parametrize("seed,n,lo,hi", [(5, 6, -1.0, 1.0), (6, 9, 0.25, 3.0), (7, 12, -2.0, -0.5)])
def test_conversion_1d_matches_scipy_bpoly(seed, n, lo, hi):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(n + 1)
    # scipy's power-basis piecewise polynomial uses (x - lo)^k coefficients, highest
    # first: build the coefficients of p(lo + s) in s by numpy polynomial products
    c = np.zeros(n + 1)
    base = np.array([1.0])
    lin = np.array([lo, 1.0])
    for k in range(n + 1):
        c[:len(base)] += a[k] * base
        base = npoly.polymul(base, lin)
    pp = PPoly(c[::-1].reshape(-1, 1), [lo, hi])
    bp = BPoly.from_power_basis(pp)
    expected = bp.c[:, 0]
    got = oracle.bernstein_from_monomial(a, [lo], [hi])
    assert np.allclose(got, expected, rtol=1e-12, atol=1e-12 * np.abs(expected).max())


@pytest.mark.parametrize("seed,shape", [(11, (5, 5)), (12, (4, 7)), (13, (3, 3, 3)), (14, (2, 3, 2, 3))])
def test_bernstein_form_reproduces_polynomial(seed, shape):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(shape)
    l = a.ndim
    lo = rng.uniform(-2, 0, size=l)
    hi = lo + rng.uniform(0.5, 3, size=l)
    b = oracle.bernstein_from_monomial(a, lo, hi)
    x = rng.uniform(lo, hi, size=(50, l))
    assert np.allclose(eval_bernstein_form(b, lo, hi, x), eval_monomial(a, x),
                       rtol=1e-11, atol=1e-11 * np.abs(a).sum())


def test_vertex_coefficients_equal_corner_values():
    rng = np.random.default_rng(21)
    a = rng.standard_normal((5, 4, 3))
    lo, hi = np.array([-1.0, 0.5, -3.0]), np.array([0.5, 2.0, -1.0])
    b = oracle.bernstein_from_monomial(a, lo, hi)
    for corner in itertools.product([0, 1], repeat=3):
        idx = tuple(0 if c == 0 else s - 1 for c, s in zip(corner, a.shape))
        pt = np.where(np.array(corner) == 0, lo, hi)
        assert b[idx] == pytest.approx(eval_monomial(a, pt)[0], rel=1e-12, abs=1e-12)


def test_linear_precision_and_constants():
    # p(x) = x_2 on a box: coefficients are the Greville abscissae lo + w i / n
    N = (3, 5)
    a = np.zeros((N[0] + 1, N[1] + 1))
    a[0, 1] = 1.0
    lo, hi = np.array([-1.0, 0.25]), np.array([2.0, 4.25])
    b = oracle.bernstein_from_monomial(a, lo, hi)
    grev = lo[1] + (hi[1] - lo[1]) * np.arange(N[1] + 1) / N[1]
    for i in range(N[0] + 1):
        assert np.allclose(b[i], grev, rtol=0, atol=1e-14)
    c = np.zeros((4, 4))
    c[0, 0] = 3.25
    assert np.all(oracle.bernstein_from_monomial(c, lo, hi) == 3.25)


# --------------------------------------------------------------------------
# range enclosure (Thm. 1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed,shape", [(31, (5, 5)), (32, (7, 7)), (33, (4, 4, 4))])
def test_enclosure_on_dense_grid(seed, shape):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(shape)
    l = a.ndim
    lo, hi = -np.ones(l), np.ones(l)
    b = oracle.bernstein_from_monomial(a, lo, hi)
    pts = 101 if l == 2 else 21
    grid = np.stack(np.meshgrid(*[np.linspace(-1, 1, pts)] * l, indexing="ij"), -1).reshape(-1, l)
    v = eval_monomial(a, grid)
    slack = 1e-12 * np.abs(b).max()
    assert v.min() >= b.min() - slack
    assert v.max() <= b.max() + slack


# --------------------------------------------------------------------------
# subdivision (Sec. II-E)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed,shape,r", [(41, (5, 5), 0), (42, (5, 5), 1), (43, (3, 6, 4), 1),
                                          (44, (4, 3, 3, 5), 3)])
def test_children_reproduce_parent_polynomial(seed, shape, r):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(shape)
    l = a.ndim
    lo = rng.uniform(-2, 0, size=l)
    hi = lo + rng.uniform(0.5, 2, size=l)
    b = oracle.bernstein_from_monomial(a, lo, hi)
    left, right = oracle.subdivide_patch(b, r)
    mid = 0.5 * (lo[r] + hi[r])
    hiL, loR = hi.copy(), lo.copy()
    hiL[r] = mid
    loR[r] = mid
    xL = rng.uniform(lo, hiL, size=(40, l))
    xR = rng.uniform(loR, hi, size=(40, l))
    tol = 1e-11 * np.abs(a).sum()
    assert np.allclose(eval_bernstein_form(left, lo, hiL, xL), eval_monomial(a, xL), atol=tol)
    assert np.allclose(eval_bernstein_form(right, loR, hi, xR), eval_monomial(a, xR), atol=tol)
    # (ii) the children equal a direct conversion over the child boxes
    assert np.allclose(left, oracle.bernstein_from_monomial(a, lo, hiL), atol=tol)
    assert np.allclose(right, oracle.bernstein_from_monomial(a, loR, hi), atol=tol)
    # (iii) nesting of the enclosures
    assert left.min() >= b.min() and left.max() <= b.max()
    assert right.min() >= b.min() and right.max() <= b.max()


def test_subdivision_1d_matches_scipy_on_subintervals():
    rng = np.random.default_rng(45)
    n = 8
    bcoef = rng.standard_normal(n + 1)
    bp = BPoly(bcoef.reshape(-1, 1), [0.0, 1.0])
    left, right = oracle.subdivide_patch(bcoef, 0)
    xs = np.linspace(0, 1, 33)
    assert np.allclose(BPoly(left.reshape(-1, 1), [0.0, 0.5])(xs / 2), bp(xs / 2), atol=1e-13)
    assert np.allclose(BPoly(right.reshape(-1, 1), [0.5, 1.0])(0.5 + xs / 2), bp(0.5 + xs / 2),
                       atol=1e-13)
    # the end coefficients of the children are the values at the split point
    assert left[-1] == pytest.approx(bp(0.5), abs=1e-14)
    assert right[0] == pytest.approx(bp(0.5), abs=1e-14)


def test_bound_gap_shrinks_quadratically():
    """Thm. 2 / Cor. 1: on boxes of width 2^-n around an interior minimiser,
    min p - min B = O(4^-n).  p >= 0 with p(c) = 0 is built so that the
    minimum over every box containing c is exactly 0."""
    x1, x2 = sp.symbols("x1 x2")
    c = (sp.Rational(137, 1000), sp.Rational(-411, 1000))
    e = ((x1 - c[0]) ** 2 * (1 + x2 ** 2 / 2) + (x2 - c[1]) ** 2 * (2 + x1)
         + sp.Rational(3, 10) * (x1 - c[0]) ** 2 * (x2 - c[1]) ** 2)
    a = np.zeros((5, 5))
    for m, coef in sp.Poly(sp.expand(e), x1, x2).terms():
        a[m] = float(coef)
    target = np.array([float(c[0]), float(c[1])])
    b = oracle.bernstein_from_monomial(a, [-1, -1], [1, 1])
    lo, hi = np.array([-1.0, -1.0]), np.array([1.0, 1.0])
    gaps = []
    for sweep in range(10):
        for r in range(2):
            left, right = oracle.subdivide_patch(b, r)
            mid = 0.5 * (lo[r] + hi[r])
            if target[r] <= mid:
                b, hi = left, hi.copy()
                hi[r] = mid
            else:
                b, lo = right, lo.copy()
                lo[r] = mid
        gaps.append(0.0 - b.min())
    gaps = np.array(gaps)
    assert np.all(gaps > 0)
    rate = (gaps[1] / gaps[9]) ** (1.0 / 8.0)
    assert 3.3 < rate < 4.8, rate            # linear convergence would give 2
    scaled = gaps * 4.0 ** np.arange(1, 11)
    assert scaled.max() / scaled.min() < 10.0  # gap <= zeta 4^-n with one zeta


def test_memory_per_item_matches_formula_table():
    """Eq. (memory_per_item): 2l + Pi(P+1) + alpha Pi(G+1) + beta Pi(H+1)."""
    assert oracle.memory_per_item(2, [4, 4], 10, [4, 4], 0, None) == 279
    assert oracle.memory_per_item(2, [6, 6], 512, [6, 6], 0, None) == 25141
    assert oracle.memory_per_item(4, [4] * 4, 64, [3] * 4, 2, [2] * 4) == 17179
