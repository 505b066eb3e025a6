"""Pins for the oracle's two point evaluators against evaluators that do not
come from the oracle: exact rational arithmetic (sympy) and numpy's and
scipy's polynomial routines.

or_eval_monomial is the judge of every feasibility and cost check of the GPU
tests, so it is pinned on non-square multi-degrees for l = 1..4: an axis or
stride mix-up, a dropped term or a wrong power changes the value at a generic
point.  or_eval_bernstein (Sec. II-D, Eq. (BF)) is pinned the same way, and
against scipy's Bernstein polynomials in one variable."""
import itertools

import numpy as np
import pytest
import sympy as sp
from numpy.polynomial import polynomial as npoly
from scipy.interpolate import BPoly

import oracle

SHAPES = [(4,), (3, 6), (6, 3), (4, 2, 5), (2, 3, 4, 3)]   # multi-degree + 1 per axis


def exact_monomial_value(a_int, x_rat):
    """sum_J a_J prod_r x_r^j_r in rationals (Eq. (poly_monomial_basis))."""
    total = sp.Integer(0)
    for J in itertools.product(*[range(s) for s in a_int.shape]):
        term = sp.Integer(int(a_int[J]))
        for r, j in enumerate(J):
            term *= x_rat[r] ** j
        total += term
    return total


def exact_bernstein_value(b_int, lo, hi, x_rat):
    """sum_J b_J prod_r C(n_r, j_r) t_r^j_r (1 - t_r)^(n_r - j_r) in rationals,
    t_r = (x_r - lo_r) / (hi_r - lo_r) (Eq. (BF))."""
    N = [s - 1 for s in b_int.shape]
    t = [(x_rat[r] - lo[r]) / (hi[r] - lo[r]) for r in range(len(N))]
    total = sp.Integer(0)
    for J in itertools.product(*[range(n + 1) for n in N]):
        term = sp.Integer(int(b_int[J]))
        for r, j in enumerate(J):
            term *= sp.binomial(N[r], j) * t[r] ** j * (1 - t[r]) ** (N[r] - j)
        total += term
    return total


def rational_points(rng, l, m, lo=-1, hi=1):
    """m random points with coordinates k/64 in [lo, hi] (exact in binary)."""
    ks = rng.integers(int(lo * 64), int(hi * 64) + 1, size=(m, l))
    return ks / 64.0, [[sp.Rational(int(k), 64) for k in row] for row in ks]


@pytest.mark.parametrize("shape", SHAPES)
def test_eval_monomial_matches_exact_rationals(shape):
    rng = np.random.default_rng(sum(shape))
    a = rng.integers(-9, 10, size=shape).astype(np.float64)
    xs, xr = rational_points(rng, len(shape), 6)
    for x, xq in zip(xs, xr):
        ref = float(exact_monomial_value(a, xq))
        got = oracle.eval_monomial(a, x)
        assert abs(got - ref) <= 1e-13 * max(1.0, np.abs(a).sum())


@pytest.mark.parametrize("shape", [(3, 6), (6, 3), (4, 2, 5)])
def test_eval_monomial_matches_numpy_polyval(shape):
    rng = np.random.default_rng(7 + len(shape))
    a = rng.standard_normal(shape)
    x = rng.uniform(-1.3, 1.3, size=(20, len(shape)))
    if len(shape) == 2:
        ref = npoly.polyval2d(x[:, 0], x[:, 1], a)
    else:
        ref = npoly.polyval3d(x[:, 0], x[:, 1], x[:, 2], a)
    got = np.array([oracle.eval_monomial(a, pt) for pt in x])
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13)


def test_eval_monomial_axes_are_not_interchangeable():
    """x_1^2 x_2 has tensor entry [2, 1]; at (2, 3) it is 12, not 18."""
    a = np.zeros((3, 2))
    a[2, 1] = 1.0
    assert oracle.eval_monomial(a, [2.0, 3.0]) == 12.0
    assert oracle.eval_monomial(a.T.copy(), [2.0, 3.0]) == 18.0


@pytest.mark.parametrize("shape", SHAPES)
def test_eval_bernstein_matches_exact_rationals(shape):
    rng = np.random.default_rng(100 + sum(shape))
    l = len(shape)
    b = rng.integers(-9, 10, size=shape).astype(np.float64)
    lo = [sp.Rational(-1, 2)] * l
    hi = [sp.Rational(3, 2)] * l
    xs, xr = rational_points(rng, l, 5, lo=-0.5, hi=1.5)
    lo_f, hi_f = np.full(l, -0.5), np.full(l, 1.5)
    for x, xq in zip(xs, xr):
        ref = float(exact_bernstein_value(b, lo, hi, xq))
        got = oracle.eval_bernstein(b, lo_f, hi_f, x)
        assert abs(got - ref) <= 1e-13 * max(1.0, np.abs(b).sum())


@pytest.mark.parametrize("n,lo,hi", [(3, -1.0, 1.0), (6, 0.0, 5.0), (9, -2.0, 0.5)])
def test_eval_bernstein_1d_matches_scipy_bpoly(n, lo, hi):
    rng = np.random.default_rng(n)
    b = rng.standard_normal(n + 1)
    poly = BPoly(b.reshape(-1, 1), [lo, hi])
    for x in rng.uniform(lo, hi, size=15):
        assert oracle.eval_bernstein(b, [lo], [hi], [x]) == pytest.approx(float(poly(x)),
                                                                          rel=1e-12, abs=1e-12)


def test_eval_bernstein_vertex_and_partition_of_unity():
    """At a corner only the corner coefficient counts; all-ones patches are 1."""
    b = np.arange(12, dtype=np.float64).reshape(3, 4)
    lo, hi = np.array([-1.0, 2.0]), np.array([1.0, 5.0])
    assert oracle.eval_bernstein(b, lo, hi, [-1.0, 2.0]) == 0.0
    assert oracle.eval_bernstein(b, lo, hi, [-1.0, 5.0]) == 3.0
    assert oracle.eval_bernstein(b, lo, hi, [1.0, 2.0]) == 8.0
    assert oracle.eval_bernstein(b, lo, hi, [1.0, 5.0]) == 11.0
    ones = np.ones((4, 2, 3))
    x = [0.3, -0.2, 0.9]
    assert oracle.eval_bernstein(ones, -np.ones(3), np.ones(3), x) == pytest.approx(1.0, abs=1e-15)
