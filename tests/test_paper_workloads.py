"""The paper-shaped workloads (Sec. VI-A RTD* planning POPs, Sec. V-C
increasing constraints): their shapes and structure, and small instances
certified by the oracle."""
import numpy as np
import pytest

import oracle
from paper_2003_01758_b300 import workloads as W
from tests import benchmarks


def total_degree(a):
    idx = np.indices(a.shape).sum(axis=0)
    nz = np.abs(a) > 0
    return int(idx[nz].max()) if nz.any() else 0


@pytest.mark.parametrize("n_wp", [1, 2])
def test_rtd_star_shape(n_wp):
    """Sec. VI-A: Q = [0,1] x [-1,1], constraints of degree 12, cost of
    degree 10 N_wp (8 N_wp with two waypoints, see the module docstring)."""
    p = W.rtd_star(31, n_ineq=120, n_wp=n_wp)
    np.testing.assert_array_equal(p.lo, [0.0, -1.0])
    np.testing.assert_array_equal(p.hi, [1.0, 1.0])
    assert p.n_ineq == 120 and p.n_eq == 0
    assert all(total_degree(g) == 12 for g in p.ineq)
    assert total_degree(p.cost) == (10 if n_wp == 1 else 16)
    assert max(p.cost.shape) - 1 <= 16 and max(p.ineq.shape[1:]) - 1 <= 16


@pytest.mark.parametrize("n_wp", [1, 2])
def test_rtd_star_pieces_agree(n_wp):
    """The cost is the waypoint product and every constraint is
    r^2 + eps - ||x_i - y(q)||^2, also as the linear family."""
    p = W.rtd_star(32, n_ineq=40, n_wp=n_wp)
    m = p.meta
    shared, weight, offset = m["linear"]
    rng = np.random.default_rng(0)
    for q in rng.uniform(p.lo, p.hi, size=(6, 2)):
        x = np.array([W.poly_value(c, q) for c in m["x"]])
        y = np.array([W.poly_value(c, q) for c in m["y"]])
        cost = np.prod([float((x - wp) @ (x - wp)) for wp in m["waypoints"]])
        assert W.poly_value(p.cost, q) == pytest.approx(cost, rel=1e-12, abs=1e-12)
        g = np.array([W.poly_value(gi, q) for gi in p.ineq])
        ref = m["radius"] ** 2 + 1e-4 - ((m["points"] - y) ** 2).sum(1)
        np.testing.assert_allclose(g, ref, rtol=0, atol=1e-12)
        s = np.array([W.poly_value(sm, q) for sm in shared])
        np.testing.assert_allclose(offset + weight @ s, ref, rtol=0, atol=1e-12)


def test_rtd_star_arc_is_the_unicycle_endpoint():
    """Without perturbation the endpoint map is the Taylor polynomial of
    (v sin(wT)/w, v (1 - cos(wT))/w)."""
    T = 1.7
    x1, x2 = W._arc(1, T, 1.0, 15)
    for v, w in ((0.7, 0.3), (1.0, -0.9), (0.2, 0.05)):
        ex = (v * np.sin(w * T) / w, v * (1.0 - np.cos(w * T)) / w)
        assert W.poly_value(x1, [v, w]) == pytest.approx(ex[0], abs=1e-6)
        assert W.poly_value(x2, [v, w]) == pytest.approx(ex[1], abs=1e-6)


def test_rtd_star_oracle_certifies_small_instances():
    for seed, n_wp in ((40, 1), (41, 2)):
        p = W.rtd_star(seed, n_ineq=30, n_wp=n_wp)
        o = oracle.solve(p.cost, p.ineq, p.eq, p.lo, p.hi, opt_tol=1e-3)
        assert o["status"] == oracle.OPTIMAL
        assert o["upper"] - o["lower"] <= 1e-3
        assert max(oracle.eval_monomial(g, o["x"]) for g in p.ineq) <= 0.0


def test_increasing_constraints_structure():
    """Sec. V-C: total degree <= 2, coefficients in [-5, 5], x* strictly
    feasible with the margin."""
    b = benchmarks.load("Powell")
    p = W.increasing_constraints(b["cost"], b["lo"], b["hi"], b["x_opt"], 50, seed=3)
    assert p.ineq.shape == (50, 3, 3, 3, 3)
    assert all(total_degree(g) <= 2 for g in p.ineq)
    nonconst = p.ineq.copy()
    nonconst[:, 0, 0, 0, 0] = 0.0
    assert np.abs(nonconst).max() <= 5.0
    for g in p.ineq:
        assert W.poly_value(g, b["x_opt"]) == pytest.approx(-1.0, abs=1e-9)
    p0 = W.increasing_constraints(b["cost"], b["lo"], b["hi"], b["x_opt"], 5, seed=3, margin=0.0)
    for g in p0.ineq:
        assert W.poly_value(g, b["x_opt"]) == pytest.approx(0.0, abs=1e-9)


@pytest.mark.parametrize("name", ["EVD", "Beale", "Bukin02", "DixonPrice2", "DixonPrice3"])
def test_increasing_constraints_oracle_brackets_the_optimum(name):
    """x* stays feasible, so the constrained optimum is the objective's value
    at x* (the printed optimum, up to its printed digits)."""
    b = benchmarks.load(name)
    p = W.increasing_constraints(b["cost"], b["lo"], b["hi"], b["x_opt"], 100, seed=7)
    eps = 1e-3 * max(1.0, abs(b["optimum"]))
    o = oracle.solve(p.cost, p.ineq, p.eq, p.lo, p.hi, opt_tol=eps, max_iters=28)
    assert o["status"] == oracle.OPTIMAL
    v = oracle.eval_monomial(p.cost, b["x_opt"])
    assert o["lower"] <= v + 1e-9 * max(1.0, abs(v))
    assert o["upper"] - o["lower"] <= eps
    assert v == pytest.approx(b["optimum"], rel=1e-6, abs=1e-6)
