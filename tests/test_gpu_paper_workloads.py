"""The paper-shaped workloads on the GPU against the FP64 oracle:
RTD* planning POPs (Sec. VI-A: Q = [0,1] x [-1,1], degree-12 constraints,
waypoint-product cost) and the increasing-constraints problems (Sec. V-C).

Parity is status equality and certified intervals that overlap the
oracle's, each of width <= opt_tol; a returned point must be feasible in the
oracle's FP64 evaluation."""
import math

import numpy as np
import pytest

import oracle
from paper_2003_01758_b300 import pcba
from paper_2003_01758_b300 import workloads as W
from tests import benchmarks

pytestmark = pytest.mark.gpu

MEM = 2 << 30


def oracle_solve(p, **kw):
    return oracle.solve(p.cost, p.ineq, p.eq, p.lo, p.hi, **kw)


def rounding_slack(p):
    """Plain FP64 (the oracle, and the library's FP64 mode) rounds the
    Bernstein coefficients with errors of the order of 2^-46 max |B| over the
    root box; on E-V-D's [-100,100]^2 (|B| ~ 1e12) that is ~1e-2, more than
    opt_tol, so intervals are compared with this slack."""
    B = oracle.bernstein_from_monomial(p.cost, p.lo, p.hi)
    return 2.0 ** -46 * float(np.abs(B).max())


def assert_parity(g, o, p, opt_tol):
    assert g["status"] == o["status"], (g["status"], o["status"], g["lower"], g["upper"],
                                        o["lower"], o["upper"])
    if o["status"] == oracle.OPTIMAL:
        d = rounding_slack(p)
        assert g["upper"] - g["lower"] <= opt_tol
        assert g["lower"] <= o["upper"] + d and o["lower"] <= g["upper"] + d, (g, o, d)
        assert max(oracle.eval_monomial(gi, g["x"]) for gi in p.ineq) <= 0.0
        v = oracle.eval_monomial(p.cost, g["x"])
        assert g["lower"] - 1e-9 - d <= v <= g["upper"] + 1e-9 + d


RTD_STAR = [(500, 30, 1), (501, 150, 1), (502, 300, 1), (503, 60, 2), (504, 200, 2),
            (505, 300, 2)]


@pytest.mark.parametrize("precision", [pcba.FP64, pcba.FP32])
@pytest.mark.parametrize("seed,n_ineq,n_wp", RTD_STAR)
def test_rtd_star_linear_family_matches_oracle(precision, seed, n_ineq, n_wp):
    """The degree-12 constraints as a linear family in (||y||^2, y_1, y_2):
    FP32 certifies as FP64 does (re-centred shared patches)."""
    p = W.rtd_star(seed, n_ineq=n_ineq, n_wp=n_wp)
    o = oracle_solve(p, opt_tol=1e-3)
    g = pcba.linear_solver_from_problem(p, precision).solve(opt_tol=1e-3, mem_cap=MEM)
    assert_parity(g, o, p, 1e-3)


@pytest.mark.parametrize("seed,n_ineq,n_wp", RTD_STAR[:4])
def test_rtd_star_dense_fp64_matches_oracle(seed, n_ineq, n_wp):
    p = W.rtd_star(seed, n_ineq=n_ineq, n_wp=n_wp)
    o = oracle_solve(p, opt_tol=1e-3)
    g = pcba.solver_from_problem(p, pcba.FP64).solve(opt_tol=1e-3, mem_cap=4 * MEM)
    assert_parity(g, o, p, 1e-3)


def test_rtd_star_batch_all_certified():
    """64 planning POPs, 30..300 constraints (log-uniform), one or two
    waypoints, as one FP32 batch of linear families; a sample against the
    oracle."""
    rng = np.random.default_rng(9)
    counts = np.floor(np.exp(rng.uniform(math.log(30), math.log(300), 64))).astype(int)
    probs = [W.rtd_star(7000 + k, n_ineq=int(c), n_wp=1 + k % 2) for k, c in enumerate(counts)]
    b = pcba.Batch([pcba.linear_solver_from_problem(p, pcba.FP32) for p in probs], 16 << 30)
    res = b.solve(opt_tol=1e-3)
    bad = [(k, r["status"]) for k, r in enumerate(res)
           if r["status"] not in (pcba.OPTIMAL, pcba.INFEASIBLE)]
    assert not bad, bad
    for k in range(0, 64, 9):
        assert_parity(res[k], oracle_solve(probs[k], opt_tol=1e-3), probs[k], 1e-3)


INCREASING = [("EVD", 10), ("EVD", 200), ("Beale", 100), ("Bukin02", 200),
              ("DeckkersAarts", 200), ("DixonPrice2", 200), ("DixonPrice3", 100),
              ("DixonPrice4", 200), ("Powell", 10)]


@pytest.mark.parametrize("precision", [pcba.FP64, pcba.FP32])
@pytest.mark.parametrize("name,n", INCREASING)
def test_increasing_constraints_match_oracle(precision, name, n):
    """Sec. V-C: the constrained optimum is the objective's value at the
    feasible optimizer x*, so both intervals must also bracket it."""
    bm = benchmarks.load(name)
    p = W.increasing_constraints(bm["cost"], bm["lo"], bm["hi"], bm["x_opt"], n, seed=11 + n)
    eps = 1e-3 * max(1.0, abs(bm["optimum"]))
    o = oracle_solve(p, opt_tol=eps, max_iters=28, max_items=1 << 21)
    g = pcba.solver_from_problem(p, precision).solve(opt_tol=eps, max_iters=28, mem_cap=4 * MEM)
    assert_parity(g, o, p, eps)
    v = oracle.eval_monomial(p.cost, bm["x_opt"])
    if precision == pcba.FP32:
        # directed rounding: the certified lower bound holds without slack
        assert g["lower"] <= v
    else:
        assert g["lower"] <= v + rounding_slack(p)
