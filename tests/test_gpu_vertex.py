"""Vertex incumbents (batch flag 8, linear families) against the FP64 oracle.

A patch's corner coefficients are the polynomial's values at the box's
corners (Sec. II-D).  With the flag, a child's corner at which every active
constraint's corner value plus its rounding bound is <= 0 is a feasible point
whose cost bound can lower p_up in the same step.  The oracle runs Alg. 1-5
without it, so the lists differ; what must hold:
  - equal status, certified intervals of width <= opt_tol that overlap the
    oracle's, and p_up never below the oracle's p_lo;
  - the returned point (a corner when the incumbent is one) is feasible in
    the oracle's FP64 evaluation, with its cost inside the interval."""
import numpy as np
import pytest

import oracle
from paper_2003_01758_b300 import pcba
from paper_2003_01758_b300 import workloads as W

pytestmark = pytest.mark.gpu

MEM = 2 << 30


def oracle_solve(p, **kw):
    return oracle.solve(p.cost, p.ineq, p.eq, p.lo, p.hi, **kw)


def check(g, o, p, opt_tol):
    assert g["status"] == o["status"], (g["status"], o["status"])
    if o["status"] == oracle.OPTIMAL:
        assert g["upper"] - g["lower"] <= opt_tol
        assert g["lower"] <= o["upper"] and o["lower"] <= g["upper"], (g, o)
        assert g["upper"] >= o["lower"] - 1e-12
        x = g["x"]
        assert np.all(x >= p.lo) and np.all(x <= p.hi)
        assert max(oracle.eval_monomial(gi, x) for gi in p.ineq) <= 0.0
        v = oracle.eval_monomial(p.cost, x)
        assert g["lower"] - 1e-9 <= v <= g["upper"] + 1e-9


def vertex_batch(probs, precision, flags=pcba.Batch.VERTEX, mem=None):
    return pcba.Batch([pcba.linear_solver_from_problem(q, precision) for q in probs],
                      mem or MEM * len(probs), flags=flags)


@pytest.mark.parametrize("precision", [pcba.FP64, pcba.FP32])
@pytest.mark.parametrize("seed,n_obs", [(2000, 37), (2001, 512), (2002, 1500), (2003, 100)])
def test_rtd_vertex_incumbents_match_oracle(precision, seed, n_obs):
    p = W.rtd(seed, n_obstacles=n_obs)
    o = oracle_solve(p, opt_tol=1e-3)
    g = vertex_batch([p], precision).solve(opt_tol=1e-3)[0]
    check(g, o, p, 1e-3)


@pytest.mark.parametrize("precision", [pcba.FP64, pcba.FP32])
@pytest.mark.parametrize("seed,n_ineq,n_wp", [(500, 30, 1), (502, 300, 1), (504, 200, 2)])
def test_rtd_star_vertex_incumbents_match_oracle(precision, seed, n_ineq, n_wp):
    p = W.rtd_star(seed, n_ineq=n_ineq, n_wp=n_wp)
    o = oracle_solve(p, opt_tol=1e-3)
    g = vertex_batch([p], precision).solve(opt_tol=1e-3)[0]
    check(g, o, p, 1e-3)


def test_corner_incumbent_is_returned():
    """Some problem of the workload must end with a corner as its incumbent
    (with no warm start given, a point that is not a box's centre can only be
    a corner: from_warm_start is set), and the flag never costs steps: a
    lower p_up only removes items earlier and stops no later."""
    counts = W.batch_obstacle_counts(64, 4000)
    probs = [W.rtd(4000 + k, n_obstacles=int(c)) for k, c in enumerate(counts)]
    with_v = vertex_batch(probs, pcba.FP32, mem=16 << 30).solve(opt_tol=1e-3)
    without = vertex_batch(probs, pcba.FP32, flags=0, mem=16 << 30).solve(opt_tol=1e-3)
    corners = 0
    for a, b in zip(with_v, without):
        assert a["status"] == b["status"]
        assert a["steps"] <= b["steps"]
        assert not b["from_warm_start"]
        corners += a["status"] == pcba.OPTIMAL and a["from_warm_start"]
    assert corners > 0


def test_uneven_batch_with_vertex_incumbents():
    counts = W.batch_obstacle_counts(256, 4000)
    probs = [W.rtd(4000 + k, n_obstacles=int(c)) for k, c in enumerate(counts)]
    res = vertex_batch(probs, pcba.FP32, mem=64 << 30).solve(opt_tol=1e-3)
    bad = [(k, r["status"]) for k, r in enumerate(res)
           if r["status"] not in (pcba.OPTIMAL, pcba.INFEASIBLE)]
    assert not bad, bad
    for k in (0, 5, 69, 86, 141, 200, 255):
        check(res[k], oracle_solve(probs[k], opt_tol=1e-3), probs[k], 1e-3)


def test_host_loop_equals_graph_loop_with_vertex():
    probs = [W.rtd(2000 + k, n_obstacles=128) for k in range(4)]
    g = vertex_batch(probs, pcba.FP32).solve(opt_tol=1e-3)
    h = vertex_batch(probs, pcba.FP32,
                     flags=pcba.Batch.VERTEX | pcba.Batch.HOST_LOOP).solve(opt_tol=1e-3)
    for a, b in zip(g, h):
        for key in ("status", "lower", "upper", "steps"):
            assert a[key] == b[key]
        np.testing.assert_array_equal(a["x"], b["x"])


def test_dense_batches_reject_the_flag():
    p = W.rtd(2000, n_obstacles=16)
    with pytest.raises(pcba.PcbaError, match="linear"):
        pcba.Batch([pcba.solver_from_problem(p, pcba.FP32)], MEM, flags=pcba.Batch.VERTEX)
