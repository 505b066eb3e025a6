"""Limits of a solve and the failure paths of the device loop, exercised with
no GPU fault: the time limit (PCBA_TIMEOUT, the robot's real-time budget of
Sec. VI), the device loop's step guard (PCBA_ERR_DEVICE_TIMEOUT, made to fire
early by a host-side test hook), and the FP32 point check of the warm-start
certification in its generic and unrolled forms."""
import numpy as np
import pytest

import oracle
from paper_2003_01758_b300 import pcba
from paper_2003_01758_b300 import workloads as W

pytestmark = pytest.mark.gpu

MEM = 1 << 30


def test_time_limit_returns_the_certified_interval_so_far():
    p = W.rtd(2000)
    o = oracle.solve(p.cost, p.ineq, p.eq, p.lo, p.hi, opt_tol=1e-3)
    for prec in (pcba.FP64, pcba.FP32):
        s = pcba.solver_from_problem(p, prec)
        s.set_time_limit(1e-9)          # runs out during the first step
        r = s.solve(opt_tol=1e-3, mem_cap=MEM)
        assert r["status"] == pcba.TIMEOUT and r["steps"] == 1, r
        # the interval of one step still brackets the optimum
        assert r["lower"] <= o["upper"] and o["lower"] <= r["upper"]
        s.set_time_limit(0.0)           # no limit again
        r = s.solve(opt_tol=1e-3, mem_cap=MEM)
        assert r["status"] == o["status"] == pcba.OPTIMAL
        s.set_time_limit(10.0)          # a limit the solve never reaches
        assert s.solve(opt_tol=1e-3, mem_cap=MEM)["status"] == pcba.OPTIMAL


def test_time_limit_stops_every_running_problem_of_a_batch():
    probs = [W.rtd(2000 + k, n_obstacles=n) for k, n in enumerate((512, 64, 300))]
    b = pcba.Batch([pcba.solver_from_problem(q) for q in probs], 4 << 30)
    b.set_time_limit(1e-9)
    res = b.solve(opt_tol=1e-3)
    for q, r in zip(probs, res):
        assert r["status"] == pcba.TIMEOUT and r["steps"] == 1
        o = oracle.solve(q.cost, q.ineq, q.eq, q.lo, q.hi, opt_tol=1e-3)
        assert r["lower"] <= o["upper"] and o["lower"] <= r["upper"]
    b.set_time_limit(0.0)
    assert all(r["status"] == pcba.OPTIMAL for r in b.solve(opt_tol=1e-3))


@pytest.mark.parametrize("loop", [pcba.Batch.GRAPH, pcba.Batch.HOST_LOOP])
def test_step_guard_reports_device_timeout_and_the_context_survives(monkeypatch, loop):
    p = W.rtd(2001, n_obstacles=128)
    b = pcba.Batch([pcba.solver_from_problem(p)], MEM, flags=loop)
    monkeypatch.setenv("PCBA_TEST_STEP_GUARD", "3")
    with pytest.raises(pcba.PcbaError, match="ERR_DEVICE_TIMEOUT"):
        b.solve(opt_tol=1e-3)
    monkeypatch.delenv("PCBA_TEST_STEP_GUARD")
    r = b.solve(opt_tol=1e-3)[0]
    assert r["status"] == pcba.OPTIMAL and r["steps"] > 3


@pytest.mark.parametrize("deg", [(2, 2), (3, 3), (4, 4), (6, 6), (8, 8), (5, 5), (3, 6)])
def test_fp32_point_check_unrolled_equals_generic_and_is_rigorous(deg):
    import torch
    rng = np.random.default_rng(sum(deg))
    a = rng.standard_normal(tuple(d + 1 for d in deg))
    x = rng.uniform(-1.0, 1.0, size=(256, 2)).astype(np.float32)
    d_a = torch.from_numpy(a.astype(np.float32).ravel()).cuda()
    d_x = torch.from_numpy(x.ravel()).cuda()
    out = {}
    for unrolled in (False, True):
        v = torch.empty(256, dtype=torch.float32, device="cuda")
        e = torch.empty(256, dtype=torch.float32, device="cuda")
        pcba.eval_points_f32(d_a.data_ptr(), deg, d_x.data_ptr(), 256, unrolled,
                             v.data_ptr(), e.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        out[unrolled] = (v.cpu().numpy(), e.cpu().numpy())
    np.testing.assert_array_equal(out[True][0].view(np.uint32), out[False][0].view(np.uint32))
    np.testing.assert_array_equal(out[True][1].view(np.uint32), out[False][1].view(np.uint32))
    v, e = out[False]
    for k in range(0, 256, 8):
        exact = oracle.eval_monomial(a, x[k].astype(np.float64))
        assert abs(float(v[k]) - exact) <= float(e[k]) + 1e-12 * max(1.0, abs(exact))
