"""Linear-family constraints (pcba_create_linear) against the FP64 oracle.

The library stores the shared patches B(||F||^2), B(F_1), B(F_2) per item and
bounds every obstacle constraint g_i = c_i + w_i . s from them; the oracle gets
the expanded dense constraints and bounds each of their patches.  In exact
arithmetic both compute the same coefficients (the Bernstein transform is
linear, Sec. II-D), so:
  - in FP64 the list (boxes, in the order of Alg. 2 and Alg. 5) is the
    oracle's after every step, its shared patches are the oracle's conversion
    of the shared polynomials on each box, and every constraint an item has
    dropped is one whose oracle patch proves g_i <= 0 on that box (Thm. 1);
  - certified intervals overlap the oracle's with width <= opt_tol and the
    returned point is feasible in the oracle's FP64 evaluation, in FP64 and in
    FP32 (whose bounds carry a rigorous rounding-error bound).
Floating point decides a box's fate from values that the two sides round
differently, so the list comparison is exact only away from ties; the
problems below have none within 1e-9."""
import numpy as np
import pytest

import oracle
from paper_2003_01758_b300 import pcba
from paper_2003_01758_b300 import workloads as W

pytestmark = pytest.mark.gpu

MEM = 1 << 30


def lin(p, prec):
    return pcba.linear_solver_from_problem(p, prec)


def oracle_solve(p, **kw):
    return oracle.solve(p.cost, p.ineq, p.eq, p.lo, p.hi, **kw)


def assert_interval_parity(g, o, opt_tol):
    assert g["status"] == o["status"], (g, o)
    if o["status"] == oracle.OPTIMAL:
        assert g["upper"] - g["lower"] <= opt_tol
        assert g["lower"] <= o["upper"] and o["lower"] <= g["upper"], (g, o)


@pytest.mark.parametrize("seed,n_obs", [(2000, 37), (2001, 100), (2002, 300)])
def test_fp64_lists_follow_the_oracle(seed, n_obs):
    p = W.rtd(seed, n_obstacles=n_obs)
    shared = p.meta["linear"][0]
    o = oracle.Solver(p.cost, p.ineq, p.eq, p.lo, p.hi)
    g = lin(p, pcba.FP64)
    for steps in range(1, 15):
        st = o.step(opt_tol=1e-9, max_iters=28)
        res = g.solve(opt_tol=1e-9, max_iters=28, mem_cap=MEM, max_steps=steps)
        ol, gl = o.get_list(), g.get_list()
        np.testing.assert_array_equal(gl["index"], ol["index"])
        np.testing.assert_array_equal(gl["level"], ol["level"])
        K = ol["index"].shape[0]
        w = (p.hi - p.lo) / 2.0 ** ol["level"]
        act = g.get_active()
        assert act.shape == (K, p.n_ineq)
        for k in range(0, K, max(1, K // 12)):
            blo = p.lo + ol["index"][k] * w
            bhi = blo + w
            np.testing.assert_allclose(gl["cost"][k], ol["cost"][k], rtol=0,
                                       atol=1e-12 * np.abs(ol["cost"][k]).max())
            # (an item with every constraint proven to hold keeps no shared patches)
            for m in range(shared.shape[0] if act[k].any() else 0):
                ref = oracle.bernstein_from_monomial(shared[m], blo, bhi)
                assert np.abs(gl["ineq"][k, m] - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max())
            # a dropped constraint is proven to hold on the box
            gmax = ol["ineq"][k].reshape(p.n_ineq, -1).max(1)
            dropped = ~act[k]
            assert np.all(gmax[dropped] <= 1e-11), (steps, k, gmax[dropped].max())
        tr = o.trace()[-1]
        assert res["upper"] == pytest.approx(tr[2], rel=1e-12, abs=1e-12) or (
            np.isinf(res["upper"]) and np.isinf(tr[2]))
        assert res["lower"] == pytest.approx(tr[3], rel=1e-12, abs=1e-12)
        if st != oracle.RUNNING:
            assert res["status"] == st
            break
        assert res["status"] == pcba.STEPLIMIT


@pytest.mark.parametrize("precision", [pcba.FP64, pcba.FP32])
@pytest.mark.parametrize("seed,n_obs", [(2000, 512), (2001, 512), (2002, 100), (2003, 37),
                                        (4005, 2000)])
def test_end_to_end_matches_oracle(precision, seed, n_obs):
    p = W.rtd(seed, n_obstacles=n_obs)
    o = oracle_solve(p, opt_tol=1e-3)
    g = lin(p, precision).solve(opt_tol=1e-3, mem_cap=MEM)
    assert_interval_parity(g, o, 1e-3)
    if g["status"] == pcba.OPTIMAL:
        assert max(oracle.eval_monomial(gi, g["x"]) for gi in p.ineq) <= 0.0
        v = oracle.eval_monomial(p.cost, g["x"])
        assert g["lower"] - 1e-9 <= v <= g["upper"] + 1e-9
        assert g["verify_max_g"] <= 1e-9


def test_fp32_shared_patches_enclose_the_shared_polynomials():
    p = W.rtd(2001, n_obstacles=64)
    shared = p.meta["linear"][0]
    s = lin(p, pcba.FP32)
    s.solve(opt_tol=1e-12, mem_cap=MEM, max_steps=9)
    L = s.get_list()
    rng = np.random.default_rng(3)
    K = L["cost"].shape[0]
    w = (p.hi - p.lo) / 2.0 ** L["level"]
    act = s.get_active().any(1)
    live = np.flatnonzero(act)
    assert live.size > 0
    for k in rng.choice(live, size=min(live.size, 12), replace=False):
        lo = p.lo + L["index"][k] * w
        for x in rng.uniform(lo, lo + w, size=(4, p.l)):
            for m in range(shared.shape[0]):
                v = oracle.eval_monomial(shared[m], x)
                e = float(L["err"][k, 1 + m])
                assert L["ineq"][k, m].min() - e <= v + 1e-12 <= L["ineq"][k, m].max() + e + 2e-12


@pytest.mark.parametrize("precision", [pcba.FP64, pcba.FP32])
def test_batch_equals_single_solves(precision):
    probs = [W.rtd(2000 + k, n_obstacles=n) for k, n in enumerate((512, 64, 300, 1500, 16))]
    singles = [lin(p, precision).solve(opt_tol=1e-3, mem_cap=MEM) for p in probs]
    res = pcba.Batch([lin(p, precision) for p in probs], MEM * len(probs)).solve(opt_tol=1e-3)
    for a, b in zip(singles, res):
        for key in ("status", "lower", "upper", "steps", "sweeps"):
            assert a[key] == b[key], key


def test_host_loop_equals_graph_loop():
    probs = [W.rtd(2000 + k, n_obstacles=128) for k in range(4)]
    g = pcba.Batch([lin(p, pcba.FP32) for p in probs], 4 << 30)
    h = pcba.Batch([lin(p, pcba.FP32) for p in probs], 4 << 30, flags=pcba.Batch.HOST_LOOP)
    for a, b in zip(g.solve(), h.solve()):
        for key in ("status", "lower", "upper", "steps"):
            assert a[key] == b[key]


def test_uneven_batch_sampled_against_oracle():
    """The 256-problem batch workload (obstacle counts log-uniform in
    [16, 4096]) with linear families: every problem certified, a sample of
    them checked by the oracle."""
    counts = W.batch_obstacle_counts(256, 4000)
    probs = [W.rtd(4000 + k, n_obstacles=int(c)) for k, c in enumerate(counts)]
    b = pcba.Batch([lin(p, pcba.FP32) for p in probs], 64 << 30)
    res = b.solve(opt_tol=1e-3)
    bad = [(k, int(counts[k]), r["status"]) for k, r in enumerate(res)
           if r["status"] not in (pcba.OPTIMAL, pcba.INFEASIBLE)]
    assert not bad, bad
    for k in (0, 5, 69, 86, 95, 141, 200, 255):
        o = oracle_solve(probs[k], opt_tol=1e-3)
        assert_interval_parity(res[k], o, 1e-3)


def test_mixed_batches_and_polish_are_rejected():
    p = W.rtd(2000, n_obstacles=16)
    with pytest.raises(pcba.PcbaError, match="mix"):
        pcba.Batch([lin(p, pcba.FP32), pcba.solver_from_problem(p, pcba.FP32)], MEM)
    b = pcba.Batch([lin(p, pcba.FP32)], MEM)
    b.solve()
    with pytest.raises(pcba.PcbaError, match="dense"):
        b.polish()


def test_guided_solve_on_linear_families():
    """The learned warm start certifies its candidates against the linear
    rows (FP32 with a rigorous bound, FP64 where undecided)."""
    import torch
    from paper_2003_01758_b300 import warmstart
    probs = [W.rtd(6000 + k, n_obstacles=n) for k, n in enumerate((64, 300, 900, 128))]
    b = pcba.Batch([lin(q, pcba.FP32) for q in probs], 4 << 30)
    pk = warmstart.pack_batch(probs, b)
    y = warmstart.predict(warmstart.load_model(), pk)
    torch.cuda.synchronize()
    res = b.solve_guided(y.data_ptr(), 2, warmstart.default_stencil(), opt_tol=1e-3)
    for k, (q, r) in enumerate(zip(probs, res)):
        o = oracle_solve(q, opt_tol=1e-3)
        assert_interval_parity(r, o, 1e-3)
        seed = b.warm_point(k)
        if seed is not None:
            assert max(oracle.eval_monomial(gi, seed) for gi in q.ineq) <= 0.0


def test_uploads_from_library_pinned_buffers():
    """New rows and coefficients queued from pcba_host_alloc buffers
    (pcba.host_empty) give the same results as the batch built from them."""
    probs = [W.rtd(2100 + k, n_obstacles=n) for k, n in enumerate((64, 300, 37))]
    b = pcba.Batch([pcba.linear_solver_from_problem(q, pcba.FP32) for q in probs], 3 << 30)
    ref = b.solve(opt_tol=1e-3)
    rows = pcba.linear_rows(probs)
    h = pcba.host_empty(rows.size)
    h[:] = rows.ravel()
    assert h.ctypes.data % 16 == 0
    b.upload_rows(h)
    again = b.solve(opt_tol=1e-3)
    for a, r in zip(again, ref):
        for key in ("status", "lower", "upper", "steps"):
            assert a[key] == r[key]
    # other rows (a constraint moved off its obstacle) change the result
    h2 = pcba.host_empty(rows.size)
    h2[:] = rows.ravel()
    h2[0] -= 1e3  # the first constraint of the first problem holds everywhere
    b.upload_rows(h2)
    moved = b.solve(opt_tol=1e-3)
    assert moved[1]["lower"] == ref[1]["lower"] and moved[2]["lower"] == ref[2]["lower"]
    b.close()


def test_packed_rows_equal_padded_rows():
    """pcba_batch_upload_rows_packed: 1 + K doubles per constraint, padded on
    the device, gives the lists and results of the padded upload."""
    probs = [W.rtd(2200 + k, n_obstacles=n) for k, n in enumerate((128, 40))]
    b = pcba.Batch([pcba.linear_solver_from_problem(q, pcba.FP32) for q in probs], 2 << 30)
    assert b.rows_packed_doubles() * 8 == b.rows_doubles() * 4  # K = 3: 4 of 8 doubles
    packed = pcba.linear_rows_packed(probs)
    h = pcba.host_empty(packed.size)
    h[:] = packed
    b.upload_rows(pcba.linear_rows(probs))
    ref = b.solve(opt_tol=1e-3)
    b.upload_rows_packed(h)
    got = b.solve(opt_tol=1e-3)
    for a, r in zip(got, ref):
        for key in ("status", "lower", "upper", "steps"):
            assert a[key] == r[key]
        np.testing.assert_array_equal(a["x"], r["x"])
    b.close()


def test_items_with_many_chunks_are_windowed_soundly():
    """12,000 obstacles: 47 chunks of 256 constraints, many with more active
    constraints at the first steps than one window takes, so that they are cut
    into word-range windows (up to four each, the window list sized for 64
    such chunks).  The linear family in FP32 certifies an interval that
    overlaps the dense FP64 solve's (an independent path), and its point is
    feasible."""
    p = W.rtd(2300, n_obstacles=12000)
    g = lin(p, pcba.FP32).solve(opt_tol=1e-3, mem_cap=4 << 30)
    d = pcba.solver_from_problem(p, pcba.FP64).solve(opt_tol=1e-3, mem_cap=8 << 30)
    assert g["status"] == d["status"], (g["status"], d["status"])
    if d["status"] == pcba.OPTIMAL:
        assert g["upper"] - g["lower"] <= 1e-3
        assert g["lower"] <= d["upper"] and d["lower"] <= g["upper"], (g, d)
        assert max(oracle.eval_monomial(gi, g["x"]) for gi in p.ineq) <= 0.0
