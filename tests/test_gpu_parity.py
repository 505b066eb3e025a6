"""Parity of the CUDA library (through its C ABI) with the FP64 oracle.

FP64 mode performs exactly the oracle's arithmetic (round-to-nearest adds and
exact halvings in the de Casteljau triangle, the same list order from Alg. 2
and Alg. 5), so starting both from the same Bernstein patches the whole list
must agree bit for bit after every step.  From monomial inputs the two
conversions round differently (the library applies per-axis matrices, the
oracle sums the definition), so there the bar is the stated tolerance:
root patches within 1e-12 of max|b| per patch, and certified intervals that
overlap with width <= opt_tol.  FP32 mode carries a rigorous error bound per
patch, so its intervals must contain the optimum the oracle brackets."""
import numpy as np
import pytest

import oracle
from paper_2003_01758_b300 import pcba
from paper_2003_01758_b300 import workloads as W
from tests import benchmarks

pytestmark = pytest.mark.gpu

MEM = 1 << 30


def gpu_solver(p, precision, form="monomial"):
    return pcba.Solver(p.cost, p.ineq, p.eq, p.lo, p.hi, precision=precision, form=form)


def oracle_solve(p, **kw):
    return oracle.solve(p.cost, p.ineq, p.eq, p.lo, p.hi, **kw)


def assert_interval_parity(g, o, opt_tol):
    assert g["status"] == o["status"], (g, o)
    if o["status"] == oracle.OPTIMAL:
        assert g["upper"] - g["lower"] <= opt_tol
        # both intervals contain p*, so they overlap
        assert g["lower"] <= o["upper"] and o["lower"] <= g["upper"], (g, o)


def random_bernstein_problem(seed, l=2, deg=4, n_ineq=6, n_eq=0, eq_deg=2):
    """Random patches given directly in Bernstein form: noise plus a ramp over
    the coefficient grid, so that every inequality holds near the lower corner
    and every equality has a zero set crossing the box."""
    cost = W.random_patches(seed, (deg + 1,) * l)
    ramp = sum(np.meshgrid(*[np.arange(deg + 1) / deg] * l, indexing="ij"))
    ineq = 0.5 * W.random_patches(seed + 1, (n_ineq,) + (deg + 1,) * l) + 2.0 * (ramp - 0.45 * l)
    eramp = np.meshgrid(*[np.arange(eq_deg + 1) / eq_deg] * l, indexing="ij")[0]
    eq = 0.3 * W.random_patches(seed + 2, (n_eq,) + (eq_deg + 1,) * l) + (eramp - 0.4)
    return W.Problem(cost, ineq, eq, -np.ones(l), np.ones(l))


# --------------------------------------------------------------------------
# K1: monomial -> Bernstein on the device
# --------------------------------------------------------------------------

@pytest.mark.parametrize("maker,seed", [(W.tiny, 1000), (W.rtd, 2000), (W.dim4, 3000)])
def test_root_patches_match_oracle(maker, seed):
    p = maker(seed)
    s = gpu_solver(p, pcba.FP64)
    cost, ineq, eq = s.root_patches()
    ref = oracle.bernstein_from_monomial(p.cost, p.lo, p.hi)
    assert np.abs(cost - ref).max() <= 1e-12 * np.abs(ref).max()
    for i in range(p.n_ineq):
        ref = oracle.bernstein_from_monomial(p.ineq[i], p.lo, p.hi)
        assert np.abs(ineq[i] - ref).max() <= 1e-12 * np.abs(ref).max()
    for j in range(p.n_eq):
        ref = oracle.bernstein_from_monomial(p.eq[j], p.lo, p.hi)
        assert np.abs(eq[j] - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("name", ["P1", "P4", "P6", "P8"])
def test_root_patches_on_paper_problems(name):
    b = benchmarks.load(name)
    p = W.Problem(b["cost"], b["ineq"], b["eq"], b["lo"], b["hi"])
    cost, ineq, _ = gpu_solver(p, pcba.FP64).root_patches()
    ref = oracle.bernstein_from_monomial(p.cost, p.lo, p.hi)
    assert np.abs(cost - ref).max() <= 1e-12 * np.abs(ref).max()
    for i in range(p.n_ineq):
        ref = oracle.bernstein_from_monomial(p.ineq[i], p.lo, p.hi)
        assert np.abs(ineq[i] - ref).max() <= 1e-12 * max(np.abs(ref).max(), 1e-300)


# --------------------------------------------------------------------------
# K2-K4: bit-exact lists in FP64 from the same Bernstein roots
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed,l,deg,n_ineq,n_eq", [
    (11, 2, 4, 6, 0), (12, 2, 6, 37, 0), (13, 3, 3, 300, 0), (14, 2, 5, 4, 1), (15, 1, 7, 3, 0),
    (16, 4, 2, 5, 1)])
def test_fp64_lists_bit_exact(seed, l, deg, n_ineq, n_eq):
    p = random_bernstein_problem(seed, l, deg, n_ineq, n_eq)
    o = oracle.Solver(p.cost, p.ineq, p.eq, p.lo, p.hi, form="bernstein")
    g = gpu_solver(p, pcba.FP64, form="bernstein")
    for steps in range(1, 4 * l + 1):
        st = o.step(opt_tol=1e-9, eq_tol=0.05, max_iters=28)
        res = g.solve(opt_tol=1e-9, eq_tol=0.05, max_iters=28, mem_cap=MEM, max_steps=steps)
        ol, gl = o.get_list(), g.get_list()
        assert gl["cost"].shape == ol["cost"].shape, steps
        np.testing.assert_array_equal(gl["index"], ol["index"])
        np.testing.assert_array_equal(gl["level"], ol["level"])
        np.testing.assert_array_equal(gl["cost"], ol["cost"])
        np.testing.assert_array_equal(gl["ineq"], ol["ineq"])
        np.testing.assert_array_equal(gl["eq"], ol["eq"])
        tr = o.trace()[-1]
        assert res["upper"] == tr[2] or (np.isinf(res["upper"]) and np.isinf(tr[2]))
        assert res["lower"] == tr[3] or (np.isinf(res["lower"]) and np.isinf(tr[3]))
        if st != oracle.RUNNING:
            assert res["status"] == st
            break
        assert res["status"] == pcba.STEPLIMIT


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_fp64_full_solve_trace_bit_exact(seed):
    p = random_bernstein_problem(seed, 2, 6, 64, 0)
    o = oracle.Solver(p.cost, p.ineq, p.eq, p.lo, p.hi, form="bernstein")
    ores = o.solve(opt_tol=1e-6)
    g = gpu_solver(p, pcba.FP64, form="bernstein")
    b = pcba.Batch([g], MEM)
    gres = b.solve(opt_tol=1e-6)[0]
    assert gres["status"] == ores["status"]
    assert gres["steps"] == ores["steps"] and gres["sweeps"] == ores["sweeps"]
    assert gres["lower"] == ores["lower"] and gres["upper"] == ores["upper"]
    np.testing.assert_array_equal(b.trace(0), o.trace())
    if ores["status"] == oracle.OPTIMAL:
        np.testing.assert_array_equal(gres["box_lo"], ores["box_lo"])
        np.testing.assert_array_equal(gres["x"], ores["x"])


# --------------------------------------------------------------------------
# end to end from monomials
# --------------------------------------------------------------------------

@pytest.mark.parametrize("precision", [pcba.FP64, pcba.FP32])
@pytest.mark.parametrize("seed", [1000, 1001, 1002, 1003, 1004, 1005])
def test_tiny_end_to_end(precision, seed):
    p = W.tiny(seed)
    o = oracle_solve(p, opt_tol=1e-3)
    g = gpu_solver(p, precision).solve(opt_tol=1e-3, mem_cap=MEM)
    assert_interval_parity(g, o, 1e-3)
    x = g["x"]
    assert max(oracle.eval_monomial(gi, x) for gi in p.ineq) <= 0.0
    v = oracle.eval_monomial(p.cost, x)
    assert g["lower"] - 1e-9 <= v <= g["upper"] + 1e-9
    assert g["verify_max_g"] <= 1e-9
    assert abs(g["verify_cost"] - v) <= 1e-9 * max(1.0, abs(v))


@pytest.mark.parametrize("precision", [pcba.FP64, pcba.FP32])
@pytest.mark.parametrize("seed,n_obs", [(2000, 512), (2001, 512), (2002, 100), (2003, 37)])
def test_rtd_end_to_end(precision, seed, n_obs):
    p = W.rtd(seed, n_obstacles=n_obs)
    o = oracle_solve(p, opt_tol=1e-3)
    g = gpu_solver(p, precision).solve(opt_tol=1e-3, mem_cap=MEM)
    assert_interval_parity(g, o, 1e-3)
    if g["status"] == pcba.OPTIMAL:
        assert max(oracle.eval_monomial(gi, g["x"]) for gi in p.ineq) <= 0.0


def test_dim4_with_equalities_end_to_end():
    p = W.dim4(3000, n_ineq=8, n_eq=1)
    kw = dict(opt_tol=1e-2, eq_tol=1e-2, max_iters=10)
    o = oracle_solve(p, max_items=1 << 16, **kw)
    for prec in (pcba.FP64, pcba.FP32):
        s = gpu_solver(p, prec)
        g = s.solve(mem_cap=(1 << 16) * s.item_bytes(), **kw)
        if prec == pcba.FP64:
            assert g["status"] == o["status"]
        assert g["lower"] <= o["upper"] + 1e-9
        if g["status"] == pcba.OPTIMAL:
            assert abs(oracle.eval_monomial(p.eq[0], g["x"])) <= 1e-2 + 1e-9


@pytest.mark.parametrize("name", ["P1", "P2", "P3", "P4", "P6", "P8"])
def test_paper_problems_fp64(name):
    b = benchmarks.load(name)
    p = W.Problem(b["cost"], b["ineq"], b["eq"], b["lo"], b["hi"])
    B = oracle.bernstein_from_monomial(p.cost, p.lo, p.hi)
    eps = 1e-7 * (B.max() - B.min())
    o = oracle_solve(p, opt_tol=eps, max_iters=28, max_items=1 << 22)
    g = gpu_solver(p, pcba.FP64).solve(opt_tol=eps, max_iters=28, mem_cap=MEM)
    assert_interval_parity(g, o, eps)


def test_p7_equality_fp32_and_fp64():
    b = benchmarks.load("P7")
    p = W.Problem(b["cost"], b["ineq"], b["eq"], b["lo"], b["hi"])
    o = oracle_solve(p, opt_tol=1e-3, eq_tol=0.1, max_iters=28, max_items=1 << 20)
    g = gpu_solver(p, pcba.FP64).solve(opt_tol=1e-3, eq_tol=0.1, max_iters=28, mem_cap=4 * MEM)
    assert g["status"] == pcba.OPTIMAL
    assert g["lower"] <= b["optimum"] + 1e-9
    assert g["lower"] <= o["upper"] and o["lower"] <= g["upper"]
    # FP32: h reaches ~4e5 on [0,5]^4; stored relative to per-patch offsets,
    # its rounding error scales with each patch's range, so FP32 certifies
    # the same interval
    g = gpu_solver(p, pcba.FP32).solve(opt_tol=1e-3, eq_tol=0.1, max_iters=28, mem_cap=MEM)
    assert g["status"] == pcba.OPTIMAL
    assert g["lower"] <= b["optimum"] + 1e-9
    assert g["lower"] <= o["upper"] and o["lower"] <= g["upper"]


def test_fp32_contains_optimum_where_plain_fp64_misses():
    """E-V-D on [-100,100]^2: plain FP64 (oracle and library) misses the
    optimum by ~1e-3 through rounding; the FP32 directed-rounding interval
    must still contain it."""
    b = benchmarks.load("EVD")
    p = W.Problem(b["cost"], b["ineq"], b["eq"], b["lo"], b["hi"])
    g = gpu_solver(p, pcba.FP32).solve(opt_tol=1e-1, max_iters=40, mem_cap=MEM)
    assert g["lower"] <= b["optimum"] <= g["upper"]


# --------------------------------------------------------------------------
# FP32 rigour: stored patch +- error encloses the polynomial on its box
# --------------------------------------------------------------------------

@pytest.mark.parametrize("maker,seed,steps", [(W.tiny, 1001, 9), (W.rtd, 2001, 7)])
def test_fp32_patches_enclose_polynomials(maker, seed, steps):
    p = maker(seed) if maker is W.tiny else maker(seed, n_obstacles=64)
    s = gpu_solver(p, pcba.FP32)
    s.solve(opt_tol=1e-12, mem_cap=MEM, max_steps=steps)
    L = s.get_list()
    rng = np.random.default_rng(seed)
    K = L["cost"].shape[0]
    w = (p.hi - p.lo) / 2.0 ** L["level"]
    for k in rng.choice(K, size=min(K, 12), replace=False):
        lo = p.lo + L["index"][k] * w
        for x in rng.uniform(lo, lo + w, size=(4, p.l)):
            v = oracle.eval_monomial(p.cost, x)
            e = float(L["err"][k, 0])
            assert L["cost"][k].min() - e - 1e-12 * abs(v) <= v <= L["cost"][k].max() + e + 1e-12 * abs(v)
            for i in range(p.n_ineq):
                gv = oracle.eval_monomial(p.ineq[i], x)
                e = float(L["err"][k, 1 + i])
                assert L["ineq"][k, i].min() - e <= gv + 1e-12 <= L["ineq"][k, i].max() + e + 2e-12


# --------------------------------------------------------------------------
# batching, loop modes, edge cases
# --------------------------------------------------------------------------

def test_batch_equals_single_solves_fp64():
    probs = [W.tiny(1000), W.rtd(2000, n_obstacles=64), W.tiny(1003), W.rtd(2002, n_obstacles=300),
             W.dim4(3001, n_ineq=4, n_eq=0)]
    kw = dict(opt_tol=1e-3, max_iters=12)
    singles = []
    for p in probs:
        s = gpu_solver(p, pcba.FP64)
        singles.append(s.solve(mem_cap=MEM, **kw))
    solvers = [gpu_solver(p, pcba.FP64) for p in probs]
    batch = pcba.Batch(solvers, MEM * len(probs))
    res = batch.solve(**kw)
    for a, b in zip(singles, res):
        for key in ("status", "lower", "upper", "steps", "sweeps"):
            assert a[key] == b[key], key


@pytest.mark.parametrize("flags", [pcba.Batch.HOST_LOOP, pcba.Batch.INSTRUMENT])
def test_host_loop_equals_graph_loop(flags):
    probs = [W.rtd(2000 + k, n_obstacles=128) for k in range(4)]
    g = pcba.Batch([gpu_solver(p, pcba.FP32) for p in probs], 4 << 30)
    h = pcba.Batch([gpu_solver(p, pcba.FP32) for p in probs], 4 << 30, flags=flags)
    rg, rh = g.solve(), h.solve()
    for a, b in zip(rg, rh):
        for key in ("status", "lower", "upper", "steps"):
            assert a[key] == b[key]
    # the graph runs two iterations per body; one after the loop's end is not
    # a step, so both loops count the same steps: those of the longest solve
    its = max(r["steps"] for r in rg)
    assert g.stats()["loop_iters"] == h.stats()["loop_iters"] == its
    if flags == pcba.Batch.INSTRUMENT:
        t = h.timing()
        assert t["subdiv_launches"] > 0 and t["subdiv_bytes"] > 0 and t["subdiv_ms"] > 0


def test_batch_repeat_and_from_host_are_stable():
    probs = [W.rtd(2000 + k, n_obstacles=64) for k in range(3)]
    b = pcba.Batch([gpu_solver(p, pcba.FP32) for p in probs], 1 << 30)
    r1 = b.solve()
    r2 = b.solve()
    host = np.concatenate([np.concatenate([p.cost.ravel(), p.ineq.ravel(), p.eq.ravel()])
                           for p in probs])
    r3 = b.solve_from_host(host)
    for a, c, d in zip(r1, r2, r3):
        assert a["lower"] == c["lower"] == d["lower"]
        assert a["upper"] == c["upper"] == d["upper"]


def test_unconstrained_and_infeasible_and_caps():
    # unconstrained separable quadratic: p* = 0
    a = np.zeros((3, 3))
    a[2, 0], a[1, 0], a[0, 0] = 1.0, -0.6, 0.09 + 0.16
    a[0, 2], a[0, 1] = 1.0, 0.8
    for prec, tol in ((pcba.FP64, 1e-6), (pcba.FP32, 1e-4)):
        # FP32 certifies down to its accumulated rounding bound (~1e-6 here)
        s = pcba.Solver(a, None, None, -1, 1, precision=prec)
        r = s.solve(opt_tol=tol, max_iters=30, mem_cap=MEM)
        assert r["status"] == pcba.OPTIMAL and r["lower"] <= 0.0 <= r["upper"], prec
    # infeasible: x1 <= 0.2 and x1 >= 0.3
    g = np.zeros((2, 2, 1))
    g[0, 1, 0], g[0, 0, 0] = 1.0, -0.2
    g[1, 1, 0], g[1, 0, 0] = -1.0, 0.3
    c = np.zeros((2, 2))
    c[1, 1] = 1.0
    for prec in (pcba.FP64, pcba.FP32):
        r = pcba.Solver(c, g, None, -1, 1, precision=prec).solve(mem_cap=MEM)
        assert r["status"] == pcba.INFEASIBLE and np.isnan(r["x"]).all()
    # memory cap and iteration cap agree with the oracle
    p = W.rtd(2002, n_obstacles=32)
    s = gpu_solver(p, pcba.FP64)
    r = s.solve(mem_cap=16 * s.item_bytes())
    o = oracle_solve(p, max_items=16)
    assert r["status"] == o["status"] == pcba.MEMCAP
    # the two conversions round differently, so the bounds agree to rounding
    assert r["lower"] == pytest.approx(o["lower"], rel=1e-12) and r["steps"] == o["steps"]
    r = s.solve(mem_cap=MEM, max_iters=3)
    assert r["status"] == pcba.MAXITER and r["steps"] == 4
    r = s.solve(mem_cap=s.item_bytes())  # M = 1 < 2: no room for the first split
    assert r["status"] == pcba.MEMCAP and r["steps"] == 0


def test_high_degree_rtd_star_shape():
    """Degree-12 constraints as in the hardware POPs (Sec. VI)."""
    rng = np.random.default_rng(5)
    l = 2
    cost = rng.standard_normal((3, 3))
    ineq = rng.standard_normal((40, 13, 13)) * 0.05
    ineq[:, 0, 0] -= 0.3
    p = W.Problem(cost, ineq, W._empty_family(l), -np.ones(l), np.ones(l))
    o = oracle_solve(p, opt_tol=1e-3)
    g = gpu_solver(p, pcba.FP64).solve(opt_tol=1e-3, mem_cap=MEM)
    assert_interval_parity(g, o, 1e-3)
    # FP32 (patches re-centred on per-patch offsets): the same certificate
    g = gpu_solver(p, pcba.FP32).solve(opt_tol=1e-3, mem_cap=MEM)
    assert_interval_parity(g, o, 1e-3)


def test_warm_start_only_tightens():
    p = W.rtd(2003, n_obstacles=128)
    o = oracle_solve(p, opt_tol=1e-3)
    s = gpu_solver(p, pcba.FP32)
    cold = s.solve(mem_cap=MEM)
    s.set_warm_start(o["x"])            # a certified-feasible point near the optimum
    warm = s.solve(mem_cap=MEM)
    assert warm["status"] == pcba.OPTIMAL
    assert warm["lower"] <= o["upper"] and o["lower"] <= warm["upper"]
    assert warm["steps"] <= cold["steps"]
    s.set_warm_start(np.array([0.0, 0.0]))  # feasible or not, certification is unchanged
    r = s.solve(mem_cap=MEM)
    assert r["lower"] <= o["upper"] and o["lower"] <= r["upper"]


def test_full_size_batch_sampled_against_oracle():
    """The benchmark's workload (rtd, 512 obstacles, FP32, one batch of 64)
    checked on a sample of problems the oracle solves one by one."""
    probs = [W.rtd(2000 + k) for k in range(64)]
    b = pcba.Batch([gpu_solver(p, pcba.FP32) for p in probs], 64 << 30)
    res = b.solve(opt_tol=1e-3)
    for k in (0, 17, 31, 41, 63):
        o = oracle_solve(probs[k], opt_tol=1e-3)
        assert_interval_parity(res[k], o, 1e-3)
    assert [r["status"] for r in res] == [pcba.OPTIMAL] * 64


@pytest.mark.parametrize("precision", [pcba.FP64, pcba.FP32])
def test_tma_and_direct_subdivision_agree(precision):
    """The TMA-staged subdivision kernel and the direct-load one perform the
    same arithmetic, so every result must be identical."""
    probs = [W.rtd(2000 + k, n_obstacles=n) for k, n in enumerate((512, 37, 300, 100))]
    probs.append(W.dim4(3002, n_ineq=40, n_eq=1))
    kw = dict(opt_tol=1e-3, eq_tol=1e-2, max_iters=10)
    a = pcba.Batch([gpu_solver(p, precision) for p in probs], 8 << 30).solve(**kw)
    b = pcba.Batch([gpu_solver(p, precision) for p in probs], 8 << 30,
                   flags=pcba.Batch.NO_TMA).solve(**kw)
    for x, y in zip(a, b):
        for key in ("status", "lower", "upper", "steps", "peak_items"):
            assert x[key] == y[key], key


def test_fp64_lists_bit_exact_without_tma(monkeypatch):
    monkeypatch.setenv("PCBA_NO_TMA", "1")
    test_fp64_lists_bit_exact(12, 2, 6, 37, 0)


def test_autotune_keeps_results_and_picks_a_config():
    probs = [W.rtd(2000 + k, n_obstacles=n) for k, n in enumerate((512, 64, 700, 200, 33, 1000))]
    base = pcba.Batch([gpu_solver(p, pcba.FP32) for p in probs], 8 << 30).solve()
    b = pcba.Batch([gpu_solver(p, pcba.FP32) for p in probs], 8 << 30)
    tune = b.autotune()
    assert len(tune["ms_per_config"]) >= 2 and 0 <= tune["chosen"] < len(tune["ms_per_config"])
    assert b.config()["index"] == tune["chosen"]
    for x, y in zip(base, b.solve()):
        for key in ("status", "lower", "upper", "steps"):
            assert x[key] == y[key]


def test_uneven_batch_sampled_against_oracle():
    """Obstacle counts log-uniform in [16, 4096]: a 48-problem slice of the
    256-problem batch workload, every sixth problem checked by the oracle."""
    counts = W.batch_obstacle_counts(256, 4000)
    ks = list(range(0, 256, 16)) + [5, 77, 130, 201] + list(range(3, 256, 9))[:28]
    probs = [W.rtd(4000 + k, n_obstacles=int(counts[k])) for k in ks]
    b = pcba.Batch([gpu_solver(p, pcba.FP32) for p in probs], 48 << 30)
    b.autotune()
    res = b.solve()
    for j in range(0, len(ks), 6):
        o = oracle_solve(probs[j], opt_tol=1e-3)
        assert_interval_parity(res[j], o, 1e-3)
    bad = [(ks[j], int(counts[ks[j]]), r["status"], r["steps"], r["peak_items"], r["lower"], r["upper"])
           for j, r in enumerate(res) if r["status"] not in (pcba.OPTIMAL, pcba.INFEASIBLE)]
    assert not bad, bad
