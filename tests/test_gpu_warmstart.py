"""The learned warm start on the device: the network kernels (forward,
backward, Adam) against the FP64 network oracle, and the guided solve
(candidate evaluation and incumbent seeding) against the PCBA oracle.

Tolerances.  Precision 32 computes every product in FP32 with FP32 sums over
at most a few thousand terms: relative error ~1e-6; bars 1e-5 on the outputs
and 1e-4 on the gradient.  Precision 16 is compared with the oracle run with
the same bfloat16 operand rounding (oracle.mlp.bf16_round at the same places),
so the two differ by FP32 accumulation order and by the rare activation whose
FP32 and FP64 values round to neighbouring bfloat16 numbers (about one element
in 10^3 to 10^4, each off by 2^-8 relative): bars 2e-3 on the outputs and 1e-2
on the gradient."""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp as omlp
from paper_2003_01758_b300 import pcba, warmstart
from paper_2003_01758_b300 import workloads as W

pytestmark = pytest.mark.gpu


def sets(seed, B, dims, size_lo=1, size_hi=300):
    dp, dg, _, _ = dims
    rng = np.random.default_rng(seed)
    sizes = rng.integers(size_lo, size_hi + 1, size=B)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    points = rng.normal(size=(offsets[-1], dp)).astype(np.float32)
    glob = rng.normal(size=(B, dg)).astype(np.float32)
    target = rng.uniform(-0.9, 0.9, size=(B, 2)).astype(np.float32)
    return points, offsets, glob, target


def network(dims, precision, seed):
    dp, dg, H, _ = dims
    m = pcba.Mlp(dp, dg, H, precision, seed)
    # biases away from zero so that no layer starts dead
    theta = omlp.init_params(seed, dims) + np.random.default_rng(seed).normal(
        0, 0.05, omlp.n_params(*dims))
    m.set_params(theta.astype(np.float32))
    return m, m.get_params().astype(np.float64)


CASES = [((2, 5, 32, 2), 7, 1, 300), ((2, 34, 128, 2), 40, 64, 1024), ((3, 0, 48, 2), 5, 1, 70)]


RND = {32: None, 16: omlp.bf16_round}


@pytest.mark.parametrize("precision,tol", [(32, 1e-5), (16, 2e-3)])
@pytest.mark.parametrize("dims,B,lo,hi", CASES)
def test_forward_matches_oracle(dims, B, lo, hi, precision, tol):
    m, theta = network(dims, precision, 11)
    points, offsets, glob, target = sets(5, B, dims, lo, hi)
    pk = warmstart.Packed(points, offsets, glob.reshape(B, dims[1]))
    y = warmstart.predict(m, pk)
    torch.cuda.synchronize()
    y_ref, _ = omlp.forward(theta, points.astype(np.float64), offsets, glob.astype(np.float64),
                            dims, RND[precision])
    assert np.max(np.abs(y.cpu().numpy() - y_ref)) <= tol


@pytest.mark.parametrize("precision,tol", [(32, 1e-4), (16, 1e-2)])
@pytest.mark.parametrize("dims,B,lo,hi", CASES)
def test_gradient_matches_oracle(dims, B, lo, hi, precision, tol):
    m, theta = network(dims, precision, 12)
    points, offsets, glob, target = sets(6, B, dims, lo, hi)
    pk = warmstart.Packed(points, offsets, glob.reshape(B, dims[1]), target)
    g, loss = m.gradient(*pk.args(), pk.target.data_ptr())
    y_ref, cache = omlp.forward(theta, points.astype(np.float64), offsets,
                                glob.astype(np.float64), dims, RND[precision])
    g_ref = omlp.backward(theta, cache, target.astype(np.float64), dims, RND[precision])
    assert abs(loss - omlp.loss(y_ref, target)) <= tol * max(1.0, omlp.loss(y_ref, target))
    # every parameter block, element by element: each entry within tol of its
    # own magnitude plus the block's largest entry.  An entry is a sum over
    # points whose terms cancel; the rounding of the BF16 operands (and of the
    # FP32 accumulation) bounds its error by tol times the sum of the absolute
    # terms, which is of the block's scale, not of the entry's
    o = 0
    for shp in omlp.layer_shapes(*dims):
        n = int(np.prod(shp))
        a, r = g[o:o + n].astype(np.float64), g_ref[o:o + n]
        scale = max(np.abs(r).max(), 1e-3 * np.abs(g_ref).max())
        bad = np.abs(a - r) > tol * (np.abs(r) + scale)
        assert not bad.any(), (shp, np.flatnonzero(bad)[:5], a[bad][:5], r[bad][:5])
        assert np.linalg.norm(a - r) <= tol * max(np.linalg.norm(r), 1e-3 * np.linalg.norm(g_ref)), shp
        o += n


def test_adam_steps_match_oracle():
    """Two train steps in FP32 against the oracle's Adam applied to the
    library's own gradients (the gradient itself is checked above)."""
    dims = (2, 5, 32, 2)
    m, theta = network(dims, 32, 13)
    points, offsets, glob, target = sets(7, 6, dims)
    pk = warmstart.Packed(points, offsets, glob, target)
    mo, vo = np.zeros_like(theta), np.zeros_like(theta)
    th = theta.copy()
    for t, lr in ((1, 1e-2), (2, 5e-3)):
        g, _ = m.gradient(*pk.args(), pk.target.data_ptr())
        m.train_step(*pk.args(), pk.target.data_ptr(), lr)
        th, mo, vo = omlp.adam_step(th, g.astype(np.float64), mo, vo, t, lr)
        got = m.get_params().astype(np.float64)
        assert np.max(np.abs(got - th) / (lr + np.abs(th))) <= 1e-5, t
        th = got


def test_training_reduces_loss():
    """BF16 training on a learnable synthetic target (a max over the set plus
    a linear term of the global vector) lowers the loss by a large factor."""
    dims = (2, 4, 64, 2)
    rng = np.random.default_rng(3)
    B = 64
    points, offsets, glob, _ = sets(8, B, dims, 5, 60)
    mx = np.stack([points[offsets[b]:offsets[b + 1]].max(0) for b in range(B)])
    target = np.clip(0.3 * mx + 0.2 * glob[:, :2], -0.9, 0.9).astype(np.float32)
    pk = warmstart.Packed(points, offsets, glob, target)
    m = pcba.Mlp(*dims[:3], 16, int(rng.integers(1 << 30)))
    first = m.train_step(*pk.args(), pk.target.data_ptr(), 1e-3)
    for _ in range(400):
        last = m.train_step(*pk.args(), pk.target.data_ptr(), 1e-3)
    assert last < 0.2 * first, (first, last)


# --------------------------------------------------------------------------
# guided solves
# --------------------------------------------------------------------------

# Candidates are certified in FP32: for these constraints (sum of |terms|
# about 10) the bound is below 1e-4, so "clearly feasible" means g < -CLEAR.
CLEAR = 1e-3
# Candidates are ranked by an FP32 upper bound on their cost (bound about
# 1e-5 of sum |a_J x^J|), so the chosen one may cost a little more than the
# cheapest feasible candidate.
RANK_TOL = 1e-3


def oracle_values(p, x):
    cost = oracle.eval_monomial(p.cost, x)
    g = max((oracle.eval_monomial(gi, x) for gi in p.ineq), default=-np.inf)
    h = max((abs(oracle.eval_monomial(hj, x)) for hj in p.eq), default=0.0)
    return cost, g, h


def test_guided_solve_seeds_best_certified_candidate():
    probs = [W.rtd(2100 + k, n_obstacles=n) for k, n in enumerate((512, 64, 1000, 200))]
    refs = [oracle.solve(p.cost, p.ineq, p.eq, p.lo, p.hi, opt_tol=1e-3) for p in probs]
    b = pcba.Batch([pcba.solver_from_problem(p, pcba.FP32) for p in probs], 16 << 30)
    cold = b.solve(opt_tol=1e-3)
    guess = np.stack([warmstart.normalise(r["x"], p) for r, p in zip(refs, probs)])
    d_guess = torch.as_tensor(guess.astype(np.float32), device="cuda")
    stencil = warmstart.default_stencil()
    res = b.solve_guided(d_guess.data_ptr(), 2, stencil, opt_tol=1e-3)
    for k, (p, r, c, o) in enumerate(zip(probs, res, cold, refs)):
        assert r["status"] == pcba.OPTIMAL and o["status"] == oracle.OPTIMAL
        assert r["lower"] <= o["upper"] and o["lower"] <= r["upper"]
        assert r["upper"] - r["lower"] <= 1e-3
        assert r["steps"] <= c["steps"]
        x, seed_cost = b.warm_point(k, with_cost=True)
        # the seed is one of the candidates (in FP32 coordinates)
        cands = np.clip(guess[k].astype(np.float32).astype(np.float64) + stencil, -1, 1)
        pts = (p.lo + 0.5 * (cands + 1.0) * (p.hi - p.lo)).astype(np.float32).astype(np.float64)
        d = np.min(np.max(np.abs(pts - x), axis=1))
        assert d == 0.0
        # it is feasible, and no clearly feasible candidate is clearly cheaper
        cx, gx, _ = oracle_values(p, x)
        assert gx <= 1e-12
        assert cx <= seed_cost <= cx + 1e-9 * (1.0 + abs(cx))
        vals = [oracle_values(p, q) for q in pts]
        clear = [v[0] for v in vals if v[1] < -CLEAR]
        if clear:       # a crowded problem may have no candidate that clear of all obstacles
            assert cx <= min(clear) + RANK_TOL * (1.0 + abs(cx))
        # the seed cannot beat the certified lower bound
        assert cx >= r["lower"] - 1e-9


def test_guided_solve_is_sound_for_any_guess():
    probs = [W.rtd(2200 + k, n_obstacles=300) for k in range(3)]
    refs = [oracle.solve(p.cost, p.ineq, p.eq, p.lo, p.hi, opt_tol=1e-3) for p in probs]
    b = pcba.Batch([pcba.solver_from_problem(p, pcba.FP32) for p in probs], 8 << 30)
    guess = torch.tensor([[np.nan, 0.0], [5.0, -5.0], [0.3, -0.7]], dtype=torch.float32,
                         device="cuda")
    res = b.solve_guided(guess.data_ptr(), 2, warmstart.default_stencil(), opt_tol=1e-3)
    for r, o in zip(res, refs):
        assert r["status"] == pcba.OPTIMAL
        assert r["lower"] <= o["upper"] and o["lower"] <= r["upper"]


def test_guided_solve_rejects_infeasible_seed():
    p = W.rtd(2300, n_obstacles=256)
    # a point mapped by F inside an obstacle: search the grid with the oracle
    xs = np.linspace(-1, 1, 41)
    bad = next(np.array([a, c]) for a in xs for c in xs
               if oracle_values(p, np.array([a, c]))[1] > 1e-3)
    b = pcba.Batch([pcba.solver_from_problem(p, pcba.FP64)], 4 << 30)
    guess = torch.as_tensor(warmstart.normalise(bad, p)[None].astype(np.float32), device="cuda")
    x_used = p.lo + 0.5 * (guess.cpu().numpy()[0].astype(np.float64) + 1) * (p.hi - p.lo)
    assert oracle_values(p, x_used)[1] > 0
    r = b.solve_guided(guess.data_ptr(), 2, np.zeros((1, 2)), opt_tol=1e-3)[0]
    assert b.warm_point(0) is None
    assert r["status"] == pcba.OPTIMAL


def test_cost_grid_matches_oracle():
    probs = [W.rtd(2400, n_obstacles=64), W.tiny(1001), W.dim4(3001, n_ineq=8, n_eq=1)]
    b = pcba.Batch([pcba.solver_from_problem(p, pcba.FP64) for p in probs], 4 << 30)
    G, ld, col0 = 7, 60, 5
    out = torch.full((len(probs), ld), -7.0, dtype=torch.float32, device="cuda")
    b.cost_grid(G, out.data_ptr(), ld, col0)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for k, p in enumerate(probs):
        x0 = p.lo[0] + (p.hi[0] - p.lo[0]) * np.arange(G) / (G - 1)
        x1 = p.lo[1] + (p.hi[1] - p.lo[1]) * np.arange(G) / (G - 1)
        c = np.empty((G, G))
        for i in range(G):
            for j in range(G):
                x = 0.5 * (p.lo + p.hi)
                x[0], x[1] = x0[i], x1[j]
                c[i, j] = oracle.eval_monomial(p.cost, x)
        ref = np.log(c - c.min() + 1e-3).ravel()
        assert np.allclose(got[k, col0:col0 + G * G], ref, rtol=1e-6, atol=1e-6)
        assert np.all(got[k, :col0] == -7.0) and np.all(got[k, col0 + G * G:] == -7.0)


def test_guided_full_stencil_and_grid_candidates():
    """1024 candidates (the limit) over a grid of the box: the seed is the
    cheapest certified-feasible grid node."""
    p = W.rtd(2500, n_obstacles=128)
    b = pcba.Batch([pcba.solver_from_problem(p, pcba.FP32)], 4 << 30)
    st = warmstart.grid_stencil(32)
    zero = torch.zeros((1, 2), dtype=torch.float32, device="cuda")
    r = b.solve_guided(zero.data_ptr(), 2, st, opt_tol=1e-3)[0]
    assert r["status"] == pcba.OPTIMAL
    x, cost = b.warm_point(0, with_cost=True)
    pts = (p.lo + 0.5 * (st + 1) * (p.hi - p.lo)).astype(np.float32).astype(np.float64)
    vals = [oracle_values(p, q) for q in pts]
    clear = [v[0] for v in vals if v[1] < -CLEAR]
    assert min(clear) >= cost - RANK_TOL * (1 + abs(cost))
    assert oracle_values(p, x)[1] <= 1e-12
    with pytest.raises(pcba.PcbaError, match="n_stencil"):
        b.solve_guided(zero.data_ptr(), 2, warmstart.grid_stencil(33))


@pytest.mark.parametrize("margin", [1e-9, 1e-6, 1e-3, -0.5])
def test_fp32_certification_never_accepts_an_infeasible_point(margin):
    """A constraint placed through the candidate with value +margin (in exact
    arithmetic on its FP64 coefficients) must be rejected for every positive
    margin, however small; a comfortably negative one must be accepted."""
    rng = np.random.default_rng(int(abs(margin) * 1e9) + 11)
    x0 = np.array([0.3125, -0.6875])                   # FP32 numbers
    for trial in range(8):
        cost = rng.standard_normal((5, 5))
        g = 3.0 * rng.standard_normal((7, 7))
        g[0, 0] += margin - W.poly_value(g, x0)
        p = W.Problem(cost, g[None], W._empty_family(2), -np.ones(2), np.ones(2))
        exact = oracle.eval_monomial(g, x0)
        assert (exact > 0) == (margin > 0)
        b = pcba.Batch([pcba.solver_from_problem(p, pcba.FP32)], 1 << 30)
        guess = torch.tensor([[x0[0], x0[1]]], dtype=torch.float32, device="cuda")
        b.solve_guided(guess.data_ptr(), 2, np.zeros((1, 2)), opt_tol=1e-3, max_iters=4)
        seed = b.warm_point(0)
        if margin > 0:
            assert seed is None
        else:
            assert seed is not None and np.array_equal(seed, x0)


def test_refinement_never_worsens_the_seed():
    """The second round around the seed (its stencil holds the centre) gives,
    problem by problem, a seed at most as costly, and the solves stay certified."""
    probs = [W.rtd(2600 + k, n_obstacles=n) for k, n in enumerate((512, 128, 300, 900))]
    b = pcba.Batch([pcba.solver_from_problem(p, pcba.FP32) for p in probs], 16 << 30)
    guess = torch.zeros((len(probs), 2), dtype=torch.float32, device="cuda")
    st = warmstart.default_stencil()
    b.solve_guided(guess.data_ptr(), 2, st)
    first = [b.warm_point(k, with_cost=True) for k in range(len(probs))]
    b.set_refine_stencil(warmstart.refine_stencil())
    res = b.solve_guided(guess.data_ptr(), 2, st)
    second = [b.warm_point(k, with_cost=True) for k in range(len(probs))]
    for p, f, g, r in zip(probs, first, second, res):
        assert r["status"] == pcba.OPTIMAL
        if f is not None:
            assert g is not None and g[1] <= f[1] + RANK_TOL * (1.0 + abs(f[1]))
            assert oracle_values(p, g[0])[1] <= 1e-12
            assert g[1] >= r["lower"] - 1e-9
    with pytest.raises(pcba.PcbaError, match="dimensions"):
        b.set_refine_stencil(np.zeros((3, 1)), guess_dim=1)
        b.solve_guided(guess.data_ptr(), 2, st)
