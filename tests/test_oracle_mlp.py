"""Pins for the FP64 reference of the warm-start network (oracle/mlp.py):
central finite differences of the loss against the analytic gradient, set
permutation invariance of the max-pool, and closed-form outputs."""
import numpy as np
import pytest

from oracle import mlp

DIMS = (2, 3, 8, 2)  # small network for the finite-difference pin


def batch(seed, B=3):
    rng = np.random.default_rng(seed)
    sizes = rng.integers(2, 7, size=B)
    offsets = np.concatenate([[0], np.cumsum(sizes)])
    points = rng.normal(size=(offsets[-1], DIMS[0]))
    glob = rng.normal(size=(B, DIMS[1]))
    target = rng.uniform(-0.9, 0.9, size=(B, 2))
    return points, offsets, glob, target


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_gradient_matches_central_differences(seed):
    theta = mlp.init_params(seed, DIMS) + np.random.default_rng(seed + 10).normal(
        0, 0.05, mlp.n_params(*DIMS))
    points, offsets, glob, target = batch(seed)
    y, cache = mlp.forward(theta, points, offsets, glob, DIMS)
    g = mlp.backward(theta, cache, target, DIMS)
    h = 1e-6
    rng = np.random.default_rng(seed)
    for i in rng.choice(len(theta), size=60, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fp = mlp.loss(mlp.forward(tp, points, offsets, glob, DIMS)[0], target)
        fm = mlp.loss(mlp.forward(tm, points, offsets, glob, DIMS)[0], target)
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_set_order_does_not_matter():
    theta = mlp.init_params(5, DIMS)
    points, offsets, glob, _ = batch(5, B=2)
    y, _ = mlp.forward(theta, points, offsets, glob, DIMS)
    perm = points.copy()
    perm[offsets[0]:offsets[1]] = perm[offsets[0]:offsets[1]][::-1]
    y2, _ = mlp.forward(theta, perm, offsets, glob, DIMS)
    assert np.array_equal(y, y2)


def test_bias_only_network_outputs_tanh_of_bias():
    theta = np.zeros(mlp.n_params(*DIMS))
    theta[-2:] = [0.3, -1.2]
    points, offsets, glob, _ = batch(7)
    y, _ = mlp.forward(theta, points, offsets, glob, DIMS)
    assert np.allclose(y, np.tanh([0.3, -1.2]))


def test_adam_first_step_is_signed_learning_rate():
    """From zero moments the bias-corrected first Adam step is lr * g / (|g| + eps),
    i.e. lr * sign(g) wherever |g| >> eps; a second step with the same gradient
    is again lr * sign(g)."""
    rng = np.random.default_rng(7)
    th = rng.normal(size=50)
    g = rng.normal(size=50)
    g[0] = 0.0
    z = np.zeros(50)
    t1, m, v = mlp.adam_step(th, g, z, z, 1, 0.01)
    tol = 0.01 * 2e-8 / np.abs(g[1:]) + 1e-14   # the eps term, relative to |g|
    assert np.all(np.abs(t1[1:] - (th[1:] - 0.01 * np.sign(g[1:]))) <= tol)
    assert t1[0] == th[0]
    t2, _, _ = mlp.adam_step(t1, g, m, v, 2, 0.01)
    assert np.all(np.abs(t2[1:] - (t1[1:] - 0.01 * np.sign(g[1:]))) <= tol)


def test_bf16_round_special_values_and_torch():
    """Ties go to the even significand; the result equals torch's own
    float64 -> bfloat16 conversion on random normal-range values."""
    import torch
    u = 2.0 ** -7                       # one bf16 ulp at 1
    assert mlp.bf16_round(1.0 + u / 2) == 1.0            # tie -> even (1.0)
    assert mlp.bf16_round(1.0 + 3 * u / 2) == 1.0 + 2 * u  # tie -> even (1 + 2u)
    assert mlp.bf16_round(1.0 + 0.6 * u) == 1.0 + u
    assert mlp.bf16_round(-3.0) == -3.0 and mlp.bf16_round(0.0) == 0.0
    x = np.random.default_rng(0).normal(size=10000) * 10.0 ** np.random.default_rng(1).integers(
        -20, 20, size=10000)
    ref = torch.tensor(x, dtype=torch.float64).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(x), ref)


def test_bf16_network_stays_near_the_plain_network():
    """Operand rounding is piecewise constant in the weights, so finite
    differences do not apply to it; with weights and inputs on the bf16 grid,
    rounding only the hidden activations moves the outputs by a few bf16 ulps
    and the gradient by a few percent."""
    theta = mlp.bf16_round(mlp.init_params(4, DIMS))
    points, offsets, glob, target = batch(4)
    points = mlp.bf16_round(points)
    y0, _ = mlp.forward(theta, points, offsets, glob, DIMS)
    y1, _ = mlp.forward(theta, points, offsets, glob, DIMS, rnd=mlp.bf16_round)
    assert np.max(np.abs(y1 - y0)) <= 6 * 2.0 ** -8 * (1.0 + np.max(np.abs(y0)))
    g0 = mlp.backward(theta, mlp.forward(theta, points, offsets, glob, DIMS)[1], target, DIMS)
    g1 = mlp.backward(theta, mlp.forward(theta, points, offsets, glob, DIMS, mlp.bf16_round)[1],
                      target, DIMS, mlp.bf16_round)
    assert np.linalg.norm(g1 - g0) <= 0.1 * np.linalg.norm(g0)
