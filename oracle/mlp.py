"""FP64 reference of the learned warm start's set-encoder network.

TEST INFRASTRUCTURE: only tests/ use this module; it shares no code with the
CUDA kernels of paper_2003_01758_b300 (the network is not part of the paper;
its definition here is the plain one, written out layer by layer).

Network (per problem: a set of points x_p in R^dp and a global vector u in R^dg):
    h1_p = relu(x_p W1 + b1)          dp  -> H
    h2_p = relu(h1_p W2 + b2)         H   -> H
    h3_p = relu(h2_p W3 + b3)         H   -> H
    z    = max_p h3_p                 (elementwise max over the set)
    h4   = relu([z, u] W4 + b4)       H+dg -> H
    h5   = relu(h4 W5 + b5)           H   -> H
    y    = tanh(h5 W6 + b6)           H   -> 2
Loss over a batch of B problems with targets t: L = (1/B) sum_b ||y_b - t_b||^2.

Parameters are kept in one flat vector in the order
W1, b1, W2, b2, W3, b3, W4, b4, W5, b5, W6, b6 (weights row-major [in][out]).

Operand rounding: with rnd=bf16_round, both operands of every matrix product
of the forward pass, and of the weight-gradient and input-gradient products of
layers 1-5 in the backward pass, are rounded to bfloat16 before an exact (FP64)
product; sums, biases, activations and the output layer's backward stay FP64.
This is the definition of the network's BF16 precision; rnd=None is the plain
FP64 network.
"""
from __future__ import annotations

import numpy as np


def layer_shapes(dp=2, dg=34, H=128, dout=2):
    return [(dp, H), (H,), (H, H), (H,), (H, H), (H,), (H + dg, H), (H,), (H, H), (H,),
            (H, dout), (dout,)]


def unflatten(theta, dp=2, dg=34, H=128, dout=2):
    out, o = [], 0
    for shp in layer_shapes(dp, dg, H, dout):
        n = int(np.prod(shp))
        out.append(np.asarray(theta[o:o + n], dtype=np.float64).reshape(shp))
        o += n
    return out


def n_params(dp=2, dg=34, H=128, dout=2):
    return int(sum(np.prod(s) for s in layer_shapes(dp, dg, H, dout)))


def relu(v):
    return np.maximum(v, 0.0)


def bf16_round(a):
    """Round to the nearest bfloat16 value (8-bit significand, ties to even),
    returned as float64.  Finite normal-range inputs only."""
    m, e = np.frexp(np.asarray(a, dtype=np.float64))    # a = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0), e - 8)


def _ident(a):
    return a


def forward(theta, points, offsets, glob, dims=(2, 34, 128, 2), rnd=None):
    """points [P, dp], offsets [B+1] (set b = points[offsets[b]:offsets[b+1]]),
    glob [B, dg]; returns y [B, 2] and the cache for backward."""
    r = rnd or _ident
    W1, b1, W2, b2, W3, b3, W4, b4, W5, b5, W6, b6 = unflatten(theta, *dims)
    h1 = relu(r(points) @ r(W1) + b1)
    h2 = relu(r(h1) @ r(W2) + b2)
    h3 = relu(r(h2) @ r(W3) + b3)
    B = len(offsets) - 1
    z = np.empty((B, h3.shape[1]))
    arg = np.empty((B, h3.shape[1]), dtype=np.int64)
    for b in range(B):
        seg = h3[offsets[b]:offsets[b + 1]]
        k = np.argmax(seg, axis=0)
        arg[b] = offsets[b] + k
        z[b] = seg[k, np.arange(seg.shape[1])]
    u = np.concatenate([z, glob], axis=1)
    h4 = relu(r(u) @ r(W4) + b4)
    h5 = relu(r(h4) @ r(W5) + b5)
    y = np.tanh(r(h5) @ r(W6) + b6)
    return y, (points, h1, h2, h3, arg, u, h4, h5, y)


def loss(y, target):
    return float(np.sum((y - target) ** 2) / y.shape[0])


def backward(theta, cache, target, dims=(2, 34, 128, 2), rnd=None):
    """Gradient of the loss with respect to the flat parameter vector."""
    r = rnd or _ident
    W1, b1, W2, b2, W3, b3, W4, b4, W5, b5, W6, b6 = unflatten(theta, *dims)
    points, h1, h2, h3, arg, u, h4, h5, y = cache
    B = y.shape[0]
    H = h1.shape[1]
    dy = 2.0 * (y - target) / B
    d6 = dy * (1.0 - y * y)
    gW6, gb6 = h5.T @ d6, d6.sum(0)
    d5 = (d6 @ W6.T) * (h5 > 0)
    gW5, gb5 = r(h4).T @ r(d5), d5.sum(0)
    d4 = (r(d5) @ r(W5).T) * (h4 > 0)
    gW4, gb4 = r(u).T @ r(d4), d4.sum(0)
    du = r(d4) @ r(W4).T
    dz = du[:, :H]
    dh3 = np.zeros_like(h3)
    for b in range(B):
        dh3[arg[b], np.arange(H)] += dz[b]
    d3 = dh3 * (h3 > 0)
    gW3, gb3 = r(h2).T @ r(d3), d3.sum(0)
    d2 = (r(d3) @ r(W3).T) * (h2 > 0)
    gW2, gb2 = r(h1).T @ r(d2), d2.sum(0)
    d1 = (r(d2) @ r(W2).T) * (h1 > 0)
    gW1, gb1 = r(points).T @ r(d1), d1.sum(0)
    return np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4, gW5, gb5,
                                               gW6, gb6)])


def init_params(seed, dims=(2, 34, 128, 2)):
    """He-style initialisation with a seeded generator (the layout above)."""
    rng = np.random.default_rng(seed)
    out = []
    for shp in layer_shapes(*dims):
        if len(shp) == 2:
            out.append(rng.normal(0.0, np.sqrt(2.0 / shp[0]), size=shp).ravel())
        else:
            out.append(np.zeros(shp))
    return np.concatenate(out)


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One step of Adam (Kingma & Ba, 2015, Algorithm 1) at step count t >= 1:
    moments updated, bias-corrected, parameters moved.  Returns the new
    (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return theta - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
