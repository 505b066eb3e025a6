"""Seeded synthetic polynomial optimisation problems (POPs, Eq. (P)).

This module only builds inputs: dense monomial coefficient tensors of the cost,
the inequality constraints and the equality constraints, plus the box domain.
It holds none of the PCBA arithmetic (no Bernstein form, no subdivision, no
bounds); both the CUDA library and the CPU oracle receive exactly the arrays
built here.

Tensor convention: a polynomial of multi-degree N in l variables is a float64
array of shape (N_1+1, ..., N_l+1); entry [j_1, ..., j_l] is the coefficient
of x_1^j_1 ... x_l^j_l (Sec. II-A, Eq. (poly_monomial_basis)).  A family of
constraints is stacked along a leading axis at one common multi-degree
(Sec. IV-C): shorter constraints are zero-padded, which leaves the polynomial
unchanged.

Workloads (numpy ``default_rng(seed)``):
  tiny      l=2 on [-1,1]^2, cost degree (4,4) ~ N(0,1), 10 inequalities of
            degree (4,4) ~ N(0,1) shifted so g_i(q*) = -0.1 at a uniform q*.
  rtd       l=2 on [-1,1]^2, a map F: [-1,1]^2 -> R^2 of degree (3,3) with
            N(0, 0.5^2) coefficients, obstacle points o_i ~ U([-2,2]^2),
            g_i = r^2 - ||F(q) - o_i||^2 (degree (6,6), r = 0.15), cost
            ||F(q) - goal||^2 with goal ~ U([-2,2]^2).  This stands in for the
            reachability-based trajectory design POP of Sec. II-C, whose FRS
            polynomial w is not available.  The constraints are also given
            as a linear family in the shared polynomials (||F||^2, F_1, F_2)
            (meta["linear"] = (shared, weight, offset)).
  dim4      l=4 on [-1,1]^4, cost degree 4 per axis ~ N(0,1), 64 inequalities of
            degree 3 per axis shifted so g_i(q*) = -0.1, 2 equalities of degree 2
            per axis with h_j(q*) = 0.
  batch     rtd problems with obstacle counts floor(exp U(ln 16, ln 4096)).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy import signal


@dataclasses.dataclass
class Problem:
    """One POP (Eq. (P)) in dense monomial form over the box [lo, hi]."""
    cost: np.ndarray            # (P+1)
    ineq: np.ndarray            # (alpha, G+1)
    eq: np.ndarray              # (beta, H+1)
    lo: np.ndarray              # (l,)
    hi: np.ndarray              # (l,)
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def l(self) -> int:
        return self.cost.ndim

    @property
    def n_ineq(self) -> int:
        return int(self.ineq.shape[0])

    @property
    def n_eq(self) -> int:
        return int(self.eq.shape[0])


def _empty_family(l: int) -> np.ndarray:
    return np.zeros((0,) + (1,) * l)


def poly_mul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Product of two dense monomial tensors (full n-D convolution)."""
    return signal.convolve(a, b, mode="full", method="direct")


def poly_add(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    shape = tuple(max(x, y) for x, y in zip(a.shape, b.shape))
    out = np.zeros(shape)
    out[tuple(slice(0, s) for s in a.shape)] += a
    out[tuple(slice(0, s) for s in b.shape)] += b
    return out


def pad_to(a: np.ndarray, shape) -> np.ndarray:
    out = np.zeros(tuple(shape))
    out[tuple(slice(0, s) for s in a.shape)] = a
    return out


def poly_value(a: np.ndarray, x) -> float:
    """Value of a dense monomial tensor at x, as a tensor contraction of the
    coefficients with the power vectors of each coordinate (used only to place
    constraints through a chosen point)."""
    out = np.asarray(a, dtype=np.float64)
    for r in range(a.ndim):
        pw = float(x[r]) ** np.arange(a.shape[r])
        out = np.tensordot(pw, out, axes=([0], [0]))
    return float(out)


def _shifted(rng, shape, q_star, value):
    """Random N(0,1) tensor whose polynomial takes ``value`` at q_star (the
    constant coefficient absorbs the shift)."""
    g = rng.standard_normal(shape)
    g[(0,) * len(shape)] += value - poly_value(g, q_star)
    return g


def tiny(seed: int, n_ineq: int = 10, degree: int = 4) -> Problem:
    """l=2, degree-4 cost and 10 degree-4 inequalities feasible at q*."""
    rng = np.random.default_rng(seed)
    l = 2
    q_star = rng.uniform(-1.0, 1.0, size=l)
    cost = rng.standard_normal((degree + 1,) * l)
    ineq = np.stack([_shifted(rng, (degree + 1,) * l, q_star, -0.1) for _ in range(n_ineq)])
    return Problem(cost, ineq, _empty_family(l), -np.ones(l), np.ones(l),
                   {"q_star": q_star, "workload": "tiny", "seed": seed})


def rtd(seed: int, n_obstacles: int = 512, radius: float = 0.15, f_degree: int = 3,
        f_sigma: float = 0.5) -> Problem:
    """RTD-shaped planning POP on [-1,1]^2 (see module docstring)."""
    rng = np.random.default_rng(seed)
    shape = (f_degree + 1, f_degree + 1)
    F = [rng.normal(0.0, f_sigma, size=shape) for _ in range(2)]
    obstacles = rng.uniform(-2.0, 2.0, size=(n_obstacles, 2))
    goal = rng.uniform(-2.0, 2.0, size=2)
    FF = poly_add(poly_mul(F[0], F[0]), poly_mul(F[1], F[1]))          # ||F||^2
    one = np.ones((1, 1))
    # cost = ||F||^2 - 2 goal.F + ||goal||^2
    cost = poly_add(FF, -2.0 * goal[0] * F[0] - 2.0 * goal[1] * F[1])
    cost = poly_add(cost, float(goal @ goal) * one)
    # g_i = r^2 - ||o_i||^2 - ||F||^2 + 2 o_i.F, all obstacles at once
    ineq = np.zeros((n_obstacles,) + FF.shape)
    ineq += -FF
    sl = (slice(None),) + tuple(slice(0, s) for s in shape)
    ineq[sl] += (2.0 * obstacles[:, 0])[:, None, None] * F[0] \
        + (2.0 * obstacles[:, 1])[:, None, None] * F[1]
    offset = np.array([radius * radius - float(o @ o) for o in obstacles])
    ineq[:, 0, 0] += offset
    # the same constraints as a linear family: g_i = offset_i + w_i . (||F||^2, F_1, F_2)
    shared = np.stack([FF, pad_to(F[0], FF.shape), pad_to(F[1], FF.shape)])
    weight = np.stack([-np.ones(n_obstacles), 2.0 * obstacles[:, 0], 2.0 * obstacles[:, 1]], 1)
    return Problem(pad_to(cost, FF.shape), ineq, _empty_family(2), -np.ones(2), np.ones(2),
                   {"F": F, "obstacles": obstacles, "goal": goal, "radius": radius,
                    "workload": "rtd", "seed": seed, "linear": (shared, weight, offset)})


def dim4(seed: int, n_ineq: int = 64, n_eq: int = 2) -> Problem:
    """l=4 POP with 64 inequalities and 2 equalities through a seeded q*."""
    rng = np.random.default_rng(seed)
    l = 4
    q_star = rng.uniform(-1.0, 1.0, size=l)
    cost = rng.standard_normal((5,) * l)
    ineq = np.stack([_shifted(rng, (4,) * l, q_star, -0.1) for _ in range(n_ineq)]) \
        if n_ineq else _empty_family(l)
    eq = np.stack([_shifted(rng, (3,) * l, q_star, 0.0) for _ in range(n_eq)]) \
        if n_eq else _empty_family(l)
    return Problem(cost, ineq, eq, -np.ones(l), np.ones(l),
                   {"q_star": q_star, "workload": "dim4", "seed": seed})


def batch_obstacle_counts(n: int, seed: int, lo: int = 16, hi: int = 4096) -> np.ndarray:
    """Obstacle counts floor(exp U(ln lo, ln hi)) for a batch of rtd problems."""
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n))).astype(int)


def batch(n: int = 256, base_seed: int = 4000, lo: int = 16, hi: int = 4096):
    """n rtd problems with log-uniform obstacle counts and seeds base_seed + k."""
    counts = batch_obstacle_counts(n, base_seed, lo, hi)
    return [rtd(base_seed + k, n_obstacles=int(c)) for k, c in enumerate(counts)]


def random_patches(seed: int, shape, scale: float = 1.0) -> np.ndarray:
    """Random N(0, scale^2) coefficient tensors, used as Bernstein patches in
    kernel-level tests (any array of coefficients is a valid Bernstein patch)."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(shape)
