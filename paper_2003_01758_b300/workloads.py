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
  rtd_star  the hardware planning POP of Sec. VI-A, Eq. (online_trajopt_POP):
            q = (speed, yaw rate) in Q = [0,1] x [-1,1]; cost the waypoint
            product prod_n ||x(q) - x_n||^2 with x(q) the endpoint of a
            unicycle arc of duration T ~ U(1, 2) s (its Taylor polynomial of
            total degree 5, so the cost has degree 10 N_wp, plus N(0, 0.02^2)
            perturbations of every monomial; total degree 4 when N_wp = 2, so
            that the product stays within the per-axis degree limit of 16);
            waypoints 1.5 m ahead.  Constraints w(x_i, q) + 1e-4 <= 0 for
            n_ineq obstacle points x_i on the perimeters of 0.3 m boxes
            (centres U([0.7, 2.2] x [-1, 1]), 20 points per box), with the
            synthetic FRS bound w(x, q) = r^2 - ||x - y(q)||^2: y(q) the arc's
            point at 0.6 T (Taylor, total degree 6, perturbed likewise) and
            r ~ U(0.35, 0.5), so every constraint has degree 12.  The FRS
            polynomial of the paper comes from an offline sums-of-squares
            program and is not available; this bound has its degree and its
            sign convention (w >= 0 where a point may be hit).  Also given as
            a linear family in (||y||^2, y_1, y_2).
  increasing_constraints  Sec. V-C, Setup: n random constraints of total
            degree <= 2 with coefficients ~ U[-5, 5], each shifted so that a
            given optimizer x* of the objective stays feasible, here with a
            margin: g(x*) = -1 (the paper's g(x*) = 0 puts x* on every
            constraint's boundary, and 10 or more random constraints through
            one point leave no box around it that a bound can prove feasible).
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


def _total_degree_mask(l: int, d: int) -> np.ndarray:
    """1 where the monomial of the (d+1)^l tensor has total degree <= d."""
    idx = np.indices((d + 1,) * l).sum(axis=0)
    return (idx <= d).astype(float)


def _arc(v_pow: int, T: float, frac: float, degree: int):
    """Taylor polynomials (in q = (v, w)) of the position of a unicycle that
    starts at the origin heading +x and drives at speed v and yaw rate w for
    time frac * T: x1 = v sin(w t) / w, x2 = v (1 - cos(w t)) / w, truncated
    to total degree `degree`; tensors of shape (degree+1, degree+1)."""
    t = frac * T
    x1 = np.zeros((degree + 1, degree + 1))
    x2 = np.zeros((degree + 1, degree + 1))
    for m in range(degree):  # terms v w^m, total degree 1 + m
        c = t ** (m + 1) / math.factorial(m + 1)
        if m % 2 == 0:
            x1[v_pow, m] = (-1) ** (m // 2) * c
        else:
            x2[v_pow, m] = (-1) ** ((m - 1) // 2) * c
    return x1, x2


def rtd_star(seed: int, n_ineq: int = 100, n_wp: int = 1, eps: float = 1e-4,
             sigma: float = 0.02) -> Problem:
    """RTD*-shaped planning POP of Sec. VI-A (see module docstring)."""
    if n_wp not in (1, 2):
        raise ValueError("n_wp must be 1 or 2")
    rng = np.random.default_rng(seed)
    T = rng.uniform(1.0, 2.0)
    dx = 5 if n_wp == 1 else 4
    x = [c + sigma * rng.standard_normal(c.shape) * _total_degree_mask(2, dx)
         for c in _arc(1, T, 1.0, dx)]
    y = [c + sigma * rng.standard_normal(c.shape) * _total_degree_mask(2, 6)
         for c in _arc(1, T, 0.6, 6)]
    if n_wp == 1:
        wps = [np.array([1.5, rng.uniform(-0.5, 0.5)])]
    else:
        wps = [np.array([1.5, 0.5]) + rng.normal(0.0, 0.05, 2),
               np.array([1.5, -0.5]) + rng.normal(0.0, 0.05, 2)]
    xx = poly_add(poly_mul(x[0], x[0]), poly_mul(x[1], x[1]))
    cost = np.ones((1, 1))
    for wp in wps:
        f = poly_add(xx, -2.0 * wp[0] * x[0] - 2.0 * wp[1] * x[1])
        f = poly_add(f, float(wp @ wp) * np.ones((1, 1)))
        cost = poly_mul(cost, f)
    # obstacle points on the perimeters of 0.3 m boxes
    n_box = max(1, -(-n_ineq // 20))
    centres = np.stack([rng.uniform(0.7, 2.2, n_box), rng.uniform(-1.0, 1.0, n_box)], 1)
    box = rng.integers(0, n_box, n_ineq)
    s = rng.uniform(0.0, 4.0, n_ineq)  # position along the perimeter (side 1)
    side, f = np.floor(s).astype(int), s - np.floor(s)
    zero, one = np.zeros_like(f), np.ones_like(f)
    local = np.stack([np.choose(side, [f, one, 1.0 - f, zero]),
                      np.choose(side, [zero, f, one, 1.0 - f])], 1)
    pts = centres[box] + 0.3 * (local - 0.5)
    radius = rng.uniform(0.35, 0.5)
    yy = poly_add(poly_mul(y[0], y[0]), poly_mul(y[1], y[1]))   # ||y||^2, degree 12
    # g_i = w(x_i, q) + eps = r^2 + eps - ||x_i||^2 + 2 x_i . y(q) - ||y(q)||^2
    ineq = np.zeros((n_ineq,) + yy.shape)
    ineq += -yy
    sl = (slice(None),) + tuple(slice(0, d) for d in y[0].shape)
    ineq[sl] += (2.0 * pts[:, 0])[:, None, None] * y[0] + (2.0 * pts[:, 1])[:, None, None] * y[1]
    offset = radius * radius + eps - (pts ** 2).sum(1)
    ineq[:, 0, 0] += offset
    shared = np.stack([yy, pad_to(y[0], yy.shape), pad_to(y[1], yy.shape)])
    weight = np.stack([-np.ones(n_ineq), 2.0 * pts[:, 0], 2.0 * pts[:, 1]], 1)
    return Problem(cost, ineq, _empty_family(2), np.array([0.0, -1.0]), np.array([1.0, 1.0]),
                   {"workload": "rtd_star", "seed": seed, "n_wp": n_wp, "T": T,
                    "waypoints": wps, "points": pts, "radius": radius, "x": x, "y": y,
                    "linear": (shared, weight, offset)})


def increasing_constraints(cost: np.ndarray, lo, hi, x_star, n_ineq: int, seed: int,
                           margin: float = 1.0) -> Problem:
    """Sec. V-C, Setup: the objective (cost on [lo, hi], a known optimizer
    x_star) with n_ineq random constraints; each is the sum of the monomials
    of total degree <= 2 with coefficients ~ U[-5, 5], minus its value at
    x_star and minus `margin`, so that x_star stays strictly feasible
    (g(x_star) = -margin; with margin 0 every constraint passes through x_star
    and the feasible set near it is the single point)."""
    l = cost.ndim
    rng = np.random.default_rng(seed)
    mask = _total_degree_mask(l, 2)
    ineq = rng.uniform(-5.0, 5.0, size=(n_ineq,) + mask.shape) * mask
    for g in ineq:
        g[(0,) * l] -= poly_value(g, x_star) + margin
    return Problem(np.array(cost, dtype=float), ineq, _empty_family(l),
                   np.array(lo, dtype=float), np.array(hi, dtype=float),
                   {"workload": "increasing_constraints", "seed": seed,
                    "x_star": np.array(x_star, dtype=float)})


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
