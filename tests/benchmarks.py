"""Loads the paper's printed benchmark problems (tests/golden/benchmark_problems.json)
into dense monomial tensors, using sympy to expand the printed expressions."""
import json
import os

import numpy as np
import sympy as sp

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                     "benchmark_problems.json")


def _matrix_form(syms, mf):
    A = sp.Matrix(mf["A"])
    b, y, z = (sp.Matrix([sp.nsimplify(v) for v in mf[k]]) for k in ("b", "y", "z"))
    x = sp.Matrix(syms)
    expr = (-(x.T * A.T * A * x) + 2 * (y.T * A * x))[0, 0] - (y.T * y)[0, 0] \
        + sp.Rational(1, 4) * ((b - z).T * (b - z))[0, 0]
    return sp.expand(expr)


def _to_tensor(expr, syms, degree):
    poly = sp.Poly(sp.expand(expr), *syms)
    out = np.zeros(tuple(d + 1 for d in degree))
    for monom, coeff in poly.terms():
        out[monom] += float(coeff)
    return out


def _degree(expr, syms):
    poly = sp.Poly(sp.expand(expr), *syms)
    deg = [0] * len(syms)
    for monom, _ in poly.terms():
        deg = [max(a, b) for a, b in zip(deg, monom)]
    return deg


def names():
    with open(_PATH) as f:
        return [k for k in json.load(f) if not k.startswith("_")]


def load(name):
    """Returns dict(cost, ineq, eq, lo, hi, optimum, x_opt, cite) with each
    constraint family stacked at its common multi-degree."""
    with open(_PATH) as f:
        spec = json.load(f)[name]
    syms = sp.symbols(spec["vars"])
    loc = {s.name: s for s in syms}
    loc["pi"] = sp.pi
    loc["Rational"] = sp.Rational
    for k, v in spec.get("defs", {}).items():
        loc[k] = sp.sympify(v, locals=loc)

    def parse(e):
        if e == "MATRIX_FORM":
            return _matrix_form(syms, spec["matrix_form"])
        return sp.sympify(e, locals=loc)

    cost = parse(spec["cost"])
    ineq = [parse(e) for e in spec["ineq"]]
    eq = [parse(e) for e in spec["eq"]]
    l = len(syms)

    def family(exprs):
        if not exprs:
            return np.zeros((0,) + (1,) * l)
        deg = [0] * l
        for e in exprs:
            deg = [max(a, b) for a, b in zip(deg, _degree(e, syms))]
        return np.stack([_to_tensor(e, syms, deg) for e in exprs])

    return {
        "cost": _to_tensor(cost, syms, _degree(cost, syms)),
        "ineq": family(ineq), "eq": family(eq),
        "lo": np.array(spec["lo"], dtype=float), "hi": np.array(spec["hi"], dtype=float),
        "optimum": spec["optimum"], "x_opt": np.array(spec["x_opt"], dtype=float),
        "cite": spec["cite"],
    }
