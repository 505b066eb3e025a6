"""PCBA oracle: plain FP64 CPU implementation of the Parallel Constrained
Bernstein Algorithm (arXiv 2003.01758), used only to check the CUDA library.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with ``paper_2003_01758_b300`` and never imports
it; the CUDA library never imports this package.

The arithmetic lives in ``pcba_oracle.c`` (plain C, one thread); this module
only compiles it with gcc and marshals numpy arrays through ctypes.  Each C
routine cites the section, definition, theorem or algorithm it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pcba_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

OPTIMAL, INFEASIBLE, MEMCAP, MAXITER, RUNNING = 0, 1, 2, 3, 10
STATUS_NAMES = {0: "OPTIMAL", 1: "INFEASIBLE", 2: "MEMCAP", 3: "MAXITER", 10: "RUNNING"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/liboracle.so``."""
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-fno-fast-math", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        D, I, L, P = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_void_p
        lib.or_bernstein_from_monomial.argtypes = [I, P, P, P, P, P]
        lib.or_bernstein_from_monomial.restype = I
        lib.or_subdivide_patch.argtypes = [I, P, P, I, P, P]
        lib.or_subdivide_patch.restype = I
        lib.or_eval_monomial.argtypes = [I, P, P, P]
        lib.or_eval_monomial.restype = D
        lib.or_eval_bernstein.argtypes = [I, P, P, P, P, P]
        lib.or_eval_bernstein.restype = D
        lib.or_create.argtypes = [I, P, P, P, P, I, P, P, I, P, P, I, ctypes.c_longlong]
        lib.or_create.restype = P
        lib.or_destroy.argtypes = [P]
        lib.or_step.argtypes = [P, D, D, I, D]
        lib.or_step.restype = I
        lib.or_solve.argtypes = [P, D, D, I, D, P]
        lib.or_solve.restype = I
        lib.or_list_length.argtypes = [P]
        lib.or_list_length.restype = L
        lib.or_item_len.argtypes = [P]
        lib.or_item_len.restype = L
        lib.or_trace_length.argtypes = [P]
        lib.or_trace_length.restype = L
        lib.or_status.argtypes = [P]
        lib.or_status.restype = I
        lib.or_get_list.argtypes = [P, P, P, P]
        lib.or_get_keep.argtypes = [P, P, L]
        lib.or_get_trace.argtypes = [P, P]
        lib.or_memory_per_item.argtypes = [I, P, I, P, I, P]
        lib.or_memory_per_item.restype = ctypes.c_longlong
        _lib = lib
        return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# primitives
# --------------------------------------------------------------------------

def bernstein_from_monomial(a, lo, hi):
    """Bernstein patch over the box [lo, hi] of the polynomial whose dense
    monomial tensor is ``a`` (shape N+1 per axis)."""
    a = _f64(a)
    l = a.ndim
    N = _i32(np.array(a.shape) - 1)
    lo, hi = _f64(np.broadcast_to(lo, (l,))), _f64(np.broadcast_to(hi, (l,)))
    b = np.empty_like(a)
    rc = _load().or_bernstein_from_monomial(l, _ptr(N), _ptr(a), _ptr(lo), _ptr(hi), _ptr(b))
    if rc:
        raise ValueError("or_bernstein_from_monomial failed: %d" % rc)
    return b


def subdivide_patch(b, r):
    """(left, right) Bernstein patches after bisecting axis r (0-based)."""
    b = _f64(b)
    l = b.ndim
    N = _i32(np.array(b.shape) - 1)
    left, right = np.empty_like(b), np.empty_like(b)
    rc = _load().or_subdivide_patch(l, _ptr(N), _ptr(b), int(r), _ptr(left), _ptr(right))
    if rc:
        raise ValueError("or_subdivide_patch failed: %d" % rc)
    return left, right


def eval_monomial(a, x):
    a = _f64(a)
    l = a.ndim
    N = _i32(np.array(a.shape) - 1)
    x = _f64(np.broadcast_to(x, (l,)))
    return _load().or_eval_monomial(l, _ptr(N), _ptr(a), _ptr(x))


def eval_bernstein(b, lo, hi, x):
    b = _f64(b)
    l = b.ndim
    N = _i32(np.array(b.shape) - 1)
    lo, hi = _f64(np.broadcast_to(lo, (l,))), _f64(np.broadcast_to(hi, (l,)))
    x = _f64(np.broadcast_to(x, (l,)))
    return _load().or_eval_bernstein(l, _ptr(N), _ptr(b), _ptr(lo), _ptr(hi), _ptr(x))


def memory_per_item(l, P, n_ineq, G, n_eq, H):
    """Entries per item, Eq. (memory_per_item)."""
    P, G, H = _i32(P), _i32(G if G is not None else [0] * l), _i32(H if H is not None else [0] * l)
    return int(_load().or_memory_per_item(l, _ptr(P), n_ineq, _ptr(G), n_eq, _ptr(H)))


# --------------------------------------------------------------------------
# solver
# --------------------------------------------------------------------------

class Solver:
    """Algorithm 1 on one problem.

    ``cost`` is a tensor of multi-degree P; ``ineq`` is an array of shape
    (alpha, G+1...) and ``eq`` of shape (beta, H+1...), each family at one
    common multi-degree.  ``form`` is "monomial" (coefficients of x over the
    box, converted here) or "bernstein" (root patches over the box)."""

    def __init__(self, cost, ineq, eq, lo, hi, form="monomial", max_items=1 << 40):
        lib = _load()
        cost = _f64(cost)
        l = cost.ndim
        self.l = l
        self._keep = []
        ineq = _f64(ineq) if ineq is not None and len(ineq) else np.zeros((0,) + (1,) * l)
        eq = _f64(eq) if eq is not None and len(eq) else np.zeros((0,) + (1,) * l)
        self.n_ineq, self.n_eq = ineq.shape[0], eq.shape[0]
        P = _i32(np.array(cost.shape) - 1)
        G = _i32(np.array(ineq.shape[1:]) - 1) if self.n_ineq else _i32([0] * l)
        H = _i32(np.array(eq.shape[1:]) - 1) if self.n_eq else _i32([0] * l)
        lo, hi = _f64(np.broadcast_to(lo, (l,))), _f64(np.broadcast_to(hi, (l,)))
        self._arrs = (cost, ineq, eq, P, G, H, lo, hi)
        self.P, self.G, self.H = P, G, H
        self.lo, self.hi = lo, hi
        h = lib.or_create(l, _ptr(lo), _ptr(hi), _ptr(P), _ptr(cost), self.n_ineq, _ptr(G),
                          _ptr(ineq), self.n_eq, _ptr(H), _ptr(eq),
                          0 if form == "monomial" else 1, int(max_items))
        if not h:
            raise ValueError("or_create rejected the problem")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _load().or_destroy(h)
            self._h = None

    def step(self, opt_tol=1e-3, eq_tol=1e-4, max_iters=28, step_tol=0.0):
        return _load().or_step(self._h, opt_tol, eq_tol, max_iters, step_tol)

    def solve(self, opt_tol=1e-3, eq_tol=1e-4, max_iters=28, step_tol=0.0):
        l = self.l
        out = np.zeros(6 + 3 * l)
        _load().or_solve(self._h, opt_tol, eq_tol, max_iters, step_tol, _ptr(out))
        return {
            "status": int(out[0]), "lower": out[1], "upper": out[2],
            "steps": int(out[3]), "sweeps": int(out[4]), "peak_items": int(out[5]),
            "x": out[6:6 + l].copy(), "box_lo": out[6 + l:6 + 2 * l].copy(),
            "box_hi": out[6 + 2 * l:6 + 3 * l].copy(),
        }

    @property
    def status(self):
        return _load().or_status(self._h)

    def list_length(self):
        return int(_load().or_list_length(self._h))

    def item_len(self):
        return int(_load().or_item_len(self._h))

    def get_list(self):
        """Current list: dict with 'cost' (K, P+1...), 'ineq' (K, alpha, G+1...),
        'eq' (K, beta, H+1...), 'index' (K, l) uint32 and 'level' (l,)."""
        lib = _load()
        K, L = self.list_length(), self.item_len()
        flat = np.empty((K, L))
        idx = np.empty((K, self.l), dtype=np.uint32)
        lev = np.empty(self.l, dtype=np.int32)
        lib.or_get_list(self._h, _ptr(flat), _ptr(idx), _ptr(lev))
        cp = int(np.prod(self.P + 1))
        cg = int(np.prod(self.G + 1)) if self.n_ineq else 0
        ch = int(np.prod(self.H + 1)) if self.n_eq else 0
        out = {"cost": flat[:, :cp].reshape((K,) + tuple(self.P + 1)),
               "index": idx, "level": lev}
        o = cp
        out["ineq"] = flat[:, o:o + self.n_ineq * cg].reshape(
            (K, self.n_ineq) + tuple(self.G + 1))
        o += self.n_ineq * cg
        out["eq"] = flat[:, o:o + self.n_eq * ch].reshape((K, self.n_eq) + tuple(self.H + 1))
        return out

    def get_keep(self, count):
        buf = np.empty(count, dtype=np.uint8)
        _load().or_get_keep(self._h, _ptr(buf), count)
        return buf

    def trace(self):
        """One row per step: (K before subdivision, K_save, p_up, p_lo)."""
        n = int(_load().or_trace_length(self._h))
        rows = np.empty((n, 4))
        if n:
            _load().or_get_trace(self._h, _ptr(rows))
        return rows


def solve(cost, ineq=None, eq=None, lo=-1.0, hi=1.0, opt_tol=1e-3, eq_tol=1e-4,
          max_iters=28, max_items=1 << 40, form="monomial", step_tol=0.0):
    """Convenience: build a Solver and run Algorithm 1 to the end."""
    s = Solver(cost, ineq, eq, lo, hi, form=form, max_items=max_items)
    res = s.solve(opt_tol=opt_tol, eq_tol=eq_tol, max_iters=max_iters, step_tol=step_tol)
    res["trace"] = s.trace()
    return res
