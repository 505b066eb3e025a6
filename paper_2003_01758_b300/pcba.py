"""Python binding of libpcba.so (include/pcba.h): argument marshalling only.

Every step of a solve runs in the library's CUDA kernels; this module turns
numpy arrays into the C structs of the ABI and back.  It loads the in-tree
``libpcba.so`` and raises if it is missing: there is no fallback.

Tensor convention as in ``workloads``: a polynomial of multi-degree N is a
float64 array of shape N+1; a constraint family is stacked on a leading axis.
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpcba.so")
MAX_DIM = 8

OPTIMAL, INFEASIBLE, MEMCAP, MAXITER, TIMEOUT, STEPLIMIT = 0, 1, 2, 3, 4, 5
FP64, FP32 = 64, 32
STATUS_NAMES = {0: "OPTIMAL", 1: "INFEASIBLE", 2: "MEMCAP", 3: "MAXITER", 4: "TIMEOUT",
                5: "STEPLIMIT"}


class PcbaError(RuntimeError):
    pass


class pcba_poly(ctypes.Structure):
    _fields_ = [("nvars", ctypes.c_int), ("degree", ctypes.POINTER(ctypes.c_int)),
                ("coeff", ctypes.POINTER(ctypes.c_double))]


# numpy image of an array of pcba_poly (x86-64 layout: int, padding, two pointers)
_POLY_DTYPE = np.dtype([("nvars", np.int32), ("pad", np.int32), ("degree", np.uint64),
                        ("coeff", np.uint64)])
assert _POLY_DTYPE.itemsize == ctypes.sizeof(pcba_poly)
assert pcba_poly.degree.offset == 8 and pcba_poly.coeff.offset == 16


class pcba_box(ctypes.Structure):
    _fields_ = [("nvars", ctypes.c_int), ("lo", ctypes.POINTER(ctypes.c_double)),
                ("hi", ctypes.POINTER(ctypes.c_double))]


class pcba_linear_family(ctypes.Structure):
    _fields_ = [("n_shared", ctypes.c_int), ("shared", ctypes.c_void_p),
                ("n_constraints", ctypes.c_int), ("weight", ctypes.POINTER(ctypes.c_double)),
                ("offset", ctypes.POINTER(ctypes.c_double))]


class pcba_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("steps", ctypes.c_int), ("sweeps", ctypes.c_int),
                ("from_warm_start", ctypes.c_int),
                ("lower", ctypes.c_double), ("upper", ctypes.c_double),
                ("x", ctypes.c_double * MAX_DIM), ("box_lo", ctypes.c_double * MAX_DIM),
                ("box_hi", ctypes.c_double * MAX_DIM),
                ("peak_items", ctypes.c_longlong), ("peak_bytes", ctypes.c_longlong),
                ("verify_cost", ctypes.c_double), ("verify_max_g", ctypes.c_double),
                ("verify_max_abs_h", ctypes.c_double), ("time_ms", ctypes.c_double),
                ("upper_err", ctypes.c_double)]


_lib = None


def lib():
    """The loaded libpcba.so (raises PcbaError if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise PcbaError("libpcba.so is not built (run paper_2003_01758_b300/build.py); "
                        "there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    LL = ctypes.c_longlong
    sigs = {
        "pcba_create": ([P, P, P, I, P, I, P, I], I),
        "pcba_create_bernstein": ([P, P, P, I, P, I, P, I], I),
        "pcba_solve": ([P, D, D, I, S, P], I),
        "pcba_solve_steps": ([P, D, D, I, S, I, P], I),
        "pcba_solve_batch": ([P, I, D, D, I, S, P, P], I),
        "pcba_batch_create": ([P, P, I, S, I], I),
        "pcba_batch_solve": ([P, D, D, I, P, P], I),
        "pcba_batch_solve_from_host": ([P, P, D, D, I, P, P], I),
        "pcba_batch_input_doubles": ([P], LL),
        "pcba_batch_trace": ([P, I, P, I], I),
        "pcba_batch_timing": ([P, P, P, P, P], I),
        "pcba_batch_stats": ([P, P, P, P, P], I),
        "pcba_batch_launch_bytes": ([P, P, I], I),
        "pcba_batch_autotune": ([P, D, D, I, P, I, P], I),
        "pcba_batch_config": ([P, P, P, P, P], I),
        "pcba_batch_refresh_stats": ([P, P, P], I),
        "pcba_batch_set_stream": ([P, P], I),
        "pcba_batch_set_time_limit": ([P, D], I),
        "pcba_set_time_limit": ([P, D], I),
        "pcba_eval_points_f32": ([P, I, P, P, I, I, P, P, P], I),
        "pcba_create_linear": ([P, P, P, P, I], I),
        "pcba_get_active": ([P, P, LL], I),
        "pcba_batch_linear_stats": ([P, P, P, P], I),
        "pcba_batch_upload_rows": ([P, P], I),
        "pcba_batch_rows_doubles": ([P], LL),
        "pcba_batch_upload_rows_packed": ([P, P], I),
        "pcba_batch_rows_packed_doubles": ([P], LL),
        "pcba_host_alloc": ([S], P),
        "pcba_host_free": ([P], I),
        "pcba_batch_polish": ([P, D, D, D, I, P], I),
        "pcba_batch_solve_polished": ([P, D, D, D, D, I, P], I),
        "pcba_batch_destroy": ([P], None),
        "pcba_get_list": ([P, P, P, P, P, P, P, P], I),
        "pcba_root_patches": ([P, P, P, P], I),
        "pcba_item_bytes": ([P], LL),
        "pcba_set_stream": ([P, P], I),
        "pcba_set_warm_start": ([P, P], I),
        "pcba_destroy": ([P], None),
        "pcba_bernstein_convert_noalloc": ([P, I, I, P, P, P, P, P], I),
        "pcba_status_string": ([I], ctypes.c_char_p),
        "pcba_last_error": ([], ctypes.c_char_p),
        "pcba_version": ([], I),
        "pcba_batch_solve_guided": ([P, D, D, I, P, I, P, I, P], I),
        "pcba_batch_warm_point": ([P, I, P, P], I),
        "pcba_batch_cost_grid": ([P, I, P, I, I], I),
        "pcba_batch_upload": ([P, P], I),
        "pcba_batch_set_refine_stencil": ([P, I, P, I, I], I),
        "pcba_mlp_kernel_launches": ([P], LL),
        "pcba_mlp_create": ([P, I, I, I, I, ctypes.c_ulonglong], I),
        "pcba_mlp_destroy": ([P], None),
        "pcba_mlp_num_params": ([P], LL),
        "pcba_mlp_set_params": ([P, P, LL], I),
        "pcba_mlp_get_params": ([P, P, LL], I),
        "pcba_mlp_forward": ([P, P, P, I, I, P, P, P], I),
        "pcba_mlp_gradient": ([P, P, P, I, I, P, P, P, P, P], I),
        "pcba_mlp_train_step": ([P, P, P, I, I, P, P, ctypes.c_float, P, P], I),
    }
    for name, (args, res) in sigs.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def exported_symbols():
    """Names the binding expects libpcba.so to export."""
    return ["pcba_create", "pcba_create_bernstein", "pcba_solve", "pcba_solve_steps",
            "pcba_solve_batch", "pcba_batch_create", "pcba_batch_solve",
            "pcba_batch_solve_from_host", "pcba_batch_input_doubles", "pcba_batch_trace",
            "pcba_batch_timing", "pcba_batch_stats", "pcba_batch_launch_bytes",
            "pcba_batch_autotune", "pcba_batch_config", "pcba_batch_refresh_stats", "pcba_batch_set_stream", "pcba_batch_destroy",
            "pcba_batch_polish", "pcba_batch_solve_polished",
            "pcba_get_list", "pcba_root_patches", "pcba_item_bytes", "pcba_set_stream",
            "pcba_set_warm_start", "pcba_destroy", "pcba_status_string", "pcba_last_error",
            "pcba_version", "pcba_bernstein_convert_noalloc", "pcba_batch_solve_guided",
            "pcba_batch_warm_point", "pcba_batch_cost_grid", "pcba_batch_upload", "pcba_batch_set_refine_stencil",
            "pcba_mlp_kernel_launches",
            "pcba_mlp_create", "pcba_mlp_destroy", "pcba_mlp_num_params", "pcba_mlp_set_params",
            "pcba_mlp_get_params", "pcba_mlp_forward", "pcba_mlp_gradient",
            "pcba_mlp_train_step", "pcba_set_time_limit", "pcba_batch_set_time_limit",
            "pcba_eval_points_f32", "pcba_create_linear", "pcba_get_active",
            "pcba_batch_linear_stats", "pcba_batch_upload_rows", "pcba_batch_rows_doubles",
            "pcba_host_alloc", "pcba_host_free", "pcba_batch_upload_rows_packed",
            "pcba_batch_rows_packed_doubles"]


def _check(rc):
    if rc < 0:
        raise PcbaError("%s: %s" % (lib().pcba_status_string(rc).decode(),
                                    lib().pcba_last_error().decode()))
    return rc


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _result_dict(r: pcba_result, l: int) -> dict:
    return {
        "status": r.status, "steps": r.steps, "sweeps": r.sweeps,
        "from_warm_start": bool(r.from_warm_start), "lower": r.lower, "upper": r.upper,
        "x": np.array(r.x[:l]), "box_lo": np.array(r.box_lo[:l]), "box_hi": np.array(r.box_hi[:l]),
        "peak_items": r.peak_items, "peak_bytes": r.peak_bytes, "verify_cost": r.verify_cost,
        "verify_max_g": r.verify_max_g, "verify_max_abs_h": r.verify_max_abs_h,
        "time_ms": r.time_ms, "upper_err": r.upper_err,
    }


class Solver:
    """One problem (pcba_create) and its single-problem solves (pcba_solve)."""

    def __init__(self, cost, ineq=None, eq=None, lo=-1.0, hi=1.0, precision=FP32,
                 form="monomial"):
        cost = np.ascontiguousarray(cost, dtype=np.float64)
        l = cost.ndim
        self.l = l
        ineq = np.zeros((0,) + (1,) * l) if ineq is None else np.ascontiguousarray(ineq, np.float64)
        eq = np.zeros((0,) + (1,) * l) if eq is None else np.ascontiguousarray(eq, np.float64)
        self.n_ineq, self.n_eq = int(ineq.shape[0]), int(eq.shape[0])
        self.precision = precision
        lo = np.ascontiguousarray(np.broadcast_to(lo, (l,)), dtype=np.float64)
        hi = np.ascontiguousarray(np.broadcast_to(hi, (l,)), dtype=np.float64)
        keep = [cost, ineq, eq, lo, hi]

        def poly(a):
            deg = np.ascontiguousarray(np.array(a.shape) - 1, dtype=np.int32)
            a = np.ascontiguousarray(a)
            keep.extend([deg, a])
            return pcba_poly(l, deg.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                             a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))

        def family(a):
            # one pcba_poly record per stacked constraint, built without a Python loop
            deg = np.ascontiguousarray(np.array(a.shape[1:]) - 1, dtype=np.int32)
            n = a.shape[0]
            rec = np.zeros(max(1, n), dtype=_POLY_DTYPE)
            rec["nvars"][:n] = l
            rec["degree"][:n] = deg.ctypes.data
            rec["coeff"][:n] = a.ctypes.data + a.strides[0] * np.arange(n, dtype=np.uint64)
            keep.extend([deg, rec])
            return rec.ctypes.data_as(ctypes.c_void_p)

        c = poly(cost)
        gi = family(ineq)
        hj = family(eq)
        box = pcba_box(l, lo.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       hi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        h = ctypes.c_void_p()
        fn = lib().pcba_create if form == "monomial" else lib().pcba_create_bernstein
        _check(fn(ctypes.byref(h), ctypes.byref(c), gi, self.n_ineq, hj, self.n_eq,
                  ctypes.byref(box), precision))
        self._h = h
        self.P = np.array(cost.shape) - 1
        self.G = np.array(ineq.shape[1:]) - 1 if self.n_ineq else np.zeros(l, int)
        self.H = np.array(eq.shape[1:]) - 1 if self.n_eq else np.zeros(l, int)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().pcba_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def item_bytes(self) -> int:
        return int(lib().pcba_item_bytes(self._h))

    def set_warm_start(self, x):
        if x is None:
            _check(lib().pcba_set_warm_start(self._h, None))
        else:
            x = np.ascontiguousarray(x, dtype=np.float64)
            _check(lib().pcba_set_warm_start(self._h, _p(x)))

    def set_time_limit(self, seconds):
        """pcba_set_time_limit: device-time limit of this handle's solves (0: none)."""
        _check(lib().pcba_set_time_limit(self._h, float(seconds)))

    def solve(self, opt_tol=1e-3, eq_tol=1e-4, max_iters=28, mem_cap=1 << 30, max_steps=0):
        r = pcba_result()
        _check(lib().pcba_solve_steps(self._h, opt_tol, eq_tol, max_iters, mem_cap, max_steps,
                                      ctypes.byref(r)))
        return _result_dict(r, self.l)

    def get_list(self):
        """List of the last solve, in the oracle's layout."""
        K = ctypes.c_longlong()
        lev = np.zeros(MAX_DIM, dtype=np.int32)
        _check(lib().pcba_get_list(self._h, ctypes.byref(K), None, None, None, None, None,
                                   _p(lev)))
        K = K.value
        cp = int(np.prod(self.P + 1))
        cg = int(np.prod(self.G + 1)) if self.n_ineq else 0
        ch = int(np.prod(self.H + 1)) if self.n_eq else 0
        cost = np.empty((K, cp))
        ineq = np.empty((K, self.n_ineq, cg))
        eq = np.empty((K, self.n_eq, ch))
        err = np.empty((K, 1 + self.n_ineq + self.n_eq), dtype=np.float32)
        idx = np.empty((K, self.l), dtype=np.uint32)
        _check(lib().pcba_get_list(self._h, ctypes.byref(ctypes.c_longlong()), _p(cost),
                                   _p(ineq), _p(eq), _p(err), _p(idx), _p(lev)))
        return {"cost": cost.reshape((K,) + tuple(self.P + 1)),
                "ineq": ineq.reshape((K, self.n_ineq) + tuple(self.G + 1)),
                "eq": eq.reshape((K, self.n_eq) + tuple(self.H + 1)),
                "err": err, "index": idx, "level": lev[:self.l].copy()}

    def root_patches(self):
        """FP64 root Bernstein patches computed on the device (Alg. 1 line 1)."""
        cp = int(np.prod(self.P + 1))
        cg = int(np.prod(self.G + 1)) if self.n_ineq else 0
        ch = int(np.prod(self.H + 1)) if self.n_eq else 0
        cost = np.empty(cp)
        ineq = np.empty(max(1, self.n_ineq * cg))
        eq = np.empty(max(1, self.n_eq * ch))
        _check(lib().pcba_root_patches(self._h, _p(cost), _p(ineq), _p(eq)))
        return (cost.reshape(tuple(self.P + 1)),
                ineq[:self.n_ineq * cg].reshape((self.n_ineq,) + tuple(self.G + 1)),
                eq[:self.n_eq * ch].reshape((self.n_eq,) + tuple(self.H + 1)))


class LinearSolver(Solver):
    """A problem whose inequalities are affine in K shared polynomials
    (pcba_create_linear): g_i = offset[i] + sum_m weight[i, m] shared[m].

    shared is an array (K, G+1...) of monomial tensors at one common
    multi-degree, weight (alpha, K), offset (alpha,).  The list's "ineq"
    patches (get_list, root_patches) are the K shared patches."""

    def __init__(self, cost, shared, weight, offset, lo=-1.0, hi=1.0, precision=FP32):
        cost = np.ascontiguousarray(cost, dtype=np.float64)
        shared = np.ascontiguousarray(shared, dtype=np.float64)
        l = cost.ndim
        self.l = l
        K = int(shared.shape[0])
        weight = np.ascontiguousarray(weight, dtype=np.float64).reshape(-1, K)
        offset = np.ascontiguousarray(offset, dtype=np.float64).reshape(-1)
        assert weight.shape[0] == offset.shape[0]
        self.n_ineq, self.n_eq, self.n_lin = K, 0, int(offset.shape[0])
        self.precision = precision
        lo = np.ascontiguousarray(np.broadcast_to(lo, (l,)), dtype=np.float64)
        hi = np.ascontiguousarray(np.broadcast_to(hi, (l,)), dtype=np.float64)
        cdeg = np.ascontiguousarray(np.array(cost.shape) - 1, dtype=np.int32)
        sdeg = np.ascontiguousarray(np.array(shared.shape[1:]) - 1, dtype=np.int32)
        rec = np.zeros(K, dtype=_POLY_DTYPE)
        rec["nvars"] = l
        rec["degree"] = sdeg.ctypes.data
        rec["coeff"] = shared.ctypes.data + shared.strides[0] * np.arange(K, dtype=np.uint64)
        self._keep = [cost, shared, weight, offset, lo, hi, cdeg, sdeg, rec]
        c = pcba_poly(l, cdeg.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                      cost.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        fam = pcba_linear_family(K, rec.ctypes.data_as(ctypes.c_void_p), self.n_lin,
                                 weight.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 offset.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        box = pcba_box(l, lo.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       hi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        h = ctypes.c_void_p()
        _check(lib().pcba_create_linear(ctypes.byref(h), ctypes.byref(c), ctypes.byref(fam),
                                        ctypes.byref(box), precision))
        self._h = h
        self.P = np.array(cost.shape) - 1
        self.G = np.array(shared.shape[1:]) - 1
        self.H = np.zeros(l, int)

    def get_active(self):
        """Activity bits of the last solve's list as a bool array (K, alpha):
        True where constraint i is still undecided (or violated) on item k."""
        words = _check(lib().pcba_get_active(self._h, None, 0))
        K = ctypes.c_longlong()
        _check(lib().pcba_get_list(self._h, ctypes.byref(K), None, None, None, None, None, None))
        K = K.value
        bits = np.zeros(max(1, K * words), dtype=np.uint32)
        _check(lib().pcba_get_active(self._h, _p(bits), bits.size))
        b = np.unpackbits(bits[:K * words].view(np.uint8), bitorder="little").reshape(K, -1)
        return b[:, :self.n_lin].astype(bool)


LIN_STRIDE = 8


def host_empty(n, dtype=np.float64):
    """A 1-D numpy array of n elements in page-locked host memory from
    pcba_host_alloc (freed when the array and its views are gone): the
    buffer for pcba_batch_upload / pcba_batch_upload_rows."""
    dt = np.dtype(dtype)
    nbytes = max(1, int(n) * dt.itemsize)
    ptr = lib().pcba_host_alloc(nbytes)
    if not ptr:
        raise PcbaError(lib().pcba_last_error().decode())
    buf = (ctypes.c_uint8 * nbytes).from_address(ptr)
    weakref.finalize(buf, lib().pcba_host_free, ctypes.c_void_p(ptr))
    return np.frombuffer(buf, dtype=dt, count=int(n))


def linear_rows(problems):
    """Host layout of pcba_batch_upload_rows for workloads problems with a
    linear form: per constraint (offset, weights..., zero padding)."""
    blocks = []
    for prob in problems:
        _, weight, offset = prob.meta["linear"]
        r = np.zeros((offset.shape[0], LIN_STRIDE))
        r[:, 0] = offset
        r[:, 1:1 + weight.shape[1]] = weight
        blocks.append(r.ravel())
    return np.ascontiguousarray(np.concatenate(blocks), dtype=np.float64)


def linear_rows_packed(problems):
    """Host layout of pcba_batch_upload_rows_packed: per constraint (offset,
    weights...), 1 + K doubles."""
    blocks = []
    for prob in problems:
        _, weight, offset = prob.meta["linear"]
        blocks.append(np.column_stack([offset, weight]).ravel())
    return np.ascontiguousarray(np.concatenate(blocks), dtype=np.float64)


def linear_solver_from_problem(prob, precision=FP32):
    """LinearSolver of a workloads problem that carries its linear form
    (meta["linear"] = (shared, weight, offset))."""
    shared, weight, offset = prob.meta["linear"]
    return LinearSolver(prob.cost, shared, weight, offset, prob.lo, prob.hi, precision=precision)


def bernstein_convert_noalloc(d_mono_ptr: int, n_patches: int, degree, lo, hi, d_out_ptr: int,
                              stream_ptr: int = 0):
    """pcba_bernstein_convert_noalloc on caller-owned device buffers (raw
    device pointers, e.g. torch's data_ptr()); queues the work on the stream."""
    degree = np.ascontiguousarray(degree, dtype=np.int32)
    l = degree.size
    lo = np.ascontiguousarray(np.broadcast_to(lo, (l,)), dtype=np.float64)
    hi = np.ascontiguousarray(np.broadcast_to(hi, (l,)), dtype=np.float64)
    _check(lib().pcba_bernstein_convert_noalloc(ctypes.c_void_p(d_mono_ptr), int(n_patches), l,
                                                _p(degree), _p(lo), _p(hi),
                                                ctypes.c_void_p(d_out_ptr),
                                                ctypes.c_void_p(stream_ptr)))


def eval_points_f32(d_coeff_ptr: int, degree, d_points_ptr: int, n_points: int, unrolled: bool,
                    d_val_ptr: int, d_err_ptr: int, stream_ptr: int = 0):
    """pcba_eval_points_f32 on caller-owned device buffers (raw device pointers)."""
    degree = np.ascontiguousarray(degree, dtype=np.int32)
    _check(lib().pcba_eval_points_f32(ctypes.c_void_p(d_coeff_ptr), degree.size, _p(degree),
                                      ctypes.c_void_p(d_points_ptr), int(n_points),
                                      1 if unrolled else 0, ctypes.c_void_p(d_val_ptr),
                                      ctypes.c_void_p(d_err_ptr), ctypes.c_void_p(stream_ptr)))


def solver_from_problem(prob, precision=FP32):
    return Solver(prob.cost, prob.ineq, prob.eq, prob.lo, prob.hi, precision=precision)


class Batch:
    """A reusable batch of problems solved together (pcba_batch_*)."""

    GRAPH, HOST_LOOP, INSTRUMENT, NO_TMA, VERTEX = 0, 1, 3, 4, 8

    def __init__(self, solvers, mem_cap_total, flags=0):
        self.solvers = list(solvers)
        self.n = len(self.solvers)
        arr = (ctypes.c_void_p * self.n)(*[s.handle for s in self.solvers])
        b = ctypes.c_void_p()
        _check(lib().pcba_batch_create(ctypes.byref(b), arr, self.n, int(mem_cap_total), flags))
        self._b = b
        self._results = (pcba_result * self.n)()

    def close(self):
        if getattr(self, "_b", None):
            lib().pcba_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _warm(self, warm):
        if warm is None:
            return None
        w = np.full((self.n, MAX_DIM), np.nan)
        for k, x in enumerate(warm):
            if x is not None:
                w[k, :len(x)] = x
        return w

    def solve(self, opt_tol=1e-3, eq_tol=1e-4, max_iters=28, warm=None, raw=False):
        w = self._warm(warm)
        _check(lib().pcba_batch_solve(self._b, opt_tol, eq_tol, max_iters,
                                      None if w is None else _p(w), self._results))
        if raw:
            return self._results
        return [_result_dict(self._results[k], self.solvers[k].l) for k in range(self.n)]

    def solve_guided(self, guess_ptr: int, guess_dim: int, stencil, opt_tol=1e-3, eq_tol=1e-4,
                     max_iters=28, raw=False):
        """pcba_batch_solve_guided: guess_ptr is a device pointer to [n][guess_dim]
        float32 normalised guesses; stencil a [n_stencil][guess_dim] array."""
        st = np.ascontiguousarray(stencil, dtype=np.float64).reshape(-1, guess_dim)
        _check(lib().pcba_batch_solve_guided(self._b, opt_tol, eq_tol, max_iters,
                                             ctypes.c_void_p(guess_ptr), guess_dim, _p(st),
                                             st.shape[0], self._results))
        if raw:
            return self._results
        return [_result_dict(self._results[k], self.solvers[k].l) for k in range(self.n)]

    def warm_point(self, k, with_cost=False):
        """The certified-feasible seed of problem k in the last solve (its point,
        and its certified cost bound if with_cost), or None."""
        x = np.empty(MAX_DIM)
        c = ctypes.c_double()
        if _check(lib().pcba_batch_warm_point(self._b, k, _p(x), ctypes.byref(c))) == 0:
            return None
        return (x[:self.solvers[k].l].copy(), c.value) if with_cost else x[:self.solvers[k].l].copy()

    def polish(self, mu0=1e-2, gap=1e-4, eq_tol=1e-4, iters=30):
        """pcba_batch_polish: the locally polished point of every problem's last
        solve (None where there is none), as a list of arrays."""
        x = np.empty((self.n, MAX_DIM))
        _check(lib().pcba_batch_polish(self._b, mu0, gap, eq_tol, iters, _p(x)))
        return [None if not np.all(np.isfinite(x[k, :self.solvers[k].l]))
                else x[k, :self.solvers[k].l].copy() for k in range(self.n)]

    def solve_polished(self, opt_tol=1e-3, eq_tol=1e-4, relax_opt_tol=3e-2, relax_eq_tol=1e-1,
                       max_iters=28, raw=False):
        """pcba_batch_solve_polished: a solve at (relax_opt_tol, relax_eq_tol),
        the polish of its points, then the certified solve at (opt_tol, eq_tol)
        seeded with them."""
        _check(lib().pcba_batch_solve_polished(self._b, opt_tol, eq_tol, relax_opt_tol,
                                               relax_eq_tol, max_iters, self._results))
        if raw:
            return self._results
        return [_result_dict(self._results[k], self.solvers[k].l) for k in range(self.n)]

    def set_refine_stencil(self, stencil, guess_dim=2, round=0):
        """pcba_batch_set_refine_stencil for one round (None or an empty array
        removes this round and the later ones)."""
        if stencil is None or len(stencil) == 0:
            _check(lib().pcba_batch_set_refine_stencil(self._b, round, None, 0, guess_dim))
            return
        st = np.ascontiguousarray(stencil, dtype=np.float64).reshape(-1, guess_dim)
        _check(lib().pcba_batch_set_refine_stencil(self._b, round, _p(st), st.shape[0],
                                                   guess_dim))

    def set_refine_stencils(self, stencils, guess_dim=2):
        """All refinement rounds at once (an empty list: none)."""
        self.set_refine_stencil(None, guess_dim, 0)
        for r, st in enumerate(stencils):
            self.set_refine_stencil(st, guess_dim, r)

    def upload(self, host_coeffs):
        """pcba_batch_upload: queue the host->device copy of all coefficients."""
        assert host_coeffs.dtype == np.float64 and host_coeffs.size == self.input_doubles()
        _check(lib().pcba_batch_upload(self._b, _p(host_coeffs)))

    def upload_rows(self, host_rows):
        """pcba_batch_upload_rows: queue the host->device copy of the linear
        constraint rows (see linear_rows)."""
        assert host_rows.dtype == np.float64 and host_rows.size == self.rows_doubles()
        _check(lib().pcba_batch_upload_rows(self._b, _p(host_rows)))

    def upload_rows_packed(self, host_rows):
        """pcba_batch_upload_rows_packed: the rows without padding (see
        linear_rows_packed)."""
        assert host_rows.dtype == np.float64 and host_rows.size == self.rows_packed_doubles()
        _check(lib().pcba_batch_upload_rows_packed(self._b, _p(host_rows)))

    def rows_packed_doubles(self) -> int:
        return int(lib().pcba_batch_rows_packed_doubles(self._b))

    def rows_doubles(self) -> int:
        return int(lib().pcba_batch_rows_doubles(self._b))

    def cost_grid(self, G, out_ptr, ld, col0=0):
        """pcba_batch_cost_grid into a device float buffer (queued on the batch stream)."""
        _check(lib().pcba_batch_cost_grid(self._b, G, ctypes.c_void_p(out_ptr), ld, col0))

    def input_doubles(self) -> int:
        return int(lib().pcba_batch_input_doubles(self._b))

    def solve_from_host(self, host_coeffs, opt_tol=1e-3, eq_tol=1e-4, max_iters=28, warm=None,
                        raw=False):
        assert host_coeffs.dtype == np.float64 and host_coeffs.size == self.input_doubles()
        w = self._warm(warm)
        _check(lib().pcba_batch_solve_from_host(self._b, _p(host_coeffs), opt_tol, eq_tol,
                                                max_iters, None if w is None else _p(w),
                                                self._results))
        if raw:
            return self._results
        return [_result_dict(self._results[k], self.solvers[k].l) for k in range(self.n)]

    def trace(self, k, max_rows=4096):
        rows = np.empty((max_rows, 4))
        n = _check(lib().pcba_batch_trace(self._b, k, _p(rows), max_rows))
        return rows[:n].copy()

    def timing(self):
        t, s, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong()
        _check(lib().pcba_batch_timing(self._b, ctypes.byref(t), ctypes.byref(s), ctypes.byref(b),
                                       ctypes.byref(n)))
        return {"total_ms": t.value, "subdiv_ms": s.value, "subdiv_bytes": b.value,
                "subdiv_launches": n.value}

    def stats(self):
        it, kl, hd, dh = (ctypes.c_longlong() for _ in range(4))
        _check(lib().pcba_batch_stats(self._b, ctypes.byref(it), ctypes.byref(kl),
                                      ctypes.byref(hd), ctypes.byref(dh)))
        return {"loop_iters": it.value, "kernel_launches": kl.value, "h2d_bytes": hd.value,
                "d2h_bytes": dh.value}

    def autotune(self, opt_tol=1e-3, eq_tol=1e-4, max_iters=28):
        """Times every subdivision configuration on this batch, keeps the fastest."""
        ms = np.full(16, np.nan)
        chosen = ctypes.c_int()
        n = _check(lib().pcba_batch_autotune(self._b, opt_tol, eq_tol, max_iters, _p(ms), 16,
                                             ctypes.byref(chosen)))
        return {"chosen": chosen.value, "ms_per_config": ms[:n].tolist(), "config": self.config()}

    def config(self):
        t, w, s, g = (ctypes.c_int() for _ in range(4))
        idx = _check(lib().pcba_batch_config(self._b, ctypes.byref(t), ctypes.byref(w),
                                             ctypes.byref(s), ctypes.byref(g)))
        return {"index": idx, "tma": bool(t.value), "warps_per_block": w.value,
                "stages": s.value, "grid": g.value}

    def launch_bytes(self, max_launches=4096):
        out = np.empty(max_launches)
        n = _check(lib().pcba_batch_launch_bytes(self._b, _p(out), max_launches))
        return out[:n].copy()

    def refresh_stats(self):
        m, r = ctypes.c_longlong(), ctypes.c_longlong()
        _check(lib().pcba_batch_refresh_stats(self._b, ctypes.byref(m), ctypes.byref(r)))
        return {"marked": m.value, "refreshed": r.value}

    def linear_stats(self):
        """pcba_batch_linear_stats of the last solve."""
        a, f, c = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(lib().pcba_batch_linear_stats(self._b, ctypes.byref(a), ctypes.byref(f),
                                             ctypes.byref(c)))
        return {"pairs": a.value, "full": f.value, "coeffs": c.value}

    def set_stream(self, stream_ptr: int):
        _check(lib().pcba_batch_set_stream(self._b, ctypes.c_void_p(stream_ptr)))

    def set_time_limit(self, seconds):
        """pcba_batch_set_time_limit: device-time limit of every solve (0: none)."""
        _check(lib().pcba_batch_set_time_limit(self._b, float(seconds)))


def solve_batch(solvers, opt_tol=1e-3, eq_tol=1e-4, max_iters=28, mem_cap_total=1 << 32,
                warm=None):
    b = Batch(solvers, mem_cap_total)
    try:
        return b.solve(opt_tol, eq_tol, max_iters, warm)
    finally:
        b.close()


class Mlp:
    """The warm-start set-encoder network (pcba_mlp_*, include/pcba_warmstart.h).

    Batch inputs are device pointers (e.g. torch CUDA tensors' data_ptr()):
    points [P][point_dim] float32, offsets [B+1] int32, glob [B][global_dim]
    float32, target / out [B][2] float32."""

    BF16, FP32 = 16, 32

    def __init__(self, point_dim=2, global_dim=34, hidden=128, precision=16, seed=0):
        m = ctypes.c_void_p()
        _check(lib().pcba_mlp_create(ctypes.byref(m), point_dim, global_dim, hidden, precision,
                                     seed))
        self._m = m
        self.dims = (point_dim, global_dim, hidden, 2)
        self.n_params = int(lib().pcba_mlp_num_params(m))

    def close(self):
        if getattr(self, "_m", None):
            lib().pcba_mlp_destroy(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def kernel_launches(self):
        return int(lib().pcba_mlp_kernel_launches(self._m))

    def get_params(self):
        out = np.empty(self.n_params, dtype=np.float32)
        _check(lib().pcba_mlp_get_params(self._m, _p(out), self.n_params))
        return out

    def set_params(self, theta):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        assert t.size == self.n_params
        _check(lib().pcba_mlp_set_params(self._m, _p(t), self.n_params))

    def forward(self, points, offsets, n_sets, n_points, glob, out, stream=0):
        _check(lib().pcba_mlp_forward(self._m, ctypes.c_void_p(points), ctypes.c_void_p(offsets),
                                      n_sets, n_points, ctypes.c_void_p(glob),
                                      ctypes.c_void_p(out), ctypes.c_void_p(stream)))

    def gradient(self, points, offsets, n_sets, n_points, glob, target, stream=0):
        g = np.empty(self.n_params, dtype=np.float32)
        loss = ctypes.c_float()
        _check(lib().pcba_mlp_gradient(self._m, ctypes.c_void_p(points), ctypes.c_void_p(offsets),
                                       n_sets, n_points, ctypes.c_void_p(glob),
                                       ctypes.c_void_p(target), _p(g), ctypes.byref(loss),
                                       ctypes.c_void_p(stream)))
        return g, loss.value

    def train_step(self, points, offsets, n_sets, n_points, glob, target, lr, want_loss=True,
                   stream=0):
        loss = ctypes.c_float()
        _check(lib().pcba_mlp_train_step(self._m, ctypes.c_void_p(points),
                                         ctypes.c_void_p(offsets), n_sets, n_points,
                                         ctypes.c_void_p(glob), ctypes.c_void_p(target),
                                         ctypes.c_float(lr),
                                         ctypes.byref(loss) if want_loss else None,
                                         ctypes.c_void_p(stream)))
        return loss.value if want_loss else None
