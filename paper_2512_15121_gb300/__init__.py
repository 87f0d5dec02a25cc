"""Python binding of the GB300 GIAMG solver (C ABI in include/giamg.h, libgiamg.so).

Argument marshalling only: every step of setup and solve runs in the library's CUDA kernels.
The functions keep the C names (giamg_setup, giamg_solve, ...); `Solver` wraps a handle.
Vectors are numpy arrays (host mode, device_ptrs = 0) or CUDA torch tensors (device mode,
device_ptrs = 1); PyTorch only supplies device memory and the stream.

Importing succeeds without the shared library (so the CPU test suite can inspect the
package); every call raises RuntimeError until `build()` has produced libgiamg.so.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgiamg.so")

GIAMG_OK, GIAMG_ERR_ARG, GIAMG_ERR_ORDER, GIAMG_ERR_MAP, GIAMG_ERR_OOM = 0, -1, -2, -3, -4
GIAMG_ERR_CUDA, GIAMG_ERR_NOT_SPD, GIAMG_ERR_BREAKDOWN, GIAMG_ERR_MAXITER, GIAMG_ERR_TIMEOUT = -5, -6, -7, -8, -9
GIAMG_LEVEL_P, GIAMG_LEVEL_H, GIAMG_LEVEL_COARSEST = 0, 1, 2

# every entry point the header declares (checked by the CPU tests against the .so)
EXPORTS = ["giamg_default_options", "giamg_setup", "giamg_solve", "giamg_solve_ex", "giamg_solve_stats",
           "giamg_solve_async", "giamg_solve_batch", "giamg_solve_batch_ex", "giamg_solve_block", "giamg_solve_grouped",
           "giamg_num_levels", "giamg_level_info", "giamg_level_templates", "giamg_level_kernel", "giamg_export_level", "giamg_export_prolongation",
           "giamg_level_rho", "giamg_set_cheb_degree", "giamg_set_row_kernel", "giamg_set_batch_rows", "giamg_apply_vcycle", "giamg_level_spmv", "giamg_level_spmv32", "giamg_level_smooth",
           "giamg_level_restrict", "giamg_level_prolong", "giamg_coarse_solve", "giamg_level_residual",
           "giamg_level_residual32", "giamg_level_smooth32", "giamg_level_restrict32", "giamg_level_prolong32",
           "giamg_coarse_solve32", "giamg_free",
           "giamg_last_error", "giamg_set_device_ptrs", "giamg_profile_enable", "giamg_profile_read",
           "giamg_launch_count", "giamg_true_relres_noalloc"]


class GiamgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("cheb_degree", ctypes.c_int), ("cheb_lo", ctypes.c_double), ("cheb_hi", ctypes.c_double),
                ("lanczos_steps", ctypes.c_int), ("coarse_max", ctypes.c_int), ("max_levels", ctypes.c_int),
                ("strength_theta", ctypes.c_double), ("precision", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("force_iters", ctypes.c_int), ("device_ptrs", ctypes.c_int), ("hash_kind", ctypes.c_int),
                ("compress_patterns", ctypes.c_int), ("autotune", ctypes.c_int), ("row_form", ctypes.c_int),
                ("row_threads", ctypes.c_int), ("prefetch_rows", ctypes.c_int), ("row_chains", ctypes.c_int),
                ("graphs", ctypes.c_int), ("p_schedule", ctypes.c_int), ("basis", ctypes.c_int)]


_lib = None


def build(force: bool = False, verbose: bool = False) -> str:
    from . import nvcc_build
    return nvcc_build.build(force=force, verbose=verbose)


def lib():
    """Load libgiamg.so; raise if it is missing (there is no fallback implementation)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgiamg.so not built ({LIB_PATH}); run paper_2512_15121_gb300.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        P = ctypes.POINTER
        L.giamg_default_options.argtypes = [P(Options)]
        L.giamg_default_options.restype = None
        L.giamg_setup.argtypes = [i64, vp, vp, vp, ctypes.c_int32, vp, vp, vp, P(Options), vp, P(vp)]
        L.giamg_solve.argtypes = [vp, vp, vp, dbl, P(i32), P(dbl)]
        L.giamg_solve_ex.argtypes = [vp, i32, i32, vp, vp, dbl, P(i32), P(dbl)]
        L.giamg_solve_stats.argtypes = [vp, vp, i32, P(dbl)]
        L.giamg_solve_batch.argtypes = [vp, i32, vp, vp, dbl, vp, vp]
        L.giamg_solve_batch_ex.argtypes = [vp, i32, i32, i32, vp, vp, dbl, vp, vp]
        L.giamg_solve_block.argtypes = [vp, i32, i32, i32, vp, vp, dbl, vp, vp]
        L.giamg_solve_async.argtypes = [vp, i32, vp, vp, dbl, vp, vp, vp]
        L.giamg_solve_grouped.argtypes = [i32, vp, vp, vp, vp, dbl, vp, vp, vp]
        L.giamg_num_levels.argtypes = [vp, P(i32)]
        L.giamg_level_info.argtypes = [vp, i32, P(i32), P(i64), P(i64), P(i32), P(i64), P(i64)]
        L.giamg_export_level.argtypes = [vp, i32, vp, vp, vp, vp]
        L.giamg_export_prolongation.argtypes = [vp, i32, vp, vp, vp]
        L.giamg_level_rho.argtypes = [vp, i32, P(dbl)]
        L.giamg_level_templates.argtypes = [vp, i32, P(i64), P(i64)]
        L.giamg_level_kernel.argtypes = [vp, i32, i32, P(i32), P(i32)]
        L.giamg_set_row_kernel.argtypes = [vp, i32, i32, i32, i32]
        L.giamg_set_batch_rows.argtypes = [vp, i32, i32]
        L.giamg_apply_vcycle.argtypes = [vp, i32, vp, vp]
        L.giamg_level_spmv.argtypes = [vp, i32, vp, vp]
        L.giamg_level_smooth.argtypes = [vp, i32, vp, vp, i32]
        L.giamg_level_restrict.argtypes = [vp, i32, vp, vp]
        L.giamg_level_prolong.argtypes = [vp, i32, vp, vp]
        L.giamg_coarse_solve.argtypes = [vp, vp, vp]
        L.giamg_level_residual.argtypes = [vp, i32, vp, vp, vp]
        L.giamg_level_residual32.argtypes = [vp, i32, vp, vp, vp]
        L.giamg_level_smooth32.argtypes = [vp, i32, vp, vp, i32]
        L.giamg_level_restrict32.argtypes = [vp, i32, vp, vp]
        L.giamg_level_prolong32.argtypes = [vp, i32, vp, vp]
        L.giamg_coarse_solve32.argtypes = [vp, vp, vp]
        L.giamg_free.argtypes = [vp]
        L.giamg_set_device_ptrs.argtypes = [vp, i32]
        L.giamg_profile_enable.argtypes = [vp, i32]
        L.giamg_profile_read.argtypes = [vp, i32, P(dbl), P(i64), P(dbl)]
        L.giamg_launch_count.argtypes = [P(i64)]
        L.giamg_true_relres_noalloc.argtypes = [vp, vp, vp, P(dbl)]
        L.giamg_last_error.argtypes = []
        L.giamg_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(rc: int):
    if rc != GIAMG_OK:
        raise GiamgError(rc, lib().giamg_last_error().decode())


def _ptr(a):
    """Pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


def default_options(**over) -> Options:
    o = Options()
    lib().giamg_default_options(ctypes.byref(o))
    for k, v in over.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


# ---------------------------------------------------------------- C-named functions
def giamg_setup(n, row_ptr, col_idx, val, n_elem, elem_dof, elem_order, coords=None, options=None, stream=None):
    h = ctypes.c_void_p()
    opt = options if options is not None else default_options()
    _check(lib().giamg_setup(n, _ptr(row_ptr), _ptr(col_idx), _ptr(val), n_elem, _ptr(elem_dof), _ptr(elem_order),
                             _ptr(coords), ctypes.byref(opt), ctypes.c_void_p(stream) if stream else None,
                             ctypes.byref(h)))
    return h


def giamg_solve(h, b, x, rtol):
    it, rr = ctypes.c_int(), ctypes.c_double()
    rc = lib().giamg_solve(h, _ptr(b), _ptr(x), rtol, ctypes.byref(it), ctypes.byref(rr))
    return rc, it.value, rr.value


def giamg_solve_ex(h, precision, force_iters, b, x, rtol):
    it, rr = ctypes.c_int(), ctypes.c_double()
    rc = lib().giamg_solve_ex(h, precision, force_iters, _ptr(b), _ptr(x), rtol, ctypes.byref(it), ctypes.byref(rr))
    return rc, it.value, rr.value


def launch_count() -> int:
    c = ctypes.c_int64()
    _check(lib().giamg_launch_count(ctypes.byref(c)))
    return c.value


def solve_grouped(solvers, Bs, rtol=1e-8, Xs=None):
    """The multi-RHS solves of several hierarchies at once (giamg_solve_grouped): one kernel launch
    per phase for all of them, each with the bits of its own solve_batch (FP32 V-cycle).  solvers:
    Solver objects in device mode on one device; Bs: CUDA float64 tensors n_i x m_i (m_i <= 32).
    Returns [(X, iters, relres, status)] in solver order."""
    import torch
    k = len(solvers)
    if k == 0 or len(Bs) != k:
        raise ValueError("one right-hand-side block per solver is needed")
    Bs = [B.to("cuda", torch.float64).contiguous() for B in Bs]
    for S, B in zip(solvers, Bs):
        if not S.device:
            raise GiamgError(GIAMG_ERR_ARG, "solve_grouped needs device=True solvers")
        if len(B.shape) != 2 or B.shape[0] != S.n or not 1 <= B.shape[1] <= 32:
            raise ValueError(f"B: shape {tuple(B.shape)}, expected ({S.n}, m) with 1 <= m <= 32")
    Xs = [torch.empty_like(B) for B in Bs] if Xs is None else Xs
    for S, B, X in zip(solvers, Bs, Xs):
        S._check_out("X", X, tuple(B.shape))
    ms = np.array([B.shape[1] for B in Bs], np.int32)
    hs = (ctypes.c_void_p * k)(*[S._h.value for S in solvers])
    bp = (ctypes.c_void_p * k)(*[B.data_ptr() for B in Bs])
    xp = (ctypes.c_void_p * k)(*[X.data_ptr() for X in Xs])
    it = np.zeros(int(ms.sum()), np.int32)
    rr = np.zeros(int(ms.sum()), np.float64)
    st = np.zeros(k, np.int32)
    _check(lib().giamg_solve_grouped(k, hs, _ptr(ms), bp, xp, rtol, _ptr(it), _ptr(rr), _ptr(st)))
    out, o = [], 0
    for i in range(k):
        out.append((Xs[i], it[o:o + ms[i]], rr[o:o + ms[i]], int(st[i])))
        o += int(ms[i])
    return out


def giamg_free(h):
    _check(lib().giamg_free(h))


def _check_inputs(n, row_ptr, col, val, elem_dof, p, coords, device):
    """Shapes, lengths and (device mode) dtypes of the setup arrays, checked before the C call:
    the ABI takes plain pointers and cannot see how long a buffer is."""
    if device:
        want = (("row_ptr", row_ptr, "int64"), ("col", col, "int32"), ("val", val, "float64"),
                ("elem_dof", elem_dof, "int32"), ("coords", coords, "float64"))
        for name, a, dt in want:
            if a is None:
                continue
            if not hasattr(a, "is_cuda") or not a.is_cuda:
                raise TypeError(f"{name}: device_ptrs=1 needs a CUDA tensor")
            if str(a.dtype) != "torch." + dt:
                raise TypeError(f"{name}: dtype {a.dtype}, expected torch.{dt}")
            if not a.is_contiguous():
                raise ValueError(f"{name}: not contiguous")
    shape = lambda a: tuple(a.shape)
    if len(shape(row_ptr)) != 1 or shape(row_ptr)[0] != n + 1:
        raise ValueError(f"row_ptr: shape {shape(row_ptr)}, expected ({n + 1},)")
    nnz = int(row_ptr[n])
    for name, a in (("col", col), ("val", val)):
        if len(shape(a)) != 1 or shape(a)[0] < nnz:
            raise ValueError(f"{name}: shape {shape(a)}, expected at least row_ptr[n] = {nnz} entries")
    if elem_dof is not None and (len(shape(elem_dof)) != 2 or shape(elem_dof)[1] != (p + 1) ** 3):
        raise ValueError(f"elem_dof: shape {shape(elem_dof)}, expected (n_elem, {(p + 1) ** 3}) for p = {p}")
    if coords is not None and shape(coords) != (n, 3):
        raise ValueError(f"coords: shape {shape(coords)}, expected ({n}, 3)")


class Solver:
    """A GIAMG hierarchy on the GPU (one handle)."""

    def __init__(self, n, row_ptr, col, val, elem_dof=None, p=1, coords=None, stream=None, **opts):
        self.opts = default_options(**opts)
        self.device = bool(self.opts.device_ptrs)
        self.n = int(n)
        p = int(p)
        if not self.device:
            row_ptr = np.ascontiguousarray(row_ptr, np.int64)
            col = np.ascontiguousarray(col, np.int32)
            val = np.ascontiguousarray(val, np.float64)
            elem_dof = None if elem_dof is None else np.ascontiguousarray(elem_dof, np.int32)
            coords = None if coords is None else np.ascontiguousarray(coords, np.float64)
        if self.n >= 1:
            _check_inputs(self.n, row_ptr, col, val, elem_dof, p, coords, self.device)
        if self.device:
            import torch
            ed = elem_dof
            n_elem = int(ed.shape[0]) if ed is not None else 0
            cur = torch.cuda.current_stream(row_ptr.device)
            order = torch.full((max(n_elem, 1),), p, dtype=torch.int32, device=row_ptr.device)
            if stream is None:
                stream = cur.cuda_stream
            elif int(stream) != int(cur.cuda_stream):
                cur.synchronize()  # inputs written on torch's stream are read on `stream`
        else:
            ed = elem_dof
            n_elem = int(ed.shape[0]) if ed is not None else 0
            order = np.full(max(n_elem, 1), p, np.int32)
        self._h = giamg_setup(self.n, row_ptr, col, val, n_elem, ed, order if n_elem else None, coords,
                              self.opts, stream)

    @classmethod
    def from_problem(cls, prob, device=False, coords=False, **opts):
        if device:
            import torch
            dev = torch.device("cuda", torch.cuda.current_device())
            t = lambda a: torch.from_numpy(a).to(dev)
            return cls(prob.n, t(prob.row_ptr), t(prob.col), t(prob.val), t(prob.elem_dof), prob.p,
                       t(prob.coords) if coords else None, device_ptrs=1, **opts)
        return cls(prob.n, prob.row_ptr, prob.col, prob.val, prob.elem_dof, prob.p,
                   prob.coords if coords else None, **opts)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            giamg_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- allocation helpers
    def _vec(self, n):
        if self.device:
            import torch
            return torch.empty(n, dtype=torch.float64, device="cuda")
        return np.empty(n, np.float64)

    def _in(self, v):
        if self.device:
            import torch
            if not isinstance(v, torch.Tensor):
                v = torch.from_numpy(np.ascontiguousarray(v, np.float64))
            return v.to("cuda", torch.float64).contiguous()
        return np.ascontiguousarray(v, np.float64)

    def _check_shape(self, name, a, shape):
        if tuple(a.shape) != tuple(shape):
            raise ValueError(f"{name}: shape {tuple(a.shape)}, expected {tuple(shape)}")

    def _check_out(self, name, a, shape):
        """A buffer the caller passes for the library to write: the right shape, float64, contiguous,
        and on the device in device mode (the C call only sees a pointer)."""
        self._check_shape(name, a, shape)
        if self.device:
            import torch
            ok = isinstance(a, torch.Tensor) and a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()
        else:
            ok = isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
        if not ok:
            kind = "CUDA tensor" if self.device else "numpy array"
            raise TypeError(f"{name}: expected a contiguous float64 {kind}")

    # -------------------------------------------------------------- solve
    def solve(self, b, rtol=1e-8, precision=None, force_iters=None, x=None):
        """Returns (x, iters, relres); raises GiamgError on failure other than max_iter."""
        b = self._in(b)
        self._check_shape("b", b, (self.n,))
        if x is not None:
            self._check_out("x", x, (self.n,))
        x = self._vec(self.n) if x is None else x
        prec = self.opts.precision if precision is None else precision
        force = self.opts.force_iters if force_iters is None else force_iters
        rc, it, rr = giamg_solve_ex(self._h, prec, force, b, x, rtol)
        if rc not in (GIAMG_OK, GIAMG_ERR_MAXITER):
            _check(rc)
        self.last_status = rc
        return x, it, rr

    def solve_async(self, b, rtol=1e-8, precision=None, x=None):
        """Enqueue a solve on the handle's stream (device mode, graphs on).  Returns device tensors
        (x, iters, relres, status), valid once the stream has passed the solve."""
        import torch
        if not self.device:
            raise GiamgError(GIAMG_ERR_ARG, "solve_async needs device=True")
        b = b.to("cuda", torch.float64).contiguous()
        self._check_shape("b", b, (self.n,))
        if x is not None:
            self._check_out("x", x, (self.n,))
        x = torch.empty_like(b) if x is None else x
        it = torch.zeros(1, dtype=torch.int32, device="cuda")
        rr = torch.zeros(1, dtype=torch.float64, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        prec = self.opts.precision if precision is None else precision
        _check(lib().giamg_solve_async(self._h, prec, _ptr(b), _ptr(x), rtol, _ptr(it), _ptr(rr), _ptr(st)))
        return x, it, rr, st

    def solve_batch(self, B, rtol=1e-8, precision=None, force_iters=None, X=None, block=False):
        """B: n x m (row-major, m <= 32).  Returns (X, iters[m], relres[m]).  block=True: the
        columns as one block in block CG (giamg_solve_block) instead of independent CGs."""
        if len(B.shape) != 2 or B.shape[0] != self.n:
            raise ValueError(f"B: shape {tuple(B.shape)}, expected ({self.n}, m)")
        m = int(B.shape[1])
        if X is not None:
            self._check_out("X", X, (self.n, m))
        if self.device:
            import torch
            B = B.to("cuda", torch.float64).contiguous()
            X = torch.empty_like(B) if X is None else X
        else:
            B = np.ascontiguousarray(B, np.float64)
            X = np.empty_like(B) if X is None else X
        it = np.zeros(m, np.int32)
        rr = np.zeros(m, np.float64)
        prec = self.opts.precision if precision is None else precision
        force = self.opts.force_iters if force_iters is None else force_iters
        fn = lib().giamg_solve_block if block else lib().giamg_solve_batch_ex
        rc = fn(self._h, prec, force, m, _ptr(B), _ptr(X), rtol, _ptr(it), _ptr(rr))
        if rc not in (GIAMG_OK, GIAMG_ERR_MAXITER):
            _check(rc)
        self.last_status = rc
        return X, it, rr

    def solve_block(self, B, rtol=1e-8, precision=None, force_iters=None, X=None):
        """Block CG on the columns of B (n x m, m <= 32).  Returns (X, iters[m], relres[m])."""
        return self.solve_batch(B, rtol=rtol, precision=precision, force_iters=force_iters, X=X, block=True)

    def true_relres_noalloc(self, b, x):
        """||b - A x|| / ||b|| on the finest level through giamg_true_relres_noalloc, which allocates
        no device memory.  b and x: contiguous float64 CUDA tensors of length n on the handle's
        device (whatever the handle's pointer mode)."""
        import torch
        for name, a in (("b", b), ("x", x)):
            if not isinstance(a, torch.Tensor) or not a.is_cuda:
                raise TypeError(f"{name}: giamg_true_relres_noalloc needs a CUDA tensor")
            if a.dtype != torch.float64 or not a.is_contiguous():
                raise TypeError(f"{name}: expected a contiguous float64 CUDA tensor")
            self._check_shape(name, a, (self.n,))
        out = ctypes.c_double()
        _check(lib().giamg_true_relres_noalloc(self._h, _ptr(b), _ptr(x), ctypes.byref(out)))
        return out.value

    def stats(self, hist_len=0):
        hist = np.zeros(max(hist_len, 1))
        tr = ctypes.c_double()
        _check(lib().giamg_solve_stats(self._h, _ptr(hist), hist_len, ctypes.byref(tr)))
        return hist[:hist_len], tr.value

    # -------------------------------------------------------------- profiling
    def set_device_ptrs(self, on: bool):
        _check(lib().giamg_set_device_ptrs(self._h, 1 if on else 0))
        self.device = bool(on)

    def profile(self, enable: bool):
        _check(lib().giamg_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self, category: int):
        ms, cnt, by = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        _check(lib().giamg_profile_read(self._h, category, ctypes.byref(ms), ctypes.byref(cnt), ctypes.byref(by)))
        return ms.value, cnt.value, by.value

    # -------------------------------------------------------------- hierarchy
    @property
    def num_levels(self):
        k = ctypes.c_int()
        _check(lib().giamg_num_levels(self._h, ctypes.byref(k)))
        return k.value

    def level_info(self, l):
        k, o = ctypes.c_int(), ctypes.c_int()
        n, nnz, pn, nn = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().giamg_level_info(self._h, l, ctypes.byref(k), ctypes.byref(n), ctypes.byref(nnz),
                                      ctypes.byref(o), ctypes.byref(pn), ctypes.byref(nn)))
        return dict(kind=k.value, n=n.value, nnz=nnz.value, order=o.value, p_nnz=pn.value, n_next=nn.value)

    def _arrays(self, shapes):
        if self.device:
            import torch
            td = {np.int64: torch.int64, np.int32: torch.int32, np.float64: torch.float64}
            return [torch.empty(max(s, 1), dtype=td[d], device="cuda") for s, d in shapes]
        return [np.empty(max(s, 1), d) for s, d in shapes]

    def _host(self, a, n):
        if self.device:
            return a[:n].cpu().numpy()
        return a[:n]

    def level(self, l):
        info = self.level_info(l)
        rp, ci, v, agg = self._arrays([(info["n"] + 1, np.int64), (info["nnz"], np.int32), (info["nnz"], np.float64),
                                       (info["n"], np.int32)])
        want_agg = info["kind"] == GIAMG_LEVEL_H
        _check(lib().giamg_export_level(self._h, l, _ptr(rp), _ptr(ci), _ptr(v), _ptr(agg) if want_agg else None))
        return (self._host(rp, info["n"] + 1), self._host(ci, info["nnz"]), self._host(v, info["nnz"]),
                self._host(agg, info["n"]) if want_agg else None)

    def prolongation(self, l):
        info = self.level_info(l)
        rp, ci, v = self._arrays([(info["n"] + 1, np.int64), (info["p_nnz"], np.int32), (info["p_nnz"], np.float64)])
        _check(lib().giamg_export_prolongation(self._h, l, _ptr(rp), _ptr(ci), _ptr(v)))
        return (self._host(rp, info["n"] + 1), self._host(ci, info["p_nnz"]), self._host(v, info["p_nnz"]),
                info["n_next"])

    def templates(self, l):
        t, o = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().giamg_level_templates(self._h, l, ctypes.byref(t), ctypes.byref(o)))
        return t.value, o.value

    def kernel(self, l, precision):
        t, p = ctypes.c_int(), ctypes.c_int()
        _check(lib().giamg_level_kernel(self._h, l, precision, ctypes.byref(t), ctypes.byref(p)))
        return t.value, ["csr", "pattern", "groups", "hybrid", "vector", "sliced"][p.value]

    def set_cheb_degree(self, k: int):
        """Smoother degree k on every level, keeping the hierarchy (giamg_set_cheb_degree)."""
        _check(lib().giamg_set_cheb_degree(self._h, int(k)))
        self.opts.cheb_degree = int(k)

    def set_row_kernel(self, l, precision, form, threads=0):
        """Switch level l's row kernel for precision 0/1 (form as the row_form option)."""
        _check(lib().giamg_set_row_kernel(self._h, int(l), int(precision), int(form), int(threads)))

    def set_batch_rows(self, l, rows_per_item):
        """Rows per work item of level l's multi-RHS FP32 products (0 automatic, 1, 2)."""
        _check(lib().giamg_set_batch_rows(self._h, int(l), int(rows_per_item)))

    def rho_hat(self, l):
        r = ctypes.c_double()
        _check(lib().giamg_level_rho(self._h, l, ctypes.byref(r)))
        return r.value

    # -------------------------------------------------------------- single steps
    def vcycle(self, r, precision=0):
        r = self._in(r)
        self._check_shape("r", r, (self.n,))
        z = self._vec(self.n)
        _check(lib().giamg_apply_vcycle(self._h, precision, _ptr(r), _ptr(z)))
        return z

    def spmv(self, l, x):
        x = self._in(x)
        self._check_shape("x", x, (self.level_info(l)["n"],))
        y = self._vec(self.level_info(l)["n"])
        _check(lib().giamg_level_spmv(self._h, l, _ptr(x), _ptr(y)))
        return y

    def spmv32(self, l, x):
        """y = A_l x in FP32 (the FP32 V-cycle's product)."""
        if self.device:
            import torch
            x = (x if isinstance(x, torch.Tensor) else torch.from_numpy(np.asarray(x))).to("cuda", torch.float32).contiguous()
            y = torch.empty(self.level_info(l)["n"], dtype=torch.float32, device="cuda")
        else:
            x = np.ascontiguousarray(x, np.float32)
            y = np.empty(self.level_info(l)["n"], np.float32)
        self._check_shape("x", x, tuple(y.shape))
        _check(lib().giamg_level_spmv32(self._h, l, _ptr(x), _ptr(y)))
        return y

    def smooth(self, l, b, x=None):
        b = self._in(b)
        self._check_shape("b", b, (self.level_info(l)["n"],))
        if x is not None:
            self._check_shape("x", x, (self.level_info(l)["n"],))
        xo = self._vec(self.level_info(l)["n"]) if x is None else self._in(x).clone() if self.device else self._in(x).copy()
        _check(lib().giamg_level_smooth(self._h, l, _ptr(b), _ptr(xo), 1 if x is None else 0))
        return xo

    def restrict(self, l, rf):
        rf = self._in(rf)
        self._check_shape("rf", rf, (self.level_info(l)["n"],))
        rc = self._vec(self.level_info(l)["n_next"])
        _check(lib().giamg_level_restrict(self._h, l, _ptr(rf), _ptr(rc)))
        return rc

    def prolong(self, l, ec, xf):
        ec = self._in(ec)
        info = self.level_info(l)
        self._check_shape("ec", ec, (info["n_next"],))
        self._check_shape("xf", xf, (info["n"],))
        xo = self._in(xf).clone() if self.device else self._in(xf).copy()
        _check(lib().giamg_level_prolong(self._h, l, _ptr(ec), _ptr(xo)))
        return xo

    def residual(self, l, b, x):
        """r = b - A_l x (FP64)."""
        n = self.level_info(l)["n"]
        b, x = self._in(b), self._in(x)
        self._check_shape("b", b, (n,))
        self._check_shape("x", x, (n,))
        r = self._vec(n)
        _check(lib().giamg_level_residual(self._h, l, _ptr(b), _ptr(x), _ptr(r)))
        return r

    # ---- single steps of the FP32 V-cycle (float32 vectors)
    def _in32(self, v):
        if self.device:
            import torch
            if not isinstance(v, torch.Tensor):
                v = torch.from_numpy(np.ascontiguousarray(v))
            return v.to("cuda", torch.float32).contiguous()
        return np.ascontiguousarray(v, np.float32)

    def _vec32(self, n):
        if self.device:
            import torch
            return torch.empty(n, dtype=torch.float32, device="cuda")
        return np.empty(n, np.float32)

    def _copy32(self, v):
        v = self._in32(v)
        return v.clone() if self.device else v.copy()

    def residual32(self, l, b, x):
        n = self.level_info(l)["n"]
        b, x = self._in32(b), self._in32(x)
        self._check_shape("b", b, (n,))
        self._check_shape("x", x, (n,))
        r = self._vec32(n)
        _check(lib().giamg_level_residual32(self._h, l, _ptr(b), _ptr(x), _ptr(r)))
        return r

    def smooth32(self, l, b, x=None):
        n = self.level_info(l)["n"]
        b = self._in32(b)
        self._check_shape("b", b, (n,))
        xo = self._vec32(n) if x is None else self._copy32(x)
        self._check_shape("x", xo, (n,))
        _check(lib().giamg_level_smooth32(self._h, l, _ptr(b), _ptr(xo), 1 if x is None else 0))
        return xo

    def restrict32(self, l, rf):
        info = self.level_info(l)
        rf = self._in32(rf)
        self._check_shape("rf", rf, (info["n"],))
        rc = self._vec32(info["n_next"])
        _check(lib().giamg_level_restrict32(self._h, l, _ptr(rf), _ptr(rc)))
        return rc

    def prolong32(self, l, ec, xf):
        info = self.level_info(l)
        ec = self._in32(ec)
        self._check_shape("ec", ec, (info["n_next"],))
        xo = self._copy32(xf)
        self._check_shape("xf", xo, (info["n"],))
        _check(lib().giamg_level_prolong32(self._h, l, _ptr(ec), _ptr(xo)))
        return xo

    def coarse_solve32(self, r):
        n = self.level_info(self.num_levels - 1)["n"]
        r = self._in32(r)
        self._check_shape("r", r, (n,))
        x = self._vec32(n)
        _check(lib().giamg_coarse_solve32(self._h, _ptr(r), _ptr(x)))
        return x

    def coarse_solve(self, r):
        r = self._in(r)
        self._check_shape("r", r, (self.level_info(self.num_levels - 1)["n"],))
        x = self._vec(self.level_info(self.num_levels - 1)["n"])
        _check(lib().giamg_coarse_solve(self._h, _ptr(r), _ptr(x)))
        return x
