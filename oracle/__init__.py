"""CPU oracle of GIAMG-preconditioned CG: plain FP64 C (oracle.c) behind ctypes, and block PCG
for several right-hand sides in numpy (block_cg.py).

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  The CUDA library (`paper_2512_15121_gb300`) never imports
it and shares no source with it.

The C source is compiled on first use if the shared library is missing or stale.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "oracle.h")]
_lock = threading.Lock()
_L = None

KIND_P, KIND_H, KIND_COARSEST = 0, 1, 2
STATUS = {0: "ok", -1: "arg", -2: "order", -3: "map", -4: "oom", -6: "not_spd", -7: "breakdown",
          -8: "maxiter"}


def build(force: bool = False) -> str:
    stale = force or not os.path.exists(_SO) or any(
        os.path.getmtime(s) > os.path.getmtime(_SO) for s in _SRC)
    if not stale:
        return _SO
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-o", _SO + ".tmp",
            os.path.join(_HERE, "oracle.c"), "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


class Options(ctypes.Structure):
    _fields_ = [("cheb_degree", ctypes.c_int), ("cheb_lo", ctypes.c_double),
                ("cheb_hi", ctypes.c_double), ("lanczos_steps", ctypes.c_int),
                ("coarse_max", ctypes.c_int), ("max_levels", ctypes.c_int),
                ("strength_theta", ctypes.c_double), ("hash_kind", ctypes.c_int), ("p_schedule", ctypes.c_int),
                ("basis", ctypes.c_int)]


class _CSR(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("rp", ctypes.c_void_p),
                ("ci", ctypes.c_void_p), ("v", ctypes.c_void_p)]


def _lib():
    global _L
    with _lock:
        if _L is None:
            build()
            L = ctypes.CDLL(_SO)
            vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
            L.orc_default_options.argtypes = [ctypes.POINTER(Options)]
            L.orc_hash.argtypes = [i32, i64]
            L.orc_hash.restype = ctypes.c_uint32
            L.orc_gll_nodes.argtypes = [i32, vp]
            L.orc_next_order.argtypes = [i32]
            L.orc_next_order_sched.argtypes = [i32, i32]
            L.orc_anchor_index.argtypes = [i32, i32, i32, ctypes.POINTER(i32)]
            L.orc_p1d.argtypes = [i32, i32, vp]
            L.orc_spgemm.argtypes = [ctypes.POINTER(_CSR)] * 3
            L.orc_transpose.argtypes = [ctypes.POINTER(_CSR)] * 2
            L.orc_csr_free.argtypes = [ctypes.POINTER(_CSR)]
            L.orc_mis2.argtypes = [i64, vp, vp, i32, vp, ctypes.POINTER(i32)]
            L.orc_aggregate.argtypes = [i64, vp, vp, vp, vp, ctypes.POINTER(i64)]
            L.orc_sa_prolongation_csr.argtypes = [ctypes.POINTER(_CSR), vp, i64, ctypes.POINTER(_CSR)]
            L.orc_lanczos_rho.argtypes = [ctypes.POINTER(_CSR), i32, i32]
            L.orc_lanczos_rho.restype = dbl
            L.orc_tridiag_max_eig.argtypes = [i32, vp, vp]
            L.orc_tridiag_max_eig.restype = dbl
            L.orc_cholesky.argtypes = [i32, vp]
            L.orc_chol_solve.argtypes = [i32, vp, vp, vp]
            L.orc_setup.argtypes = [i64, vp, vp, vp, ctypes.c_int32, vp, i32, ctypes.POINTER(Options),
                                    ctypes.POINTER(vp)]
            L.orc_num_levels.argtypes = [vp]
            L.orc_level_info.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i64),
                                         ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i64),
                                         ctypes.POINTER(i64)]
            L.orc_export_level.argtypes = [vp, i32, vp, vp, vp, vp]
            L.orc_export_prolongation.argtypes = [vp, i32, vp, vp, vp]
            L.orc_level_extra.argtypes = [vp, i32, ctypes.POINTER(dbl), vp]
            L.orc_free.argtypes = [vp]
            L.orc_vcycle.argtypes = [vp, i32, vp, vp]
            L.orc_level_spmv.argtypes = [vp, i32, vp, vp]
            L.orc_level_cheb.argtypes = [vp, i32, vp, vp, i32]
            L.orc_level_restrict.argtypes = [vp, i32, vp, vp]
            L.orc_level_prolong.argtypes = [vp, i32, vp, vp]
            L.orc_coarse_solve.argtypes = [vp, vp, vp]
            L.orc_level_residual.argtypes = [vp, i32, vp, vp, vp]
            L.orc_level_spmv32.argtypes = [vp, i32, vp, vp]
            L.orc_level_residual32.argtypes = [vp, i32, vp, vp, vp]
            L.orc_level_cheb32.argtypes = [vp, i32, vp, vp, i32]
            L.orc_level_restrict32.argtypes = [vp, i32, vp, vp]
            L.orc_level_prolong32.argtypes = [vp, i32, vp, vp]
            L.orc_coarse_solve32.argtypes = [vp, vp, vp]
            L.orc_solve.argtypes = [vp, vp, vp, dbl, i32, i32, i32, i32, ctypes.POINTER(i32),
                                    ctypes.POINTER(dbl), vp]
            L.orc_num_threads.restype = i32
            L.orc_set_num_threads.argtypes = [i32]
            _L = L
    return _L


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def default_options(**over) -> Options:
    o = Options()
    _lib().orc_default_options(ctypes.byref(o))
    for k, v in over.items():
        setattr(o, k, v)
    return o


# ------------------------------------------------------------------ building blocks
def hash32(i: int, kind: int = 0) -> int:
    return _lib().orc_hash(kind, i)


def gll_nodes(p: int) -> np.ndarray:
    x = np.empty(p + 1)
    _lib().orc_gll_nodes(p, _p(x))
    return x


def next_order(p: int, schedule: int = 0) -> int:
    return _lib().orc_next_order_sched(p, schedule)


def anchor_index(p: int, q: int, s: int):
    """(fine index, tie) labelling coarse index s: see orc_anchor_index."""
    tie = ctypes.c_int()
    a = _lib().orc_anchor_index(p, q, s, ctypes.byref(tie))
    return a, bool(tie.value)


def p1d(p: int, q: int) -> np.ndarray:
    t = np.empty((p + 1, q + 1))
    _lib().orc_p1d(p, q, _p(t))
    return t


def _csr_in(A):
    """(rp, ci, v, ncols) numpy CSR -> ctypes struct (arrays kept alive by the caller)."""
    rp, ci, v, m = A
    return _CSR(len(rp) - 1, m, rp.ctypes.data, ci.ctypes.data, v.ctypes.data)


def _csr_out(C: _CSR):
    n = C.n
    rp = np.ctypeslib.as_array((ctypes.c_int64 * (n + 1)).from_address(C.rp)).copy()
    nnz = int(rp[-1])
    ci = np.ctypeslib.as_array((ctypes.c_int32 * max(nnz, 1)).from_address(C.ci))[:nnz].copy()
    v = np.ctypeslib.as_array((ctypes.c_double * max(nnz, 1)).from_address(C.v))[:nnz].copy()
    _lib().orc_csr_free(ctypes.byref(C))
    return rp, ci, v, C.m if C.m else None


def spgemm(A, B):
    """C = A B for CSR tuples (rp int64, ci int32, v float64, ncols)."""
    A = (np.ascontiguousarray(A[0], np.int64), np.ascontiguousarray(A[1], np.int32), _f64(A[2]), A[3])
    B = (np.ascontiguousarray(B[0], np.int64), np.ascontiguousarray(B[1], np.int32), _f64(B[2]), B[3])
    a, b, c = _csr_in(A), _csr_in(B), _CSR()
    rc = _lib().orc_spgemm(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    if rc:
        raise RuntimeError(f"orc_spgemm: {STATUS.get(rc, rc)}")
    m = c.m
    rp, ci, v, _ = _csr_out(c)
    return rp, ci, v, m


def mis2(rp, ci, hash_kind: int = 0):
    """MIS-2 on the symmetric graph (rp, ci) without self loops; returns (in_set bool, rounds)."""
    rp = np.ascontiguousarray(rp, np.int64)
    ci = np.ascontiguousarray(ci, np.int32)
    n = len(rp) - 1
    out = np.zeros(max(n, 1), np.uint8)
    rounds = ctypes.c_int()
    _lib().orc_mis2(n, _p(rp), _p(ci), hash_kind, _p(out), ctypes.byref(rounds))
    return out[:n].astype(bool), rounds.value


def aggregate(rp, ci, in_set):
    rp = np.ascontiguousarray(rp, np.int64)
    ci = np.ascontiguousarray(ci, np.int32)
    n = len(rp) - 1
    ins = np.ascontiguousarray(in_set, np.uint8)
    agg = np.empty(max(n, 1), np.int32)
    na = ctypes.c_int64()
    rc = _lib().orc_aggregate(n, _p(rp), _p(ci), _p(ins), _p(agg), ctypes.byref(na))
    if rc:
        raise RuntimeError("orc_aggregate: node without a phase-1 neighbour")
    return agg[:n], na.value


def sa_prolongation(rp, ci, v, agg, n_agg):
    """P = T - M A T for aggregates agg (SPAI-0 M), as a CSR tuple."""
    A = (np.ascontiguousarray(rp, np.int64), np.ascontiguousarray(ci, np.int32), _f64(v), len(rp) - 1)
    agg = np.ascontiguousarray(agg, np.int32)
    a, c = _csr_in(A), _CSR()
    rc = _lib().orc_sa_prolongation_csr(ctypes.byref(a), _p(agg), n_agg, ctypes.byref(c))
    if rc:
        raise RuntimeError(f"orc_sa_prolongation: {STATUS.get(rc, rc)}")
    m = c.m
    rp2, ci2, v2, _ = _csr_out(c)
    return rp2, ci2, v2, m


def lanczos_rho(rp, ci, v, steps: int = 20, hash_kind: int = 0) -> float:
    A = (np.ascontiguousarray(rp, np.int64), np.ascontiguousarray(ci, np.int32), _f64(v), len(rp) - 1)
    a = _csr_in(A)
    return _lib().orc_lanczos_rho(ctypes.byref(a), steps, hash_kind)


def tridiag_max_eig(alpha, beta) -> float:
    alpha, beta = _f64(alpha), _f64(beta)
    return _lib().orc_tridiag_max_eig(len(alpha), _p(alpha), _p(beta))


def cholesky(a: np.ndarray) -> np.ndarray:
    L = np.array(a, dtype=np.float64, order="C", copy=True)
    rc = _lib().orc_cholesky(L.shape[0], _p(L))
    if rc:
        raise RuntimeError(f"orc_cholesky: {STATUS.get(rc, rc)}")
    return L


def chol_solve(L: np.ndarray, b: np.ndarray) -> np.ndarray:
    L, b = _f64(L), _f64(b)
    x = np.empty_like(b)
    _lib().orc_chol_solve(L.shape[0], _p(L), _p(b), _p(x))
    return x


def num_threads() -> int:
    return _lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    """Threads of the OpenMP row loops; results are bitwise the same for any count."""
    _lib().orc_set_num_threads(int(n))


# ------------------------------------------------------------------ hierarchy
class Hierarchy:
    """The oracle's GIAMG hierarchy for an assembled system (Sec. 2)."""

    def __init__(self, n, row_ptr, col, val, elem_dof, p, **opts):
        L = _lib()
        self.opt = default_options(**opts)
        self._keep = [np.ascontiguousarray(row_ptr, np.int64), np.ascontiguousarray(col, np.int32),
                      _f64(val), np.ascontiguousarray(elem_dof, np.int32)]
        rp, ci, v, ed = self._keep
        self.n = n
        self._h = ctypes.c_void_p()
        n_elem = ed.shape[0] if ed.ndim == 2 else 0
        rc = L.orc_setup(n, _p(rp), _p(ci), _p(v), n_elem, _p(ed), p, ctypes.byref(self.opt),
                         ctypes.byref(self._h))
        self._keep = None
        if rc:
            raise RuntimeError(f"orc_setup: {STATUS.get(rc, rc)}")

    @classmethod
    def from_problem(cls, prob, **opts):
        return cls(prob.n, prob.row_ptr, prob.col, prob.val, prob.elem_dof, prob.p, **opts)

    def close(self):
        if self._h is not None and self._h.value:
            _lib().orc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_levels(self) -> int:
        return _lib().orc_num_levels(self._h)

    def level_info(self, l: int) -> dict:
        k, o = ctypes.c_int(), ctypes.c_int()
        n, nnz, pn, nn = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        rc = _lib().orc_level_info(self._h, l, ctypes.byref(k), ctypes.byref(n), ctypes.byref(nnz),
                                   ctypes.byref(o), ctypes.byref(pn), ctypes.byref(nn))
        if rc:
            raise IndexError(l)
        return dict(kind=k.value, n=n.value, nnz=nnz.value, order=o.value, p_nnz=pn.value,
                    n_next=nn.value)

    def level(self, l: int):
        """(row_ptr, col, val, aggregates or None) of A_l."""
        info = self.level_info(l)
        rp = np.empty(info["n"] + 1, np.int64)
        ci = np.empty(max(info["nnz"], 1), np.int32)
        v = np.empty(max(info["nnz"], 1), np.float64)
        agg = np.full(info["n"], -1, np.int32) if info["kind"] == KIND_H else None
        _lib().orc_export_level(self._h, l, _p(rp), _p(ci), _p(v), _p(agg))
        return rp, ci[:info["nnz"]], v[:info["nnz"]], agg

    def prolongation(self, l: int):
        info = self.level_info(l)
        rp = np.empty(info["n"] + 1, np.int64)
        ci = np.empty(max(info["p_nnz"], 1), np.int32)
        v = np.empty(max(info["p_nnz"], 1), np.float64)
        rc = _lib().orc_export_prolongation(self._h, l, _p(rp), _p(ci), _p(v))
        if rc:
            raise IndexError(l)
        return rp, ci[:info["p_nnz"]], v[:info["p_nnz"]], info["n_next"]

    def rho_hat(self, l: int) -> float:
        r = ctypes.c_double()
        _lib().orc_level_extra(self._h, l, ctypes.byref(r), None)
        return r.value

    def vcycle(self, r, precision: int = 0) -> np.ndarray:
        r = _f64(r)
        z = np.empty_like(r)
        _lib().orc_vcycle(self._h, precision, _p(r), _p(z))
        return z

    def spmv(self, l, x):
        x = _f64(x)
        n = self.level_info(l)["n"]
        y = np.empty(n)
        _lib().orc_level_spmv(self._h, l, _p(x), _p(y))
        return y

    def cheb(self, l, b, x=None):
        b = _f64(b)
        x0 = np.zeros_like(b) if x is None else _f64(x).copy()
        _lib().orc_level_cheb(self._h, l, _p(b), _p(x0), 1 if x is None else 0)
        return x0

    def restrict(self, l, rf):
        rf = _f64(rf)
        rc = np.empty(self.level_info(l)["n_next"])
        _lib().orc_level_restrict(self._h, l, _p(rf), _p(rc))
        return rc

    def prolong(self, l, ec, xf):
        ec = _f64(ec)
        xf = _f64(xf).copy()
        _lib().orc_level_prolong(self._h, l, _p(ec), _p(xf))
        return xf

    def coarse_solve(self, r):
        r = _f64(r)
        x = np.empty_like(r)
        _lib().orc_coarse_solve(self._h, _p(r), _p(x))
        return x

    def residual(self, l, b, x):
        """r = b - A_l x (FP64)."""
        b, x = _f64(b), _f64(x)
        r = np.empty_like(b)
        _lib().orc_level_residual(self._h, l, _p(b), _p(x), _p(r))
        return r

    # FP32 single steps: inputs rounded to float32, results float32
    def spmv32(self, l, x):
        x = np.ascontiguousarray(x, np.float32)
        y = np.empty(self.level_info(l)["n"], np.float32)
        _lib().orc_level_spmv32(self._h, l, _p(x), _p(y))
        return y

    def residual32(self, l, b, x):
        b, x = np.ascontiguousarray(b, np.float32), np.ascontiguousarray(x, np.float32)
        r = np.empty_like(b)
        _lib().orc_level_residual32(self._h, l, _p(b), _p(x), _p(r))
        return r

    def cheb32(self, l, b, x=None):
        b = np.ascontiguousarray(b, np.float32)
        x0 = np.zeros_like(b) if x is None else np.array(x, dtype=np.float32, copy=True)
        _lib().orc_level_cheb32(self._h, l, _p(b), _p(x0), 1 if x is None else 0)
        return x0

    def restrict32(self, l, rf):
        rf = np.ascontiguousarray(rf, np.float32)
        rc = np.empty(self.level_info(l)["n_next"], np.float32)
        _lib().orc_level_restrict32(self._h, l, _p(rf), _p(rc))
        return rc

    def prolong32(self, l, ec, xf):
        ec = np.ascontiguousarray(ec, np.float32)
        xf = np.array(xf, dtype=np.float32, copy=True)
        _lib().orc_level_prolong32(self._h, l, _p(ec), _p(xf))
        return xf

    def coarse_solve32(self, r):
        r = np.ascontiguousarray(r, np.float32)
        x = np.empty_like(r)
        _lib().orc_coarse_solve32(self._h, _p(r), _p(x))
        return x

    def solve(self, b, rtol=1e-8, max_iter=1000, force_iters=0, precision=0, flexible=None):
        """Returns (x, iters, relres, history, status)."""
        b = _f64(b)
        x = np.empty_like(b)
        if flexible is None:
            flexible = 1 if precision else 0
        it, rr = ctypes.c_int(), ctypes.c_double()
        hist = np.zeros(max(max_iter, force_iters) + 2)
        rc = _lib().orc_solve(self._h, _p(b), _p(x), rtol, max_iter, force_iters, precision, flexible,
                              ctypes.byref(it), ctypes.byref(rr), _p(hist))
        return x, it.value, rr.value, hist[:it.value + 1], STATUS.get(rc, rc)

    def solve_block(self, B, rtol=1e-8, max_iter=1000, force_iters=0, precision=0):
        """Block PCG (oracle/block_cg.py) on the n x m block B with this hierarchy's V-cycle as M.
        Returns (X, iters, relres per column, status, kept directions per iteration)."""
        from .block_cg import block_pcg

        def apply_A(P):
            return np.stack([self.spmv(0, P[:, j]) for j in range(P.shape[1])], axis=1)

        def apply_M(R):
            return np.stack([self.vcycle(R[:, j], precision) for j in range(R.shape[1])], axis=1)

        return block_pcg(apply_A, apply_M, B, rtol=rtol, max_iter=max_iter, force_iters=force_iters)
