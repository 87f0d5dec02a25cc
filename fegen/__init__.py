"""Seeded synthetic finite-element inputs (mesh, element map, assembled CSR, right-hand sides).

This package stands in for the finite-element library of the paper (Sec. 2, "Required geometric
information": the FE library assembles A and supplies the element-to-dof map).  It contains no
step of the multigrid method.  Both the CUDA library's tests/benchmark and the CPU oracle take
its arrays as *inputs*; it imports neither of them.

The C core (fegen.c) is compiled on first use if the shared library is missing or older than
its source.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libfegen.so")
_SRC = [os.path.join(_HERE, "fegen.c"), os.path.join(_HERE, "fegen.h")]
_lock = threading.Lock()
_lib_handle = None

MESH = {"uniform": 0, "jitter": 1, "graded": 2}
RHS = {"none": 0, "manufactured": 1, "fourier": 2, "one": 3}


def build(force: bool = False) -> str:
    """Compile fegen.c into libfegen.so (OpenMP when the compiler supports it)."""
    stale = force or not os.path.exists(_SO) or any(
        os.path.getmtime(s) > os.path.getmtime(_SO) for s in _SRC)
    if not stale:
        return _SO
    base = ["gcc", "-O3", "-fPIC", "-shared", "-ffp-contract=off", "-o", _SO + ".tmp",
            os.path.join(_HERE, "fegen.c"), "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("p", ctypes.c_int), ("nq", ctypes.c_int), ("mesh_kind", ctypes.c_int),
                ("jitter", ctypes.c_double), ("mesh_seed", ctypes.c_uint64),
                ("grade_first", ctypes.c_double), ("kappa_kind", ctypes.c_int),
                ("lambda_", ctypes.c_double), ("dirichlet", ctypes.c_int),
                ("rhs_kind", ctypes.c_int), ("rhs_seed", ctypes.c_uint64),
                ("perm_seed", ctypes.c_uint64), ("sym_seed", ctypes.c_uint64), ("basis", ctypes.c_int)]


def _lib():
    global _lib_handle
    with _lock:
        if _lib_handle is None:
            build()
            L = ctypes.CDLL(_SO)
            vp = ctypes.c_void_p
            L.fegen_create.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(vp)]
            L.fegen_create.restype = ctypes.c_int
            L.fegen_sizes.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
            L.fegen_fill.argtypes = [vp] + [vp] * 6
            L.fegen_fill.restype = ctypes.c_int
            L.fegen_rhs.argtypes = [vp, ctypes.c_int, ctypes.c_uint64, vp]
            L.fegen_rhs.restype = ctypes.c_int
            L.fegen_l2_error.argtypes = [vp, vp]
            L.fegen_l2_error.restype = ctypes.c_double
            L.fegen_free.argtypes = [vp]
            L.fegen_num_threads.restype = ctypes.c_int
            L.fegen_gauss_rule.argtypes = [ctypes.c_int, vp, vp]
            L.fegen_gauss_rule.restype = ctypes.c_int
            L.fegen_fourier_coef.argtypes = [ctypes.c_uint64, vp]
            _lib_handle = L
    return _lib_handle


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


@dataclasses.dataclass
class Problem:
    """An assembled system with the data the solver's setup call takes."""
    nx: int
    ny: int
    nz: int
    p: int
    n: int
    nnz: int
    row_ptr: np.ndarray      # int64 [n+1]
    col: np.ndarray          # int32 [nnz], ascending within each row
    val: np.ndarray          # float64 [nnz]
    elem_dof: np.ndarray     # int32 [n_elem, (p+1)^3], local index (p+1)^2 i + (p+1) j + k
    coords: np.ndarray       # float64 [n, 3]
    boundary: np.ndarray     # uint8 [n]
    b: np.ndarray | None     # float64 [n]
    params: dict
    _ctx: object = None

    @property
    def n_elem(self) -> int:
        return self.elem_dof.shape[0]

    @property
    def elem_order(self) -> np.ndarray:
        return np.full(self.n_elem, self.p, dtype=np.int32)

    def rhs(self, kind: str = "fourier", seed: int = 1000) -> np.ndarray:
        out = np.empty(self.n, dtype=np.float64)
        rc = _lib().fegen_rhs(self._ctx.value, RHS[kind], seed, _ptr(out))
        if rc != 0:
            raise RuntimeError(f"fegen_rhs failed ({rc})")
        return out

    def rhs_nodal(self, seed: int = 1000) -> np.ndarray:
        """The smooth Fourier field of rhs("fourier") -- sum over k1, k2, k3 in 1..4 of
        c_k sin(k1 pi x) sin(k2 pi y) sin(k3 pi z), c ~ N(0, 1) drawn from `seed` (numpy's PCG64) --
        evaluated at the nodes instead of loaded by quadrature, zero on Dirichlet rows.  Costs
        O(64 n), for streams of many right-hand sides on large meshes."""
        c = np.random.default_rng(seed).standard_normal((4, 4, 4))
        k = np.arange(1, 5)[:, None] * np.pi
        sx, sy, sz = (np.sin(k * self.coords[None, :, d]) for d in range(3))  # 4 x n each
        f = np.einsum("abc,an,bn,cn->n", c, sx, sy, sz, optimize=True)
        f[self.boundary != 0] = 0.0
        return f

    def l2_error(self, uh: np.ndarray) -> float:
        """L2 distance of the nodal field uh to the manufactured solution."""
        uh = np.ascontiguousarray(uh, dtype=np.float64)
        return _lib().fegen_l2_error(self._ctx.value, _ptr(uh))

    def scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.n, self.n))

    def close(self):
        if self._ctx is not None and self._ctx.value:
            _lib().fegen_free(self._ctx.value)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make(n: int | tuple = 4, p: int = 4, mesh: str = "uniform", lam: float = 1.0, kappa: int = 0,
         mesh_seed: int = 1, jitter: float = 0.2, grade_first: float = 0.0, nq: int = 0,
         dirichlet: bool = True, rhs: str = "manufactured", rhs_seed: int = 1000,
         perm_seed: int = 0, sym_seed: int = 0, with_values: bool = True, basis: str = "nodal") -> Problem:
    """Assemble -div(kappa grad u) + lam u = f on an n^3 (or nx*ny*nz) hex mesh of order p, in the
    nodal GLL basis or the modal (hierarchical) one.  For the modal basis, `coords` holds the GLL
    lattice positions the modes are numbered by, not nodes of the functions."""
    nx, ny, nz = (n, n, n) if isinstance(n, int) else tuple(n)
    L = _lib()
    prm = _Params(nx, ny, nz, p, nq, MESH[mesh], jitter, mesh_seed, grade_first, kappa, lam,
                  1 if dirichlet else 0, RHS[rhs], rhs_seed, perm_seed, sym_seed,
                  {"nodal": 0, "modal": 1}[basis])
    ctx = ctypes.c_void_p()
    rc = L.fegen_create(ctypes.byref(prm), ctypes.byref(ctx))
    if rc != 0:
        raise RuntimeError(f"fegen_create failed ({rc})")
    N, NNZ = ctypes.c_int64(), ctypes.c_int64()
    NE, NL = ctypes.c_int32(), ctypes.c_int32()
    L.fegen_sizes(ctx, ctypes.byref(N), ctypes.byref(NNZ), ctypes.byref(NE), ctypes.byref(NL))
    N, NNZ, NE, NL = N.value, NNZ.value, NE.value, NL.value
    row_ptr = np.empty(N + 1, dtype=np.int64)
    col = np.empty(NNZ, dtype=np.int32)
    val = np.empty(NNZ, dtype=np.float64) if with_values else None
    elem_dof = np.empty((NE, NL), dtype=np.int32)
    coords = np.empty((N, 3), dtype=np.float64)
    bnd = np.empty(N, dtype=np.uint8)
    rc = L.fegen_fill(ctx, _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(elem_dof), _ptr(coords), _ptr(bnd))
    if rc != 0:
        L.fegen_free(ctx)
        raise RuntimeError(f"fegen_fill failed ({rc})")
    prob = Problem(nx, ny, nz, p, N, NNZ, row_ptr, col, val, elem_dof, coords, bnd, None,
                   dict(n=(nx, ny, nz), p=p, mesh=mesh, lam=lam, kappa=kappa, mesh_seed=mesh_seed,
                        jitter=jitter, nq=nq, dirichlet=dirichlet, rhs=rhs, rhs_seed=rhs_seed,
                        perm_seed=perm_seed, sym_seed=sym_seed, basis=basis), ctx)
    if rhs != "none":
        prob.b = prob.rhs(rhs, rhs_seed)
    return prob


# Workloads, named by what they are (mesh, order, operator).  The Helmholtz and Poisson
# operators are the paper's problem classes (Sec. 3.1, Eq. 2; Sec. 3.2 pressure Poisson and
# velocity Helmholtz of the velocity-correction scheme); the meshes are synthetic stand-ins
# for the paper's Nektar++ meshes, which are not available.
WORKLOADS = {
    # unit-cube Helmholtz, lambda = 1, uniform 4^3, p = 4: 4913 dofs
    "helmholtz_4cube_p4": dict(n=4, p=4, mesh="uniform", lam=1.0, rhs="manufactured", k=3),
    # Helmholtz lambda = 10 on a jittered 16^3 mesh, p = 6: 912,673 dofs
    "helmholtz_16cube_jitter_p6": dict(n=16, p=6, mesh="jitter", mesh_seed=1, lam=10.0,
                                       rhs="manufactured", k=3),
    # the same operator and order on an 8^3 mesh (117,649 dofs, 5.1e7 nonzeros: larger than L2),
    # used for detailed kernel profiles
    "helmholtz_8cube_jitter_p6": dict(n=8, p=6, mesh="jitter", mesh_seed=1, lam=10.0, rhs="manufactured", k=3),
    # and on a 12^3 mesh (389,017 dofs, 1.7e8 nonzeros, about 3.5 GB on the device with the
    # hierarchy): the smallest of these on which the hybrid row form is the default, for its
    # detailed profiles
    "helmholtz_12cube_jitter_p6": dict(n=12, p=6, mesh="jitter", mesh_seed=1, lam=10.0, rhs="manufactured", k=3),
    # pressure Poisson on a jittered 24^3 mesh, p = 4: 912,673 dofs, 32 Fourier right-hand sides
    "poisson_24cube_jitter_p4": dict(n=24, p=4, mesh="jitter", mesh_seed=2, lam=0.0,
                                     rhs="fourier", k=2),
    # velocity Helmholtz lambda = 1000, variable kappa, 12^3 graded to z = 0, p = 8
    "helmholtz_12cube_graded_p8": dict(n=12, p=8, mesh="graded", lam=1000.0, kappa=1,
                                       rhs="manufactured", k=2),
}


def workload(name: str, **over) -> Problem:
    cfg = dict(WORKLOADS[name])
    cfg.pop("k", None)
    cfg.update(over)
    return make(**cfg)


def num_threads() -> int:
    return _lib().fegen_num_threads()


def gauss_rule(n: int):
    """The n-point Gauss-Legendre rule the assembly integrates with: (nodes, weights) on [-1, 1]."""
    x, w = np.empty(n), np.empty(n)
    if _lib().fegen_gauss_rule(n, _ptr(x), _ptr(w)) != 0:
        raise ValueError(f"no Gauss-Legendre rule with {n} points")
    return x, w


def fourier_coef(seed: int) -> np.ndarray:
    """The coefficients c[k1-1, k2-1, k3-1] of rhs("fourier", seed) (the generator's own
    counter-based normal draws, not numpy's)."""
    c = np.empty(64)
    _lib().fegen_fourier_coef(seed, _ptr(c))
    return c.reshape(4, 4, 4)
