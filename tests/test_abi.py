"""The C ABI library loads and exports every entry point include/giamg.h declares (no GPU needed).

Only host-side logic runs here: the default options and the argument checks that return before
any CUDA call.  Compute calls are in the -m gpu tests.
"""
import ctypes
import os
import re

import pytest

import paper_2512_15121_gb300 as g

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    with open(os.path.join(ROOT, "include", "giamg.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"GIAMG_API\s+[\w\s\*]*?\b(giamg_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(g.LIB_PATH):
        g.build()
    return g.lib()


def test_header_and_binding_agree():
    assert declared() == sorted(g.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in declared():
        assert hasattr(lib, name), name


def test_default_options(lib):
    o = g.default_options()
    assert (o.cheb_degree, o.cheb_lo, o.cheb_hi, o.lanczos_steps) == (3, 0.1, 1.1, 20)
    assert (o.coarse_max, o.max_levels, o.strength_theta, o.precision) == (500, 16, 0.0, 0)
    assert (o.max_iter, o.force_iters, o.device_ptrs, o.hash_kind) == (1000, 0, 0, 0)


def test_argument_errors_without_a_gpu(lib):
    h = ctypes.c_void_p()
    opt = g.default_options()
    assert lib.giamg_setup(4, None, None, None, 0, None, None, None, ctypes.byref(opt), None, None) == g.GIAMG_ERR_ARG
    assert b"out" in lib.giamg_last_error()
    assert lib.giamg_setup(0, None, None, None, 0, None, None, None, ctypes.byref(opt), None,
                           ctypes.byref(h)) == g.GIAMG_ERR_ARG
    assert lib.giamg_solve(None, None, None, 1e-8, None, None) == g.GIAMG_ERR_ARG
    assert b"handle" in lib.giamg_last_error()
    for rc in (lib.giamg_solve_async(None, 0, None, None, 1e-8, None, None, None),
               lib.giamg_solve_block(None, 0, 0, 4, None, None, 1e-8, None, None),
               lib.giamg_solve_batch_ex(None, 0, 0, 4, None, None, 1e-8, None, None)):
        assert rc == g.GIAMG_ERR_ARG and b"handle" in lib.giamg_last_error()
    assert lib.giamg_free(None) == g.GIAMG_OK
    assert lib.giamg_launch_count(None) == g.GIAMG_ERR_ARG
    c = ctypes.c_int64(-1)
    assert lib.giamg_launch_count(ctypes.byref(c)) == g.GIAMG_OK and c.value >= 0
    bad = g.default_options(cheb_degree=0)
    assert lib.giamg_setup(4, None, None, None, 0, None, None, None, ctypes.byref(bad), None,
                           ctypes.byref(h)) == g.GIAMG_ERR_ARG


def test_oracle_is_not_imported_by_the_product():
    # the product package never names the oracle
    pkg = os.path.join(ROOT, "paper_2512_15121_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                with open(os.path.join(dirpath, fn)) as f:
                    text = f.read()
                assert "import oracle" not in text and "orc_" not in text, fn


def test_setup_input_checks_without_a_gpu(lib):
    """Host-mode setup rejects malformed inputs before its first CUDA call: options out of range,
    non-uniform or unsupported element orders, a missing element map, and a row pointer that
    cannot hold a diagonal per row (return code and message)."""
    import numpy as np
    n = 27
    rp = np.arange(n + 1, dtype=np.int64)
    ci = np.arange(n, dtype=np.int32)
    v = np.ones(n)
    dofs = np.zeros((2, 27), np.int32)
    ptr = lambda a: None if a is None else a.ctypes.data

    def setup(opt=None, n_elem=2, order=(2, 2), elem_dof=dofs, row_ptr=rp, coords=None):
        h = ctypes.c_void_p()
        o = opt if opt is not None else g.default_options()
        ords = np.array(order, np.int32)
        rc = lib.giamg_setup(n, ptr(row_ptr), ptr(ci), ptr(v), n_elem, ptr(elem_dof), ptr(ords), ptr(coords),
                             ctypes.byref(o), None, ctypes.byref(h))
        assert h.value is None
        return rc, lib.giamg_last_error().decode()

    cases = [
        (dict(order=(2, 3)), g.GIAMG_ERR_ORDER, "not uniform"),
        (dict(order=(13, 13)), g.GIAMG_ERR_ORDER, "outside 1..12"),
        (dict(order=(0, 0)), g.GIAMG_ERR_ORDER, "outside 1..12"),
        (dict(elem_dof=None), g.GIAMG_ERR_MAP, "elem_dof is required"),
        (dict(n_elem=-1, order=()), g.GIAMG_ERR_ARG, "n_elem must be positive"),
        (dict(row_ptr=np.zeros(n + 1, np.int64)), g.GIAMG_ERR_ARG, "row_ptr[n]"),
        (dict(opt=g.default_options(precision=2)), g.GIAMG_ERR_ARG, "precision"),
        (dict(opt=g.default_options(row_form=7)), g.GIAMG_ERR_ARG, "row_form"),
        (dict(opt=g.default_options(row_threads=3)), g.GIAMG_ERR_ARG, "row_threads"),
        (dict(opt=g.default_options(row_chains=3)), g.GIAMG_ERR_ARG, "row_chains"),
        (dict(opt=g.default_options(graphs=3)), g.GIAMG_ERR_ARG, "graphs"),
        (dict(opt=g.default_options(p_schedule=3)), g.GIAMG_ERR_ARG, "p_schedule"),
        (dict(opt=g.default_options(basis=2)), g.GIAMG_ERR_ARG, "basis"),
        (dict(opt=g.default_options(cheb_degree=65)), g.GIAMG_ERR_ARG, "cheb_degree"),
        (dict(opt=g.default_options(cheb_lo=0.0)), g.GIAMG_ERR_ARG, "cheb_lo"),
        (dict(opt=g.default_options(cheb_lo=1.2, cheb_hi=1.1)), g.GIAMG_ERR_ARG, "cheb_lo"),
        (dict(opt=g.default_options(max_levels=0)), g.GIAMG_ERR_ARG, "max_levels"),
        (dict(opt=g.default_options(lanczos_steps=0)), g.GIAMG_ERR_ARG, "lanczos_steps"),
        (dict(opt=g.default_options(prefetch_rows=-2)), g.GIAMG_ERR_ARG, "prefetch_rows"),
        (dict(opt=g.default_options(basis=1), coords=np.zeros((n, 3))), g.GIAMG_ERR_ARG, "modal"),
    ]
    for kw, code, text in cases:
        rc, msg = setup(**kw)
        assert rc == code and text in msg, (kw, rc, msg)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libgiamg.so every entry into the package raises: there is no fallback path."""
    monkeypatch.setattr(g, "_lib", None)
    monkeypatch.setattr(g, "LIB_PATH", str(tmp_path / "libgiamg.so"))
    with pytest.raises(RuntimeError, match="not built"):
        g.lib()
    with pytest.raises(RuntimeError, match="not built"):
        g.default_options()


def test_solver_checks_array_shapes_and_device_tensors():
    """The binding checks what the C ABI cannot (buffer lengths, shapes, dtypes of device tensors)
    and raises before any library or CUDA call."""
    import numpy as np
    import torch
    n, p = 27, 2
    rp = np.arange(n + 1, dtype=np.int64)
    ci = np.arange(n, dtype=np.int32)
    v = np.ones(n)
    ed = np.zeros((1, 27), np.int32)
    bad = [
        (dict(row_ptr=rp[:-1]), ValueError, "row_ptr"),
        (dict(col=ci[:-1]), ValueError, "col"),
        (dict(val=v[:-3]), ValueError, "val"),
        (dict(elem_dof=np.zeros((1, 26), np.int32)), ValueError, "elem_dof"),
        (dict(coords=np.zeros((n, 2))), ValueError, "coords"),
    ]
    for kw, exc, text in bad:
        args = dict(row_ptr=rp, col=ci, val=v, elem_dof=ed, coords=None)
        args.update(kw)
        with pytest.raises(exc, match=text):
            g.Solver(n, args["row_ptr"], args["col"], args["val"], args["elem_dof"], p, coords=args["coords"])
    # device mode: host tensors, or the wrong dtype, are refused before touching CUDA
    t = torch.from_numpy
    with pytest.raises(TypeError, match="CUDA tensor"):
        g.Solver(n, t(rp), t(ci), t(v), t(ed), p, device_ptrs=1)
    with pytest.raises(TypeError, match="CUDA tensor"):
        g.Solver(n, rp, ci, v, ed, p, device_ptrs=1)


def test_solve_calls_check_their_buffers():
    """solve / solve_batch refuse right-hand sides and output buffers of the wrong shape, dtype or
    layout before calling the library (checked on an object that was never set up)."""
    import numpy as np
    S = g.Solver.__new__(g.Solver)
    S.n, S.device, S.opts, S._h = 10, False, g.default_options(), ctypes.c_void_p()
    with pytest.raises(ValueError, match="b: shape"):
        S.solve(np.zeros(9))
    with pytest.raises(ValueError, match="x: shape"):
        S.solve(np.zeros(10), x=np.zeros(11))
    with pytest.raises(TypeError, match="float64"):
        S.solve(np.zeros(10), x=np.zeros(10, np.float32))
    with pytest.raises(ValueError, match="B: shape"):
        S.solve_batch(np.zeros((9, 2)))
    with pytest.raises(ValueError, match="B: shape"):
        S.solve_batch(np.zeros(10))
    with pytest.raises(ValueError, match="X: shape"):
        S.solve_batch(np.zeros((10, 2)), X=np.zeros((10, 3)))
    with pytest.raises(TypeError, match="contiguous"):
        S.solve_batch(np.zeros((10, 2)), X=np.zeros((2, 10)).T)


def test_single_step_calls_check_lengths(monkeypatch):
    """The per-step entry points refuse vectors whose length is not the level's (level sizes
    stubbed on an object that was never set up)."""
    import numpy as np
    S = g.Solver.__new__(g.Solver)
    S.n, S.device, S.opts, S._h = 10, False, g.default_options(), ctypes.c_void_p()
    S.level_info = lambda l: {"n": 10 if l == 0 else 4, "n_next": 4}
    monkeypatch.setattr(g.Solver, "num_levels", property(lambda self: 2))
    short, fine, coarse = np.zeros(9), np.zeros(10), np.zeros(4)
    calls = [lambda: S.vcycle(short), lambda: S.spmv(0, short), lambda: S.spmv32(0, short),
             lambda: S.smooth(0, short), lambda: S.smooth(0, fine, short), lambda: S.restrict(0, short),
             lambda: S.prolong(0, np.zeros(3), fine), lambda: S.prolong(0, coarse, short),
             lambda: S.coarse_solve(short)]
    for call in calls:
        with pytest.raises(ValueError, match="shape"):
            call()


class _AsCuda:
    """A CPU tensor that reports itself as a CUDA tensor (everything else forwarded), to run the
    binding's device-mode checks on the path that accepts the arrays from_problem builds."""

    def __init__(self, t):
        self._t = t

    is_cuda = True

    def __getattr__(self, name):
        return getattr(self._t, name)

    def __getitem__(self, i):
        return self._t[i]


def test_device_mode_checks_accept_what_from_problem_builds():
    import numpy as np
    import torch

    import fegen
    prob = fegen.make(2, 2, mesh="jitter", lam=1.0)
    t = lambda a: _AsCuda(torch.from_numpy(a))
    g._check_inputs(prob.n, t(prob.row_ptr), t(prob.col), t(prob.val), t(prob.elem_dof), prob.p,
                    t(prob.coords), True)
    with pytest.raises(TypeError, match="int64"):
        g._check_inputs(prob.n, t(prob.row_ptr.astype(np.int32)), t(prob.col), t(prob.val), None, 2, None, True)
    with pytest.raises(TypeError, match="float64"):
        g._check_inputs(prob.n, t(prob.row_ptr), t(prob.col), t(prob.val.astype(np.float32)), None, 2, None, True)
    nc = _AsCuda(torch.from_numpy(np.ascontiguousarray(prob.elem_dof.T)).T)
    with pytest.raises(ValueError, match="contiguous"):
        g._check_inputs(prob.n, t(prob.row_ptr), t(prob.col), t(prob.val), nc, 2, None, True)


def test_every_entry_point_is_documented_in_the_header():
    """Each declared entry point has a comment of its own just above it, or is named in one (the
    header states argument meaning, layout, ownership and errors there)."""
    with open(os.path.join(ROOT, "include", "giamg.h")) as f:
        text = f.read()
    comments = " ".join(re.findall(r"/\*.*?\*/", text, re.S))
    lines = text.splitlines()
    for name in declared():
        i = next(k for k, l in enumerate(lines) if "GIAMG_API" in l and re.search(r"\b" + name + r"\s*\(", l))
        above = "\n".join(lines[max(0, i - 4):i])
        assert name in comments or "*/" in above, name
