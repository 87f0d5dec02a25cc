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
