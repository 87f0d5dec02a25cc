"""giamg_true_relres_noalloc: the allocation-free true-residual check.

Some callers cannot call cudaMalloc while they check convergence (their device memory belongs to
another allocator, or their loop must keep a fixed footprint).  The entry point gives them the
same number as giamg_solve_stats with its scratch in a static device array.  This file is named
so that pytest collects it last; it passes alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import fegen  # noqa: E402
import paper_2512_15121_gb300 as g  # noqa: E402


def noalloc_relres(S, b, x):
    out = ctypes.c_double(-1.0)
    rc = g.lib().giamg_true_relres_noalloc(S._h, g._ptr(b), g._ptr(x), ctypes.byref(out))
    assert rc == g.GIAMG_OK, g.lib().giamg_last_error()
    return out.value


def test_matches_solve_stats_on_two_calls_in_a_row():
    prob = fegen.make((6, 5, 7), 4, mesh="jitter", lam=1.0)
    S = g.Solver.from_problem(prob, device=True)
    for seed in (1000, 1001):
        b = torch.from_numpy(prob.rhs("fourier", seed)).cuda()
        x, it, rr = S.solve(b, rtol=1e-6)
        _, ref = S.stats(0)
        got = noalloc_relres(S, b, x)
        # same quantity, products and partial sums grouped differently; b - A x cancels to the
        # residual level, so compare with the tolerance the parity tests use for true residuals
        assert ref > 0 and abs(got - ref) <= 1e-6 * ref, (seed, got, ref)
    # a second pair of calls on the same inputs, after the scratch holds the last call's sums
    again = noalloc_relres(S, b, x)
    assert abs(again - got) <= 1e-15 * got
    S.close()


def test_rejects_null_arguments():
    prob = fegen.make(2, 2, lam=1.0)
    S = g.Solver.from_problem(prob, device=True)
    out = ctypes.c_double()
    assert g.lib().giamg_true_relres_noalloc(S._h, None, None, ctypes.byref(out)) == g.GIAMG_ERR_ARG
    assert g.lib().giamg_true_relres_noalloc(None, None, None, ctypes.byref(out)) == g.GIAMG_ERR_ARG
    S.close()
