"""giamg_true_relres_noalloc: the allocation-free true-residual check.

Some callers cannot call cudaMalloc while they check convergence: their device memory belongs to
another allocator that has reserved the GPU, or their loop must keep a fixed device-memory
footprint.  The entry point gives them ||b - A x|| / ||b|| with its scratch in a static device
array that giamg_setup loads.  The checks here:
  * two calls in a row against the existing entry point (giamg_solve_stats) and against the
    residual computed in FP64 numpy from the oracle's CSR of the same matrix;
  * in a fresh process, the device's free memory is the same before and after the first and the
    second call (nothing is loaded or allocated by a call);
  * host arrays and NULL arguments are refused with GIAMG_ERR_ARG before any kernel runs.
This file is named so that pytest collects it last; it passes alone in a fresh process and after
the other tests.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import fegen  # noqa: E402
import paper_2512_15121_gb300 as g  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def numpy_relres(prob, b, x):
    """||b - A x|| / ||b|| in FP64 from the assembled CSR (scipy product), independent of the library."""
    import scipy.sparse as sp
    A = sp.csr_matrix((prob.val, prob.col, prob.row_ptr), shape=(prob.n, prob.n))
    r = b - A @ x
    return np.linalg.norm(r) / np.linalg.norm(b)


def test_matches_solve_stats_and_numpy_on_two_calls_in_a_row():
    prob = fegen.make((6, 5, 7), 4, mesh="jitter", lam=1.0)
    S = g.Solver.from_problem(prob, device=True)
    try:
        for seed in (1000, 1001):
            b = torch.from_numpy(prob.rhs("fourier", seed)).cuda()
            x, it, rr = S.solve(b, rtol=1e-6)
            _, ref = S.stats(0)
            got = S.true_relres_noalloc(b, x)
            want = numpy_relres(prob, b.cpu().numpy(), x.cpu().numpy())
            # b - A x cancels down to the residual (1e-6 of b), so two summation orders of the same
            # FP64 quantity agree to about 1e-16 |A||x| / |r|: a few 1e-10 relative at most
            assert ref > 0 and abs(got - ref) <= 1e-9 * ref, (seed, got, ref)
            assert abs(got - want) <= 1e-9 * want, (seed, got, want)
        # the scratch now holds the last call's sums; the same inputs again give the same bits
        again = S.true_relres_noalloc(b, x)
        assert again == got
    finally:
        S.close()


def test_refuses_host_arrays_and_null_arguments():
    prob = fegen.make(2, 2, lam=1.0)
    S = g.Solver.from_problem(prob, device=True)
    try:
        out = ctypes.c_double(-1.0)
        L = g.lib()
        assert L.giamg_true_relres_noalloc(S._h, None, None, ctypes.byref(out)) == g.GIAMG_ERR_ARG
        assert L.giamg_true_relres_noalloc(None, None, None, ctypes.byref(out)) == g.GIAMG_ERR_ARG
        # host arrays (pageable and pinned) are refused by the pointer check, before any launch
        bh = np.ones(prob.n)
        xd = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
        rc = L.giamg_true_relres_noalloc(S._h, g._ptr(bh), g._ptr(xd), ctypes.byref(out))
        assert rc == g.GIAMG_ERR_ARG and b"device memory" in L.giamg_last_error()
        pinned = torch.ones(prob.n, dtype=torch.float64).pin_memory()
        rc = L.giamg_true_relres_noalloc(S._h, g._ptr(xd), g._ptr(pinned), ctypes.byref(out))
        assert rc == g.GIAMG_ERR_ARG
        assert out.value == -1.0
        # the binding refuses what is not a CUDA float64 tensor of length n
        with pytest.raises(TypeError):
            S.true_relres_noalloc(bh, xd)
        with pytest.raises(ValueError):
            S.true_relres_noalloc(xd[:-1], xd[:-1])
        # the library still works after the refusals
        b = torch.from_numpy(prob.b).cuda()
        x, _, _ = S.solve(b, rtol=1e-8)
        assert S.true_relres_noalloc(b, x) <= 1.5e-8
    finally:
        S.close()


_FRESH = r"""
import sys, torch
sys.path.insert(0, sys.argv[1])
import fegen, paper_2512_15121_gb300 as g
prob = fegen.make(4, 4, mesh="jitter", lam=1.0)
S = g.Solver.from_problem(prob, device=True)
b = torch.from_numpy(prob.b).cuda()
x, _, _ = S.solve(b, rtol=1e-8)
torch.cuda.synchronize()
free = [torch.cuda.mem_get_info()[0]]
vals = []
for _ in range(2):
    vals.append(S.true_relres_noalloc(b, x))
    torch.cuda.synchronize()
    free.append(torch.cuda.mem_get_info()[0])
print("FREE", *free)
print("VALS", *vals)
S.close()
"""


def test_first_call_in_a_fresh_process_allocates_nothing():
    out = subprocess.run([sys.executable, "-c", _FRESH, ROOT], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    free = [int(v) for v in next(l for l in out.stdout.splitlines() if l.startswith("FREE")).split()[1:]]
    vals = [float(v) for v in next(l for l in out.stdout.splitlines() if l.startswith("VALS")).split()[1:]]
    assert free[0] == free[1] == free[2], free
    assert vals[0] == vals[1] and 0.0 < vals[0] <= 1.5e-8, vals
