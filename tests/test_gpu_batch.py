"""Multi-right-hand-side PCG (giamg_solve_batch): m independent CG recurrences sharing every
matrix pass.  Each column is checked against the oracle's single-vector solve of that column
(the oracle runs the columns one after another: independent recurrences are the definition).

Bars: FP64 with the oracle's iteration count forced, every column within 1e-10 of the oracle;
free stopping, per-column iterations within +-1 and relres <= rtol; FP32 V-cycle, true relative
residual of every column <= 1.5e-8 (computed by the oracle's product)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import fegen  # noqa: E402
import oracle  # noqa: E402
import paper_2512_15121_gb300 as g  # noqa: E402

CASES = {
    "jitter5_p4": dict(n=5, p=4, mesh="jitter", lam=0.0, k=2),
    "jitter8_p2_hlevels": dict(n=8, p=2, mesh="jitter", lam=1.0, k=2),
    "graded3_p6": dict(n=(3, 3, 4), p=6, mesh="graded", lam=1000.0, kappa=1, k=3),
}
_cache = {}


def case(name, m):
    key = (name, m)
    if key not in _cache:
        cfg = dict(CASES[name])
        k = cfg.pop("k")
        prob = fegen.make(**cfg, rhs="none")
        B = np.stack([prob.rhs("fourier", 1000 + j) for j in range(m)], axis=1)
        orc = oracle.Hierarchy.from_problem(prob, cheb_degree=k)
        gpu = g.Solver.from_problem(prob, device=True, cheb_degree=k)
        _cache[key] = (prob, B, orc, gpu)
    return _cache[key]


@pytest.fixture(scope="module", autouse=True)
def _release():
    yield
    for _, _, _, gpu in _cache.values():
        gpu.close()
    _cache.clear()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("m", [1, 5, 32])
def test_batch_forced_matches_oracle_columns(name, m):
    prob, B, orc, gpu = case(name, m)
    its = [orc.solve(B[:, j], rtol=1e-8)[1] for j in range(m)]
    N = max(its)
    X, it, rr = gpu.solve_batch(torch.from_numpy(B).cuda(), rtol=1e-8, force_iters=N)
    X = X.cpu().numpy()
    assert np.all(it == N)
    for j in range(m):
        xo = orc.solve(B[:, j], force_iters=N)[0]
        assert np.linalg.norm(X[:, j] - xo) <= 1e-10 * np.linalg.norm(xo), j


@pytest.mark.parametrize("name", list(CASES))
def test_batch_free_stopping_per_column(name):
    prob, B, orc, gpu = case(name, 5)
    X, it, rr = gpu.solve_batch(torch.from_numpy(B).cuda(), rtol=1e-8)
    assert np.all(rr <= 1e-8)
    for j in range(5):
        _, ito, _, _, _ = orc.solve(B[:, j], rtol=1e-8)
        assert abs(int(it[j]) - ito) <= 1, (j, it[j], ito)


@pytest.mark.parametrize("name", list(CASES))
def test_batch_mixed_precision_reaches_tolerance(name):
    prob, B, orc, gpu = case(name, 5)
    X, it, rr = gpu.solve_batch(torch.from_numpy(B).cuda(), rtol=1e-8, precision=1)
    X = X.cpu().numpy()
    assert np.all(rr <= 1e-8)
    for j in range(5):
        r = B[:, j] - orc.spmv(0, X[:, j])
        assert np.linalg.norm(r) <= 1.5e-8 * np.linalg.norm(B[:, j]), j


def test_batch_column_equals_single_solve():
    prob, B, orc, gpu = case("jitter5_p4", 5)
    X, it, rr = gpu.solve_batch(torch.from_numpy(B).cuda(), rtol=1e-8, force_iters=7)
    X = X.cpu().numpy()
    for j in range(5):
        x, i1, _ = gpu.solve(torch.from_numpy(B[:, j].copy()).cuda(), rtol=1e-8, force_iters=7)
        x = x.cpu().numpy()
        assert np.linalg.norm(X[:, j] - x) <= 1e-12 * np.linalg.norm(x), j


def test_batch_is_reproducible_and_host_mode_agrees():
    prob, B, orc, gpu = case("jitter8_p2_hlevels", 5)
    Bd = torch.from_numpy(B).cuda()
    X1, i1, _ = gpu.solve_batch(Bd, rtol=1e-9)
    X2, i2, _ = gpu.solve_batch(Bd, rtol=1e-9)
    assert np.array_equal(i1, i2) and torch.equal(X1, X2)
    gpu.set_device_ptrs(False)
    try:
        Xh, ih, _ = gpu.solve_batch(B, rtol=1e-9)
    finally:
        gpu.set_device_ptrs(True)
    assert np.array_equal(ih, i1) and np.array_equal(Xh, X1.cpu().numpy())


def test_batch_argument_errors():
    prob, B, orc, gpu = case("jitter5_p4", 5)
    Bd = torch.from_numpy(B).cuda()
    import ctypes
    it = np.zeros(40, np.int32)
    rr = np.zeros(40)
    for m in (0, 33):
        rc = g.lib().giamg_solve_batch_ex(gpu._h, 0, 0, m, g._ptr(Bd), g._ptr(Bd), 1e-8, g._ptr(it), g._ptr(rr))
        assert rc == g.GIAMG_ERR_ARG


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_graph_equals_host_loop(precision):
    """The batch solve captured as one CUDA graph and the host-driven loop: same per-column
    iterations, relres and solution bits; graphs are captured per column count and recaptured
    after the work buffers grow."""
    prob, B, orc, _ = case("jitter8_p2_hlevels", 32)
    gpu = g.Solver.from_problem(prob, device=True, cheb_degree=2, graphs=2)
    host_loop = g.Solver.from_problem(prob, device=True, cheb_degree=2, graphs=0)
    try:
        for m in (5, 32, 5, 1):
            Bd = torch.from_numpy(np.ascontiguousarray(B[:, :m])).cuda()
            for force in (None, 4):
                Xg, itg, rrg = gpu.solve_batch(Bd, rtol=1e-8, precision=precision, force_iters=force)
                Xh, ith, rrh = host_loop.solve_batch(Bd, rtol=1e-8, precision=precision, force_iters=force)
                assert np.array_equal(itg, ith) and np.array_equal(rrg, rrh), m
                assert torch.equal(Xg, Xh), m
    finally:
        gpu.close()
        host_loop.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_column_bits_independent_of_width(precision):
    """A column's arithmetic does not depend on how many columns share the batch (the group width
    of the batched row kernels changes with m): the same right-hand side gives the same bits in
    batches of 1, 3, 9 and 20 columns."""
    prob, B, orc, gpu = case("jitter5_p4", 32)
    ref = None
    for m in (1, 3, 9, 20):
        X, it, rr = gpu.solve_batch(torch.from_numpy(np.ascontiguousarray(B[:, :m])).cuda(), rtol=1e-8,
                                    precision=precision)
        if ref is None:
            ref = (X[:, 0].clone(), int(it[0]))
        else:
            assert int(it[0]) == ref[1] and torch.equal(X[:, 0], ref[0]), m
