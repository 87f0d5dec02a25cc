"""Block CG (giamg_solve_block): the m right-hand sides as one block sharing one Krylov space,
against the oracle's block PCG (oracle/block_cg.py) on the same hierarchy.

Bars: FP64 V-cycle with the oracle's iteration count forced, X within 1e-10 of the oracle's
(Frobenius, relative); free stopping, the block iteration count within +-1 and every column at
rtol; FP32 V-cycle (and FP32 Gram products), the true relative residual of every column
<= 1.5e-8 (the oracle's product); dependent, duplicate and zero columns give the oracle's
iterates and relations; the graph and the host loop agree bit for bit."""
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


def case(name):
    if name not in _cache:
        cfg = dict(CASES[name])
        k = cfg.pop("k")
        prob = fegen.make(**cfg, rhs="none")
        orc = oracle.Hierarchy.from_problem(prob, cheb_degree=k)
        gpu = g.Solver.from_problem(prob, device=True, cheb_degree=k)
        _cache[name] = (prob, orc, gpu)
    return _cache[name]


def rhs(prob, m, seed=1000):
    return np.stack([prob.rhs("fourier", seed + j) for j in range(m)], axis=1)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module", autouse=True)
def _release():
    yield
    for _, _, gpu in _cache.values():
        gpu.close()
    _cache.clear()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("m", [1, 5, 32])
def test_block_forced_matches_oracle(name, m):
    prob, orc, gpu = case(name)
    B = rhs(prob, m)
    Xo, N, rro, st, _ = orc.solve_block(B, rtol=1e-8)
    assert st == "ok"
    X, it, rr = gpu.solve_block(dev(B), rtol=1e-8, force_iters=N)
    assert np.all(it == N)
    Xo = orc.solve_block(B, force_iters=N)[0]
    assert np.linalg.norm(X.cpu().numpy() - Xo) <= 1e-10 * np.linalg.norm(Xo)


@pytest.mark.parametrize("name", list(CASES))
def test_block_free_stopping(name):
    prob, orc, gpu = case(name)
    B = rhs(prob, 7, seed=300)
    _, ito, _, st, _ = orc.solve_block(B, rtol=1e-8)
    X, it, rr = gpu.solve_block(dev(B), rtol=1e-8)
    assert gpu.last_status == g.GIAMG_OK
    assert np.all(it == it[0]) and abs(int(it[0]) - ito) <= 1
    assert np.all(rr <= 1e-8)


@pytest.mark.parametrize("name", list(CASES))
def test_block_mixed_precision_reaches_tolerance(name):
    prob, orc, gpu = case(name)
    B = rhs(prob, 32)
    X, it, rr = gpu.solve_block(dev(B), rtol=1e-8, precision=1)
    X = X.cpu().numpy()
    assert np.all(rr <= 1e-8)
    for j in range(32):
        r = B[:, j] - orc.spmv(0, X[:, j])
        assert np.linalg.norm(r) <= 1.5e-8 * np.linalg.norm(B[:, j]), j


def test_block_dependent_duplicate_and_zero_columns():
    prob, orc, gpu = case("jitter5_p4")
    b0, b1, b2 = (prob.rhs("fourier", s) for s in (7, 8, 9))
    B = np.stack([b0, b1, b0, np.zeros_like(b0), b0 + 2.0 * b1, b2], axis=1)
    Xo, ito, _, st, ranks = orc.solve_block(B, rtol=1e-8)
    assert st == "ok" and max(ranks) == 3
    X, it, rr = gpu.solve_block(dev(B), rtol=1e-8, force_iters=ito)
    X = X.cpu().numpy()
    scale = np.linalg.norm(Xo)
    assert np.linalg.norm(X - Xo) <= 1e-10 * scale
    assert np.all(X[:, 3] == 0.0) and rr[3] == 0.0
    assert np.linalg.norm(X[:, 2] - X[:, 0]) <= 1e-10 * scale
    assert np.linalg.norm(X[:, 4] - X[:, 0] - 2.0 * X[:, 1]) <= 1e-10 * scale
    X, it, rr = gpu.solve_block(dev(B), rtol=1e-8)
    assert gpu.last_status == g.GIAMG_OK and np.all(rr <= 1e-8)
    # FP32 V-cycle and FP32 Gram products: the dependent directions are dropped at the FP32
    # threshold, every column still reaches rtol with an FP64-consistent residual
    X, it, rr = gpu.solve_block(dev(B), rtol=1e-8, precision=1)
    assert gpu.last_status == g.GIAMG_OK and np.all(rr <= 1e-8)
    X = X.cpu().numpy()
    assert np.all(X[:, 3] == 0.0)
    for j in (0, 1, 2, 4, 5):
        r = B[:, j] - orc.spmv(0, X[:, j])
        assert np.linalg.norm(r) <= 1.5e-8 * np.linalg.norm(B[:, j]), j
    # all columns zero: no iteration
    Xz, itz, rrz = gpu.solve_block(dev(np.zeros((prob.n, 3))), rtol=1e-8)
    assert np.all(itz == 0) and np.all(Xz.cpu().numpy() == 0.0)


def test_block_one_column_equals_single_solve():
    prob, orc, gpu = case("graded3_p6")
    b = prob.rhs("fourier", 55)
    x, it, rr = gpu.solve(dev(b), rtol=1e-8)
    X, itb, rrb = gpu.solve_block(dev(b[:, None]), rtol=1e-8)
    assert int(itb[0]) == it
    xn = x.cpu().numpy()
    assert np.linalg.norm(X.cpu().numpy()[:, 0] - xn) <= 1e-10 * np.linalg.norm(xn)


@pytest.mark.parametrize("precision", [0, 1])
def test_block_graph_equals_host_loop(precision):
    cfg = dict(CASES["jitter8_p2_hlevels"])
    k = cfg.pop("k")
    prob = fegen.make(**cfg, rhs="none")
    B = dev(rhs(prob, 9, seed=40))
    out = []
    for graphs in (0, 2, 2):  # host loop, then the captured graph twice
        s = g.Solver.from_problem(prob, device=True, cheb_degree=k, graphs=graphs)
        X, it, rr = s.solve_block(B, rtol=1e-8, precision=precision)
        out.append((X.cpu().numpy(), it.copy(), rr.copy()))
        if graphs == 2:
            X2, it2, rr2 = s.solve_block(B, rtol=1e-8, precision=precision)
            assert np.array_equal(X2.cpu().numpy(), out[-1][0]) and np.array_equal(it2, it)
        s.close()
    for X, it, rr in out[1:]:
        assert np.array_equal(X, out[0][0]) and np.array_equal(it, out[0][1]) and np.array_equal(rr, out[0][2])


def test_block_fewer_iterations_than_independent_columns_modal_basis():
    # the modal basis leaves outlying eigenvalues in the preconditioned operator, which the
    # shared block space removes for all columns at once
    prob = fegen.make(4, 6, mesh="jitter", lam=1.0, basis="modal", rhs="none")
    orc = oracle.Hierarchy.from_problem(prob, cheb_degree=3)
    gpu = g.Solver.from_problem(prob, device=True, cheb_degree=3)
    try:
        B = rhs(prob, 32)
        _, ito, _, st, _ = orc.solve_block(B, rtol=1e-8)
        X, it, rr = gpu.solve_block(dev(B), rtol=1e-8)
        assert np.all(rr <= 1e-8) and abs(int(it[0]) - ito) <= 2
        _, iti, _ = gpu.solve_batch(dev(B), rtol=1e-8)
        assert int(it[0]) < 0.8 * int(iti.max())
        Xm, itm, rrm = gpu.solve_block(dev(B), rtol=1e-8, precision=1)
        assert np.all(rrm <= 1e-8)
        Xm = Xm.cpu().numpy()
        for j in (0, 13, 31):
            r = B[:, j] - orc.spmv(0, Xm[:, j])
            assert np.linalg.norm(r) <= 1.5e-8 * np.linalg.norm(B[:, j]), j
    finally:
        gpu.close()


def test_block_argument_errors():
    prob, orc, gpu = case("jitter8_p2_hlevels")
    B = dev(np.zeros((prob.n, 33)))
    with pytest.raises(g.GiamgError):
        gpu.solve_block(B)
    with pytest.raises(g.GiamgError):
        gpu.solve_block(dev(np.zeros((prob.n, 2))), precision=2)
