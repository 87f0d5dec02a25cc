"""giamg_solve_grouped: the multi-right-hand-side solves of several hierarchies at once, one kernel
launch per phase over all of them.  Each hierarchy's results are bit for bit those of its own
giamg_solve_batch (host loop and graph alike) and independent of the group it runs in; the
hierarchies differ in order, level count (p-levels only, or with aggregation), smoother degree
and column count.  Every column is also checked against the oracle's product (true residual)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import fegen  # noqa: E402
import oracle  # noqa: E402
import paper_2512_15121_gb300 as g  # noqa: E402

CASES = [  # (mesh, p, lambda, Chebyshev degree, columns)
    (dict(n=4, p=4, mesh="uniform", lam=1.0), 3, 5),
    (dict(n=6, p=2, mesh="jitter", lam=0.0), 2, 17),        # FP32 products in row pairs (m > 16)
    (dict(n=(5, 4, 6), p=3, mesh="jitter", lam=1000.0), 3, 1),
    (dict(n=8, p=2, mesh="jitter", lam=1.0), 2, 32),         # aggregation levels (h-transfers)
]


@pytest.fixture(scope="module")
def members():
    out = []
    for cfg, k, m in CASES:
        prob = fegen.make(**cfg)
        S = g.Solver.from_problem(prob, device=True, cheb_degree=k)
        B = np.stack([prob.rhs("fourier", 300 + j) for j in range(m)], axis=1)
        out.append((prob, S, torch.from_numpy(B).cuda()))
    yield out
    for _, S, _ in out:
        S.close()


def test_grouped_equals_each_batch_solve_bit_for_bit(members):
    alone = []
    for prob, S, B in members:
        X, it, rr = S.solve_batch(B, rtol=1e-8, precision=1)
        assert S.last_status == g.GIAMG_OK
        alone.append((X.clone(), it.copy(), rr.copy()))
    res = g.solve_grouped([S for _, S, _ in members], [B for _, _, B in members], rtol=1e-8)
    assert [r[3] for r in res] == [g.GIAMG_OK] * len(members)
    for (prob, S, B), (X, it, rr, st), (Xa, ita, rra) in zip(members, res, alone):
        assert torch.equal(X, Xa), prob.params
        assert np.array_equal(it, ita) and np.array_equal(rr, rra)
        Xh = X.cpu().numpy()
        Bh = B.cpu().numpy()
        for j in range(B.shape[1]):
            r = Bh[:, j] - prob.scipy() @ Xh[:, j]
            assert np.linalg.norm(r) <= 1.5e-8 * np.linalg.norm(Bh[:, j]), (prob.params, j)


def test_a_member_gives_the_same_bits_in_any_group(members):
    idx = [3, 1]
    first = g.solve_grouped([members[i][1] for i in idx], [members[i][2] for i in idx])
    solo = g.solve_grouped([members[1][1]], [members[1][2]])
    rev = g.solve_grouped([members[i][1] for i in (1, 0, 2)], [members[i][2] for i in (1, 0, 2)])
    assert torch.equal(first[1][0], solo[0][0]) and torch.equal(rev[0][0], solo[0][0])
    assert np.array_equal(first[1][1], solo[0][1])


def test_grouped_edge_cases(members):
    # a zero right-hand side column retires at once; the others converge
    prob, S, B = members[0]
    Bz = B.clone()
    Bz[:, 1] = 0.0
    (X, it, rr, st), = g.solve_grouped([S], [Bz])
    assert st == g.GIAMG_OK and it[1] == 0 and rr[1] == 0.0 and torch.count_nonzero(X[:, 1]) == 0
    assert np.all(rr <= 1e-8)
    # the iteration limit: MAXITER reported for that member only
    capped = g.Solver.from_problem(prob, device=True, cheb_degree=3, max_iter=2)
    try:
        res = g.solve_grouped([capped, members[2][1]], [B, members[2][2]], rtol=1e-12)
        assert res[0][3] == g.GIAMG_ERR_MAXITER and np.all(res[0][1] == 2)
        Xc, itc, rrc = capped.solve_batch(B, rtol=1e-12, precision=1)
        assert torch.equal(res[0][0], Xc)
    finally:
        capped.close()
    # refusals: the same hierarchy twice, host-mode hierarchies, a wrong block shape
    with pytest.raises(g.GiamgError):
        g.solve_grouped([S, S], [B, B])
    host = g.Solver.from_problem(prob, device=False)
    try:
        with pytest.raises(g.GiamgError):
            g.solve_grouped([host], [B])
    finally:
        host.close()
    with pytest.raises(ValueError):
        g.solve_grouped([S], [B[:, :0]])
