"""The GPU's Galerkin products against the oracle's sparse product on the same operands, bit for bit.

Every coarse operator the GPU builds is R (A P) with R = P^T (Sec. 2).  Here the oracle's
`spgemm` (the plain definition: the symbolic union over the inner index, each entry summed in
ascending inner index from 0, one rounded product added at a time) is applied to the GPU's own
A_l and P_l, and the result must equal the GPU's A_{l+1} exactly: pattern and every bit of every
value.  This pins the numeric passes themselves (warp work items for groups of many rows, a warp
per row otherwise, the plain hash pass of the aggregation levels) apart from the operands: the
GLL nodes behind P come from two independent Newton iterations, which may differ in the last bit
at p = 8, so the hierarchies are compared with the oracle's own in test_gpu_parity.py to 1e-12.

Cases: p = 8 (large row groups: warp items with one lane per row), p = 6, p = 4 with relabelled
dofs (coarse rows of one row each: the per-row pass), an order-1 input (aggregation levels only),
the modal basis (injection P).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import scipy.sparse as sp  # noqa: E402

import fegen  # noqa: E402
import oracle  # noqa: E402
import paper_2512_15121_gb300 as g  # noqa: E402

CASES = {
    "jitter2_p8": (dict(n=2, p=8, mesh="jitter", lam=1000.0), {}),
    "graded223_p8_kappa": (dict(n=(2, 2, 3), p=8, mesh="graded", lam=10.0, kappa=1), {}),
    "jitter4_p6": (dict(n=4, p=6, mesh="jitter", lam=10.0), {}),
    "jitter6_p4_relabelled": (dict(n=6, p=4, mesh="jitter", lam=1.0, perm_seed=5, sym_seed=6), {}),
    "jitter10_p1": (dict(n=10, p=1, mesh="jitter", lam=1.0), {}),
    "jitter4_p4_modal": (dict(n=4, p=4, mesh="jitter", lam=1.0, basis="modal"), dict(basis=1)),
}


def transpose(rp, ci, v, ncols):
    """P^T with ascending columns (values copied, so exact)."""
    T = sp.csr_matrix((v, ci, rp), shape=(len(rp) - 1, ncols)).T.tocsr()
    T.sort_indices()
    return T.indptr.astype(np.int64), T.indices.astype(np.int32), T.data, T.shape[1]


@pytest.mark.parametrize("name", list(CASES))
def test_coarse_operators_are_the_oracle_product_of_the_gpu_operands(name):
    cfg, opts = CASES[name]
    prob = fegen.make(**cfg)
    S = g.Solver.from_problem(prob, device=True, cheb_degree=2, **opts)
    try:
        assert S.num_levels >= 2
        for l in range(S.num_levels - 1):
            rp, ci, v, _ = S.level(l)
            n = len(rp) - 1
            prp, pci, pv, m = S.prolongation(l)
            AP = oracle.spgemm((rp, ci, v, n), (prp, pci, pv, m))
            C = oracle.spgemm(transpose(prp, pci, pv, m), AP)
            crp, cci, cv, _ = S.level(l + 1)
            assert np.array_equal(C[0], crp) and np.array_equal(C[1], cci), (name, l)
            same = C[2] == cv
            assert same.all(), (name, l, int((~same).sum()), float(np.max(np.abs(C[2] - cv))))
    finally:
        S.close()
        prob.close()
