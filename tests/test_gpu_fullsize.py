"""GPU parity at the full workload sizes, with the default options bench.py times.

Workloads (seeded, synthetic; fegen.WORKLOADS):
  helmholtz_4cube_p4           4,913 dofs       p 4 -> 2 -> 1, Chebyshev degree 3
  helmholtz_16cube_jitter_p6   912,673 dofs     p 6 -> 3 -> 1 -> aggregation, degree 3
  poisson_24cube_jitter_p4     912,673 dofs     p 4 -> 2 -> 1 -> aggregation, degree 2, 32 RHS
  helmholtz_12cube_graded_p8   912,673 dofs     p 8 -> 4 -> 2 -> 1 -> aggregation, degree 2

At these sizes the oracle still builds the whole hierarchy and runs the whole solve in seconds
to a minute on the host cores, so the checks are the ones of the small cases:
  hierarchy structure (sizes, row pointers, columns, aggregates, P patterns)   bit-exact
  hierarchy values                                                              1e-12 relative
  FP64 PCG with the oracle's iteration count forced                             x within 1e-10
  FP64 PCG stopping freely                                                      iterations +-1
  FP32 V-cycle in FP64 flexible CG: true relative residual (oracle product)     <= 1.5e-8
  FP32 V-cycle against the oracle's FP32 V-cycle, element by element            1e-5 of max |z|
  finest level's FP32 residual and smoother (the headline kernels: the vector
    hybrid row form at p = 6 and 8) against the oracle's, row by row            rounding bounds
    (tests/fp32_bounds.py)
  32-column batch (Poisson): three columns against the oracle's single solves   x within 1e-10
                             every column's true residual (oracle product)      <= 1.5e-8
  32-column block CG (Poisson), both V-cycle precisions: every column's true
                             residual (oracle product)                          <= 1.5e-8
                             (the oracle's block PCG couples all 32 columns through 32 V-cycles
                             per iteration, too slow at this size; it is compared element by
                             element on the smaller cases of test_gpu_block.py)
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import fegen  # noqa: E402
import oracle  # noqa: E402
import paper_2512_15121_gb300 as g  # noqa: E402
from fp32_bounds import fp32_step_checks  # noqa: E402

NAMES = ["helmholtz_4cube_p4", "helmholtz_16cube_jitter_p6", "poisson_24cube_jitter_p4",
         "helmholtz_12cube_graded_p8"]


class Full:
    def __init__(self, name):
        self.name = name
        self.k = fegen.WORKLOADS[name]["k"]
        self.prob = fegen.workload(name)
        self.orc = oracle.Hierarchy.from_problem(self.prob, cheb_degree=self.k)
        self.gpu = g.Solver.from_problem(self.prob, device=True, cheb_degree=self.k)
        self._fp64 = None

    def oracle_fp64(self):
        """The oracle's FP64 PCG, stopping freely at 1e-8 (x, iterations)."""
        if self._fp64 is None:
            xo, ito, _, _, st = self.orc.solve(self.prob.b, rtol=1e-8)
            assert st == "ok"
            self._fp64 = (xo, ito)
        return self._fp64

    def close(self):
        self.gpu.close()
        self.orc.close()
        self.prob.close()


@pytest.fixture(scope="module", params=NAMES)
def full(request):
    f = Full(request.param)
    yield f
    f.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_structure_bit_exact(full):
    orc, gpu = full.orc, full.gpu
    assert gpu.num_levels == orc.num_levels
    for l in range(orc.num_levels):
        a, b = gpu.level_info(l), orc.level_info(l)
        assert a == b, (l, a, b)
        grp, gci, gv, gagg = gpu.level(l)
        orp, oci, ov, oagg = orc.level(l)
        assert np.array_equal(grp, orp) and np.array_equal(gci, oci), l
        assert np.max(np.abs(gv - ov)) <= 1e-12 * np.max(np.abs(ov)), l
        del gv, ov, gci, oci
        if oagg is not None:
            assert np.array_equal(gagg, oagg), l
        if b["kind"] != oracle.KIND_COARSEST:
            prp, pci, pv, _ = gpu.prolongation(l)
            qrp, qci, qv, _ = orc.prolongation(l)
            assert np.array_equal(prp, qrp) and np.array_equal(pci, qci), l
            assert np.max(np.abs(pv - qv)) <= 1e-12 * np.max(np.abs(qv)), l


def test_fp64_pcg_forced_and_free(full):
    xo, ito = full.oracle_fp64()
    b = dev(full.prob.b)
    x, it, _ = full.gpu.solve(b, rtol=1e-8, force_iters=ito)
    assert it == ito
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-10 * np.linalg.norm(xo)
    assert np.max(np.abs(x.cpu().numpy() - xo)) <= 1e-10 * np.max(np.abs(xo))
    x2, it2, rr2 = full.gpu.solve(b, rtol=1e-8)
    assert abs(it2 - ito) <= 1 and rr2 <= 1e-8


def test_mixed_precision_true_residual(full):
    b = full.prob.b
    x, it, rr = full.gpu.solve(dev(b), rtol=1e-8, precision=1)
    assert rr <= 1e-8
    r_true = b - full.orc.spmv(0, x.cpu().numpy())
    assert np.linalg.norm(r_true) <= 1.5e-8 * np.linalg.norm(b)


def test_fp32_vcycle_and_finest_steps(full):
    rng = np.random.default_rng(21)
    r = rng.standard_normal(full.prob.n)
    z32 = full.gpu.vcycle(dev(r), 1).cpu().numpy()
    zo32 = full.orc.vcycle(r, 1)
    assert np.max(np.abs(z32 - zo32)) <= 1e-5 * np.max(np.abs(zo32))
    form = full.gpu.kernel(0, 1)[1]
    fp32_step_checks(full.orc, full.gpu, full.k, rng, levels=[0], smooth_starts=(None,))
    print(f"{full.name}: FP32 finest-level form {form}")


def test_batch_32_columns(full):
    if full.name != "poisson_24cube_jitter_p4":
        pytest.skip("the 32-RHS batch is the Poisson workload's")
    prob = full.prob
    B = np.stack([prob.rhs("fourier", 1000 + j) for j in range(32)], axis=1)
    sample = (0, 17, 31)
    ref = {j: full.orc.solve(B[:, j], rtol=1e-8) for j in sample}
    N = max(ref[j][1] for j in sample)
    X, it, _ = full.gpu.solve_batch(dev(B), rtol=1e-8, force_iters=N)
    X = X.cpu().numpy()
    for j in sample:
        xo = ref[j][0] if ref[j][1] == N else full.orc.solve(B[:, j], force_iters=N)[0]
        assert np.linalg.norm(X[:, j] - xo) <= 1e-10 * np.linalg.norm(xo), j
    Xm, itm, rrm = full.gpu.solve_batch(dev(B), rtol=1e-8, precision=1)
    Xm = Xm.cpu().numpy()
    assert np.all(rrm <= 1e-8)
    for j in range(32):
        r = B[:, j] - full.orc.spmv(0, Xm[:, j])
        assert np.linalg.norm(r) <= 1.5e-8 * np.linalg.norm(B[:, j]), j


def test_block_32_columns(full):
    if full.name != "poisson_24cube_jitter_p4":
        pytest.skip("the 32-RHS batch is the Poisson workload's")
    prob = full.prob
    B = np.stack([prob.rhs("fourier", 1000 + j) for j in range(32)], axis=1)
    for precision in (1, 0):
        X, it, rr = full.gpu.solve_block(dev(B), rtol=1e-8, precision=precision)
        assert full.gpu.last_status == g.GIAMG_OK and np.all(it == it[0]) and np.all(rr <= 1e-8)
        X = X.cpu().numpy()
        for j in range(32):
            r = B[:, j] - full.orc.spmv(0, X[:, j])
            assert np.linalg.norm(r) <= 1.5e-8 * np.linalg.norm(B[:, j]), (precision, j)
