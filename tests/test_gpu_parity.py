"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same inputs.

Bars (written where they are used):
  hierarchy structure (sizes, row pointers, columns, aggregates, P patterns)   bit-exact
  hierarchy values (A_l, P_l)                                                   1e-12 relative
  level SpMV                                                                    1e-13 of |A||x|
  transfers, smoother, coarse solve, V-cycle (FP64)                             1e-10 relative
  FP32 steps (residual, smoother, restriction, prolongation, coarsest) vs the
    oracle's FP32 steps on the same FP32 inputs, row by row                     the sum of the two
                                       sides' worst-case rounding bounds (tests/fp32_bounds.py)
  V-cycle with FP32 levels vs the oracle's FP32 V-cycle, element by element     1e-5 of max |z|
    (the oracle's own FP32 V-cycle is within 1.6e-6 of max |z| of its FP64 one on these cases)
  PCG with the oracle's iteration count forced                                  x within 1e-10
  PCG stopping freely                                                           iterations +-1
The cases span several tiles and ragged sizes: uniform, jittered and graded meshes, p = 2..8,
a relabelled numbering with per-element index symmetries, and levels with aggregation.
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

CASES = {
    "cube4_p4": dict(n=4, p=4, mesh="uniform", lam=1.0, k=3),
    "jitter8_p2_poisson": dict(n=8, p=2, mesh="jitter", lam=0.0, rhs="fourier", k=2),
    "jitter6_p6": dict(n=6, p=6, mesh="jitter", lam=10.0, k=3),
    "graded345_p8_kappa": dict(n=(3, 4, 5), p=8, mesh="graded", lam=1000.0, kappa=1, k=2),
    "jitter6_p4_relabelled": dict(n=6, p=4, mesh="jitter", lam=1.0, perm_seed=5, sym_seed=6, k=3),
    "jitter12_p2_ragged": dict(n=(12, 11, 13), p=2, mesh="jitter", lam=1.0, k=2),
    "cube2_p3_odd": dict(n=2, p=3, mesh="uniform", lam=1.0, k=3),
    # non-halving p schedules: coarse nodes labelled by their nearest fine nodes
    "jitter4_p5_by_one": dict(n=4, p=5, mesh="jitter", lam=1.0, perm_seed=5, sym_seed=6, k=3, opts=dict(p_schedule=1)),
    "jitter3_p7_by_two": dict(n=3, p=7, mesh="jitter", lam=10.0, k=2, opts=dict(p_schedule=2)),
    # an order-1 input: aggregation levels only, Dirichlet identity rows isolated
    "jitter10_p1": dict(n=10, p=1, mesh="jitter", lam=1.0, k=2),
    # the modal (hierarchical) basis: prefix of modes, injection P
    "jitter4_p4_modal": dict(n=4, p=4, mesh="jitter", lam=1.0, basis="modal", k=3, opts=dict(basis=1)),
    "jitter334_p5_modal_by_one": dict(n=(3, 3, 4), p=5, mesh="jitter", lam=1.0, basis="modal", k=3,
                                      opts=dict(basis=1, p_schedule=1)),
}

_cache = {}


def setup_case(name):
    if name not in _cache:
        cfg = dict(CASES[name])
        k = cfg.pop("k")
        opts = cfg.pop("opts", {})
        prob = fegen.make(**cfg)
        orc = oracle.Hierarchy.from_problem(prob, cheb_degree=k, **opts)
        gpu = g.Solver.from_problem(prob, device=True, cheb_degree=k, **opts)
        _cache[name] = (prob, orc, gpu, k)
    return _cache[name]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()




def host(t):
    return t.cpu().numpy()


@pytest.fixture(scope="module", autouse=True)
def _release():
    yield
    for prob, orc, gpu, k in _cache.values():
        gpu.close()
    _cache.clear()


@pytest.mark.parametrize("name", list(CASES))
def test_hierarchy_structure_bit_exact(name):
    prob, orc, gpu, _ = setup_case(name)
    assert gpu.num_levels == orc.num_levels
    for l in range(orc.num_levels):
        a, b = gpu.level_info(l), orc.level_info(l)
        assert a == b, (l, a, b)
        grp, gci, gv, gagg = gpu.level(l)
        orp, oci, ov, oagg = orc.level(l)
        assert np.array_equal(grp, orp) and np.array_equal(gci, oci), l
        assert np.max(np.abs(gv - ov)) <= 1e-12 * np.max(np.abs(ov)), l
        if oagg is not None:
            assert np.array_equal(gagg, oagg), l
        if b["kind"] != oracle.KIND_COARSEST:
            prp, pci, pv, _ = gpu.prolongation(l)
            qrp, qci, qv, _ = orc.prolongation(l)
            assert np.array_equal(prp, qrp) and np.array_equal(pci, qci), l
            assert np.max(np.abs(pv - qv)) <= 1e-12 * np.max(np.abs(qv)), l


@pytest.mark.parametrize("name", list(CASES))
def test_chebyshev_bounds(name):
    prob, orc, gpu, _ = setup_case(name)
    for l in range(orc.num_levels - 1):
        assert abs(gpu.rho_hat(l) - orc.rho_hat(l)) <= 1e-10 * orc.rho_hat(l)


@pytest.mark.parametrize("name", list(CASES))
def test_level_spmv(name):
    prob, orc, gpu, _ = setup_case(name)
    rng = np.random.default_rng(1)
    for l in range(orc.num_levels):
        n = orc.level_info(l)["n"]
        x = rng.normal(size=n)
        y = host(gpu.spmv(l, dev(x)))
        yo = orc.spmv(l, x)
        rp, ci, v, _ = orc.level(l)
        import scipy.sparse as sp
        absA = sp.csr_matrix((np.abs(v), ci, rp), shape=(n, n))
        scale = absA @ np.abs(x)
        assert np.all(np.abs(y - yo) <= 1e-13 * scale + 1e-300), l


@pytest.mark.parametrize("name", list(CASES))
def test_transfers(name):
    prob, orc, gpu, _ = setup_case(name)
    rng = np.random.default_rng(2)
    for l in range(orc.num_levels - 1):
        info = orc.level_info(l)
        rf = rng.normal(size=info["n"])
        rc = host(gpu.restrict(l, dev(rf)))
        rco = orc.restrict(l, rf)
        assert np.max(np.abs(rc - rco)) <= 1e-12 * np.max(np.abs(rco)), l
        ec = rng.normal(size=info["n_next"])
        xf = rng.normal(size=info["n"])
        xo = host(gpu.prolong(l, dev(ec), dev(xf)))
        xoo = orc.prolong(l, ec, xf)
        assert np.max(np.abs(xo - xoo)) <= 1e-12 * np.max(np.abs(xoo)), l


@pytest.mark.parametrize("name", list(CASES))
def test_smoother_and_coarse_solve(name):
    prob, orc, gpu, _ = setup_case(name)
    rng = np.random.default_rng(3)
    for l in range(orc.num_levels - 1):
        n = orc.level_info(l)["n"]
        b = rng.normal(size=n)
        x0 = rng.normal(size=n)
        for start in (None, x0):
            xg = host(gpu.smooth(l, dev(b), None if start is None else dev(start)))
            xo = orc.cheb(l, b, start)
            assert np.max(np.abs(xg - xo)) <= 1e-10 * np.max(np.abs(xo)), l
    nc = orc.level_info(orc.num_levels - 1)["n"]
    r = rng.normal(size=nc)
    assert np.allclose(host(gpu.coarse_solve(dev(r))), orc.coarse_solve(r), rtol=0, atol=1e-10 * np.abs(orc.coarse_solve(r)).max())


@pytest.mark.parametrize("name", list(CASES))
def test_vcycle(name):
    prob, orc, gpu, _ = setup_case(name)
    rng = np.random.default_rng(4)
    r = rng.normal(size=prob.n)
    z = host(gpu.vcycle(dev(r), 0))
    zo = orc.vcycle(r, 0)
    assert np.linalg.norm(z - zo) <= 1e-10 * np.linalg.norm(zo)
    assert np.max(np.abs(z - zo)) <= 1e-10 * np.max(np.abs(zo))
    z32 = host(gpu.vcycle(dev(r), 1))
    zo32 = orc.vcycle(r, 1)
    assert np.max(np.abs(z32 - zo32)) <= 1e-5 * np.max(np.abs(zo32))


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_steps(name):
    prob, orc, gpu, k = setup_case(name)
    fp32_step_checks(orc, gpu, k, np.random.default_rng(13))


def test_fp64_residual_step():
    prob, orc, gpu, k = setup_case("jitter6_p6")
    rng = np.random.default_rng(14)
    for l in range(orc.num_levels):
        n = orc.level_info(l)["n"]
        b, x = rng.standard_normal(n), rng.standard_normal(n)
        rg, ro = host(gpu.residual(l, dev(b), dev(x))), orc.residual(l, b, x)
        rp, ci, v, _ = orc.level(l)
        import scipy.sparse as sp
        scale = np.abs(b) + sp.csr_matrix((np.abs(v), ci, rp), shape=(n, n)) @ np.abs(x)
        assert np.all(np.abs(rg - ro) <= 1e-13 * scale), l


@pytest.mark.parametrize("name", list(CASES))
def test_pcg_parity(name):
    prob, orc, gpu, _ = setup_case(name)
    b = prob.b
    xo, ito, rro, hist, st = orc.solve(b, rtol=1e-8)
    assert st == "ok"
    x, it, rr = gpu.solve(dev(b), rtol=1e-8, force_iters=ito)
    assert it == ito
    assert np.linalg.norm(host(x) - xo) <= 1e-10 * np.linalg.norm(xo)
    assert np.max(np.abs(host(x) - xo)) <= 1e-10 * np.max(np.abs(xo))
    x2, it2, rr2 = gpu.solve(dev(b), rtol=1e-8)
    assert abs(it2 - ito) <= 1 and rr2 <= 1e-8
    ghist, true_rr = gpu.stats(it2 + 1)
    assert np.allclose(ghist[: min(len(hist), it2 + 1)], hist[: min(len(hist), it2 + 1)], rtol=1e-6, atol=1e-14)
    r_true = b - orc.spmv(0, host(x2))
    assert abs(true_rr - np.linalg.norm(r_true) / np.linalg.norm(b)) <= 1e-6 * true_rr + 1e-15


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_precision_solve(name):
    prob, orc, gpu, _ = setup_case(name)
    b = prob.b
    x, it, rr = gpu.solve(dev(b), rtol=1e-8, precision=1)
    assert rr <= 1e-8
    r_true = b - orc.spmv(0, host(x))
    assert np.linalg.norm(r_true) <= 1.5e-8 * np.linalg.norm(b)
    xo, ito, _, _, _ = orc.solve(b, rtol=1e-8, precision=1)
    assert abs(it - ito) <= 2


def test_solve_is_bitwise_reproducible():
    prob, orc, gpu, _ = setup_case("jitter6_p6")
    b = dev(prob.b)
    x1, i1, _ = gpu.solve(b, rtol=1e-9)
    x2, i2, _ = gpu.solve(b, rtol=1e-9)
    assert i1 == i2 and torch.equal(x1, x2)


def test_host_mode_matches_device_mode():
    prob = fegen.make(3, 4, mesh="jitter", lam=1.0)
    a = g.Solver.from_problem(prob, device=False, coords=True)
    d = g.Solver.from_problem(prob, device=True, coords=True)
    xa, ia, ra = a.solve(prob.b, rtol=1e-9)
    xd, idd, rd = d.solve(dev(prob.b), rtol=1e-9)
    assert ia == idd and np.array_equal(xa, host(xd))
    a.close()
    d.close()


def test_zero_rhs_and_exact_iteration_limit():
    prob, orc, gpu, _ = setup_case("cube2_p3_odd")
    x, it, rr = gpu.solve(dev(np.zeros(prob.n)), rtol=1e-8)
    assert it == 0 and rr == 0.0 and torch.count_nonzero(x) == 0
    capped = g.Solver.from_problem(prob, device=True, max_iter=2)
    x, it, rr = capped.solve(dev(prob.b), rtol=1e-30)
    assert capped.last_status == g.GIAMG_ERR_MAXITER and it == 2 and rr > 0
    capped.close()


def test_errors_are_reported_not_raised_in_c():
    prob = fegen.make(2, 2, lam=1.0)
    # non-uniform orders
    order = np.full(prob.n_elem, 2, np.int32)
    order[1] = 3
    h = __import__("ctypes").c_void_p()
    L = g.lib()
    opt = g.default_options()
    rc = L.giamg_setup(prob.n, g._ptr(prob.row_ptr), g._ptr(prob.col), g._ptr(prob.val), prob.n_elem,
                       g._ptr(prob.elem_dof), g._ptr(order), None, __import__("ctypes").byref(opt), None,
                       __import__("ctypes").byref(h))
    assert rc == g.GIAMG_ERR_ORDER and b"uniform" in L.giamg_last_error()
    # element map pairing dofs of far-apart elements (no Dirichlet rows to excuse the pairs)
    free = fegen.make(2, 2, lam=1.0, dirichlet=False)
    bad = free.elem_dof.copy()
    bad[0, 0], bad[-1, -1] = bad[-1, -1], bad[0, 0]
    with pytest.raises(g.GiamgError) as e:
        g.Solver(free.n, free.row_ptr, free.col, free.val, bad, 2)
    assert e.value.code == g.GIAMG_ERR_MAP
    # the count reported: node pairs of one element missing from A's pattern, counted on the host
    import scipy.sparse as sp
    pat = sp.csr_matrix((np.ones(len(free.col)), free.col, free.row_ptr), shape=(free.n, free.n))
    missing = sum(int(bad.shape[1] ** 2 - pat[ids][:, ids].nnz) for ids in bad)
    assert missing > 0 and f": {missing} entries" in str(e.value), (missing, str(e.value))
    # out-of-range map entry
    bad = prob.elem_dof.copy()
    bad[0, 0] = prob.n + 7
    with pytest.raises(g.GiamgError) as e:
        g.Solver(prob.n, prob.row_ptr, prob.col, prob.val, bad, 2)
    assert e.value.code == g.GIAMG_ERR_MAP
    # not positive definite: flip the sign of the matrix
    with pytest.raises(g.GiamgError) as e:
        g.Solver(prob.n, prob.row_ptr, prob.col, -prob.val, prob.elem_dof, 2)
    assert e.value.code == g.GIAMG_ERR_NOT_SPD
    # coordinates that are not the element's GLL image
    c = prob.coords.copy()
    c[prob.elem_dof[0, 13]] += 0.01
    with pytest.raises(g.GiamgError) as e:
        g.Solver(prob.n, prob.row_ptr, prob.col, prob.val, prob.elem_dof, 2, coords=c)
    assert e.value.code == g.GIAMG_ERR_MAP
    # unsorted columns
    col = prob.col.copy()
    i = np.flatnonzero(np.diff(prob.row_ptr) > 2)[0]
    s = prob.row_ptr[i]
    col[s], col[s + 1] = col[s + 1], col[s]
    with pytest.raises(g.GiamgError) as e:
        g.Solver(prob.n, prob.row_ptr, col, prob.val, prob.elem_dof, 2)
    assert e.value.code == g.GIAMG_ERR_ARG


def test_strength_threshold_option_runs_and_matches_oracle():
    prob = fegen.make(8, 2, mesh="jitter", lam=0.0, rhs="fourier")
    orc = oracle.Hierarchy.from_problem(prob, cheb_degree=2, strength_theta=0.05)
    gpu = g.Solver.from_problem(prob, device=True, cheb_degree=2, strength_theta=0.05)
    assert gpu.num_levels == orc.num_levels
    for l in range(orc.num_levels):
        grp, gci, gv, gagg = gpu.level(l)
        orp, oci, ov, oagg = orc.level(l)
        assert np.array_equal(grp, orp) and np.array_equal(gci, oci)
        if oagg is not None:
            assert np.array_equal(gagg, oagg)
    gpu.close()


def test_pattern_compression_matches_plain_csr():
    # the compressed row kernels group the sums differently: agreement to rounding
    prob = fegen.make(6, 6, mesh="jitter", lam=10.0)
    a = g.Solver.from_problem(prob, device=True, compress_patterns=1)
    c = g.Solver.from_problem(prob, device=True, compress_patterns=0)
    assert a.templates(0)[0] > 0 and a.templates(1)[0] > 0 and c.templates(0) == (0, 0)
    b = dev(prob.b)
    for prec in (0, 1):
        xa, ia, _ = a.solve(b, rtol=1e-9, precision=prec, force_iters=8)
        xc, ic, _ = c.solve(b, rtol=1e-9, precision=prec, force_iters=8)
        tol = 1e-10 if prec == 0 else 1e-5
        assert torch.linalg.norm(xa - xc) <= tol * torch.linalg.norm(xc), prec
    a.close()
    c.close()
    # a relabelled numbering repeats no pattern: plain CSR is kept
    rel = fegen.make(6, 4, mesh="jitter", lam=1.0, perm_seed=5)
    r = g.Solver.from_problem(rel, device=True)
    assert r.templates(0) == (0, 0)
    r.close()


_forms_oracle = {}


FORMS = ["csr", "pattern", "groups", "hybrid", "vector", "sliced"]


@pytest.mark.parametrize("form", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("threads", [0, 4, 16])
def test_row_kernel_forms_match_oracle(form, threads):
    # every row-kernel form (CSR, row patterns, row groups, hybrid, vector hybrid, sliced) and
    # thread count on the same problem
    if "p" not in _forms_oracle:
        prob = fegen.make(5, 6, mesh="jitter", lam=10.0)
        _forms_oracle["p"] = (prob, oracle.Hierarchy.from_problem(prob, cheb_degree=3))
    prob, orc = _forms_oracle["p"]
    gpu = g.Solver.from_problem(prob, device=True, cheb_degree=3, row_form=form, row_threads=threads)
    try:
        for prec in (0, 1):
            assert gpu.kernel(0, prec)[1] == FORMS[form - 1]
        rng = np.random.default_rng(7)
        for l in range(orc.num_levels):
            n = orc.level_info(l)["n"]
            x = rng.normal(size=n)
            y, yo = host(gpu.spmv(l, dev(x))), orc.spmv(l, x)
            assert np.max(np.abs(y - yo)) <= 1e-12 * np.max(np.abs(yo)), l
        r = rng.normal(size=prob.n)
        zo = orc.vcycle(r, 0)
        assert np.linalg.norm(host(gpu.vcycle(dev(r), 0)) - zo) <= 1e-10 * np.linalg.norm(zo)
        zo32 = orc.vcycle(r, 1)
        assert np.max(np.abs(host(gpu.vcycle(dev(r), 1)) - zo32)) <= 1e-5 * np.max(np.abs(zo32))
        # the FP32 steps of every row form on the finest level (the form only changes level 0 and
        # the levels large enough for it)
        fp32_step_checks(orc, gpu, 3, np.random.default_rng(8), levels=[0, 1], smooth_starts=(None, "x"))
        xo, ito, _, _, _ = orc.solve(prob.b, rtol=1e-8)
        x, it, _ = gpu.solve(dev(prob.b), rtol=1e-8, force_iters=ito)
        assert np.linalg.norm(host(x) - xo) <= 1e-10 * np.linalg.norm(xo)
        B = np.stack([prob.b, prob.rhs("fourier", 1001)], axis=1)
        X, its, rr = gpu.solve_batch(torch.from_numpy(B).cuda(), rtol=1e-8, force_iters=ito)
        assert np.linalg.norm(X.cpu().numpy()[:, 0] - xo) <= 1e-10 * np.linalg.norm(xo)
    finally:
        gpu.close()


def test_autotuned_forms_match_oracle():
    """autotune = 1 times the finest level's row-kernel candidates inside the solve at setup (the
    hybrid, vector hybrid and sliced forms included) and keeps the fastest per precision; whatever
    it picks matches the oracle."""
    if "p" not in _forms_oracle:
        prob = fegen.make(5, 6, mesh="jitter", lam=10.0)
        _forms_oracle["p"] = (prob, oracle.Hierarchy.from_problem(prob, cheb_degree=3))
    prob, orc = _forms_oracle["p"]
    gpu = g.Solver.from_problem(prob, device=True, cheb_degree=3, autotune=1)
    try:
        for prec in (0, 1):
            assert gpu.kernel(0, prec)[1] in FORMS
        rng = np.random.default_rng(5)
        for l in range(orc.num_levels):
            rp, ci, v, _ = orc.level(l)
            x = rng.normal(size=len(rp) - 1)
            y, yo = host(gpu.spmv(l, dev(x))), orc.spmv(l, x)
            assert np.max(np.abs(y - yo)) <= 1e-12 * np.max(np.abs(yo)), l
            y32 = gpu.spmv32(l, dev(x)).cpu().numpy().astype(np.float64)
            ref, bound = fp32_product_bound(rp, ci, v, x)
            assert np.all(np.abs(y32 - ref) <= bound), l
        xo, ito, _, _, _ = orc.solve(prob.b, rtol=1e-8)
        x, it, _ = gpu.solve(dev(prob.b), rtol=1e-8, force_iters=ito)
        assert np.linalg.norm(host(x) - xo) <= 1e-10 * np.linalg.norm(xo)
        xm, itm, rrm = gpu.solve(dev(prob.b), rtol=1e-8, precision=1)
        assert rrm <= 1e-8
        r = prob.b - orc.spmv(0, host(xm))
        assert np.linalg.norm(r) <= 1.5e-8 * np.linalg.norm(prob.b)
    finally:
        gpu.close()


def test_switching_row_kernels_and_batch_rows_after_setup():
    """giamg_set_row_kernel switches a level's kernel after setup (dropping the captured graphs) and
    giamg_set_batch_rows the multi-RHS FP32 products: every choice matches the oracle, a switch
    back gives the original bits, and the in-solve tuners leave a valid choice set."""
    from paper_2512_15121_gb300 import tune
    if "p" not in _forms_oracle:
        prob = fegen.make(5, 6, mesh="jitter", lam=10.0)
        _forms_oracle["p"] = (prob, oracle.Hierarchy.from_problem(prob, cheb_degree=3))
    prob, orc = _forms_oracle["p"]
    gpu = g.Solver.from_problem(prob, device=True, cheb_degree=3, graphs=2)
    try:
        b = dev(prob.b)
        xo, ito, _, _, _ = orc.solve(prob.b, rtol=1e-8)
        x_ref, _, _ = gpu.solve(b, rtol=1e-8, precision=0, force_iters=ito)
        for form in (1, 2, 3, 4, 5, 6, 0):
            for prec in (0, 1):
                gpu.set_row_kernel(0, prec, form)
            assert gpu.kernel(0, 0)[1] == (FORMS[form - 1] if form else gpu.kernel(0, 0)[1])
            x, it, _ = gpu.solve(b, rtol=1e-8, precision=0, force_iters=ito)
            assert it == ito and np.max(np.abs(host(x) - xo)) <= 1e-10 * np.max(np.abs(xo)), form
            xm, itm, rrm = gpu.solve(b, rtol=1e-8, precision=1)
            assert rrm <= 1e-8, form
        x_back, _, _ = gpu.solve(b, rtol=1e-8, precision=0, force_iters=ito)
        assert torch.equal(x_back, x_ref)  # form 0 again: the setup's own kernels
        with pytest.raises(g.GiamgError):
            gpu.set_row_kernel(0, 0, 7)
        with pytest.raises(g.GiamgError):
            gpu.set_batch_rows(0, 3)
        # multi-RHS FP32 products with one and two rows per item: each column as the oracle's
        B = np.stack([prob.rhs("fourier", 1000 + j) for j in range(20)], axis=1)
        for rows in (1, 2, 0):
            gpu.set_batch_rows(0, rows)
            X, its, rr = gpu.solve_batch(dev(B), rtol=1e-8, precision=1)
            assert np.all(rr <= 1e-8), rows
            for j in (0, 19):
                r = B[:, j] - orc.spmv(0, host(X)[:, j])
                assert np.linalg.norm(r) <= 1.5e-8 * np.linalg.norm(B[:, j]), (rows, j)
        # the in-solve tuners: whatever they keep solves correctly
        best, timings = tune.tune_row_kernels(gpu, b, precision=1, candidates=((0, 0), (2, 8), (6, 0)), reps=1,
                                              warmup=1)
        assert best in ((0, 0), (2, 8), (6, 0)) and len(timings) == 3
        _, _, rr = gpu.solve(b, rtol=1e-8, precision=1)
        assert rr <= 1e-8
        rows, bt = tune.tune_batch_rows(gpu, dev(B), reps=1, warmup=1)
        assert rows in (1, 2) and len(bt) == 2
    finally:
        gpu.close()


def fp32_product_bound(rp, ci, v, x):
    """y = fl32(A) fl32(x) evaluated in FP64 from the FP32-rounded operands (the definition of the
    FP32 product up to the FP32 accumulation), and the bound n_row * 2^-23 * |fl32(A)||fl32(x)|
    on the accumulation error of any summation order."""
    import scipy.sparse as sp
    n = len(rp) - 1
    v32 = v.astype(np.float32).astype(np.float64)
    x32 = x.astype(np.float32).astype(np.float64)
    A32 = sp.csr_matrix((v32, ci, rp), shape=(n, n))
    absA = sp.csr_matrix((np.abs(v32), ci, rp), shape=(n, n))
    lens = np.diff(rp).astype(np.float64)
    return A32 @ x32, (lens + 1) * 2.0 ** -23 * (absA @ np.abs(x32))


@pytest.mark.parametrize("form", [1, 2, 3, 4, 5, 6])
def test_fp32_level_product(form):
    """The FP32 product of every level through the level's FP32 row kernel, against the product of
    the FP32-rounded operands: within the accumulation bound, row by row."""
    if "p" not in _forms_oracle:
        prob = fegen.make(5, 6, mesh="jitter", lam=10.0)
        _forms_oracle["p"] = (prob, oracle.Hierarchy.from_problem(prob, cheb_degree=3))
    prob, orc = _forms_oracle["p"]
    gpu = g.Solver.from_problem(prob, device=True, cheb_degree=3, row_form=form)
    try:
        rng = np.random.default_rng(11)
        for l in range(orc.num_levels):
            rp, ci, v, _ = orc.level(l)
            x = rng.normal(size=len(rp) - 1)
            y = gpu.spmv32(l, dev(x)).cpu().numpy().astype(np.float64)
            ref, bound = fp32_product_bound(rp, ci, v, x)
            assert np.all(np.abs(y - ref) <= bound), l
            assert np.max(np.abs(y - ref)) <= 1e-5 * np.max(np.abs(ref)), l
    finally:
        gpu.close()


@pytest.mark.parametrize("n, p", [(4, 4), (5, 5), (4, 7)])
def test_vector_hybrid_block_sizes_match_oracle(n, p):
    """The FP32 vector hybrid forced on operators whose row groups set other block sizes than the
    p = 6 forms test (5 warps): the block takes 8 warps unless they leave over 5% of the warp-rows
    idle -- 7 warps at p = 4 (interior groups of 27 rows), 8 at p = 5 and 7 (groups of 64 / 16
    and 216 / 36 rows; p = 8 runs the form by default at full size, test_gpu_fullsize.py): the
    finest level's FP32 product against the product of the FP32-rounded operands row by row
    within the accumulation bound, its FP32 residual and smoother steps against the oracle's
    within the rounding bounds, and FP64 PCG with the oracle's iteration count against the
    oracle's solution."""
    prob = fegen.make(n, p, mesh="jitter", lam=10.0)
    orc = oracle.Hierarchy.from_problem(prob, cheb_degree=2)
    gpu = g.Solver.from_problem(prob, device=True, cheb_degree=2, row_form=5)
    try:
        assert gpu.kernel(0, 1)[1] == "vector"
        rng = np.random.default_rng(13)
        rp, ci, v, _ = orc.level(0)
        x = rng.normal(size=len(rp) - 1)
        y = gpu.spmv32(0, dev(x)).cpu().numpy().astype(np.float64)
        ref, bound = fp32_product_bound(rp, ci, v, x)
        assert np.all(np.abs(y - ref) <= bound)
        fp32_step_checks(orc, gpu, 2, rng, levels=[0], smooth_starts=(None, "x"))
        xo, ito, _, _, st = orc.solve(prob.b, rtol=1e-8)
        assert st == "ok"
        xg, it, _ = gpu.solve(dev(prob.b), rtol=1e-8, force_iters=ito, precision=0)
        assert it == ito and np.max(np.abs(host(xg) - xo)) <= 1e-10 * np.max(np.abs(xo))
    finally:
        gpu.close()
        orc.close()
        prob.close()


@pytest.mark.parametrize("name", ["cube4_p4", "jitter8_p2_poisson", "graded345_p8_kappa"])
@pytest.mark.parametrize("precision", [0, 1])
def test_graph_solve_equals_host_loop(name, precision):
    """The solve captured as one CUDA graph (device-side stopping rule) and the host-driven loop give
    the same iterations, relres history and solution bits, and execute the same kernels."""
    prob, orc, _, k = setup_case(name)
    gpu = g.Solver.from_problem(prob, device=True, cheb_degree=k, graphs=2)  # graph from the first solve
    host_loop = g.Solver.from_problem(prob, device=True, cheb_degree=k, graphs=0)
    try:
        b = dev(prob.b)
        for force in (None, 3):
            c0 = g.launch_count()
            xg, itg, rrg = gpu.solve(b, rtol=1e-8, precision=precision, force_iters=force)
            c1 = g.launch_count()
            xh, ith, rrh = host_loop.solve(b, rtol=1e-8, precision=precision, force_iters=force)
            c2 = g.launch_count()
            hg, _ = gpu.stats(itg + 1)
            hh, _ = host_loop.stats(ith + 1)
            assert itg == ith and rrg == rrh and torch.equal(xg, xh)
            assert np.array_equal(hg, hh)
            # the executed kernels: the host loop's plus the graph's start and per-iteration checks
            assert c1 - c0 == (c2 - c1) + 1 + itg
    finally:
        gpu.close()
        host_loop.close()


def test_graph_solve_edge_cases():
    prob, orc, _, k = setup_case("cube4_p4")
    gpu = g.Solver.from_problem(prob, device=True, cheb_degree=k, graphs=2)
    # b = 0: no iteration, x = 0
    x, it, rr = gpu.solve(dev(np.zeros(prob.n)), rtol=1e-8)
    assert it == 0 and rr == 0.0 and torch.count_nonzero(x) == 0
    # the iteration limit: MAXITER reported, x the iterate after max_iter steps (as the host loop)
    lim = g.Solver.from_problem(prob, device=True, cheb_degree=k, max_iter=2, graphs=2)
    ref = g.Solver.from_problem(prob, device=True, cheb_degree=k, max_iter=2, graphs=0)
    try:
        xg, itg, rrg = lim.solve(dev(prob.b), rtol=1e-14)
        xh, ith, rrh = ref.solve(dev(prob.b), rtol=1e-14)
        assert lim.last_status == g.GIAMG_ERR_MAXITER == ref.last_status
        assert itg == ith == 2 and rrg == rrh and torch.equal(xg, xh)
        # more forced iterations than the captured history holds: the host loop takes over
        xf, itf, _ = lim.solve(dev(prob.b), rtol=1e-8, force_iters=4)
        xr, itr, _ = ref.solve(dev(prob.b), rtol=1e-8, force_iters=4)
        assert itf == itr == 4 and torch.equal(xf, xr)
    finally:
        lim.close()
        ref.close()
    # host pointers through the graph path
    gpu.set_device_ptrs(False)
    try:
        xh, ith, _ = gpu.solve(prob.b, rtol=1e-8)
    finally:
        gpu.set_device_ptrs(True)
    xd, itd, _ = gpu.solve(dev(prob.b), rtol=1e-8)
    assert ith == itd and np.array_equal(xh, xd.cpu().numpy())
    gpu.close()


def test_graph_captured_from_the_second_solve():
    """graphs = 1 (default): the first solve of a shape runs the host loop, later ones the graph;
    the launch count shows which ran (the graph adds its start and check kernels)."""
    prob, orc, _, k = setup_case("cube4_p4")
    s = g.Solver.from_problem(prob, device=True, cheb_degree=k)
    try:
        b = dev(prob.b)
        counts = []
        for _ in range(3):
            c0 = g.launch_count()
            x, it, _ = s.solve(b, rtol=1e-8)
            counts.append(g.launch_count() - c0)
        assert counts[1] == counts[2] == counts[0] + 1 + it
    finally:
        s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_set_cheb_degree_equals_fresh_setup(precision):
    """Changing the smoother degree after setup gives the handle a fresh setup with that degree
    would build: same iterations and solution bits (graph path, which is recaptured)."""
    prob, orc, _, k = setup_case("jitter6_p6")
    s = g.Solver.from_problem(prob, device=True, cheb_degree=k, graphs=2)
    try:
        b = dev(prob.b)
        s.solve(b, rtol=1e-8, precision=precision)  # a graph of the old degree exists
        for deg in (1, 2, 5):
            s.set_cheb_degree(deg)
            x, it, rr = s.solve(b, rtol=1e-8, precision=precision)
            fresh = g.Solver.from_problem(prob, device=True, cheb_degree=deg, graphs=2)
            try:
                xf, itf, rrf = fresh.solve(b, rtol=1e-8, precision=precision)
            finally:
                fresh.close()
            assert it == itf and rr == rrf and torch.equal(x, xf), deg
    finally:
        s.close()


def test_set_cheb_degree_matches_oracle_and_errors():
    prob, orc, _, k = setup_case("cube4_p4")
    s = g.Solver.from_problem(prob, device=True, cheb_degree=k)
    try:
        s.set_cheb_degree(5)
        o5 = oracle.Hierarchy.from_problem(prob, cheb_degree=5)
        try:
            xo, ito, _, _, _ = o5.solve(prob.b, rtol=1e-8)
        finally:
            o5.close()
        x, it, _ = s.solve(dev(prob.b), rtol=1e-8, force_iters=ito)
        assert np.linalg.norm(host(x) - xo) <= 1e-10 * np.linalg.norm(xo)
        with pytest.raises(g.GiamgError):
            s.set_cheb_degree(0)
    finally:
        s.close()


def test_tune_cheb_degree():
    from paper_2512_15121_gb300 import tune
    prob, orc, _, k = setup_case("jitter6_p6")
    s = g.Solver.from_problem(prob, device=True, cheb_degree=k)
    try:
        best, timings = tune.tune_cheb_degree(s, dev(prob.b), degrees=(1, 2, 3), reps=2, warmup=1)
        assert best in (1, 2, 3) and [t.degree for t in timings] == [1, 2, 3]
        assert all(t.ms > 0 and t.iterations > 0 for t in timings)
        chosen = next(t for t in timings if t.degree == best)
        assert chosen.relres <= 1e-8 and chosen.ms == min(t.ms for t in timings if t.relres <= 1e-8)
        assert s.opts.cheb_degree == best
        # fewer iterations with a higher degree (the polynomial smooths more per V-cycle)
        assert timings[2].iterations <= timings[0].iterations
    finally:
        s.close()


def test_async_solve_equals_the_synchronous_graph_solve():
    """giamg_solve_async enqueues the captured solve with no host round trip; its results, read
    after a stream synchronisation, are those of giamg_solve bit for bit."""
    prob, orc, _, k = setup_case("cube4_p4")
    gpu = g.Solver.from_problem(prob, device=True, cheb_degree=k, graphs=2)
    lim = g.Solver.from_problem(prob, device=True, cheb_degree=k, graphs=2, max_iter=2)
    try:
        b = dev(prob.b)
        b2 = dev(prob.rhs("fourier", 77))
        for precision in (0, 1):
            x, it, rr = gpu.solve(b, rtol=1e-8, precision=precision)
            x2, it2, rr2 = gpu.solve(b2, rtol=1e-8, precision=precision)
            # two solves queued back to back, then one synchronisation
            ya, ita, rra, sta = gpu.solve_async(b, rtol=1e-8, precision=precision)
            yb, itb, rrb, stb = gpu.solve_async(b2, rtol=1e-8, precision=precision)
            torch.cuda.synchronize()
            assert torch.equal(ya, x) and int(ita) == it and float(rra) == rr and int(sta) == g.GIAMG_OK
            assert torch.equal(yb, x2) and int(itb) == it2 and float(rrb) == rr2 and int(stb) == g.GIAMG_OK
        _, tr = gpu.stats(0)
        assert tr <= 1.5e-8
        # b = 0: no iteration
        z, itz, rrz, stz = gpu.solve_async(dev(np.zeros(prob.n)), rtol=1e-8)
        torch.cuda.synchronize()
        assert int(itz) == 0 and float(rrz) == 0.0 and int(stz) == g.GIAMG_OK and torch.count_nonzero(z) == 0
        # the iteration limit: MAXITER on the device, as giamg_solve reports it
        xl, itl, rrl = lim.solve(b, rtol=1e-14)
        za, ita, rra, sta = lim.solve_async(b, rtol=1e-14)
        torch.cuda.synchronize()
        assert lim.last_status == g.GIAMG_ERR_MAXITER == int(sta) and int(ita) == itl == 2
        assert torch.equal(za, xl) and float(rra) == rrl
    finally:
        gpu.close()
        lim.close()
    # host arrays or the host loop: refused
    host_mode = g.Solver.from_problem(prob, device=False, cheb_degree=k)
    loop = g.Solver.from_problem(prob, device=True, cheb_degree=k, graphs=0)
    try:
        with pytest.raises(g.GiamgError):
            host_mode.solve_async(torch.zeros(prob.n, dtype=torch.float64, device="cuda"))
        with pytest.raises(g.GiamgError):
            loop.solve_async(dev(prob.b))
    finally:
        host_mode.close()
        loop.close()
