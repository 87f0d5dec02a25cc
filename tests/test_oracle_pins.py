"""Pins for the CPU oracle: each part is tied to something other than itself.

  GLL nodes        Fig. 1's printed positions, closed forms, numpy's Legendre roots
  P (Alg. 2-4, 7)  partition of unity, exact reproduction of degree-q fields, coincident nodes
  RAP (Sec. 2)     equals the order-q operator assembled directly with the fine rule;
                   on affine meshes also with the coarse level's own (q+2)-point rule;
                   Table 1's 4 levels and 27/343 coarsest level
  SpGEMM           scipy's product (values) and the boolean product (pattern)
  MIS-2 (Sec. 2.5) brute-force greedy MIS of the squared graph; validity; hand-worked path
  hash             SplitMix64's published outputs from state 0
  aggregates       cover, one root each, connected; hand-worked paths (one where the second
                   phase decides between two aggregates)
  SPAI-0           minimiser of ||e_i - m a_i|| row by row
  Lanczos          dense eigenvalues (numpy) within 1%; Ritz bounds, monotone growth, finite
                   termination, one step = the start vector's Rayleigh quotient
  Chebyshev        closed-form damping T_k((theta - mu)/delta) / T_k(theta/delta)
  Cholesky         numpy's factor and solve
  V-cycle (Alg. 1) symmetric as an operator; the FP32 V-cycle applies the FP64 operator to
                   FP32 rounding
  PCG              dense direct solve; Dirichlet entries converge to zero; fewer iterations
                   than Jacobi-preconditioned CG, and nearly independent of the order where
                   Jacobi CG's count grows several times (Fig. 3); thread-count independence; flexible CG
                   follows the standard recurrence to rounding with a fixed V-cycle
  block PCG        m = 1 is the scalar PCG; finite termination; the brute-force energy
                   projection onto the block Krylov space; dependent and zero columns; energy
                   error never above each column's own PCG; the Gram pseudo-inverse
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

import fegen
import oracle
from conftest import read_golden


# ----------------------------------------------------------------------------- 1D rules
def test_gll_nodes_match_fig1():
    g = read_golden("fig1_gll_nodes_p4.txt")
    for p_s, pos in g.items():
        p = int(p_s)
        x = (oracle.gll_nodes(p) + 1.0) / 2.0
        assert np.allclose(x, [float(v) for v in pos], atol=5e-5)


@pytest.mark.parametrize("p", range(1, 13))
def test_gll_nodes_closed_forms_and_legendre_roots(p):
    x = oracle.gll_nodes(p)
    assert x[0] == -1.0 and x[-1] == 1.0
    assert np.all(np.diff(x) > 0)
    assert np.array_equal(x, -x[::-1])
    if p >= 2:
        roots = np.sort(np.polynomial.legendre.Legendre.basis(p).deriv().roots().real)
        assert np.allclose(x[1:-1], roots, atol=1e-14)
    if p == 3:
        assert np.allclose(x[1:3], [-1 / np.sqrt(5), 1 / np.sqrt(5)], atol=1e-15)
    if p == 4:
        assert np.allclose(x[1:4], [-np.sqrt(3 / 7), 0.0, np.sqrt(3 / 7)], atol=1e-15)
    if p % 2 == 0:
        assert x[p // 2] == 0.0


def test_p_schedule():
    assert [oracle.next_order(p) for p in range(1, 11)] == [1, 1, 1, 2, 1, 3, 1, 4, 3, 5]


@pytest.mark.parametrize("p,q", [(2, 1), (4, 2), (6, 3), (8, 4), (3, 1), (9, 3), (12, 6)])
def test_p1d_interpolates_degree_q_polynomials(p, q):
    T = oracle.p1d(p, q)
    xp, xq = oracle.gll_nodes(p), oracle.gll_nodes(q)
    assert np.allclose(T.sum(axis=1), 1.0, atol=1e-14)
    for deg in range(q + 1):
        assert np.allclose(T @ xq ** deg, xp ** deg, atol=1e-13)
    # endpoints interpolate exactly; every other entry of the end rows is an exact zero
    assert T[0, 0] == 1.0 and T[p, q] == 1.0
    assert np.all(T[0, 1:] == 0.0) and np.all(T[p, :q] == 0.0)
    if p % 2 == 0 and q % 2 == 0:
        row = T[p // 2]
        assert row[q // 2] == 1.0 and np.count_nonzero(row) == 1


# ----------------------------------------------------------------------------- hierarchy
def _coarse_coords(prob, H, level):
    """Positions of the order-q nodes of `level` on an affine (uniform) mesh."""
    p = prob.p
    info = H.level_info(level)
    q = info["order"]
    nlc = (q + 1) ** 3
    import ctypes
    l2g = np.empty((prob.n_elem, nlc), np.int32)
    oracle._lib().orc_level_extra(H._h, level, None, oracle._p(l2g))
    xq = oracle.gll_nodes(q)
    X = np.zeros((info["n"], 3))
    n1 = p + 1
    for e in range(prob.n_elem):
        lo = prob.coords[prob.elem_dof[e, 0]]
        hi = prob.coords[prob.elem_dof[e, n1 ** 3 - 1]]
        for b in range(nlc):
            i, j, k = b // (q + 1) ** 2, (b // (q + 1)) % (q + 1), b % (q + 1)
            t = (np.array([xq[i], xq[j], xq[k]]) + 1.0) / 2.0
            X[l2g[e, b]] = lo + t * (hi - lo)
    return X


@pytest.mark.parametrize("n,p", [(2, 4), (3, 6), (2, 8)])
def test_prolongation_reproduces_degree_q_fields(n, p):
    prob = fegen.make(n, p, mesh="uniform", lam=1.0)
    H = oracle.Hierarchy.from_problem(prob)
    q = H.level_info(1)["order"]
    Xc = _coarse_coords(prob, H, 1)
    rp, ci, v, m = H.prolongation(0)
    P = sp.csr_matrix((v, ci, rp), shape=(prob.n, m))
    assert np.allclose(P @ np.ones(m), 1.0, atol=1e-13)
    rng = np.random.default_rng(0)
    for _ in range(3):
        a, b, c = rng.integers(0, q + 1, 3)
        f = lambda X: X[:, 0] ** a * X[:, 1] ** b * X[:, 2] ** c + 0.5 * X[:, 0] ** q
        assert np.max(np.abs(P @ f(Xc) - f(prob.coords))) < 1e-12


def test_prolongation_coincident_nodes_are_unit_rows():
    prob = fegen.make(2, 4, mesh="jitter", lam=1.0)
    H = oracle.Hierarchy.from_problem(prob)
    rp, ci, v, m = H.prolongation(0)
    # fine nodes at coarse node positions of the 4 -> 2 step: every second node per direction
    N1 = 2 * 4 + 1
    I = np.arange(prob.n)
    coinc = ((I // (N1 * N1)) % 2 == 0) & (((I // N1) % N1) % 2 == 0) & ((I % N1) % 2 == 0)
    for i in np.flatnonzero(coinc):
        assert rp[i + 1] - rp[i] == 1 and v[rp[i]] == 1.0


@pytest.mark.parametrize("mesh,p,kappa,lam", [("jitter", 4, 0, 1.0), ("jitter", 6, 1, 10.0),
                                              ("graded", 2, 0, 1000.0), ("uniform", 8, 0, 1.0)])
def test_rap_equals_direct_assembly_with_the_fine_rule(mesh, p, kappa, lam):
    n = 2
    fine = fegen.make(n, p, mesh=mesh, lam=lam, kappa=kappa, dirichlet=False, rhs="none")
    H = oracle.Hierarchy.from_problem(fine, coarse_max=1)
    q = H.level_info(1)["order"]
    direct = fegen.make(n, q, mesh=mesh, lam=lam, kappa=kappa, nq=p + 2, dirichlet=False, rhs="none")
    rp, ci, v, _ = H.level(1)
    Ac = sp.csr_matrix((v, ci, rp), shape=(direct.n, direct.n)).toarray()
    Ad = direct.scipy().toarray()
    assert np.max(np.abs(Ac - Ad)) <= 1e-12 * np.max(np.abs(Ad))



@pytest.mark.parametrize("mesh,p,lam", [("uniform", 4, 1.0), ("uniform", 6, 10.0), ("graded", 8, 1000.0),
                                        ("uniform", 3, 1.0)])
def test_rap_equals_own_rule_assembly_on_affine_meshes(mesh, p, lam):
    """On elements whose map is affine (uniform or z-graded boxes) with constant kappa, the order-q
    stiffness and mass integrands are polynomials of degree <= 2q per direction, which the coarse
    level's own (q+2)-point rule integrates exactly: R A P equals that assembly too."""
    fine = fegen.make(2, p, mesh=mesh, lam=lam, dirichlet=False, rhs="none")
    H = oracle.Hierarchy.from_problem(fine, coarse_max=1)
    q = H.level_info(1)["order"]
    own = fegen.make(2, q, mesh=mesh, lam=lam, dirichlet=False, rhs="none")
    rp, ci, v, _ = H.level(1)
    Ac = sp.csr_matrix((v, ci, rp), shape=(own.n, own.n)).toarray()
    Ad = own.scipy().toarray()
    assert np.max(np.abs(Ac - Ad)) <= 1e-12 * np.max(np.abs(Ad))

def test_rap_interior_block_with_dirichlet():
    fine = fegen.make(3, 4, mesh="jitter", lam=1.0)
    H = oracle.Hierarchy.from_problem(fine, coarse_max=1)
    direct = fegen.make(3, 2, mesh="jitter", lam=1.0, nq=6)
    rp, ci, v, _ = H.level(1)
    Ac = sp.csr_matrix((v, ci, rp), shape=(direct.n, direct.n)).toarray()
    Ad = direct.scipy().toarray()
    inner = np.flatnonzero(direct.boundary == 0)
    blk = np.ix_(inner, inner)
    assert np.max(np.abs(Ac[blk] - Ad[blk])) <= 1e-12 * np.max(np.abs(Ad))


def test_table1_hierarchy():
    g = read_golden("table1_giamg_hierarchy.txt")
    n, p = int(g["elements_per_direction"][0]), int(g["order"][0])
    prob = fegen.make(n, p, lam=float(g["lambda"][0]))
    H = oracle.Hierarchy.from_problem(prob, cheb_degree=int(g["cheb_degree"][0]))
    assert H.num_levels == int(g["levels"][0])
    info = H.level_info(H.num_levels - 1)
    assert info["kind"] == oracle.KIND_COARSEST
    assert info["n"] == int(g["coarsest_rows"][0]) and info["nnz"] == int(g["coarsest_nnz"][0])
    assert [H.level_info(l)["order"] for l in range(H.num_levels)] == [8, 4, 2, 1]


def test_coarse_operators_symmetric_and_hierarchy_sizes_c2_shape():
    # a small mesh of the 16^3 p=6 workload's type, with an aggregation level
    prob = fegen.make(6, 6, mesh="jitter", lam=10.0)
    H = oracle.Hierarchy.from_problem(prob, cheb_degree=3)
    kinds = [H.level_info(l)["kind"] for l in range(H.num_levels)]
    assert kinds[:2] == [oracle.KIND_P, oracle.KIND_P] and kinds[-1] == oracle.KIND_COARSEST
    assert H.level_info(1)["n"] == (6 * 3 + 1) ** 3 and H.level_info(2)["n"] == 7 ** 3
    for l in range(1, H.num_levels):
        rp, ci, v, _ = H.level(l)
        A = sp.csr_matrix((v, ci, rp))
        assert abs(A - A.T).max() <= 1e-13 * abs(A).max()


# ----------------------------------------------------------------------------- SpGEMM
def _rand_csr(n, m, dens, rng):
    A = sp.random(n, m, density=dens, random_state=rng, format="csr")
    A.sort_indices()
    return A


def test_spgemm_matches_scipy_and_boolean_pattern():
    rng = np.random.default_rng(3)
    A, B = _rand_csr(40, 30, 0.15, rng), _rand_csr(30, 25, 0.2, rng)
    C = oracle.spgemm((A.indptr, A.indices, A.data, A.shape[1]), (B.indptr, B.indices, B.data, B.shape[1]))
    rp, ci, v, m = C
    Cs = sp.csr_matrix((v, ci, rp), shape=(40, 25))
    assert np.allclose(Cs.toarray(), (A @ B).toarray(), atol=1e-15)
    Ab, Bb = A.copy(), B.copy()
    Ab.data[:] = 1.0
    Bb.data[:] = 1.0
    pat = (Ab @ Bb).tocsr()
    pat.sort_indices()
    assert np.array_equal(rp, pat.indptr) and np.array_equal(ci, pat.indices)


def test_spgemm_keeps_exact_cancellations():
    # [1 1] x [1; -1] = [0]: the entry is structurally present and stored as 0.0
    A = (np.array([0, 2], np.int64), np.array([0, 1], np.int32), np.array([1.0, 1.0]), 2)
    B = (np.array([0, 1, 2], np.int64), np.array([0, 0], np.int32), np.array([1.0, -1.0]), 1)
    rp, ci, v, m = oracle.spgemm(A, B)
    assert rp.tolist() == [0, 1] and ci.tolist() == [0] and v.tolist() == [0.0]


# ----------------------------------------------------------------------------- MIS-2
def _graph_from_edges(n, edges):
    adj = [set() for _ in range(n)]
    for a, b in edges:
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    rp = np.zeros(n + 1, np.int64)
    ci = []
    for i in range(n):
        nb = sorted(adj[i])
        ci += nb
        rp[i + 1] = rp[i] + len(nb)
    return rp, np.array(ci, np.int32), adj


def _dist(adj, n):
    D = np.full((n, n), 99)
    for s in range(n):
        D[s, s] = 0
        front = [s]
        while front:
            nxt = []
            for u in front:
                for w in adj[u]:
                    if D[s, w] > D[s, u] + 1:
                        D[s, w] = D[s, u] + 1
                        nxt.append(w)
            front = nxt
    return D


def _greedy_mis2(n, adj, prio):
    D = _dist(adj, n)
    chosen = []
    for i in sorted(range(n), key=lambda i: prio[i], reverse=True):
        if all(D[i, j] > 2 for j in chosen):
            chosen.append(i)
    return set(chosen), D



def test_hash_is_the_splitmix64_finaliser():
    """h(i) = upper 32 bits of SplitMix64's output i + 1 from state 0 (published reference
    values, `tests/golden/splitmix64_seed0.txt`); the identity option returns i."""
    g = read_golden("splitmix64_seed0.txt")
    for i, hexval in enumerate(g["outputs"]):
        assert oracle.hash32(i, 0) == int(hexval, 16) >> 32
    assert [oracle.hash32(i, 1) for i in (0, 1, 7, 123456)] == [0, 1, 7, 123456]

def test_mis2_hand_worked_path():
    g = read_golden("mis2_path7.txt")
    n = int(g["n"][0])
    edges = [tuple(map(int, e.split("-"))) for e in g["edges"]]
    rp, ci, _ = _graph_from_edges(n, edges)
    ins, _ = oracle.mis2(rp, ci, hash_kind=1)
    assert sorted(np.flatnonzero(ins).tolist()) == [int(v) for v in g["roots"]]
    agg, na = oracle.aggregate(rp, ci, ins)
    assert agg.tolist() == [int(v) for v in g["aggregates"]] and na == 3



def test_aggregates_hand_worked_second_phase():
    """Two paths whose middle nodes lie at distance 2 from two roots: the second phase of the
    aggregation (Sec. 2.5, smallest phase-1 aggregate id) decides where they go."""
    g = read_golden("aggregates_phase2.txt")
    n = int(g["n"][0])
    edges = [tuple(map(int, e.split("-"))) for e in g["edges"]]
    rp, ci, _ = _graph_from_edges(n, edges)
    ins, rounds = oracle.mis2(rp, ci, hash_kind=1)
    assert sorted(np.flatnonzero(ins).tolist()) == [int(v) for v in g["roots"]]
    assert rounds == int(g["rounds"][0])
    agg, na = oracle.aggregate(rp, ci, ins)
    assert agg.tolist() == [int(v) for v in g["aggregates"]] and na == len(g["roots"])

@pytest.mark.parametrize("seed", range(40))
@pytest.mark.parametrize("hash_kind", [0, 1])
def test_mis2_equals_greedy_on_squared_graph(seed, hash_kind):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 13))
    dens = rng.uniform(0.05, 0.6)
    edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < dens]
    rp, ci, adj = _graph_from_edges(n, edges)
    ins, _ = oracle.mis2(rp, ci, hash_kind=hash_kind)
    prio = [(oracle.hash32(i, hash_kind), i) for i in range(n)]
    greedy, D = _greedy_mis2(n, adj, prio)
    S = set(np.flatnonzero(ins).tolist())
    assert S == greedy
    # validity: distance >= 3 inside the set, every node within distance 2 of the set
    for a in S:
        for b in S:
            assert a == b or D[a, b] >= 3
    for i in range(n):
        assert min(D[i, s] for s in S) <= 2
    # aggregates
    agg, na = oracle.aggregate(rp, ci, ins)
    roots = sorted(S)
    assert na == len(roots)
    for a_id, r in enumerate(roots):
        members = np.flatnonzero(agg == a_id)
        assert r in members
        assert all(D[r, m] <= 2 for m in members)
        # connected: every member reaches the root inside the aggregate
        seen, front = {r}, [r]
        mem = set(members.tolist())
        while front:
            front = [w for u in front for w in adj[u] if w in mem and w not in seen and not seen.add(w)]
        assert seen == mem
    for i in range(n):
        if i not in S and any(j in S for j in adj[i]):
            assert agg[i] == roots.index(next(j for j in adj[i] if j in S))


# ----------------------------------------------------------------------------- SPAI-0
def test_sa_prolongation_spai0_and_constants():
    prob = fegen.make(3, 1, mesh="jitter", lam=0.0, dirichlet=False, rhs="none")
    rp, ci, v = prob.row_ptr, prob.col, prob.val
    grp = np.zeros_like(rp)
    gci = []
    for i in range(prob.n):
        nb = [c for c in ci[rp[i]:rp[i + 1]] if c != i]
        gci += nb
        grp[i + 1] = grp[i] + len(nb)
    ins, _ = oracle.mis2(grp, np.array(gci, np.int32))
    agg, na = oracle.aggregate(grp, np.array(gci, np.int32), ins)
    Prp, Pci, Pv, m = oracle.sa_prolongation(rp, ci, v, agg, na)
    P = sp.csr_matrix((Pv, Pci, Prp), shape=(prob.n, na))
    A = prob.scipy()
    # zero row sums of A: the smoothed prolongation keeps constants exactly (to rounding)
    assert np.allclose(P @ np.ones(na), 1.0, atol=1e-13)
    # the diagonal weights minimise ||e_i - m a_i||_2 row by row (SPAI-0)
    AT = (A @ sp.csr_matrix((np.ones(prob.n), agg, np.arange(prob.n + 1)), shape=(prob.n, na))).toarray()
    Pd = P.toarray()
    checked = 0
    for i in range(0, prob.n, 7):
        j = int(np.argmax(np.abs(AT[i])))
        if abs(AT[i, j]) < 1e-8:
            continue  # the whole row lies in one aggregate: A T has no usable entry
        m_i = ((1.0 if agg[i] == j else 0.0) - Pd[i, j]) / AT[i, j]
        checked += 1
        a = A.getrow(i).toarray().ravel()
        e = np.zeros(prob.n)
        e[i] = 1.0
        f = lambda t: np.linalg.norm(e - t * a)
        assert f(m_i) <= f(m_i * (1 + 1e-6)) and f(m_i) <= f(m_i * (1 - 1e-6))
    assert checked > 3


# ----------------------------------------------------------------------------- smoother
def _dense_level(H, l):
    rp, ci, v, _ = H.level(l)
    return sp.csr_matrix((v, ci, rp)).toarray()


def test_lanczos_estimate_within_one_percent():
    prob = fegen.make(2, 4, mesh="jitter", lam=1.0)
    H = oracle.Hierarchy.from_problem(prob)
    for l in range(H.num_levels - 1):
        A = _dense_level(H, l)
        d = 1.0 / np.sqrt(np.diag(A))
        lam = np.linalg.eigvalsh(d[:, None] * A * d[None, :]).max()
        assert abs(H.rho_hat(l) - lam) <= 0.01 * lam



def test_lanczos_ritz_bounds_finite_termination_and_start_vector():
    """Lanczos on B = D^-1/2 A D^-1/2: the largest Ritz value never exceeds lambda_max(B) and
    grows with the number of steps; with as many steps as rows the Krylov space is the whole
    space and it equals lambda_max(B); after one step it is the Rayleigh quotient of the start
    vector v_i = 1 + (h(i) mod 1024) / 1024."""
    rng = np.random.default_rng(3)
    for n in (5, 12, 20):
        M = rng.normal(size=(n, n))
        A = M @ M.T + n * np.eye(n)
        S = sp.csr_matrix(A)
        d = 1.0 / np.sqrt(np.diag(A))
        lam = np.linalg.eigvalsh(d[:, None] * A * d[None, :]).max()
        assert abs(oracle.lanczos_rho(S.indptr, S.indices, S.data, steps=20) - lam) <= 1e-12 * lam
    n = 300
    A = sp.diags([-np.ones(n - 1), 2.5 + rng.random(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
    Ad = A.toarray()
    d = 1.0 / np.sqrt(np.diag(Ad))
    B = d[:, None] * Ad * d[None, :]
    lam = np.linalg.eigvalsh(B).max()
    prev = 0.0
    for steps in (1, 2, 5, 10, 20, 40):
        r = oracle.lanczos_rho(A.indptr, A.indices, A.data, steps=steps)
        assert prev - 1e-14 <= r <= lam * (1 + 1e-12)
        prev = r
    for kind in (0, 1):
        v = 1.0 + np.array([oracle.hash32(i, kind) % 1024 for i in range(n)]) / 1024.0
        v /= np.linalg.norm(v)
        r1 = oracle.lanczos_rho(A.indptr, A.indices, A.data, steps=1, hash_kind=kind)
        assert abs(r1 - v @ B @ v) <= 1e-13 * abs(r1)

def test_tridiagonal_eigenvalue_by_bisection():
    rng = np.random.default_rng(1)
    for m in [1, 2, 5, 20]:
        a, b = rng.normal(size=m), rng.normal(size=max(m - 1, 1))
        T = np.diag(a) + np.diag(b[:m - 1], 1) + np.diag(b[:m - 1], -1)
        assert abs(oracle.tridiag_max_eig(a, b) - np.linalg.eigvalsh(T).max()) < 1e-12


def test_chebyshev_damping_closed_form():
    prob = fegen.make(2, 2, mesh="jitter", lam=1.0)
    for k in [1, 2, 3, 4]:
        H = oracle.Hierarchy.from_problem(prob, cheb_degree=k)
        A = _dense_level(H, 0)
        D = np.diag(A)
        w, V = np.linalg.eig(A / D[:, None])
        rho = H.rho_hat(0)
        lo, hi = 0.1 * rho, 1.1 * rho
        theta, delta = (hi + lo) / 2, (hi - lo) / 2
        for idx in np.argsort(w.real)[:: max(1, len(w) // 6)]:
            mu, v = w[idx].real, V[:, idx].real
            # error equation: b = 0, x0 = v; after smoothing x = damping * v
            x = H.cheb(0, np.zeros(prob.n), v)
            Tk = lambda t: np.cos(k * np.arccos(t)) if abs(t) <= 1 else np.cosh(k * np.arccosh(abs(t))) * np.sign(t) ** k
            damp = Tk((theta - mu) / delta) / Tk(theta / delta)
            assert np.allclose(x, damp * v, atol=1e-11 * np.abs(v).max())



def test_chebyshev_zero_start_equals_explicit_zero():
    """Presmoothing starts from x = 0 and skips the first product (its residual is b); the general
    branch started from an explicit zero vector computes r = b - A 0 and must give the same x."""
    prob = fegen.make(3, 4, mesh="jitter", lam=1.0)
    rng = np.random.default_rng(4)
    for k in (1, 2, 3):
        H = oracle.Hierarchy.from_problem(prob, cheb_degree=k)
        for l in range(H.num_levels - 1):
            b = rng.standard_normal(H.level_info(l)["n"])
            x_fast = H.cheb(l, b)
            x_full = H.cheb(l, b, np.zeros_like(b))
            assert np.max(np.abs(x_fast - x_full)) <= 1e-14 * np.max(np.abs(x_full))


def test_single_steps_are_their_definitions():
    """The per-step entry points the GPU parity tests compare against: level product y = A_l x,
    restriction r_c = P_l^T r_f, prolongation x_f + P_l e_c, coarsest solve A_L^-1 r (with the
    levels' exported A_l and P_l, themselves pinned above)."""
    prob = fegen.make(4, 4, mesh="jitter", lam=1.0)
    H = oracle.Hierarchy.from_problem(prob, coarse_max=100)
    rng = np.random.default_rng(6)
    assert H.level_info(H.num_levels - 2)["kind"] == oracle.KIND_H
    for l in range(H.num_levels):
        info = H.level_info(l)
        rp, ci, v, _ = H.level(l)
        A = sp.csr_matrix((v, ci, rp), shape=(info["n"], info["n"]))
        x = rng.standard_normal(info["n"])
        assert np.allclose(H.spmv(l, x), A @ x, rtol=0, atol=1e-13 * np.abs(A).sum(axis=1).max() * np.abs(x).max())
        if info["kind"] == oracle.KIND_COARSEST:
            z = H.coarse_solve(x)
            assert np.linalg.norm(z - np.linalg.solve(A.toarray(), x)) <= 1e-10 * np.linalg.norm(z)
            continue
        prp, pci, pv, m = H.prolongation(l)
        P = sp.csr_matrix((pv, pci, prp), shape=(info["n"], m))
        e = rng.standard_normal(m)
        assert np.allclose(H.restrict(l, x), P.T @ x, rtol=1e-13, atol=1e-13 * np.abs(x).max())
        assert np.allclose(H.prolong(l, e, x), x + P @ e, rtol=1e-13, atol=1e-13 * np.abs(e).max())

def test_fp32_single_steps_are_their_definitions():
    """The FP32 steps of the V-cycle (the entry points the GPU's FP32 kernels are compared with):
    each equals its FP64 definition on the same FP32 inputs -- b - A_l x, P_l^T r_f, x_f + P_l e_c,
    and the Chebyshev smoother pinned above -- within the worst-case FP32 rounding bound of
    tests/fp32_bounds.py, row by row; the coarsest step is A_L^-1 r in FP64 rounded to FP32 (one
    unit in the last place).  A wrong coefficient or a dropped term moves a row by the size of a
    term, 10^4 or more times the bound."""
    from fp32_bounds import U, f32, csr, residual_bound, product_bound, cheb_bound, cheb_coeffs
    prob = fegen.make(4, 4, mesh="jitter", lam=1.0)
    for k in (2, 3):
        H = oracle.Hierarchy.from_problem(prob, coarse_max=100, cheb_degree=k)
        rng = np.random.default_rng(16 + k)
        assert H.level_info(H.num_levels - 2)["kind"] == oracle.KIND_H
        for l in range(H.num_levels):
            info = H.level_info(l)
            rp, ci, v, _ = H.level(l)
            A = csr(rp, ci, v, info["n"])
            b, x = f32(rng.standard_normal(info["n"])), f32(rng.standard_normal(info["n"]))
            y = H.spmv32(l, x).astype(np.float64)
            assert np.all(np.abs(y - A @ x) <= product_bound(A, x)), l
            r = H.residual32(l, b, x).astype(np.float64)
            assert np.all(np.abs(r - (b - A @ x)) <= residual_bound(A, b, x)), l
            r64 = H.residual(l, b, x)
            assert np.allclose(r64, b - A @ x, rtol=0, atol=1e-13 * (np.abs(b) + abs(A) @ np.abs(x)).max())
            if info["kind"] == oracle.KIND_COARSEST:
                z = H.coarse_solve32(b).astype(np.float64)
                ze = np.linalg.solve(A.toarray(), b)
                assert np.all(np.abs(z - ze) <= 2 * U * np.abs(ze) + 1e-12 * np.abs(ze).max()), l
                continue
            c1, c2 = cheb_coeffs(H.rho_hat(l), k)
            dinv = 1.0 / A.diagonal()
            for start in (None, x):
                xs = H.cheb32(l, b, start).astype(np.float64)
                xe, E = cheb_bound(A, dinv, c1, c2, b, start)
                assert np.all(np.abs(xs - xe) <= E), (l, start is None)
                # the FP64 smoother on the same inputs: the exact recurrence
                assert np.allclose(H.cheb(l, b, start), xe, rtol=0, atol=1e-12 * np.abs(xe).max())
            prp, pci, pv, m = H.prolongation(l)
            P = csr(prp, pci, pv, m)
            assert np.all(np.abs(H.restrict32(l, b).astype(np.float64) - P.T @ b) <= product_bound(P.T.tocsr(), b)), l
            e = f32(rng.standard_normal(m))
            xf = H.prolong32(l, e, x).astype(np.float64)
            bound = product_bound(P, e) + U * (np.abs(x) + abs(P) @ np.abs(e))
            assert np.all(np.abs(xf - (x + P @ e)) <= bound), l


# ----------------------------------------------------------------------------- coarsest
def test_cholesky_matches_numpy():
    rng = np.random.default_rng(5)
    for n in [1, 3, 50, 200]:
        M = rng.normal(size=(n, n))
        A = M @ M.T + n * np.eye(n)
        L = oracle.cholesky(A)
        assert np.allclose(L, np.linalg.cholesky(A), atol=1e-12 * n)
        b = rng.normal(size=n)
        assert np.allclose(oracle.chol_solve(L, b), np.linalg.solve(A, b), atol=1e-12)
    with pytest.raises(RuntimeError):
        oracle.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))


# ----------------------------------------------------------------------------- V-cycle / PCG
@pytest.mark.parametrize("n,p,mesh,k", [(4, 4, "uniform", 3), (8, 2, "jitter", 2), (3, 6, "jitter", 3)])
def test_vcycle_is_symmetric(n, p, mesh, k):
    prob = fegen.make(n, p, mesh=mesh, lam=1.0)
    H = oracle.Hierarchy.from_problem(prob, cheb_degree=k)
    rng = np.random.default_rng(2)
    u, w = rng.normal(size=prob.n), rng.normal(size=prob.n)
    u[prob.boundary == 1] = 0
    w[prob.boundary == 1] = 0
    a, b = np.dot(H.vcycle(u), w), np.dot(u, H.vcycle(w))
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))


@pytest.mark.parametrize("n,p,mesh", [(4, 4, "jitter"), (8, 2, "uniform"), (3, 6, "jitter")])
def test_fp32_vcycle_is_the_fp64_operator_to_fp32_rounding(n, p, mesh):
    """The FP32 V-cycle (FP32 values, smoother and transfers; coarsest solve in FP64) is the same
    linear operator as the FP64 one, so the two agree to FP32 rounding (unit roundoff 6e-8,
    a few hundred roundings deep): a wrong coefficient in the FP32 smoother or transfer moves
    the result by O(1)."""
    prob = fegen.make(n, p, mesh=mesh, lam=1.0)
    H = oracle.Hierarchy.from_problem(prob)
    rng = np.random.default_rng(5)
    for r in (prob.b, rng.standard_normal(prob.n)):
        z64, z32 = H.vcycle(r, 0), H.vcycle(r, 1)
        assert np.linalg.norm(z32 - z64) <= 1e-5 * np.linalg.norm(z64)

@pytest.mark.parametrize("n,p,mesh,lam", [(2, 2, "uniform", 1.0), (2, 4, "jitter", 10.0), (3, 3, "graded", 1000.0),
                                          (8, 2, "jitter", 0.0)])
def test_pcg_matches_dense_direct_solve(n, p, mesh, lam):
    prob = fegen.make(n, p, mesh=mesh, lam=lam, rhs="fourier", rhs_seed=1001)
    H = oracle.Hierarchy.from_problem(prob)
    x, it, rr, hist, st = H.solve(prob.b, rtol=1e-12)
    assert st == "ok" and rr <= 1e-12
    xd = np.linalg.solve(prob.scipy().toarray(), prob.b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    # Dirichlet entries are not frozen (the coarse correction reaches them through P), but
    # they converge to the exact value 0 with the rest of the solution
    assert np.max(np.abs(x[prob.boundary == 1])) <= 1e-10 * np.max(np.abs(xd))
    assert np.all(np.diff(hist) < 0.5) or it < 3


def test_pcg_beats_jacobi_cg_and_matches_discretisation_error():
    # the paper's qualitative result (Sec. 3.1.2): far fewer iterations than diagonally
    # preconditioned CG on a rough right-hand side
    prob = fegen.make(4, 4, mesh="jitter", lam=1.0, rhs="fourier")
    H = oracle.Hierarchy.from_problem(prob, cheb_degree=3)
    x, it, rr, hist, st = H.solve(prob.b, rtol=1e-10)
    A = prob.scipy()
    count = [0]
    sla.cg(A, prob.b, rtol=1e-10, M=sp.diags(1.0 / A.diagonal()), maxiter=5000,
           callback=lambda _: count.__setitem__(0, count[0] + 1))
    assert it * 5 < count[0]
    # on the manufactured problem the iterate carries the discretisation error of the direct solve
    prob = fegen.make(4, 4, mesh="uniform", lam=1.0)
    H = oracle.Hierarchy.from_problem(prob, cheb_degree=3)
    x = H.solve(prob.b, rtol=1e-10)[0]
    xd = sla.spsolve(prob.scipy().tocsc(), prob.b)
    assert abs(prob.l2_error(x) - prob.l2_error(xd)) <= 1e-6 * prob.l2_error(xd)



def _jacobi_cg_iterations(A, b, rtol):
    d = A.diagonal()
    r = b.copy()
    z = r / d
    p, rz, nb = z.copy(), r @ z, np.linalg.norm(b)
    for k in range(1, 10000):
        q = A @ p
        a = rz / (p @ q)
        r -= a * q
        if np.linalg.norm(r) <= rtol * nb:
            return k
        z = r / d
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return 10000


def test_iterations_nearly_independent_of_order():
    """Sec. 3.1 (Fig. 3): with the halving p schedule the iteration count to a relative residual
    of 1e-6 hardly grows with the order, while Jacobi-preconditioned CG's grows several times
    over the same orders.  Here p = 4..10 on 2^3 jittered elements, p-levels down to order 1
    and a direct solve there (no aggregation)."""
    ours, jac = [], []
    for p in (4, 6, 8, 10):
        prob = fegen.make(2, p, mesh="jitter", lam=1.0)
        H = oracle.Hierarchy.from_problem(prob, coarse_max=100000)
        assert all(H.level_info(l)["kind"] != oracle.KIND_H for l in range(H.num_levels))
        x, it, rr, _, st = H.solve(prob.b, rtol=1e-6)
        assert st == "ok"
        ours.append(it)
        jac.append(_jacobi_cg_iterations(prob.scipy().tocsr(), prob.b, 1e-6))
    assert max(ours) <= 2 * min(ours), ours
    assert max(jac) >= 3 * min(jac), jac
    assert all(a < b for a, b in zip(ours, jac))


def test_iteration_limit_and_zero_right_hand_side():
    """Stopping rules (Sec. 3.1: x0 = 0, relative residual): a limit below the needed count stops
    there with status maxiter and the recursive residual of that iterate, which for an exact
    recurrence is the true one; b = 0 returns x = 0 after no iteration with relres 0."""
    prob = fegen.make(3, 4, mesh="jitter", lam=1.0)
    H = oracle.Hierarchy.from_problem(prob)
    _, it, _, hist, st = H.solve(prob.b, rtol=1e-8)
    assert st == "ok" and it > 3 and hist[0] == 1.0 and np.all(np.diff(hist) < 0)
    x2, it2, rr2, hist2, st2 = H.solve(prob.b, rtol=1e-8, max_iter=2)
    assert (it2, st2) == (2, "maxiter") and rr2 == hist2[-1] == hist[2]
    true = np.linalg.norm(prob.b - prob.scipy() @ x2) / np.linalg.norm(prob.b)
    assert abs(true - rr2) <= 1e-10 * rr2
    x0, it0, rr0, _, st0 = H.solve(np.zeros(prob.n), rtol=1e-8)
    assert (it0, rr0, st0) == (0, 0.0, "ok") and not np.any(x0)

def test_force_iters_and_flexible_cg():
    prob = fegen.make(4, 4, mesh="jitter", lam=1.0)
    H = oracle.Hierarchy.from_problem(prob)
    x, it, rr, hist, st = H.solve(prob.b, rtol=1e-8)
    xf, itf, rrf, _, stf = H.solve(prob.b, force_iters=it + 3)
    assert itf == it + 3 and rrf < rr
    # flexible CG with the same symmetric V-cycle follows PCG to rounding
    xfl, itfl, rrfl, histfl, _ = H.solve(prob.b, rtol=1e-8, flexible=1)
    assert abs(itfl - it) <= 1
    # with a fixed SPD preconditioner <z_{k+1}, r_k> = 0, so the flexible beta equals the
    # standard one in exact arithmetic: the residual histories agree to rounding
    m = min(len(hist), len(histfl))
    assert np.allclose(histfl[:m], hist[:m], rtol=1e-8, atol=0.0)
    # FP32 V-cycle inside FP64 flexible CG reaches the same tolerance
    x32, it32, rr32, _, st32 = H.solve(prob.b, rtol=1e-8, precision=1)
    assert st32 == "ok" and rr32 <= 1e-8
    r_true = prob.b - prob.scipy() @ x32
    assert np.linalg.norm(r_true) <= 2e-8 * np.linalg.norm(prob.b)


def test_hierarchy_invariant_under_renumbering_and_element_symmetries():
    base = fegen.make(6, 2, mesh="jitter", lam=1.0)
    perm = fegen.make(6, 2, mesh="jitter", lam=1.0, perm_seed=11, sym_seed=13)
    Hb = oracle.Hierarchy.from_problem(base)
    Hp = oracle.Hierarchy.from_problem(perm)
    assert Hb.num_levels == Hp.num_levels
    # p-levels are the same operators up to relabelling (compare spectra of level 1)
    for l in range(2):
        ib, ip = Hb.level_info(l), Hp.level_info(l)
        assert (ib["n"], ib["nnz"]) == (ip["n"], ip["nnz"])
    eb = np.linalg.eigvalsh(_dense_level(Hb, 1))
    ep = np.linalg.eigvalsh(_dense_level(Hp, 1))
    assert np.allclose(eb, ep, atol=1e-12 * eb.max())
    # the solutions agree through the relabelling
    xb = Hb.solve(base.b, rtol=1e-11)[0]
    xp = Hp.solve(perm.b, rtol=1e-11)[0]
    key = lambda c: np.lexsort(np.round(c, 12).T[::-1])
    pmap = np.empty(base.n, np.int64)
    pmap[key(base.coords)] = key(perm.coords)
    assert np.allclose(xp[pmap], xb, atol=1e-9 * np.abs(xb).max())


def test_results_do_not_depend_on_thread_count():
    import os
    import subprocess
    import sys
    code = ("import fegen, oracle, numpy as np;"
            "P = fegen.make(6, 2, mesh='jitter', lam=1.0);"
            "H = oracle.Hierarchy.from_problem(P);"
            "x = H.solve(P.b, rtol=1e-10)[0];"
            "print(np.frombuffer(x.tobytes(), np.uint64).sum() % 1000003)")
    outs = []
    for t in ["1", "3"]:
        env = dict(os.environ, OMP_NUM_THREADS=t)
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        r = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        outs.append(r.stdout.strip())
    assert outs[0] == outs[1]


# ----------------------------------------------------------------------------- other p schedules
def test_p_schedules_by_one_and_two():
    assert [oracle.next_order(p, 1) for p in range(1, 9)] == [1, 1, 2, 3, 4, 5, 6, 7]
    assert [oracle.next_order(p, 2) for p in range(1, 9)] == [1, 1, 1, 2, 3, 4, 5, 6]


@pytest.mark.parametrize("p", range(2, 13))
def test_coarse_labels_injective_symmetric_and_exact_for_whole_ratios(p):
    """Labels per direction: whole ratios give r s; otherwise the nearest fine index, both
    neighbours at exactly half way; distinct coarse indices never share a candidate; reflecting
    the edge (s -> q - s) reflects the candidates (a -> p - a)."""
    for q in range(1, p):
        cands = []
        for s in range(q + 1):
            a, tie = oracle.anchor_index(p, q, s)
            c = {a, a + 1} if tie else {a}
            if p % q == 0:
                assert not tie and a == (p // q) * s
            else:
                x = s * p / q
                assert all(abs(ci - x) <= 0.5 for ci in c) and (tie == (abs(x - a) == 0.5))
            cands.append(c)
        assert all(not (cands[s] & cands[t]) for s in range(q + 1) for t in range(s))
        assert all({p - ci for ci in cands[q - s]} == cands[s] for s in range(q + 1))


def _coarse_positions(prob, H, level):
    """Physical position of every (element, coarse local node) of `level`: the trilinear image of
    the order-q GLL point in the element's own local frame (its corners are fine dofs)."""
    p = prob.p
    q = H.level_info(level)["order"]
    nlc = (q + 1) ** 3
    l2g = np.empty((prob.n_elem, nlc), np.int32)
    oracle._lib().orc_level_extra(H._h, level, None, oracle._p(l2g))
    xq = (oracle.gll_nodes(q) + 1.0) / 2.0
    n1 = p + 1
    corners = [(a * p) * n1 * n1 + (b * p) * n1 + (c * p) for a in (0, 1) for b in (0, 1) for c in (0, 1)]
    t = np.arange(nlc)
    u, v, w = xq[t // (q + 1) ** 2], xq[(t // (q + 1)) % (q + 1)], xq[t % (q + 1)]
    wts = np.stack([(u if a else 1 - u) * (v if b else 1 - v) * (w if c else 1 - w)
                    for a in (0, 1) for b in (0, 1) for c in (0, 1)], axis=1)  # nlc x 8
    C = prob.coords[prob.elem_dof[:, corners]]  # n_elem x 8 x 3, the element's local frame
    return l2g, np.einsum("tc,ecd->etd", wts, C)


@pytest.mark.parametrize("p,schedule", [(5, 1), (5, 2), (7, 1), (4, 1), (6, 2)])
def test_coarse_numbering_conforms_under_relabelling_and_symmetries(p, schedule):
    """Every element sharing a coarse dof places it at the same point, and different points get
    different dofs: on a jittered mesh with relabelled global ids and per-element index
    symmetries (reflections and axis permutations of the local order)."""
    # a third level keeps the oracle's dense coarsest factorisation small
    prob = fegen.make(3 if p <= 6 else 2, p, mesh="jitter", lam=1.0, perm_seed=3, sym_seed=4, rhs="none")
    H = oracle.Hierarchy.from_problem(prob, p_schedule=schedule, coarse_max=1, max_levels=3)
    n_c = H.level_info(1)["n"]
    l2g, pos = _coarse_positions(prob, H, 1)
    ref = np.full((n_c, 3), np.nan)
    ref[l2g.ravel()] = pos.reshape(-1, 3)  # one of the copies of each dof
    assert not np.isnan(ref).any()
    assert np.max(np.abs(ref[l2g] - pos)) < 1e-12  # every copy agrees
    assert len({tuple(np.round(x, 10)) for x in ref}) == n_c


@pytest.mark.parametrize("p,schedule", [(5, 1), (5, 2), (7, 1), (3, 1)])
def test_prolongation_reproduces_degree_q_fields_other_schedules(p, schedule):
    """P interpolates order-q fields exactly.  On a jittered (trilinear) mesh a physical field of
    degree d_x, d_y, d_z is a reference field of degree d_x + d_y + d_z per direction, so those with
    that sum <= q are reproduced; on a uniform mesh every field of degree <= q per direction."""
    prob = fegen.make(2, p, mesh="jitter", lam=1.0, sym_seed=2, rhs="none")
    H = oracle.Hierarchy.from_problem(prob, p_schedule=schedule, coarse_max=1, max_levels=3)
    q = H.level_info(1)["order"]
    assert q == oracle.next_order(p, schedule)
    l2g, pos = _coarse_positions(prob, H, 1)
    Xc = np.empty((H.level_info(1)["n"], 3))
    Xc[l2g.ravel()] = pos.reshape(-1, 3)
    rp, ci, v, m = H.prolongation(0)
    P = sp.csr_matrix((v, ci, rp), shape=(prob.n, m))
    assert np.allclose(P @ np.ones(m), 1.0, atol=1e-13)
    for a, b, c in [(1, 0, 0), (0, 1, 1), (1, 1, 1), (2, 0, 1)]:
        if a + b + c > q:
            continue
        f = lambda X: X[:, 0] ** a * X[:, 1] ** b * X[:, 2] ** c
        assert np.max(np.abs(P @ f(Xc) - f(prob.coords))) < 1e-12, (a, b, c)
    uni = fegen.make(2, p, mesh="uniform", lam=1.0, rhs="none")
    Hu = oracle.Hierarchy.from_problem(uni, p_schedule=schedule, coarse_max=1, max_levels=3)
    l2g, pos = _coarse_positions(uni, Hu, 1)
    Xc = np.empty((Hu.level_info(1)["n"], 3))
    Xc[l2g.ravel()] = pos.reshape(-1, 3)
    rp, ci, v, m = Hu.prolongation(0)
    P = sp.csr_matrix((v, ci, rp), shape=(uni.n, m))
    f = lambda X: X[:, 0] ** q * X[:, 1] ** (q - 1) * X[:, 2] + X[:, 2] ** q
    assert np.max(np.abs(P @ f(Xc) - f(uni.coords))) < 1e-12


@pytest.mark.parametrize("mesh,p,schedule,kappa,lam", [("jitter", 5, 1, 0, 1.0), ("jitter", 5, 2, 1, 10.0),
                                                       ("graded", 3, 1, 0, 1000.0), ("uniform", 7, 1, 0, 1.0)])
def test_rap_equals_direct_assembly_other_schedules(mesh, p, schedule, kappa, lam):
    """With p/q not whole the coarse space is still the order-q space on the mesh, so R A P is
    the order-q operator assembled with the fine rule (the labels keep fegen's order)."""
    n = 2
    fine = fegen.make(n, p, mesh=mesh, lam=lam, kappa=kappa, dirichlet=False, rhs="none")
    H = oracle.Hierarchy.from_problem(fine, coarse_max=1, p_schedule=schedule, max_levels=3)
    q = H.level_info(1)["order"]
    direct = fegen.make(n, q, mesh=mesh, lam=lam, kappa=kappa, nq=p + 2, dirichlet=False, rhs="none")
    rp, ci, v, _ = H.level(1)
    Ac = sp.csr_matrix((v, ci, rp), shape=(direct.n, direct.n)).toarray()
    Ad = direct.scipy().toarray()
    assert np.max(np.abs(Ac - Ad)) <= 1e-12 * np.max(np.abs(Ad))


@pytest.mark.parametrize("schedule", [1, 2])
def test_pcg_other_schedules_match_dense_direct_solve(schedule):
    prob = fegen.make(2, 5, mesh="jitter", lam=1.0)
    H = oracle.Hierarchy.from_problem(prob, p_schedule=schedule)
    orders = [H.level_info(l)["order"] for l in range(H.num_levels)]
    assert orders[:2] == [5, oracle.next_order(5, schedule)]
    x, it, rr, _, st = H.solve(prob.b, rtol=1e-10)
    assert st == "ok"
    xd = np.linalg.solve(prob.scipy().toarray(), prob.b)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


# ----------------------------------------------------------------------------- modal basis
def _modal_kept(n, p, q):
    """Fine structured ids of the order-q modes: per direction, coarse lattice index e q + i is
    fine index e p + i for i < q, and e p + p for i = q."""
    ic = np.arange(n * q + 1)
    e = np.minimum(ic // q, n - 1)
    i = ic - e * q
    fmap = e * p + np.where(i == q, p, i)
    Nf = n * p + 1
    I, J, K = np.meshgrid(fmap, fmap, fmap, indexing="ij")
    return ((I * Nf + J) * Nf + K).ravel()


@pytest.mark.parametrize("p,schedule", [(4, 0), (6, 0), (5, 1), (7, 2), (3, 0)])
def test_modal_injection_rap_is_the_principal_submatrix(p, schedule):
    """Modal basis (the paper's setting): Algorithm 2 keeps the prefix of modes of degree <= q,
    Algorithm 7 puts a 1 at each kept mode, so P is a 0/1 selection and R A P is exactly the
    fine operator restricted to the kept modes, which is also the order-q modal operator
    assembled directly with the fine rule."""
    n = 2
    fine = fegen.make(n, p, mesh="jitter", lam=10.0, kappa=1, dirichlet=False, rhs="none", basis="modal")
    H = oracle.Hierarchy.from_problem(fine, basis=1, p_schedule=schedule, coarse_max=1, max_levels=3)
    q = H.level_info(1)["order"]
    assert q == oracle.next_order(p, schedule)
    rp, ci, v, m = H.prolongation(0)
    P = sp.csr_matrix((v, ci, rp), shape=(fine.n, m))
    assert np.all(v == 1.0) and np.all(np.diff(rp) <= 1) and P.nnz == m
    kept = _modal_kept(n, p, q)
    assert np.array_equal(np.sort(P.nonzero()[0]), np.sort(kept))
    rp, ci, v, _ = H.level(1)
    Ac = sp.csr_matrix((v, ci, rp), shape=(m, m)).toarray()
    sub = fine.scipy().tocsr()[kept][:, kept].toarray()
    assert np.array_equal(Ac, sub)  # injection: every entry is one fine entry, no rounding
    direct = fegen.make(n, q, mesh="jitter", lam=10.0, kappa=1, nq=p + 2, dirichlet=False, rhs="none", basis="modal")
    Ad = direct.scipy().toarray()
    assert np.max(np.abs(Ac - Ad)) <= 1e-12 * np.max(np.abs(Ad))


@pytest.mark.parametrize("p", [4, 6])
def test_modal_pcg_matches_dense_solve_and_nodal_energy(p):
    modal = fegen.make(2, p, mesh="jitter", lam=1.0, basis="modal")
    nodal = fegen.make(2, p, mesh="jitter", lam=1.0)
    H = oracle.Hierarchy.from_problem(modal, basis=1)
    x, it, rr, _, st = H.solve(modal.b, rtol=1e-11)
    assert st == "ok"
    A = modal.scipy().toarray()
    assert np.linalg.norm(modal.b - A @ x) <= 1e-10 * np.linalg.norm(modal.b)
    # the modal matrix is worse conditioned than the nodal one: the error is bounded by
    # cond(A) times the residual
    xd = np.linalg.solve(A, modal.b)
    assert np.linalg.norm(x - xd) <= np.linalg.cond(A) * 1e-10 * np.linalg.norm(xd)
    xn = np.linalg.solve(nodal.scipy().toarray(), nodal.b)
    assert abs(x @ modal.b - xn @ nodal.b) <= 1e-10 * abs(xn @ nodal.b)


def test_sa_prolongation_keeps_isolated_rows():
    """A row with no off-diagonal entry (a Dirichlet identity row, its own aggregate) keeps its
    tentative column: SPAI-0's m_i = 1 / a_ii would make it exactly zero and the coarse operator
    singular."""
    A = sp.csr_matrix(np.array([[1.0, 0, 0, 0], [0, 2.0, -1.0, 0], [0, -1.0, 2.0, -1.0], [0, 0, -1.0, 2.0]]))
    agg = np.array([0, 1, 1, 1], np.int32)
    rp, ci, v, _ = oracle.sa_prolongation(A.indptr, A.indices, A.data, agg, 2)
    P = sp.csr_matrix((v, ci, rp), shape=(4, 2)).toarray()
    assert P[0, 0] == 1.0 and P[0, 1] == 0.0
    Ac = P.T @ A.toarray() @ P
    assert np.all(np.linalg.eigvalsh(Ac) > 0)


@pytest.mark.parametrize("n", [8, 12])
def test_order_one_input_with_dirichlet_rows(n):
    """An order-1 system goes straight to aggregation with its Dirichlet identity rows isolated;
    the hierarchy stays definite and PCG matches the direct solve."""
    prob = fegen.make(n, 1, mesh="jitter", lam=1.0)
    H = oracle.Hierarchy.from_problem(prob)
    assert H.level_info(0)["kind"] == oracle.KIND_H
    x, it, rr, _, st = H.solve(prob.b, rtol=1e-10)
    assert st == "ok"
    xd = sla.spsolve(prob.scipy().tocsc(), prob.b)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)



def test_strength_threshold_keeps_only_strong_couplings():
    """Opt-in strength graph (theta > 0): a_ij is kept when |a_ij| >= theta sqrt(a_ii a_jj).  On a
    chain whose couplings alternate between -1 and -0.01 (diagonal 2.02), theta = 0.1 keeps only
    the -1 links, the graph falls into disjoint pairs, and every pair becomes one aggregate
    (roots numbered in ascending order: pair i is aggregate i); theta = 0 keeps the chain."""
    n = 40
    off = np.array([-1.0 if i % 2 == 0 else -0.01 for i in range(n - 1)])
    A = sp.diags([off, np.full(n, 2.02), off], [-1, 0, 1]).tocsr()
    A.sort_indices()
    no_map = np.zeros((0, 1), np.int32)
    H = oracle.Hierarchy(n, A.indptr, A.indices, A.data, no_map, 1, coarse_max=5, strength_theta=0.1)
    agg = H.level(0)[3]
    assert agg.tolist() == (np.arange(n) // 2).tolist() and H.level_info(1)["n"] == n // 2
    H0 = oracle.Hierarchy(n, A.indptr, A.indices, A.data, no_map, 1, coarse_max=5, strength_theta=0.0)
    assert H0.level(0)[3].tolist() != agg.tolist()

# ----------------------------------------------------------------------------- block PCG
# oracle/block_cg.py: O'Leary's block CG with A-conjugate directions and dependent directions
# dropped.  Pins: m = 1 is the scalar PCG; finite termination after n/m steps; the iterate is
# the energy-norm projection onto the block Krylov space (brute force); dependent columns;
# never a larger energy error than the columns' own PCG; the Gram pseudo-inverse.
from oracle.block_cg import block_pcg, gram_factor, gram_solve  # noqa: E402


def _spd(n, cond, rng):
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (Qm * np.geomspace(1.0, cond, n)) @ Qm.T


def test_gram_pseudo_inverse_full_rank_and_singular():
    rng = np.random.default_rng(5)
    G = _spd(12, 1e4, rng)
    Y = rng.standard_normal((12, 5))
    F = gram_factor(G)
    assert F[1].all()
    assert np.allclose(gram_solve(F, Y), np.linalg.solve(G, Y), rtol=0, atol=1e-10 * np.abs(np.linalg.solve(G, Y)).max())
    # rank 4 of 9, with a zero direction: 5 dropped, and G x = y on the range of G
    V = rng.standard_normal((9, 4))
    V = np.insert(V, 2, 0.0, axis=0)[:9]
    G = V @ V.T
    F = gram_factor(G)
    assert F[1].sum() == np.linalg.matrix_rank(G) and not F[1][2]
    y = G @ rng.standard_normal((9, 3))
    assert np.linalg.norm(G @ gram_solve(F, y) - y) <= 1e-10 * np.linalg.norm(y)


def test_block_pcg_one_column_is_the_scalar_pcg():
    prob = fegen.make(4, 4, mesh="jitter", lam=0.0, rhs="fourier", rhs_seed=1001)
    H = oracle.Hierarchy.from_problem(prob, cheb_degree=2)
    b = prob.b
    for precision, tol in ((0, 1e-12), (1, 1e-9)):
        x, it, rr, _, st = H.solve(b, rtol=1e-8, precision=precision)
        X, itb, rrb, stb, ranks = H.solve_block(b[:, None], rtol=1e-8, precision=precision)
        assert st == stb == "ok" and itb == it and ranks == [1] * it
        assert np.linalg.norm(X[:, 0] - x) <= tol * np.linalg.norm(x)
        assert abs(rrb[0] - rr) <= 1e-6 * rr
    x = H.solve(b, force_iters=3)[0]
    X = H.solve_block(b[:, None], force_iters=3)[0]
    assert np.linalg.norm(X[:, 0] - x) <= 1e-12 * np.linalg.norm(x)


@pytest.mark.parametrize("m", [3, 4, 6])
def test_block_pcg_finite_termination(m):
    # the block Krylov space has dimension m k, so n = 24 unknowns are exhausted after 24 / m steps
    rng = np.random.default_rng(m)
    n = 24
    A = _spd(n, 50.0, rng)
    dinv = 1.0 / np.diag(A)
    B = rng.standard_normal((n, m))
    X, it, rr, st, ranks = block_pcg(lambda P: A @ P, lambda R: dinv[:, None] * R, B, force_iters=n // m)
    assert st == "ok" and it == n // m and ranks == [m] * it
    assert np.all(rr <= 1e-9)
    Xd = np.linalg.solve(A, B)
    assert np.linalg.norm(X - Xd) <= 1e-9 * np.linalg.norm(Xd)


def test_block_pcg_is_the_energy_projection_onto_the_block_krylov_space():
    rng = np.random.default_rng(11)
    n, m = 40, 3
    A = _spd(n, 1e3, rng)
    C = rng.standard_normal((n, n))
    M = C @ C.T / n + np.eye(n)  # a fixed SPD preconditioner
    B = rng.standard_normal((n, m))
    Z0 = M @ B
    for k in range(1, 5):
        Xk = block_pcg(lambda P: A @ P, lambda R: M @ R, B, force_iters=k)[0]
        # span{Z0, (MA) Z0, ..., (MA)^(k-1) Z0}, orthonormalised; X = K (K^T A K)^-1 K^T B
        blocks, W = [], Z0
        for _ in range(k):
            blocks.append(W)
            W = M @ (A @ W)
        K, _ = np.linalg.qr(np.hstack(blocks))
        Xs = K @ np.linalg.solve(K.T @ A @ K, K.T @ B)
        assert np.linalg.norm(Xk - Xs) <= 1e-9 * np.linalg.norm(Xs), k


def test_block_pcg_dependent_and_zero_columns():
    prob = fegen.make(4, 4, mesh="jitter", lam=0.0)
    H = oracle.Hierarchy.from_problem(prob, cheb_degree=2)
    b0, b1, b2 = (prob.rhs("fourier", s) for s in (7, 8, 9))
    B = np.stack([b0, b1, b0, np.zeros_like(b0), b0 + 2.0 * b1, b2], axis=1)
    X, it, rr, st, ranks = H.solve_block(B, rtol=1e-8)
    assert st == "ok" and np.all(rr <= 1e-8) and max(ranks) == 3
    X3, it3, _, _, _ = H.solve_block(B[:, [0, 1, 5]], rtol=1e-8)
    assert it == it3
    scale = np.linalg.norm(X3)
    assert np.linalg.norm(X[:, [0, 1, 5]] - X3) <= 1e-10 * scale
    assert np.linalg.norm(X[:, 2] - X[:, 0]) <= 1e-10 * scale
    assert np.all(X[:, 3] == 0.0) and rr[3] == 0.0
    assert np.linalg.norm(X[:, 4] - X[:, 0] - 2.0 * X[:, 1]) <= 1e-10 * scale
    # all columns zero: nothing to do
    Xz, itz, rrz, stz, _ = H.solve_block(np.zeros((prob.n, 2)))
    assert itz == 0 and stz == "ok" and np.all(Xz == 0.0)


def test_block_pcg_energy_error_never_above_the_columns_own_pcg():
    # the block space contains each column's own Krylov space (fixed symmetric V-cycle)
    prob = fegen.make(4, 4, mesh="jitter", lam=0.0)
    H = oracle.Hierarchy.from_problem(prob, cheb_degree=2)
    A = prob.scipy().tocsc()
    B = np.stack([prob.rhs("fourier", 20 + j) for j in range(8)], axis=1)
    Xd = np.stack([sla.spsolve(A, B[:, j]) for j in range(8)], axis=1)

    def energy(E):
        return np.sqrt(np.einsum("ij,ij->j", E, A @ E))

    for k in range(1, 7):
        eb = energy(H.solve_block(B, force_iters=k)[0] - Xd)
        es = energy(np.stack([H.solve(B[:, j], force_iters=k)[0] for j in range(8)], axis=1) - Xd)
        assert np.all(eb <= es * (1 + 1e-8) + 1e-12 * energy(Xd)), k
