"""Pins for the synthetic input generator (the assembled FE systems both sides consume).

The generator stands in for the paper's FE library (Sec. 2).  These checks tie its output to
mathematics that fixes it independently of the code: the nonzero count of the tensor-product
pattern, exact symmetry, zero row sums of the pure Laplacian, the mass matrix integrating to
the cube's volume, O(h^{p+1}) convergence to the manufactured solution of Sec. 3.1, the
Gauss-Legendre rule's exactness degree and remainder, the patch test on distorted elements, and
closed-form moments of the Fourier load.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as sla

import fegen


@pytest.mark.parametrize("n", range(1, 13))
def test_gauss_legendre_rule(n):
    """The n-point rule of the assembly: numpy's Gauss-Legendre nodes and weights, exact on the
    monomials of degree <= 2n - 1, and on x^(2n) off by exactly the Gauss remainder
    2^(2n+1) (n!)^4 / ((2n+1) ((2n)!)^2), which no rule of other points or degree has."""
    x, w = fegen.gauss_rule(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.max(np.abs(x - xr)) <= 1e-14 and np.max(np.abs(w - wr)) <= 1e-14
    for k in range(2 * n):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.dot(w, x ** k) - exact) <= 1e-14
    k = 2 * n
    rem = 2.0 ** (2 * n + 1) * math.factorial(n) ** 4 / ((2 * n + 1) * math.factorial(2 * n) ** 2)
    assert abs((2.0 / (k + 1) - np.dot(w, x ** k)) - rem) <= 1e-6 * rem


def _nnz_formula(n, p):
    nnz1 = n * (p + 1) ** 2 - (n - 1)
    # drop the rows and columns of the two end nodes; they share an element when n = 1
    inner = nnz1 - 4 * (p + 1) + 2 if n > 1 else (p - 1) ** 2
    N1 = n * p + 1
    return inner ** 3 + (N1 ** 3 - (N1 - 2) ** 3)


@pytest.mark.parametrize("n,p", [(1, 2), (2, 3), (3, 4), (4, 4), (2, 6)])
def test_pattern_size_matches_tensor_formula(n, p):
    P = fegen.make(n, p, with_values=False, rhs="none")
    assert P.n == (n * p + 1) ** 3
    assert P.nnz == _nnz_formula(n, p)
    # boundary rows keep only their diagonal
    bnd = np.flatnonzero(P.boundary)
    assert np.all(np.diff(P.row_ptr)[bnd] == 1)
    assert np.all(P.col[P.row_ptr[bnd]] == bnd)


def test_c1_nonzero_count():
    P = fegen.make(4, 4, with_values=False, rhs="none")
    assert (P.n, P.nnz) == (4913, 494577)


@pytest.mark.parametrize("mesh", ["uniform", "jitter", "graded"])
def test_exact_symmetry_and_sorted_columns(mesh):
    P = fegen.make(3, 3, mesh=mesh, lam=2.0, kappa=1)
    A = P.scipy()
    assert (A - A.T).count_nonzero() == 0
    for i in range(P.n):
        c = P.col[P.row_ptr[i]:P.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)


@pytest.mark.parametrize("mesh", ["uniform", "jitter"])
def test_laplacian_rows_sum_to_zero(mesh):
    P = fegen.make(3, 4, mesh=mesh, lam=0.0, dirichlet=False, rhs="none")
    A = P.scipy()
    rs = np.asarray(A.sum(axis=1)).ravel()
    assert np.max(np.abs(rs)) <= 1e-12 * np.max(np.abs(P.val))


@pytest.mark.parametrize("mesh", ["uniform", "jitter", "graded"])
def test_mass_matrix_integrates_volume(mesh):
    P = fegen.make(3, 3, mesh=mesh, lam=1.0, kappa=2, dirichlet=False, rhs="none")
    assert abs(P.val.sum() - 1.0) < 1e-12


def test_dense_solve_matches_sparse_direct():
    P = fegen.make(2, 3, mesh="jitter", lam=1.0)
    x = sla.spsolve(P.scipy().tocsc(), P.b)
    xd = np.linalg.solve(P.scipy().toarray(), P.b)
    assert np.linalg.norm(x - xd) <= 1e-12 * np.linalg.norm(xd)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_convergence_rate_to_manufactured_solution(p):
    errs, hs = [], []
    for n in ([4, 8] if p <= 2 else [2, 4]):
        P = fegen.make(n, p, mesh="uniform", lam=1.0)
        x = sla.spsolve(P.scipy().tocsc(), P.b)
        errs.append(P.l2_error(x))
        hs.append(1.0 / n)
    rate = np.log(errs[0] / errs[1]) / np.log(hs[0] / hs[1])
    assert abs(rate - (p + 1)) < 0.3, (p, rate, errs)


def test_variable_coefficient_manufactured_solution():
    errs = []
    for n in [2, 4]:
        P = fegen.make(n, 3, mesh="uniform", lam=1000.0, kappa=1)
        x = sla.spsolve(P.scipy().tocsc(), P.b)
        errs.append(P.l2_error(x))
    assert abs(np.log2(errs[0] / errs[1]) - 4) < 0.4


def test_renumbering_and_element_symmetries_give_the_same_operator():
    base = fegen.make(2, 3, mesh="jitter", lam=1.0)
    perm = fegen.make(2, 3, mesh="jitter", lam=1.0, perm_seed=7, sym_seed=9)
    # map base ids to permuted ids through the coordinates
    key = lambda c: np.lexsort(np.round(c, 12).T[::-1])
    ib, ip = key(base.coords), key(perm.coords)
    pmap = np.empty(base.n, np.int64)
    pmap[ib] = ip
    Ab = base.scipy().toarray()
    Ap = perm.scipy().toarray()
    assert np.array_equal(Ap[np.ix_(pmap, pmap)], Ab)
    assert np.array_equal(perm.b[pmap], base.b)
    # element maps agree as sets per element, and differ in order for some elements
    same_order = 0
    for e in range(base.n_elem):
        assert sorted(pmap[base.elem_dof[e]]) == sorted(perm.elem_dof[e])
        same_order += np.array_equal(pmap[base.elem_dof[e]], perm.elem_dof[e])
    assert same_order < base.n_elem



def test_jittered_mesh_recipe():
    """Jittered meshes: boundary vertices stay on the grid (the cube is kept), every interior
    vertex is moved per coordinate by an independent offset uniform in [-0.2 h, 0.2 h] (so at most
    0.2 h, with mean magnitude 0.1 h and no correlation between the coordinates)."""
    import numpy as np
    n = 8
    P = fegen.make(n, 1, mesh="jitter", rhs="none", with_values=False)
    X = P.coords.reshape(n + 1, n + 1, n + 1, 3)
    grid = np.stack(np.meshgrid(*[np.arange(n + 1) / n] * 3, indexing="ij"), axis=-1)
    off = (X - grid) * n
    bnd = np.zeros((n + 1,) * 3, bool)
    bnd[[0, -1], :, :] = bnd[:, [0, -1], :] = bnd[:, :, [0, -1]] = True
    assert np.all(off[bnd] == 0.0)
    inner = off[~bnd]                                  # (n-1)^3 x 3 offsets in units of h
    assert np.max(np.abs(inner)) <= 0.2
    assert abs(np.mean(np.abs(inner)) - 0.1) < 0.01    # 1029 samples: standard error 0.0018
    for d in range(3):                                 # 343 per coordinate
        assert abs(inner[:, d].mean()) < 0.03          # mean 0, standard error 0.0062
        assert abs(inner[:, d].std() - 0.2 / np.sqrt(3.0)) < 0.015
    assert abs(np.corrcoef(inner[:, 0], inner[:, 1])[0, 1]) < 0.15

def test_graded_mesh_aspect_ratio():
    P = fegen.make(12, 1, mesh="graded", rhs="none", with_values=False)
    z = np.unique(np.round(P.coords[:, 2], 12))
    h = np.diff(z)
    assert abs(h[0] - 1.0 / 120.0) < 1e-12
    assert abs(h.sum() - 1.0) < 1e-12
    assert abs(h[1] / h[0] - 1.37618) < 1e-4


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
def test_patch_test_on_jittered_elements(p):
    """Irons' patch test on trilinear (non-affine) elements: a linear field lies in the mapped
    space, and |J| J^-T is a polynomial of degree <= 2 per direction, so the p + 2 Gauss points
    integrate grad(u).grad(phi_i) exactly; integrating by parts, K u vanishes at every node away
    from the domain's boundary.  A wrong metric (J^-T J^-1 for J^-1 J^-T) or a missing
    off-diagonal metric term fails here, though not on the box-shaped elements of a uniform mesh."""
    import numpy as np
    P = fegen.make(3, p, mesh="jitter", lam=0.0, dirichlet=False, rhs="none")
    K = P.scipy()
    X = P.coords
    inner = np.flatnonzero(np.all((X > 1e-12) & (X < 1.0 - 1e-12), axis=1))
    assert len(inner) == (3 * p - 1) ** 3
    scale = abs(K).max()
    for u in (X[:, 0], X[:, 1], X[:, 2], 0.3 * X[:, 0] - 1.1 * X[:, 1] + 0.7 * X[:, 2] + 2.0):
        r = K @ u
        assert np.max(np.abs(r[inner])) <= 1e-13 * scale * np.max(np.abs(u))



@pytest.mark.parametrize("p", [2, 3, 4, 6])
def test_patch_test_modal_basis(p):
    """The patch test in the modal basis: the vertex modes are the trilinear shape functions, so a
    linear field is its vertex values on the vertex modes and zero on every bubble; K u vanishes
    at every mode whose support misses the domain's boundary.  A bubble derivative inconsistent
    with its function (the Jacobi recurrence, the P^(1,1)' = (n+3)/2 P^(2,2) identity) breaks
    the integral of phi' over an element and fails here."""
    import numpy as np
    n = 3
    P = fegen.make(n, p, mesh="jitter", lam=0.0, dirichlet=False, rhs="none", basis="modal")
    K = P.scipy()
    N1 = n * p + 1
    g = np.arange(P.n)
    I, J, L = g // (N1 * N1), (g // N1) % N1, g % N1
    vertex = (I % p == 0) & (J % p == 0) & (L % p == 0)
    inner = (I > 0) & (I < N1 - 1) & (J > 0) & (J < N1 - 1) & (L > 0) & (L < N1 - 1)
    scale = abs(K).max()
    for d in range(3):
        u = np.where(vertex, P.coords[:, d], 0.0)
        assert np.max(np.abs((K @ u)[inner])) <= 1e-13 * scale * np.max(np.abs(u))

@pytest.mark.parametrize("mesh", ["uniform", "jitter"])
def test_fourier_load_moments(mesh):
    """rhs("fourier") loads f = sum c_k sin(k1 pi x) sin(k2 pi y) sin(k3 pi z), k in 1..4, by
    quadrature.  Without Dirichlet rows the basis sums to 1 and reproduces x, so sum_i b_i is the
    integral of f and sum_i b_i x_i that of x f: per direction int_0^1 sin(k pi x) dx =
    (1 - (-1)^k) / (k pi) and int_0^1 x sin(k pi x) dx = (-1)^(k+1) / (k pi).  Fourteen Gauss
    points per direction make the quadrature error negligible."""
    import numpy as np
    P = fegen.make(3, 4, mesh=mesh, lam=1.0, dirichlet=False, nq=14, rhs="none")
    b = P.rhs("fourier", 7)
    c = fegen.fourier_coef(7)
    k = np.arange(1, 5)
    i0 = (1.0 - (-1.0) ** k) / (k * np.pi)
    i1 = (-1.0) ** (k + 1) / (k * np.pi)
    tol = 1e-12 * np.abs(c).sum()
    assert abs(b.sum() - np.einsum("abc,a,b,c->", c, i0, i0, i0)) <= tol
    assert abs(b @ P.coords[:, 0] - np.einsum("abc,a,b,c->", c, i1, i0, i0)) <= tol
    assert abs(b @ P.coords[:, 1] - np.einsum("abc,a,b,c->", c, i0, i1, i0)) <= tol
    assert abs(b @ P.coords[:, 2] - np.einsum("abc,a,b,c->", c, i0, i0, i1)) <= tol

def test_nodal_fourier_rhs():
    """rhs_nodal: the Fourier field at the nodes, zero on Dirichlet rows, seeded; against a direct
    evaluation of the defining sum at a few nodes."""
    import numpy as np
    prob = fegen.make(3, 2, mesh="jitter", lam=1.0, rhs="none")
    f = prob.rhs_nodal(5)
    assert np.array_equal(f, prob.rhs_nodal(5)) and not np.array_equal(f, prob.rhs_nodal(6))
    assert np.all(f[prob.boundary != 0] == 0.0)
    c = np.random.default_rng(5).standard_normal((4, 4, 4))
    for i in np.flatnonzero(prob.boundary == 0)[:5]:
        x, y, z = prob.coords[i]
        ref = sum(c[a, b, d] * np.sin((a + 1) * np.pi * x) * np.sin((b + 1) * np.pi * y) * np.sin((d + 1) * np.pi * z)
                  for a in range(4) for b in range(4) for d in range(4))
        assert abs(f[i] - ref) <= 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("p", [1, 2, 4, 6])
def test_modal_basis_spans_the_nodal_space(p):
    """The hierarchical modes span the same space Q_p as the GLL Lagrange basis, so the Galerkin
    solutions are the same function: the energy x^T b = integral of f u_h and the L2 error of the
    manufactured solution agree between the two discretisations."""
    a = fegen.make(3, p, mesh="jitter", lam=1.0)
    b = fegen.make(3, p, mesh="jitter", lam=1.0, basis="modal")
    xa = sla.spsolve(a.scipy().tocsc(), a.b)
    xb = sla.spsolve(b.scipy().tocsc(), b.b)
    assert abs(xa @ a.b - xb @ b.b) <= 1e-12 * abs(xa @ a.b)
    assert abs(a.l2_error(xa) - b.l2_error(xb)) <= 1e-9 * a.l2_error(xa)
    assert (a.n, a.nnz) == (b.n, b.nnz)


@pytest.mark.parametrize("p,q", [(4, 2), (5, 4), (6, 3), (3, 1)])
def test_modal_operator_is_hierarchical(p, q):
    """The order-q modal operator is the principal submatrix of the order-p one on the modes of
    degree <= q (same quadrature rule): per direction, coarse lattice index e q + i is fine index
    e p + i for i < q and e p + p for i = q."""
    n = 2
    fine = fegen.make(n, p, mesh="jitter", lam=1.0, kappa=1, dirichlet=False, rhs="none", basis="modal")
    coarse = fegen.make(n, q, mesh="jitter", lam=1.0, kappa=1, nq=p + 2, dirichlet=False, rhs="none", basis="modal")
    Nc, Nf = n * q + 1, n * p + 1
    ic = np.arange(Nc)
    # lattice index e q + i (0 <= i < q) of coarse element e, and the last vertex at n q
    e, i = np.minimum(ic // q, n - 1), ic - np.minimum(ic // q, n - 1) * q
    fmap = e * p + np.where(i == q, p, i)
    I, J, K = np.meshgrid(fmap, fmap, fmap, indexing="ij")
    kept = ((I * Nf + J) * Nf + K).ravel()
    Kf = fine.scipy().tocsr()[kept][:, kept].toarray()
    Kc = coarse.scipy().toarray()
    assert np.max(np.abs(Kf - Kc)) <= 1e-12 * np.max(np.abs(Kc))


def test_modal_basis_rejects_element_symmetries():
    with pytest.raises(RuntimeError):
        fegen.make(2, 3, basis="modal", sym_seed=5)
