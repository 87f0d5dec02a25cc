"""Forward error bounds of the FP32 steps of the V-cycle, and the GPU-against-oracle check that uses
them (test helpers: numpy, and torch only inside fp32_step_checks).

Every bound here is a first-order worst-case bound from the standard model of binary32 arithmetic
(round to nearest, unit roundoff u = 2^-24; fused multiply-adds round once and are covered): a
sum of L products computed in any order carries an error of at most (L + 1) u times the sum of the
magnitudes of its terms, and every coefficient rounded from FP64 to FP32 is off by at most u
relative.  They bound the distance of a computed FP32 result from the exact result of the same
step on the same FP32 inputs with the FP64 operator; a difference of two FP32 implementations
(the oracle's and the GPU's) is at most the sum of their two bounds.

A plausible mistake in one kernel -- a wrong coefficient, a dropped term, one mis-indexed element
class -- moves the result by the size of a term, about 1/(L u) = 10^5 times these bounds.
"""
import numpy as np
import scipy.sparse as sp

U = 2.0 ** -24
KIND_P, KIND_COARSEST = 0, 2  # level kinds of giamg_level_info / the oracle


def f32(a):
    """FP32 rounding of a (as float64 values)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def csr(rp, ci, v, ncols):
    n = len(rp) - 1
    return sp.csr_matrix((v, ci, rp), shape=(n, ncols))


def row_lengths(M):
    return np.diff(M.indptr).astype(np.float64)


def residual_bound(A, b, x, depth=0.0):
    """Bound on |fl32(b - A x) - (b - A x)| per row, b and x FP32 inputs, A's FP32 copy rounded
    from the FP64 A: (L_i + 2 + depth) u (|b| + |A||x|) + u |A||x| (the matrix rounding)."""
    Aa = abs(A)
    s = Aa @ np.abs(x)
    L = row_lengths(A)
    return (L + 2.0 + depth) * U * (np.abs(b) + s) + U * s


def product_bound(M, v, depth=0.0, entry_roundings=1.0):
    """Bound on |fl32(M v) - M v| per row for an FP32 input v: (L_i + 1 + depth) u |M||v| for the
    accumulation plus entry_roundings * u |M||v| for M's FP32 entries (one rounding each, or more
    where an entry is formed from several rounded factors)."""
    s = abs(M) @ np.abs(v)
    return (row_lengths(M) + 1.0 + depth + entry_roundings) * U * s


def cheb_bound(A, dinv, c1, c2, b, x0=None):
    """Bound on |x_computed - x_exact| after the Chebyshev smoother's steps (the recurrence of Saad's
    Algorithm 12.1 with the Jacobi preconditioner, coefficients c1[s], c2[s]): the error of every
    step propagated through the next ones.

    Per step s with r = b - A x:  d_s = c1[s] d_{s-1} + c2[s] D^-1 r,  x_s = x_{s-1} + d_s.
    The computed x carries E_x, d carries E_d; the residual of the next step inherits |A| E_x plus
    its own accumulation error; the FP32 coefficients c1, c2 and D^-1 are each off by u (plus the
    1e-10 relative by which two Lanczos estimates may differ), the products and the sum round once
    each.  Magnitudes come from the same recurrence in FP64, widened by the error bound itself."""
    Aa = abs(A)
    L = row_lengths(A)
    n = A.shape[0]
    b = np.asarray(b, np.float64)
    zero = x0 is None
    x = np.zeros(n) if zero else np.asarray(x0, np.float64).copy()
    d = np.zeros(n)
    Ex = np.zeros(n)
    Ed = np.zeros(n)
    ad = np.abs(dinv)
    coef = 1.01 * U  # rounding of a coefficient or of D^-1, and the Lanczos difference
    for s in range(len(c1)):
        if s == 0 and zero:
            r = b.copy()
            Er = np.zeros(n)
        else:
            r = b - A @ x
            ax = Aa @ (np.abs(x) + Ex)
            Er = Aa @ Ex + (L + 2.0) * U * (np.abs(b) + ax) + U * ax
        t1 = c1[s] * d
        t2 = c2[s] * dinv * r
        mag = np.abs(t1) + np.abs(c2[s]) * ad * (np.abs(r) + Er)
        Ed = abs(c1[s]) * Ed + abs(c2[s]) * ad * Er + (3 * coef + 3 * U) * (mag + abs(c1[s]) * Ed)
        d = t1 + t2
        x_new = x + d
        Ex = Ex + Ed + U * (np.abs(x_new) + Ex + Ed)
        x = x_new
    return x, Ex


def cheb_coeffs(rho, k, lo=0.1, hi=1.1):
    """The smoother's coefficients from the Lanczos estimate rho (FP64): step 0 c2 = 1/theta, step
    s >= 1 c1 = rho_s rho_{s-1}, c2 = 2 rho_s / delta, rho_s = 1 / (2 sigma - rho_{s-1})."""
    a, bb = lo * rho, hi * rho
    theta, delta = 0.5 * (bb + a), 0.5 * (bb - a)
    sigma = theta / delta
    rr = 1.0 / sigma
    c1, c2 = [0.0], [1.0 / theta]
    for _ in range(1, k):
        rn = 1.0 / (2.0 * sigma - rr)
        c1.append(rn * rr)
        c2.append(2.0 * rn / delta)
        rr = rn
    return np.array(c1), np.array(c2)


def fp32_step_checks(orc, gpu, k, rng, levels=None, smooth_starts=(None, "x")):
    """Every FP32 step of the V-cycle on the levels given (default all), GPU against oracle on the
    same FP32 inputs: each row within the sum of the two sides' worst-case rounding bounds above,
    and the largest difference within 2e-5 of the largest value (measured FP32 noise is ~1e-6 of
    it).  gpu: a paper_2512_15121_gb300.Solver in device mode; orc: an oracle.Hierarchy."""
    import torch

    def dev32(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()

    def h64(t):
        return t.cpu().numpy().astype(np.float64)

    nl = orc.num_levels
    for l in (range(nl) if levels is None else levels):
        info = orc.level_info(l)
        n = info["n"]
        rp, ci, v, _ = orc.level(l)
        A = csr(rp, ci, v, n)
        b, x = f32(rng.standard_normal(n)), f32(rng.standard_normal(n))
        rg, ro = h64(gpu.residual32(l, dev32(b), dev32(x))), orc.residual32(l, b, x).astype(np.float64)
        assert np.all(np.abs(rg - ro) <= 2 * residual_bound(A, b, x)), ("residual", l)
        assert np.max(np.abs(rg - ro)) <= 2e-5 * np.max(np.abs(ro)), ("residual", l)
        if info["kind"] == KIND_COARSEST:
            zg, zo = h64(gpu.coarse_solve32(dev32(b))), orc.coarse_solve32(b).astype(np.float64)
            # both: A_L^-1 b in FP64 (two algorithms, ~kappa 1e-16 apart) rounded to FP32
            assert np.all(np.abs(zg - zo) <= 2 * U * np.abs(zo) + 1e-10 * np.abs(zo).max()), ("coarsest", l)
            continue
        c1, c2 = cheb_coeffs(orc.rho_hat(l), k)
        dinv = 1.0 / A.diagonal()
        for start in smooth_starts:
            x0 = None if start is None else x
            xg = h64(gpu.smooth32(l, dev32(b), None if x0 is None else dev32(x0)))
            xo = orc.cheb32(l, b, x0).astype(np.float64)
            _, E = cheb_bound(A, dinv, c1, c2, b, x0)
            assert np.all(np.abs(xg - xo) <= 2 * E), ("smoother", l, start)
            assert np.max(np.abs(xg - xo)) <= 2e-5 * np.max(np.abs(xo)), ("smoother", l, start)
        prp, pci, pv, m = orc.prolongation(l)
        P = csr(prp, pci, pv, m)
        R = P.T.tocsr()
        # the GPU's p-level transfers are sum-factorised element contractions (three 1D passes of at
        # most p+1 terms, entries formed from three FP32-rounded 1D values) plus a gather over at
        # most 8 elements; the oracle's are CSR products with FP32 entries
        depth = 3 * (info["order"] + 1) + 8 if info["kind"] == KIND_P else 0
        rcg, rco = h64(gpu.restrict32(l, dev32(b))), orc.restrict32(l, b).astype(np.float64)
        bound = product_bound(R, b, depth=depth, entry_roundings=6) + product_bound(R, b)
        assert np.all(np.abs(rcg - rco) <= bound), ("restrict", l)
        e = f32(rng.standard_normal(m))
        xg = h64(gpu.prolong32(l, dev32(e), dev32(x)))
        xo = orc.prolong32(l, e, x).astype(np.float64)
        s = abs(P) @ np.abs(e)
        bound = product_bound(P, e, depth=depth, entry_roundings=6) + product_bound(P, e) + 2 * U * (np.abs(x) + s)
        assert np.all(np.abs(xg - xo) <= bound), ("prolong", l)
