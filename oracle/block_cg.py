"""Block preconditioned CG for several right-hand sides sharing one Krylov space (oracle).

TEST INFRASTRUCTURE ONLY, like the rest of `oracle/`: plain numpy in FP64, no blocking or
fusion, each step as the method states it.

The method is O'Leary's block conjugate gradient algorithm (D. P. O'Leary, "The block
conjugate gradient algorithm and related methods", Linear Algebra Appl. 29 (1980) 293-322),
preconditioned by M (the GIAMG V-cycle of Algorithm 1), with the m right-hand sides B (n x m)
as one block and X0 = 0:

    R0 = B,  Z0 = M R0,  P0 = Z0
    for k = 0, 1, ...
        Q_k     = A P_k
        G_k     = P_k^T Q_k                       (m x m, symmetric positive semidefinite)
        alpha_k = G_k^+ (P_k^T R_k)
        X_k+1   = X_k + P_k alpha_k
        R_k+1   = R_k - Q_k alpha_k
        stop when every column has ||r_j|| <= rtol ||b_j||
        Z_k+1   = M R_k+1
        beta_k  = -G_k^+ (Q_k^T Z_k+1)
        P_k+1   = Z_k+1 + P_k beta_k

beta_k makes P_k+1 A-conjugate to P_k by construction.  With a fixed symmetric positive definite
M this is O'Leary's beta_k = (Z_k^T R_k)^-1 (Z_k+1^T R_k+1) in exact arithmetic (Q_k = (R_k -
R_k+1) alpha_k^-1 and R_k^T Z_k+1 = 0); it needs no inverse of Z^T R and stays valid when M
changes from one application to the next (an FP32 V-cycle), as the flexible scalar CG does.
For m = 1 it is the scalar PCG of Algorithm 1's outer loop.

G^+ (dependent directions).  Equal or dependent right-hand sides, or a zero column, make G_k
singular.  G^+ y is defined as: S = diag(G)^-1/2, a direction with G_jj <= 0 dropped; G^ = S G S
(its lower triangle); a Cholesky factorisation of G^ taken column by column in index order, in
which a direction whose pivot is <= tau is dropped (its row and column of the factor are zero);
on the kept index set K, G^+ y = S_K (L L^T)^-1 S_K y_K, and zero on the dropped rows.  A dropped
direction lies (to tau) in the span of the kept ones, so the search space is unchanged.
"""
from __future__ import annotations

import numpy as np

# pivot below which a direction of the unit-diagonal Gram matrix counts as dependent
DROP_TOL = 1e-10


def gram_factor(G: np.ndarray, tau: float = DROP_TOL):
    """Scaled Cholesky factor of the symmetric positive semidefinite G with dependent directions
    dropped.  Returns (s, keep, L): s = diag(G)^-1/2 (0 where dropped), keep the kept mask, L the
    lower-triangular factor of S G S on the kept set (zero rows and columns elsewhere)."""
    G = np.asarray(G, dtype=np.float64)
    m = G.shape[0]
    d = np.diag(G).copy()
    keep = np.isfinite(d) & (d > 0.0)
    s = np.zeros(m)
    s[keep] = 1.0 / np.sqrt(d[keep])
    L = np.zeros((m, m))
    for j in range(m):
        if not keep[j]:
            continue
        # G^_jj = s_j G_jj s_j, less the squares of row j of the factor so far
        piv = s[j] * G[j, j] * s[j] - np.dot(L[j, :j], L[j, :j])
        if not (piv > tau):
            keep[j] = False
            s[j] = 0.0
            L[j, :] = 0.0
            continue
        L[j, j] = np.sqrt(piv)
        for i in range(j + 1, m):
            if keep[i]:
                L[i, j] = (s[i] * G[i, j] * s[j] - np.dot(L[i, :j], L[j, :j])) / L[j, j]
    return s, keep, L


def gram_solve(factor, Y: np.ndarray) -> np.ndarray:
    """G^+ Y for the factor of `gram_factor` (Y is m x c)."""
    s, keep, L = factor
    Y = np.asarray(Y, dtype=np.float64)
    m = s.shape[0]
    y = s[:, None] * Y
    z = np.zeros_like(y)
    for j in range(m):  # L z = S y on the kept rows
        if keep[j]:
            z[j] = (y[j] - L[j, :j] @ z[:j]) / L[j, j]
    w = np.zeros_like(y)
    for j in reversed(range(m)):  # L^T w = z
        if keep[j]:
            w[j] = (z[j] - L[j + 1:, j] @ w[j + 1:]) / L[j, j]
    return s[:, None] * w


def block_pcg(apply_A, apply_M, B, rtol: float = 1e-8, max_iter: int = 1000, force_iters: int = 0,
              tau: float = DROP_TOL):
    """Block PCG on the n x m block B.  apply_A and apply_M map an n x m block to an n x m block.

    force_iters > 0 runs exactly that many iterations and ignores rtol.  Returns (X, iters,
    relres, status, ranks): relres per column (||r_j|| / ||b_j||, 0 for a zero column), status
    "ok", "maxiter" or "breakdown", ranks the number of kept directions in each iteration."""
    B = np.array(B, dtype=np.float64, copy=True)
    if B.ndim == 1:
        B = B[:, None]
    n, m = B.shape
    X = np.zeros((n, m))
    R = B.copy()
    bb = np.sum(B * B, axis=0)
    limit = force_iters if force_iters > 0 else max_iter

    def relres(R):
        rr = np.sum(R * R, axis=0)
        return np.where(bb > 0.0, np.sqrt(rr / np.where(bb > 0.0, bb, 1.0)), 0.0)

    def done(R):
        return force_iters <= 0 and bool(np.all(relres(R) <= rtol))

    ranks = []
    if limit <= 0 or done(R):
        return X, 0, relres(R), "ok", ranks
    Z = apply_M(R)
    P = Z.copy()
    it = 0
    while True:
        Q = apply_A(P)
        G = P.T @ Q
        F = gram_factor(G, tau)
        ranks.append(int(np.sum(F[1])))
        alpha = gram_solve(F, P.T @ R)
        X = X + P @ alpha
        R = R - Q @ alpha
        it += 1
        rel = relres(R)
        if not np.all(np.isfinite(rel)) or (ranks[-1] == 0 and not done(R)):
            return X, it, rel, "breakdown", ranks
        if done(R):
            return X, it, rel, "ok", ranks
        if it >= limit:
            return X, it, rel, "ok" if force_iters > 0 else "maxiter", ranks
        Z = apply_M(R)
        beta = -gram_solve(F, Q.T @ Z)
        P = Z + P @ beta
