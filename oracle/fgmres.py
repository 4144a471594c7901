"""Right-preconditioned flexible GMRES(m) (oracle; test infrastructure).

Sec. 5 solves every system by GMRES preconditioned with ORAS; the side, restart
length and tolerance are not stated there.  Reading used here: right
preconditioning in the flexible form (Z_m basis kept, x = x0 + Z_m y), x0 = 0,
Hermitian inner product, modified Gram-Schmidt Arnoldi, complex Givens rotations
for the Hessenberg least-squares problem.  A cycle ends when the estimated
relative residual |g_{j+1}| / ||b|| <= tol or after m steps; the true residual
||b - A x|| / ||b|| is then recomputed in FP64 and the method restarts if it is
above tol.  Multiple right-hand sides are independent recurrences (the
pseudo-block method of Sec. 5 fuses only their arithmetic); block_fgmres() below
is the Block GMRES that Sec. 6 names for them.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla


@dataclass
class Result:
    x: np.ndarray
    iterations: int
    relres: float
    converged: bool


def givens(a, b):
    """c (real), s (complex) with [c s; -conj(s) c] [a; b] = [rho; 0]."""
    aa, bb = abs(a), abs(b)
    if bb == 0.0:
        return 1.0, 0.0j
    if aa == 0.0:
        return 0.0, np.conj(b) / bb
    den = np.hypot(aa, bb)
    return aa / den, (a / aa) * np.conj(b) / den


def fgmres(matvec, precond, b, tol=1e-8, m=50, max_iter=5000) -> Result:
    b = np.asarray(b, dtype=np.complex128)
    n = b.size
    x = np.zeros(n, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return Result(x, 0, 0.0, True)
    it = 0
    r = b.copy()
    while True:
        beta = np.linalg.norm(r)
        if beta / bnorm <= tol:
            return Result(x, it, beta / bnorm, True)
        if it >= max_iter:
            return Result(x, it, beta / bnorm, False)
        V = np.zeros((m + 1, n), dtype=np.complex128)
        Z = np.zeros((m, n), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            Z[j] = precond(V[j])
            w = matvec(Z[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j] = givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k = j + 1
            if abs(g[j + 1]) / bnorm <= tol or it >= max_iter:
                break
        y = sla.solve_triangular(H[:k, :k], g[:k])
        x = x + Z[:k].T @ y
        r = b - matvec(x)


# ---------------------------------------------------------------------------------------------
# Block flexible GMRES (Sec. 6 names Block GMRES for the several right-hand sides of one system;
# the paper prints no algorithm).  Reading used here: the block analogue of fgmres() above with
# the p right-hand sides as one block, x0 = 0, block modified Gram-Schmidt against the earlier
# blocks, each new block orthonormalised by CholQR2, the block Hessenberg least-squares problem
# min ||E1 S - Hbar Y||_F solved per iteration by a library least-squares routine, a cycle ending
# when every column's estimated relative residual is <= tol (or after m block steps), then true
# FP64 residuals per column and a restart if any column is above tol.


class BlockBreakdown(RuntimeError):
    """The new block is (numerically) rank deficient: CholQR2 cannot factor it."""


def cholqr2(W):
    """W = Q C with Q^H Q = I (Cholesky QR applied twice).  W: n x p; C: p x p upper."""
    def cholqr(X):
        G = X.conj().T @ X
        try:
            Lc = np.linalg.cholesky(G)       # G = Lc Lc^H
        except np.linalg.LinAlgError as e:
            raise BlockBreakdown(str(e)) from None
        C = Lc.conj().T                      # G = C^H C, C upper triangular
        Q = sla.solve_triangular(C, X.conj().T, trans="C", lower=False).conj().T   # X C^{-1}
        return Q, C
    Q1, C1 = cholqr(W)
    Q, C2 = cholqr(Q1)
    return Q, C2 @ C1


@dataclass
class BlockResult:
    x: np.ndarray            # n x p
    iterations: int          # block steps
    relres: np.ndarray       # p true relative residuals
    converged: bool


def block_fgmres(matvec, precond, B, tol=1e-8, m=50, max_iter=5000) -> BlockResult:
    """matvec / precond act on one vector; B: n x p."""
    B = np.asarray(B, dtype=np.complex128)
    if B.ndim == 1:
        B = B[:, None]
    n, p = B.shape
    X = np.zeros((n, p), dtype=np.complex128)
    bnorm = np.linalg.norm(B, axis=0)
    bnorm = np.where(bnorm == 0.0, 1.0, bnorm)
    apply_cols = lambda f, Y: np.stack([f(Y[:, c]) for c in range(Y.shape[1])], axis=1)
    it = 0
    R = B.copy()
    while True:
        rel = np.linalg.norm(R, axis=0) / bnorm
        if np.all(rel <= tol):
            return BlockResult(X, it, rel, True)
        if it >= max_iter:
            return BlockResult(X, it, rel, False)
        V0, S = cholqr2(R)
        V = [V0]
        Z = []
        H = np.zeros(((m + 1) * p, m * p), dtype=np.complex128)
        E1S = np.zeros(((m + 1) * p, p), dtype=np.complex128)
        E1S[:p] = S
        k = 0
        Y = None
        for j in range(m):
            Z.append(apply_cols(precond, V[j]))
            W = apply_cols(matvec, Z[j])
            for i in range(j + 1):
                Hij = V[i].conj().T @ W
                H[i * p:(i + 1) * p, j * p:(j + 1) * p] = Hij
                W = W - V[i] @ Hij
            Vn, Hn = cholqr2(W)
            H[(j + 1) * p:(j + 2) * p, j * p:(j + 1) * p] = Hn
            V.append(Vn)
            it += 1
            k = j + 1
            Hk = H[:(k + 1) * p, :k * p]
            Y = np.linalg.lstsq(Hk, E1S[:(k + 1) * p], rcond=None)[0]
            est = np.linalg.norm(E1S[:(k + 1) * p] - Hk @ Y, axis=0) / bnorm
            if np.all(est <= tol) or it >= max_iter:
                break
        X = X + np.concatenate(Z[:k], axis=1) @ Y
        R = B - apply_cols(matvec, X)
