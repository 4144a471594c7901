"""Right-preconditioned flexible GMRES(m) (oracle; test infrastructure).

Sec. 5 solves every system by GMRES preconditioned with ORAS; the side, restart
length and tolerance are not stated there.  Reading used here: right
preconditioning in the flexible form (Z_m basis kept, x = x0 + Z_m y), x0 = 0,
Hermitian inner product, modified Gram-Schmidt Arnoldi, complex Givens rotations
for the Hessenberg least-squares problem.  A cycle ends when the estimated
relative residual |g_{j+1}| / ||b|| <= tol or after m steps; the true residual
||b - A x|| / ||b|| is then recomputed in FP64 and the method restarts if it is
above tol.  Multiple right-hand sides are independent recurrences (the
pseudo-block method of Sec. 5 fuses only their arithmetic).
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
