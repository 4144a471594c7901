"""GCRO-DR(m, k): GMRES with deflated restarting and a subspace recycled across a sequence of
systems (oracle; test infrastructure).

Sec. 6 of the paper names recycling, GCRO-DR in particular, for the imaging loop: a sequence of
slowly varying systems, one per inversion step, each with its antennas' right-hand sides.  The
paper prints no algorithm; this follows the method of Parks, de Sturler, Mackey, Johnson and
Maiti (SIAM J. Sci. Comput. 28, 2006), written from its description:

* the iteration works on one operator A_hat (here A M^{-1} with a fixed preconditioner; the
  solution is x = M^{-1} y) and keeps a k-dimensional subspace U with A_hat U = C, C^H C = I;
* a cycle first projects the residual off C, then runs m - k Arnoldi steps with the operator
  (I - C C^H) A_hat, and minimises the residual over span(U) + the new Krylov space (a small
  least-squares problem in the matrix G of the cycle);
* U is refreshed from the harmonic Ritz vectors of the cycle with the k smallest harmonic Ritz
  values (deflation of the slowest components);
* for the next system the same U is kept and C recomputed from A_hat_new U by a QR
  factorisation.

With k = 0 it is restarted GMRES(m).
Dense NumPy/SciPy only: library eigen-, QR and least-squares routines serve as steps.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla


@dataclass
class GcroResult:
    y: np.ndarray            # solution of A_hat y = b
    matvecs: int             # products with A_hat in Arnoldi steps and for C = A_hat U (the true
                             # residual at each cycle end is not counted, as in fgmres)
    relres: float            # true ||b - A_hat y|| / ||b||
    converged: bool
    U: np.ndarray            # recycled subspace for the next system (n x k), or None
    history: list            # true relative residual after each cycle


def _smallest(theta, vecs, k):
    """The k eigenvectors with the smallest |theta| (ties by index), real-normalised."""
    order = np.argsort(np.abs(theta), kind="stable")[:k]
    return vecs[:, order]


def _harmonic_ritz_gmres(H, hnext, k):
    """Harmonic Ritz vectors of an m-step Arnoldi relation A V_m = V_{m+1} Hbar_m, Hbar_m =
    [H; hnext e_m^T]: (H + |hnext|^2 H^{-H} e_m e_m^T) z = theta z."""
    m = H.shape[0]
    em = np.zeros(m, dtype=np.complex128)
    em[-1] = 1.0
    f = sla.solve(H.conj().T, em)
    Hh = H + abs(hnext) ** 2 * np.outer(f, em)
    theta, Z = sla.eig(Hh)
    return _smallest(theta, Z, k)


def _harmonic_ritz_cycle(G, WhV, k):
    """Harmonic Ritz vectors of a GCRO-DR cycle: G^H G z = theta G^H (W^H V) z."""
    theta, Z = sla.eig(G.conj().T @ G, G.conj().T @ WhV)
    return _smallest(theta, Z, k)


def _qr_pair(M):
    """Reduced QR, M = Q R."""
    Q, R = np.linalg.qr(M, mode="reduced")
    return Q, R


def _right_solve(X, R):
    """X R^{-1} for upper-triangular R."""
    return sla.solve_triangular(R.T, X.T, lower=True).T


def _cycle(op, r, steps, tol, bnorm, C=None, U=None):
    """One cycle from the residual r: Arnoldi with (I - C C^H) op (plain when C is None), the
    least-squares problem re-solved after every step, stopping early once its residual estimate
    reaches tol.  Returns (dy, G, What, Vhat, nsteps) with dy the update of y."""
    n = r.size
    kk = 0 if C is None else C.shape[1]
    beta = np.linalg.norm(r)
    V = np.zeros((n, steps + 1), dtype=np.complex128)
    V[:, 0] = r / beta
    G = np.zeros((kk + steps + 1, kk + steps), dtype=np.complex128)
    if kk:
        d = 1.0 / np.linalg.norm(U, axis=0)
        G[:kk, :kk] = np.diag(d)
    c = np.zeros(kk + steps + 1, dtype=np.complex128)
    c[kk] = beta                       # r = [C, V] c exactly
    z = None
    j_done = 0
    for j in range(steps):
        w = op(V[:, j])
        if kk:
            bj = C.conj().T @ w
            G[:kk, kk + j] = bj
            w = w - C @ bj
        for i in range(j + 1):
            h = np.vdot(V[:, i], w)
            G[kk + i, kk + j] = h
            w = w - h * V[:, i]
        hn = np.linalg.norm(w)
        G[kk + j + 1, kk + j] = hn
        if hn > 0.0:
            V[:, j + 1] = w / hn
        j_done = j + 1
        Gj = G[:kk + j_done + 1, :kk + j_done]
        z = np.linalg.lstsq(Gj, c[:kk + j_done + 1], rcond=None)[0]
        est = np.linalg.norm(c[:kk + j_done + 1] - Gj @ z) / bnorm
        if est <= tol or hn == 0.0:
            break
    Vhat = V[:, :j_done] if not kk else np.concatenate([U * (1.0 / np.linalg.norm(U, axis=0)), V[:, :j_done]], axis=1)
    What = V[:, :j_done + 1] if not kk else np.concatenate([C, V[:, :j_done + 1]], axis=1)
    G = G[:kk + j_done + 1, :kk + j_done]
    return Vhat @ z, G, What, Vhat, j_done


def gcrodr(op, b, m=30, k=10, tol=1e-8, max_matvecs=5000, U=None) -> GcroResult:
    """Solves op(y) = b.  U: recycled subspace from an earlier system (or None).  k = 0 is
    restarted GMRES(m).  Cycles have m - k Arnoldi steps once a recycled subspace exists."""
    b = np.asarray(b, dtype=np.complex128)
    n = b.size
    bnorm = np.linalg.norm(b)
    y = np.zeros(n, dtype=np.complex128)
    hist = []
    if bnorm == 0.0:
        return GcroResult(y, 0, 0.0, True, U, hist)
    mv = 0
    C = None
    if k == 0:
        U = None
    if U is not None:
        AU = np.stack([op(U[:, j]) for j in range(U.shape[1])], axis=1)
        mv += U.shape[1]
        C, R = _qr_pair(AU)
        U = _right_solve(U, R)                     # op(U) = C, C^H C = I
    r = b.copy()
    while True:
        if C is not None:                          # keep r orthogonal to C: y += U C^H r
            t = C.conj().T @ r
            y = y + U @ t
            r = r - C @ t
        rel = np.linalg.norm(r) / bnorm
        if rel <= tol or mv >= max_matvecs:
            break
        if C is None:
            steps = min(m, max_matvecs - mv)
            dy, G, What, Vhat, nst = _cycle(op, r, steps, tol, bnorm)
            mv += nst
            y = y + dy
            if k > 0 and nst >= k:                 # first deflation space from the GMRES cycle
                P = _harmonic_ritz_gmres(G[:nst, :nst], G[nst, nst - 1], k)
                Q, R = _qr_pair(G @ P)
                C = What @ Q
                U = _right_solve(Vhat @ P, R)
        else:
            steps = min(m - C.shape[1], max_matvecs - mv)
            dy, G, What, Vhat, nst = _cycle(op, r, steps, tol, bnorm, C, U)
            mv += nst
            y = y + dy
            kk = C.shape[1]
            P = _harmonic_ritz_cycle(G, What.conj().T @ Vhat, kk)
            Q, R = _qr_pair(G @ P)
            C = What @ Q
            U = _right_solve(Vhat @ P, R)
        r = b - op(y)                              # true residual at the end of a cycle
        hist.append(np.linalg.norm(r) / bnorm)
    true_rel = np.linalg.norm(b - op(y)) / bnorm
    return GcroResult(y, mv, true_rel, true_rel <= tol, U, hist)
