"""Pins of the oracle's block flexible GMRES (Sec. 6: Block GMRES for the several right-hand
sides of one system) and of its CholQR2 block orthonormalisation.  All CPU.

What fixes the block method independently of its own code:
* CholQR2 is a QR factorisation: Q^H Q = I, Q C = W, C upper triangular with a positive diagonal;
* with one right-hand side the block method is GMRES, so it must reproduce fgmres();
* the block Krylov space contains every column's own Krylov space, so after j block steps each
  column's residual is at most its single-right-hand-side GMRES residual after j steps
  (minimal-residual property), and a block solve to tol needs no more block steps than the
  slowest single solve;
* the result is the direct solve.
"""
from __future__ import annotations

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import fgmres, problem


def _dense_system(n=48, seed=5):
    rng = np.random.default_rng(seed)
    A = np.eye(n) * 12 + rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    # a fixed, non-trivial linear preconditioner (Jacobi of a perturbed diagonal)
    d = np.diag(A) * (1 + 0.3 * rng.normal(size=n))
    return A, (lambda v: A @ v), (lambda v: v / d), rng


def test_cholqr2_is_a_qr_factorisation():
    rng = np.random.default_rng(1)
    n, p = 300, 8
    U, _ = np.linalg.qr(rng.normal(size=(n, p)) + 1j * rng.normal(size=(n, p)))
    Vh, _ = np.linalg.qr(rng.normal(size=(p, p)) + 1j * rng.normal(size=(p, p)))
    W = U @ np.diag(np.logspace(0, -5, p)) @ Vh          # condition number 1e5
    Q, C = fgmres.cholqr2(W)
    assert np.abs(Q.conj().T @ Q - np.eye(p)).max() <= 1e-13
    assert np.linalg.norm(Q @ C - W) <= 1e-13 * np.linalg.norm(W)
    assert np.abs(np.tril(C, -1)).max() == 0.0
    assert np.all(np.abs(np.diag(C).imag) <= 1e-14 * np.abs(np.diag(C))) and np.all(np.diag(C).real > 0)


def test_cholqr2_reports_a_rank_deficient_block():
    rng = np.random.default_rng(2)
    W = rng.normal(size=(50, 3)) + 1j * rng.normal(size=(50, 3))
    W[:, 2] = 2.0 * W[:, 0]
    with pytest.raises(fgmres.BlockBreakdown):
        fgmres.cholqr2(W)


def test_one_column_block_is_fgmres():
    A, mv, pc, rng = _dense_system()
    b = rng.normal(size=A.shape[0]) + 1j * rng.normal(size=A.shape[0])
    for m in (48, 10):                          # unrestarted, and restarted cycles
        s = fgmres.fgmres(mv, pc, b, tol=1e-10, m=m)
        blk = fgmres.block_fgmres(mv, pc, b[:, None], tol=1e-10, m=m)
        assert blk.iterations == s.iterations and blk.converged and s.converged
        assert np.linalg.norm(blk.x[:, 0] - s.x) <= 1e-9 * np.linalg.norm(s.x)


@pytest.mark.parametrize("j", [3, 7, 12])
def test_block_residual_is_at_most_each_single_residual(j):
    A, mv, pc, rng = _dense_system()
    B = rng.normal(size=(A.shape[0], 4)) + 1j * rng.normal(size=(A.shape[0], 4))
    blk = fgmres.block_fgmres(mv, pc, B, tol=0.0, m=j, max_iter=j)
    assert blk.iterations == j
    for c in range(4):
        s = fgmres.fgmres(mv, pc, B[:, c], tol=0.0, m=j, max_iter=j)
        assert s.iterations == j
        rs = np.linalg.norm(B[:, c] - A @ s.x)
        rb = np.linalg.norm(B[:, c] - A @ blk.x[:, c])
        assert rb <= rs * (1 + 1e-9)
    # and strictly better than the single recurrences for at least one column
    assert any(np.linalg.norm(B[:, c] - A @ blk.x[:, c])
               < 0.999 * np.linalg.norm(B[:, c] - A @ fgmres.fgmres(mv, pc, B[:, c], 0.0, j, j).x)
               for c in range(4))


def test_block_oras_solve_is_the_direct_solve():
    w = synth.small(n=4, r=2, nsub=8, overlap=1, nrhs=4)
    p = problem.from_workload(w)
    B = p.B
    assert B.shape[1] == 4
    mv = lambda v: p.A @ v
    blk = fgmres.block_fgmres(mv, p.oras.apply, B, tol=1e-10, m=100)
    assert blk.converged and np.all(blk.relres <= 1e-10)
    lu = spla.splu(p.A.tocsc())
    for c in range(4):
        xd = lu.solve(B[:, c])
        assert np.linalg.norm(blk.x[:, c] - xd) <= 1e-8 * np.linalg.norm(xd)
    single = [fgmres.fgmres(mv, p.oras.apply, B[:, c], tol=1e-10, m=100).iterations for c in range(4)]
    assert blk.iterations <= max(single)
