"""Pins of the oracle's GCRO-DR (Sec. 6: subspace recycling for the imaging loop's sequence of
slowly varying systems).  All CPU.

What fixes it independently of its own code:
* with k = 0 it is restarted GMRES(m), so it must reproduce fgmres() step for step;
* on a matrix whose slow convergence comes from a few isolated small eigenvalues, deflated
  restarting removes their effect (far fewer products than GMRES(m)), and recycling the
  deflation space into the next, slightly perturbed system removes it from the start;
* each cycle minimises the residual over a space containing the previous iterate's
  correction directions, so the true residual never grows from cycle to cycle;
* the result is the direct solve.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import fgmres, gcrodr


def _dense(n=48, seed=5):
    rng = np.random.default_rng(seed)
    A = np.eye(n) * 12 + rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    return A, rng


def _small_eigenvalues(n=200, seed=7):
    """A = S diag(lam) S^-1: six eigenvalues in [0.01, 0.05], the rest in [1, 3], mildly
    non-normal; E a perturbation direction for the sequence."""
    rng = np.random.default_rng(seed)
    lam = np.concatenate([np.linspace(0.01, 0.05, 6), rng.uniform(1, 3, n - 6)])
    lam = lam * np.exp(1j * rng.uniform(-0.3, 0.3, n))
    S = np.eye(n) + 0.1 * rng.normal(size=(n, n)) / np.sqrt(n)
    A = S @ np.diag(lam) @ np.linalg.inv(S)
    E = rng.normal(size=(n, n)) / np.sqrt(n)
    return A, E, rng


@pytest.mark.parametrize("m", [48, 10])
def test_no_recycling_is_restarted_gmres(m):
    A, rng = _dense()
    b = rng.normal(size=A.shape[0]) + 1j * rng.normal(size=A.shape[0])
    s = fgmres.fgmres(lambda v: A @ v, lambda v: v, b, tol=1e-10, m=m)
    g = gcrodr.gcrodr(lambda v: A @ v, b, m=m, k=0, tol=1e-10)
    assert g.converged and s.converged and g.matvecs == s.iterations
    assert np.linalg.norm(g.y - s.x) <= 1e-9 * np.linalg.norm(s.x)


def test_deflated_restarting_and_recycling():
    A, E, rng = _small_eigenvalues()
    m, k, tol = 30, 8, 1e-8
    U = None
    for t in range(3):
        At = A + 1e-3 * t * E
        op = lambda v, At=At: At @ v
        b = rng.normal(size=A.shape[0]) + 1j * rng.normal(size=A.shape[0])
        g = fgmres.fgmres(op, lambda v: v, b, tol=tol, m=m)
        fresh = gcrodr.gcrodr(op, b, m=m, k=k, tol=tol)
        rec = gcrodr.gcrodr(op, b, m=m, k=k, tol=tol, U=U)
        U = rec.U
        assert g.converged and fresh.converged and rec.converged
        assert fresh.matvecs < 0.6 * g.iterations            # deflation of the small eigenvalues
        if t > 0:
            assert rec.matvecs < 0.75 * fresh.matvecs        # recycled from the previous system
        xd = np.linalg.solve(At, b)
        assert np.linalg.norm(rec.y - xd) <= 1e-6 * np.linalg.norm(xd)
        for h0, h1 in zip(fresh.history, fresh.history[1:]):
            assert h1 <= h0 * (1 + 1e-8)


def test_zero_right_hand_side():
    A, _ = _dense()
    g = gcrodr.gcrodr(lambda v: A @ v, np.zeros(A.shape[0]), m=10, k=4)
    assert g.converged and g.matvecs == 0 and not np.any(g.y)
