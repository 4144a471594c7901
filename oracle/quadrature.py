"""Quadrature rules (oracle; test infrastructure).

Gauss-Jacobi nodes and weights come from the Golub-Welsch eigenvalue method applied
to the three-term recurrence of the Jacobi polynomials (weight (1-x)^a (1+x)^b on
[-1, 1]); a library symmetric eigensolver is the only primitive used.  Simplex rules
are Stroud's conical products: collapse the simplex onto a cube and use Gauss-Jacobi
in the collapsed directions so that the Jacobian is absorbed into the weight.
An n-point Gauss rule integrates polynomials of degree 2n-1 exactly in each
direction, so `tri_rule(n)` and `tet_rule(n)` are exact to total degree 2n-1.
"""
from __future__ import annotations

from functools import lru_cache
from math import gamma

import numpy as np


@lru_cache(maxsize=None)
def gauss_jacobi(n: int, a: float = 0.0, b: float = 0.0):
    """n-point Gauss-Jacobi rule on [-1, 1] for weight (1-x)^a (1+x)^b."""
    k = np.arange(n, dtype=np.float64)
    s = 2.0 * k + a + b
    diag = np.empty(n)
    with np.errstate(divide="ignore", invalid="ignore"):
        diag[:] = (b * b - a * a) / (s * (s + 2.0))
    if n > 0:
        diag[0] = (b - a) / (a + b + 2.0)
    kk = np.arange(1, n, dtype=np.float64)
    ss = 2.0 * kk + a + b
    off = np.sqrt(4.0 * kk * (kk + a) * (kk + b) * (kk + a + b) /
                  (ss * ss * (ss + 1.0) * (ss - 1.0)))
    J = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    x, V = np.linalg.eigh(J)
    mu0 = 2.0 ** (a + b + 1.0) * gamma(a + 1.0) * gamma(b + 1.0) / gamma(a + b + 2.0)
    w = mu0 * V[0, :] ** 2
    return x, w


def rule01(n: int, a: float = 0.0):
    """Nodes s in [0,1] and weights for the weight (1-s)^a on [0, 1]."""
    x, w = gauss_jacobi(n, a, 0.0)
    return 0.5 * (x + 1.0), w / 2.0 ** (a + 1.0)


@lru_cache(maxsize=None)
def tri_rule(n: int):
    """Conical-product rule on the reference triangle (area 1/2).

    Returns barycentrics [P,3] and weights [P] (sum 1/2).
    """
    s, ws = rule01(n, 1.0)
    t, wt = rule01(n, 0.0)
    S, Tt = np.meshgrid(s, t, indexing="ij")
    W = np.outer(ws, wt)
    u = S.ravel()
    v = (Tt * (1.0 - S)).ravel()
    lam = np.stack([1.0 - u - v, u, v], axis=1)
    return lam, W.ravel()


@lru_cache(maxsize=None)
def tet_rule(n: int):
    """Conical-product rule on the reference tetrahedron (volume 1/6).

    Returns barycentrics [P,4] and weights [P] (sum 1/6).
    """
    s1, w1 = rule01(n, 2.0)
    s2, w2 = rule01(n, 1.0)
    s3, w3 = rule01(n, 0.0)
    A, B, C = np.meshgrid(s1, s2, s3, indexing="ij")
    W = w1[:, None, None] * w2[None, :, None] * w3[None, None, :]
    u = A
    v = B * (1.0 - A)
    w = C * (1.0 - A) * (1.0 - B)
    lam = np.stack([(1.0 - u - v - w).ravel(), u.ravel(), v.ravel(), w.ravel()], axis=1)
    return lam, W.ravel()


@lru_cache(maxsize=None)
def line_rule(n: int):
    """Gauss-Legendre on [0, 1]: nodes, weights (sum 1)."""
    return rule01(n, 0.0)
