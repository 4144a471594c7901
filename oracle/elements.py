"""Element matrices of the curl-curl weak form (oracle; test infrastructure).

Weak form (Sec. 2, variational formulation):
    int_Omega [ mu_r^{-1} curl E . curl v - k0^2 eps_r E . v ]
      + int_Gamma i beta (E x n) . (v x n)  =  int_Gamma g . v .
The matrices are computed from their definition: the degree-r generators lambda^k w^{ij} of
Sec. 3 and their curls (product formula) are evaluated at the points of a conical-product
Gauss-Jacobi rule (oracle.quadrature) and the integrands are summed with its weights,

    M_T[a,b] = int_T w_a . w_b,                K_T[a,b] = int_T curl w_a . curl w_b,
    S_f[a,b] = int_f (w_a x n) . (w_b x n).

w_a is a polynomial of degree r and curl w_a of degree r - 1, so the integrands have degree at
most 2r; the n-point rule in each collapsed direction is exact to total degree 2n - 1, so
n = r + 1 points give the exact integrals up to rounding.  The affine map of the reference
simplex contributes the factor 6|T| (volume, rule weights summing to 1/6) or 2|f| (face,
weights summing to 1/2); on a face f opposite the local vertex o the unit normal is
grad(lambda_o) / |grad(lambda_o)| (its sign does not matter in S_f) and |f| = 3 |T| |grad lambda_o|.
"""
from __future__ import annotations

import numpy as np

from . import basis, quadrature

CHUNK = 2048     # tetrahedra evaluated together (bounds the memory of the point values)


def geometry(xyz, st):
    """Barycentric gradients [T,4,3], volumes [T] and Gram matrices G [T,4,4]."""
    v = xyz[st]
    J = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]], axis=2)
    Jinv = np.linalg.inv(J)
    grads = np.empty((len(st), 4, 3))
    grads[:, 1:] = Jinv
    grads[:, 0] = -Jinv.sum(axis=1)
    vol = np.abs(np.linalg.det(J)) / 6.0
    G = np.einsum("tpi,tqi->tpq", grads, grads)
    return grads, vol, G


def _gram(F, w):
    """sum_p w_p F[t,p,a,:] . F[t,p,b,:] for F [T,P,n,3] -> [T,n,n]."""
    Fw = F * np.sqrt(w)[None, :, None, None]
    Fw = Fw.transpose(0, 2, 1, 3).reshape(F.shape[0], F.shape[2], -1)   # [T, n, P*3]
    return Fw @ Fw.transpose(0, 2, 1)


def element_mass_stiffness(xyz, st, r):
    """M_T[t,a,b] = int w_a . w_b and K_T[t,a,b] = int curl w_a . curl w_b (real), by the
    (r+1)-point conical-product rule on every tetrahedron."""
    st = np.asarray(st)
    lam, w = quadrature.tet_rule(r + 1)
    n = basis.n_local(r)
    M = np.empty((len(st), n, n))
    K = np.empty((len(st), n, n))
    for c0 in range(0, len(st), CHUNK):
        grads, vol, _ = geometry(xyz, st[c0:c0 + CHUNK])
        val, cur = basis.eval_basis_batch(r, lam, grads)
        M[c0:c0 + CHUNK] = 6.0 * vol[:, None, None] * _gram(val, w)
        K[c0:c0 + CHUNK] = 6.0 * vol[:, None, None] * _gram(cur, w)
    return M, K


def element_matrices(xyz, st, r, eps_r, mu_r, k0):
    """A_T = mu_r^{-1} K_T - k0^2 eps_r M_T (complex, without boundary terms)."""
    M, K = element_mass_stiffness(xyz, st, r)
    return (1.0 / mu_r)[:, None, None] * K - (k0 ** 2) * eps_r[:, None, None] * M


def face_points(lf, r):
    """Barycentric points [P,4] of the (r+1)-point triangle rule on local face lf (the opposite
    coordinate is zero) and the rule's weights (sum 1/2)."""
    lam3, w = quadrature.tri_rule(r + 1)
    lam = np.zeros((lam3.shape[0], 4))
    lam[:, list(basis.LOCAL_FACES[lf])] = lam3
    return lam, w


def face_matrices(xyz, st, tets_idx, local_face, r):
    """S_f[a,b] = int_f (w_a x n).(w_b x n) for faces given as (tet, local face) pairs.

    Returned in the tet-local numbering (n_local x n_local; zero rows and columns for the DOFs
    whose tangential trace vanishes on the face).
    """
    tets_idx = np.asarray(tets_idx)
    local_face = np.asarray(local_face)
    n = basis.n_local(r)
    out = np.zeros((len(tets_idx), n, n))
    for lf in range(4):
        sel = np.nonzero(local_face == lf)[0]
        if len(sel) == 0:
            continue
        o = basis.FACE_OPPOSITE[lf]
        lam, w = face_points(lf, r)
        for c0 in range(0, len(sel), CHUNK):
            part = sel[c0:c0 + CHUNK]
            grads, vol, _ = geometry(xyz, st[tets_idx[part]])
            gn = np.linalg.norm(grads[:, o], axis=1)
            nrm = grads[:, o] / gn[:, None]
            area = 3.0 * vol * gn
            val, _ = basis.eval_basis_batch(r, lam, grads)
            tan = np.cross(val, nrm[:, None, None, :])
            out[part] = 2.0 * area[:, None, None] * _gram(tan, w)
    return out
