"""Element matrices by the exact monomial integration rule (test-side cross-check of the oracle).

The oracle computes its element matrices from their definition, by quadrature of the directly
evaluated basis (oracle.elements).  This module computes the same matrices a second way, without
any quadrature: every generator lambda^k w^{ij} (Sec. 3) is a sum of terms
c * lambda^alpha * grad(lambda_m) and its curl a sum of terms c * lambda^beta * (grad lambda_p x
grad lambda_m) (curl(f grad g) = grad f x grad g); products of two terms are integrated exactly
with
    int_T lambda^alpha = 6 |T| alpha! / (|alpha| + 3)!          (volume)
    int_f lambda^alpha = 2 |f| alpha! / (|alpha| + 2)!          (face, alpha_opp = 0)
and the geometric factors G_pq = grad lambda_p . grad lambda_q,
(grad l_p x grad l_m).(grad l_q x grad l_n) = G_pq G_mn - G_pn G_mq.  On a face with opposite
vertex o, (u x n).(v x n) = u.v - (u.n)(v.n), n = grad lambda_o / |grad lambda_o|, so the
tangential Gram matrix is G^T_pq = G_pq - G_po G_qo / G_oo and |f| = 3 |T| |grad lambda_o|.
"""
from functools import lru_cache
from math import factorial

import numpy as np

from oracle import basis
from oracle.elements import geometry


def _fact(alpha):
    out = 1
    for a in alpha:
        out *= factorial(a)
    return out


def vol_coef(alpha):
    """int_T lambda^alpha / |T|."""
    return 6.0 * _fact(alpha) / factorial(sum(alpha) + 3)


def face_coef(alpha):
    """int_f lambda^alpha / |f| for alpha supported on the face."""
    return 2.0 * _fact(alpha) / factorial(sum(alpha) + 2)


def _terms(d):
    """lambda^k (lambda_i grad l_j - lambda_j grad l_i) as [(c, alpha, m)]."""
    _, _, _, i, j, k = d
    a1 = list(k)
    a1[i] += 1
    a2 = list(k)
    a2[j] += 1
    return [(1.0, tuple(a1), j), (-1.0, tuple(a2), i)]


def _curl_terms(d):
    """curl of the generator as [(c, beta, p, m)] meaning c lambda^beta (grad l_p x grad l_m)."""
    out = []
    for c, alpha, m in _terms(d):
        for p in range(4):
            if alpha[p] > 0:
                beta = list(alpha)
                beta[p] -= 1
                out.append((c * alpha[p], tuple(beta), p, m))
    return out


def _add(a, b):
    return tuple(x + y for x, y in zip(a, b))


@lru_cache(maxsize=None)
def mass_coefficients(r):
    dofs = basis.local_dofs(r)
    n = len(dofs)
    C = np.zeros((n, n, 4, 4))
    for a, da in enumerate(dofs):
        for b, db in enumerate(dofs):
            for ca, aa, ma in _terms(da):
                for cb, ab, mb in _terms(db):
                    C[a, b, ma, mb] += ca * cb * vol_coef(_add(aa, ab))
    return C


@lru_cache(maxsize=None)
def stiffness_coefficients(r):
    dofs = basis.local_dofs(r)
    n = len(dofs)
    C = np.zeros((n, n, 4, 4, 4, 4))
    ct = [_curl_terms(d) for d in dofs]
    for a in range(n):
        for b in range(n):
            for ca, ba, pa, ma in ct[a]:
                for cb, bb, pb, mb in ct[b]:
                    C[a, b, pa, ma, pb, mb] += ca * cb * vol_coef(_add(ba, bb))
    return C.reshape(n, n, 16, 16)


@lru_cache(maxsize=None)
def face_coefficients(r, opp):
    dofs = basis.local_dofs(r)
    n = len(dofs)
    C = np.zeros((n, n, 4, 4))
    for a, da in enumerate(dofs):
        for b, db in enumerate(dofs):
            for ca, aa, ma in _terms(da):
                for cb, ab, mb in _terms(db):
                    al = _add(aa, ab)
                    if al[opp] != 0:
                        continue
                    C[a, b, ma, mb] += ca * cb * face_coef(tuple(al[v] for v in range(4) if v != opp))
    return C


def cross_gram(G):
    """X[t,(p,m),(q,n)] = (grad l_p x grad l_m).(grad l_q x grad l_n)."""
    X = (np.einsum("tpq,tmn->tpmqn", G, G) - np.einsum("tpn,tmq->tpmqn", G, G))
    return X.reshape(len(G), 16, 16)


def element_mass_stiffness(xyz, st, r):
    """Exact M_T[t,a,b] = int w_a.w_b and K_T[t,a,b] = int curl w_a . curl w_b (real)."""
    _, vol, G = geometry(xyz, st)
    M = vol[:, None, None] * np.einsum("abpq,tpq->tab", mass_coefficients(r), G)
    K = vol[:, None, None] * np.einsum("abxy,txy->tab", stiffness_coefficients(r), cross_gram(G))
    return M, K


def face_matrices(xyz, st, tets_idx, local_face, r):
    """S_f[a,b] = int_f (w_a x n).(w_b x n) for (tet, local face) pairs, tet-local numbering."""
    tets_idx = np.asarray(tets_idx)
    local_face = np.asarray(local_face)
    _, vol, G = geometry(xyz, st[tets_idx])
    out = np.zeros((len(tets_idx), basis.n_local(r), basis.n_local(r)))
    for lf in range(4):
        sel = np.nonzero(local_face == lf)[0]
        if len(sel) == 0:
            continue
        o = basis.FACE_OPPOSITE[lf]
        Gs = G[sel]
        goo = Gs[:, o, o]
        GT = Gs - Gs[:, :, o][:, :, None] * Gs[:, :, o][:, None, :] / goo[:, None, None]
        area = 3.0 * vol[sel] * np.sqrt(goo)
        out[sel] = area[:, None, None] * np.einsum("abpq,tpq->tab", face_coefficients(r, o), GT)
    return out
