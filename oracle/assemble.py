"""Global system A u = b of Sec. 4 (oracle; test infrastructure).

A = sum_T P_T^T A_T P_T + sum_{f on boundary} i beta_f P_f^T S_f P_f, where A_T is the
element matrix of `oracle.elements` and S_f the tangential face mass matrix.  The
impedance coefficient on an outer face is beta_f = k0 sqrt(Re mu_r Re eps_r) of the
adjacent tetrahedron (the wave number of Sec. 2 with the loss dropped).

Right-hand sides:
* plane-wave impedance data (Sec. 2, eq. for g_j): for the exact field
  E = p exp(-i gamma d.x), gamma = k0 sqrt(mu_r eps_r) (principal root),
  g = mu_r^{-1} (curl E) x n + i beta n x (E x n) on every boundary face and
  b_a = int_{boundary} g . w_a, by a conical-product rule on each face;
* point dipole: b_a = w_a(x0) . dir in the lowest-index tetrahedron containing x0
  (all barycentrics >= -1e-12).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import basis, elements, quadrature
from .topology import Topology


def impedance_beta(k0, eps_r, mu_r):
    return k0 * np.sqrt(np.real(mu_r) * np.real(eps_r))


def face_beta_table(tets, beta_face):
    """beta[t, lf] on the sorted local face lf of every tetrahedron from a caller's table
    beta_face[t, q] given on the face opposite the caller's vertex tets[t, q] (Sec. 2: beta is
    the caller's per-port wave number).  The sorted local face lf (basis.LOCAL_FACES) is the
    face opposite the sorted vertex FACE_OPPOSITE[lf]."""
    tets = np.asarray(tets)
    beta_face = np.asarray(beta_face, dtype=np.float64).reshape(-1, 4)
    st = np.sort(tets, axis=1)
    out = np.empty((len(tets), 4))
    for lf in range(4):
        opp = st[:, basis.FACE_OPPOSITE[lf]]
        q = np.argmax(tets == opp[:, None], axis=1)
        out[:, lf] = beta_face[np.arange(len(tets)), q]
    return out


def outer_beta(k0, eps_r, mu_r, t, lf, beta_lf=None):
    """beta of outer faces (t, lf): the caller's table when given, else k0 sqrt(Re mu Re eps)."""
    if beta_lf is not None:
        return np.asarray(beta_lf)[t, lf]
    return impedance_beta(k0, eps_r[t], mu_r[t])


def boundary_face_list(topo: Topology):
    """(face ids, adjacent tet, local face index) of all outer faces."""
    bf = topo.boundary_faces()
    t = topo.face_tets[bf, 0]
    lf = np.argmax(topo.tet_faces[t] == bf[:, None], axis=1)
    return bf, t, lf


def global_matrix(topo: Topology, xyz, eps_r, mu_r, k0, beta_lf=None, mask=None):
    """beta_lf: [T, 4] beta per sorted local face (face_beta_table) or None (derived).  mask:
    Boolean [ndof] of the degrees of freedom constrained by metallic faces (oracle.ports), whose
    rows and columns become identity rows and columns."""
    AT = elements.element_matrices(xyz, topo.st, topo.r, eps_r, mu_r, k0)
    bf, bt, blf = boundary_face_list(topo)
    if len(bf):
        S = elements.face_matrices(xyz, topo.st, bt, blf, topo.r)
        beta = outer_beta(k0, eps_r, mu_r, bt, blf, beta_lf)
        np.add.at(AT, bt, 1j * beta[:, None, None] * S)
    nl = AT.shape[1]
    rows = np.repeat(topo.dofmap, nl, axis=1).ravel()
    cols = np.tile(topo.dofmap, (1, nl)).ravel()
    A = sp.coo_matrix((AT.ravel(), (rows, cols)), shape=(topo.ndof, topo.ndof)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    if mask is not None and mask.any():
        from .ports import constrain
        A = constrain(A, mask)
    return A


def _basis_on_points(r, lam, grads):
    """Values [F,P,n_local,3] of the local basis at barycentric points lam[P,4] of F tetrahedra
    with barycentric gradients grads[F,4,3] (direct evaluation of the generators, Sec. 3)."""
    val, _ = basis.eval_basis_batch(r, lam, grads)
    return val


def plane_wave_load(topo: Topology, xyz, eps_r, mu_r, k0, d, p, nq=8, beta_lf=None):
    d = np.asarray(d, dtype=np.float64)
    p = np.asarray(p, dtype=np.complex128)
    b = np.zeros(topo.ndof, dtype=np.complex128)
    bf, bt, blf = boundary_face_list(topo)
    grads, vol, _ = elements.geometry(xyz, topo.st[bt])
    lam3, w = quadrature.tri_rule(nq)
    for lf in range(4):
        sel = np.nonzero(blf == lf)[0]
        if len(sel) == 0:
            continue
        fv = basis.LOCAL_FACES[lf]
        o = basis.FACE_OPPOSITE[lf]
        lam = np.zeros((lam3.shape[0], 4))
        lam[:, list(fv)] = lam3
        t = bt[sel]
        g = grads[sel]
        go = g[:, o]
        gn = np.linalg.norm(go, axis=1)
        nrm = -go / gn[:, None]                       # outward unit normal
        area = 3.0 * vol[sel] * gn
        verts = xyz[topo.st[t]]                       # [F,4,3]
        x = np.einsum("pv,fvi->fpi", lam, verts)      # [F,P,3]
        gamma = k0 * np.sqrt(mu_r[t] * eps_r[t])
        beta = outer_beta(k0, eps_r, mu_r, t, np.full(len(t), lf), beta_lf)
        phase = np.exp(-1j * gamma[:, None] * (x @ d))  # [F,P]
        E = phase[:, :, None] * p[None, None, :]
        curlE = (-1j * gamma)[:, None, None] * phase[:, :, None] * np.cross(d, p)[None, None, :]
        n3 = nrm[:, None, :]
        ET = np.cross(n3, np.cross(E, n3))
        gval = (1.0 / mu_r[t])[:, None, None] * np.cross(curlE, n3) + 1j * beta[:, None, None] * ET
        W = _basis_on_points(topo.r, lam, g)           # [F,P,n,3]
        loc = np.einsum("fpi,fpai,p->fa", gval, W, w) * (2.0 * area)[:, None]
        np.add.at(b, topo.dofmap[t].ravel(), loc.ravel())
    return b


def locate_point(topo: Topology, xyz, x0, tol=1e-12):
    """Lowest-index tetrahedron whose barycentrics of x0 are all >= -tol."""
    v = xyz[topo.st]
    J = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]], axis=2)
    lam123 = np.linalg.solve(J, (np.asarray(x0)[None, :] - v[:, 0])[:, :, None])[:, :, 0]
    lam = np.concatenate([1.0 - lam123.sum(axis=1, keepdims=True), lam123], axis=1)
    inside = np.nonzero((lam >= -tol).all(axis=1))[0]
    if len(inside) == 0:
        raise ValueError("source point outside the mesh")
    t = int(inside[0])
    return t, lam[t]


def dipole_load(topo: Topology, xyz, x0, direction):
    t, lam = locate_point(topo, xyz, x0)
    grads, _, _ = elements.geometry(xyz, topo.st[t:t + 1])
    W = _basis_on_points(topo.r, lam[None, :], grads)[0, 0]  # [n,3]
    b = np.zeros(topo.ndof, dtype=np.complex128)
    b[topo.dofmap[t]] += W @ np.asarray(direction, dtype=np.float64)
    return b
