"""Metallic walls, waveguide ports and the scattering functional (oracle; test infrastructure).

Metallic boundary (Sec. 2, eq. metallicbc): E x n = 0 on Gamma_w, and the space of the weak form
is V = {v in H(curl) : v x n = 0 on Gamma_w}.  In the edge-element space, a degree of freedom is
constrained (its coefficient is zero) when its basis function has a nonzero tangential trace on a
metallic face.  `constrained_dofs` finds these by evaluating w_a x n on every metallic face at the
points of a triangle rule: a tangential trace that is a nonzero vector polynomial of degree r
cannot vanish at the (r + 2)^2 Gauss points of the rule.  The system on V is written on all
degrees of freedom with identity rows and columns for the constrained ones and a zero right-hand
side there, so x = 0 there and the free block is the Galerkin system on V.

Ports (Sec. 2, eqs. wgj and wgi; Sec. 5.1).  A port is a planar rectangle
    {o + s u + t v : s, t in [0, 1]}
on the outer boundary, with u and v orthogonal.  Its faces are the outer faces whose centroid
((x0 + x1) + x2) / 3 lies in it: 0 <= s, t <= 1 and distance to its plane at most 1e-9 (|u| + |v|).
Its fundamental TE10 mode is
    E0(x) = sin(pi s) v / |v|,   s = (x - o).u / |u|^2,
and beta is the propagation wavenumber along the waveguide.

* Transmitting port.  The incoming mode is E_in = E0 exp(i beta zeta), with zeta = (x - o).n the
  coordinate along the outward normal n, so it travels into the domain.  For E = f e ê_v
  (f = sin(pi s), e = exp(i beta zeta), ê_u, ê_v in the port plane):
  - curl E = grad(f e) x ê_v = (pi/|u|) cos(pi s) e (ê_u x ê_v) + i beta f e (n x ê_v);
  - (curl E) x n = i beta f e ê_v, since ê_u x ê_v is parallel to n;
  - n x (E x n) = E.
  The data of eq. wgj, g = mu_r^{-1} (curl E_in) x n + i beta n x (E_in x n), is therefore
  i beta (1 + 1/mu_r) E0 on the port plane.  The load is b_a = int_port g . w_a.
* Receiving ports carry the Silver-Mueller condition (eq. wgi): the impedance term i beta on
  their faces (the caller's beta_face) and no load.
* Scattering coefficients (eq. sij):
    S_ij = int_{Gamma_i} conj(E_j) . E0_i / int_{Gamma_i} |E0_i|^2
         = sum_a conj(x_j[a]) p_i[a] / N_i,
  with p_i[a] = int_{Gamma_i} w_a . E0_i (real basis functions) and N_i = int_{Gamma_i} |E0_i|^2.
  On the transmitting port the formula is taken as printed: the total field, incident wave
  included.
* Error metric (eq. errsij): E = ||S - S_ref||_F / ||S_ref||_F.

The face integrals use the conical-product rule `quadrature.tri_rule(nq)` on each face.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import basis, elements, quadrature
from .topology import Topology

PORT_NQ = 10            # triangle-rule points per direction for the port integrals
_PLANE_TOL = 1e-9


@dataclass
class Port:
    origin: np.ndarray   # [3]
    u: np.ndarray        # [3] width edge (the mode varies along it)
    v: np.ndarray        # [3] height edge (the mode points along it)
    beta: float          # propagation wavenumber along the waveguide


def face_kind_table(tets, face_kind):
    """kind[t, lf] on the sorted local face lf of every tetrahedron from the caller's table
    face_kind[t, q] given on the face opposite the caller's vertex tets[t, q]."""
    tets = np.asarray(tets)
    fk = np.asarray(face_kind).reshape(-1, 4)
    st = np.sort(tets, axis=1)
    out = np.empty((len(tets), 4), dtype=np.int64)
    for lf in range(4):
        opp = st[:, basis.FACE_OPPOSITE[lf]]
        q = np.argmax(tets == opp[:, None], axis=1)
        out[:, lf] = fk[np.arange(len(tets)), q]
    return out


def _face_points(topo: Topology, xyz, t, lf, nq):
    """Barycentrics [P,4] of the rule on local face lf, its weights (sum 1/2), the points [F,P,3],
    outward unit normals [F,3], areas [F] and barycentric gradients [F,4,3] of tets t."""
    lam3, w = quadrature.tri_rule(nq)
    lam = np.zeros((lam3.shape[0], 4))
    lam[:, list(basis.LOCAL_FACES[lf])] = lam3
    grads, vol, _ = elements.geometry(xyz, topo.st[t])
    go = grads[:, basis.FACE_OPPOSITE[lf]]
    gn = np.linalg.norm(go, axis=1)
    nrm = -go / gn[:, None]
    area = 3.0 * vol * gn
    x = np.einsum("pv,fvi->fpi", lam, xyz[topo.st[t]])
    return lam, w, x, nrm, area, grads


def constrained_dofs(topo: Topology, xyz, kind_lf):
    """Boolean [ndof]: the degrees of freedom whose basis functions have a nonzero tangential
    trace on a metallic face (kind_lf[t, lf] == 1 on an outer face)."""
    kind_lf = np.asarray(kind_lf)
    mask = np.zeros(topo.ndof, dtype=bool)
    for lf in range(4):
        t = np.nonzero(kind_lf[:, lf] == 1)[0]
        if len(t) == 0:
            continue
        faces = topo.tet_faces[t, lf]
        if np.any(topo.face_tets[faces, 1] >= 0):
            raise ValueError("metallic condition on an interior face")
        lam, _, _, nrm, _, grads = _face_points(topo, xyz, t, lf, topo.r + 2)
        W, _ = basis.eval_basis_batch(topo.r, lam, grads)               # [F,P,n,3]
        tang = np.cross(W, nrm[:, None, None, :])                        # w_a x n
        scale = np.abs(W).max(axis=(1, 2, 3))                             # per face
        nz = np.abs(tang).max(axis=(1, 3)) > 1e-10 * scale[:, None]      # [F,n]
        mask[topo.dofmap[t][nz]] = True
    return mask


def constrain(A, mask):
    """Identity rows and columns for the constrained degrees of freedom of the CSR matrix A."""
    A = sp.csr_matrix(A, copy=True)
    free = (~mask).astype(np.float64)
    D = sp.diags(free)
    out = (D @ A @ D).tocsr()
    out = out + sp.diags(mask.astype(np.float64))
    out.sort_indices()
    return out.tocsr()


def port_faces(topo: Topology, xyz, port: Port):
    """(tets, local faces) of the outer faces whose centroid lies in the port rectangle."""
    o, u, v = (np.asarray(a, dtype=np.float64) for a in (port.origin, port.u, port.v))
    nrm = np.cross(u, v)
    nrm /= np.linalg.norm(nrm)
    tol = _PLANE_TOL * (np.linalg.norm(u) + np.linalg.norm(v))
    bf = topo.boundary_faces()
    tt = topo.face_tets[bf, 0]
    lf = np.argmax(topo.tet_faces[tt] == bf[:, None], axis=1)
    fv = xyz[topo.faces[bf]]                                              # [F,3,3]
    c = ((fv[:, 0] + fv[:, 1]) + fv[:, 2]) / 3.0
    d = c - o
    s = d @ u / (u @ u)
    t = d @ v / (v @ v)
    on = np.abs(d @ nrm) <= tol
    inside = on & (s >= 0.0) & (s <= 1.0) & (t >= 0.0) & (t <= 1.0)
    return tt[inside], lf[inside]


def _mode(port: Port, x):
    u = np.asarray(port.u, dtype=np.float64)
    v = np.asarray(port.v, dtype=np.float64)
    s = (x - np.asarray(port.origin, dtype=np.float64)) @ u / (u @ u)
    return np.sin(np.pi * s)[..., None] * (v / np.linalg.norm(v))


def port_vector(topo: Topology, xyz, port: Port, nq=PORT_NQ, coef=None):
    """p[a] = sum over the port's faces of int_f coef_f w_a . E0 (coef_f = 1 by default), and
    N = int_port |E0|^2."""
    tt, lfs = port_faces(topo, xyz, port)
    p = np.zeros(topo.ndof, dtype=np.complex128)
    norm = 0.0
    for lf in range(4):
        sel = np.nonzero(lfs == lf)[0]
        if len(sel) == 0:
            continue
        t = tt[sel]
        lam, w, x, _, area, grads = _face_points(topo, xyz, t, lf, nq)
        E0 = _mode(port, x)                                               # [F,P,3]
        W, _ = basis.eval_basis_batch(topo.r, lam, grads)                 # [F,P,n,3]
        loc = np.einsum("fpi,fpai,p->fa", E0, W, w) * (2.0 * area)[:, None]
        if coef is not None:
            loc = loc * np.asarray(coef)[t][:, None]
        np.add.at(p, topo.dofmap[t].ravel(), loc.ravel())
        norm += float(np.sum(np.einsum("fpi,fpi,p->f", E0, E0, w) * 2.0 * area))
    return p, norm


def port_load(topo: Topology, xyz, mu_r, port: Port, mask=None, nq=PORT_NQ):
    """b_a = int_port i beta (1 + 1/mu_r) E0 . w_a (incoming TE10 mode), zero on constrained
    degrees of freedom."""
    coef = 1j * port.beta * (1.0 + 1.0 / np.asarray(mu_r))
    b, _ = port_vector(topo, xyz, port, nq, coef)
    if mask is not None:
        b[mask] = 0.0
    return b


def s_matrix(topo: Topology, xyz, ports, X, nq=PORT_NQ):
    """S[i, j] = sum_a conj(X[a, j]) p_i[a] / N_i for the fields X [N, k]."""
    X = np.asarray(X).reshape(topo.ndof, -1)
    S = np.empty((len(ports), X.shape[1]), dtype=np.complex128)
    for i, port in enumerate(ports):
        p, norm = port_vector(topo, xyz, port, nq)
        S[i] = (np.conj(X) * p[:, None]).sum(axis=0) / norm
    return S


def s_error(S, S_ref):
    """Relative error of Sec. 5.2: ||S - S_ref||_F / ||S_ref||_F."""
    S = np.asarray(S)
    S_ref = np.asarray(S_ref)
    return float(np.sqrt(np.sum(np.abs(S - S_ref) ** 2)) / np.sqrt(np.sum(np.abs(S_ref) ** 2)))
