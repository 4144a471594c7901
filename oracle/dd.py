"""Overlapping domain decomposition and the ORAS preconditioner (oracle; test infrastructure).

Sec. 4:  M^{-1}_ORAS = sum_s R_s^T D_s A_s^{-1} R_s, with R_s the Boolean restriction to
the ordered unknown set N_s of the overlapping subdomain Omega_s, D_s a diagonal
partition of unity (sum_s R_s^T D_s R_s = I), and A_s the local matrix of the
subproblem with impedance transmission conditions
    (curl E) x n + i omega~ n x (E x n)
on the interfaces, omega~ being the wave number of Sec. 2 (loss dropped).

Readings where the paper is silent (the paper names the objects, not their construction):
* partition: recursive coordinate bisection of tetrahedron centroids
  c = (((v0 + v1) + v2) + v3) * 0.25 (sorted vertex order, this exact summation order);
  axis = largest centroid extent (ties -> x, then y, then z); stable order by
  (coordinate, tet id); child 0 takes floor(m * p0 / p) tets, p0 = floor(p / 2) parts;
  subdomain ids depth-first, child 0 first;
* overlap: delta layers, each adds every tetrahedron sharing a vertex with the set (a
  face-sharing variant is available as an option);
* N_s: all DOFs on entities of the tetrahedra of Omega_s^delta, ascending global id;
* D_s: Boolean ownership; a DOF belongs to the non-overlapping subdomain of the
  lowest-index tetrahedron carrying it;
* omega~ on an interface face: k0 sqrt(Re mu_r Re eps_r) of the tetrahedron inside
  Omega_s^delta; outer boundary faces keep their beta;
* A_s^{-1}: dense LU with partial pivoting (LAPACK getrf semantics).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from . import elements
from .assemble import impedance_beta, outer_beta
from .topology import Topology, dof_min_tet


def centroids(xyz, st):
    v = xyz[st]
    return (((v[:, 0] + v[:, 1]) + v[:, 2]) + v[:, 3]) * 0.25


def rcb(xyz, st, nsub):
    """Recursive coordinate bisection -> part[T] in 0..nsub-1."""
    T = st.shape[0]
    if nsub < 1 or nsub > T:
        raise ValueError("nsub must be in [1, number of tetrahedra]")
    cen = centroids(xyz, st)
    part = np.empty(T, dtype=np.int64)
    stack = [(np.arange(T), 0, nsub)]
    while stack:
        ids, base, p = stack.pop()
        if p == 1:
            part[ids] = base
            continue
        c = cen[ids]
        ext = c.max(axis=0) - c.min(axis=0)
        axis = int(np.argmax(ext))
        order = np.lexsort((ids, c[:, axis]))
        srt = ids[order]
        p0 = p // 2
        h = (len(ids) * p0) // p
        stack.append((srt[h:], base + p0, p - p0))
        stack.append((srt[:h], base, p0))
    return part


def overlap_tets(st, nv, part, nsub, delta, kind="vertex", face_tets=None, tet_faces=None):
    """Omega_s^delta for every s: ascending tet ids.  kind="vertex": a layer adds every
    tetrahedron sharing a vertex with the set; kind="face": sharing a face."""
    out = []
    for s in range(nsub):
        mark = part == s
        for _ in range(delta):
            if kind == "face":
                nxt = mark.copy()
                f = tet_faces[mark].ravel()
                for q in range(2):
                    o = face_tets[f, q]
                    nxt[o[o >= 0]] = True
                mark = nxt
            else:
                vm = np.zeros(nv, dtype=bool)
                vm[st[mark].ravel()] = True
                mark = vm[st].any(axis=1)
        out.append(np.nonzero(mark)[0])
    return out


@dataclass
class Decomposition:
    part: np.ndarray
    tets: list            # Omega_s^delta tet ids
    dofs: list            # N_s (ascending global ids)
    pou: list             # D_s diagonal (float 0/1)
    owner: np.ndarray     # owner subdomain per global DOF
    iface: list = field(default_factory=list)  # per s: (tet, local face) arrays of interface faces


def decompose(topo: Topology, xyz, nsub, delta, part=None, kind="vertex") -> Decomposition:
    if part is None:
        part = rcb(xyz, topo.st, nsub)
    part = np.asarray(part, dtype=np.int64)
    tets = overlap_tets(topo.st, topo.nv, part, nsub, delta, kind, topo.face_tets, topo.tet_faces)
    owner = part[dof_min_tet(topo)]
    dofs, pou, iface = [], [], []
    for s in range(nsub):
        Ns = np.unique(topo.dofmap[tets[s]].ravel())
        dofs.append(Ns)
        pou.append((owner[Ns] == s).astype(np.float64))
        inside = np.zeros(topo.nt, dtype=bool)
        inside[tets[s]] = True
        t_l, f_l = [], []
        for t in tets[s]:
            for lf in range(4):
                f = topo.tet_faces[t, lf]
                a, b = topo.face_tets[f]
                other = b if a == t else a
                if other >= 0 and not inside[other]:
                    t_l.append(t)
                    f_l.append(lf)
        iface.append((np.array(t_l, dtype=np.int64), np.array(f_l, dtype=np.int64)))
    return Decomposition(part=part, tets=tets, dofs=dofs, pou=pou, owner=owner, iface=iface)


def local_matrix(topo: Topology, xyz, eps_r, mu_r, k0, dec: Decomposition, s, beta_lf=None, mask=None):
    """Dense A_s: element terms of Omega_s^delta + outer impedance (beta of the caller's table
    beta_lf [T, 4] when given) + interface impedance (omega~ of the inside tetrahedron).  mask:
    Boolean [ndof] of the degrees of freedom constrained by metallic faces: their local rows and
    columns become identity rows and columns (the local problem posed on V, Sec. 2)."""
    Ns = dec.dofs[s]
    ts = dec.tets[s]
    n = len(Ns)
    A = np.zeros((n, n), dtype=np.complex128)
    AT = elements.element_matrices(xyz, topo.st[ts], topo.r, eps_r[ts], mu_r[ts], k0)
    loc = np.searchsorted(Ns, topo.dofmap[ts])
    for q in range(len(ts)):
        A[np.ix_(loc[q], loc[q])] += AT[q]
    # outer boundary faces carried by tets of the subdomain
    ft_t, ft_f, coef = [], [], []
    for t in ts:
        for lf in range(4):
            f = topo.tet_faces[t, lf]
            if topo.face_tets[f, 1] < 0:
                ft_t.append(t)
                ft_f.append(lf)
                coef.append(outer_beta(k0, eps_r, mu_r, t, lf, beta_lf))
    it, il = dec.iface[s]
    ft_t += list(it)
    ft_f += list(il)
    coef += list(impedance_beta(k0, eps_r[it], mu_r[it])) if len(it) else []
    if ft_t:
        S = elements.face_matrices(xyz, topo.st, np.array(ft_t), np.array(ft_f), topo.r)
        lt = np.searchsorted(Ns, topo.dofmap[np.array(ft_t)])
        for q in range(len(ft_t)):
            A[np.ix_(lt[q], lt[q])] += 1j * coef[q] * S[q]
    if mask is not None:
        fixed = np.nonzero(mask[Ns])[0]
        A[fixed, :] = 0.0
        A[:, fixed] = 0.0
        A[fixed, fixed] = 1.0
    return A


def restricted_matrix(A_global, dec: Decomposition, s):
    """Dense R_s A R_s^T: the rows and columns N_s of the global matrix (restricted additive
    Schwarz with Dirichlet transmission, the variant the paper compares ORAS against, Sec. 4)."""
    Ns = dec.dofs[s]
    return A_global[Ns][:, Ns].toarray()


class ORAS:
    """M^{-1} v = sum_s R_s^T D_s A_s^{-1} R_s v with LU-factored dense A_s.

    transmission "impedance": A_s of local_matrix (ORAS, Sec. 4); "dirichlet": A_s = R_s A R_s^T
    (RAS), which needs the global matrix A_global."""

    def __init__(self, topo, xyz, eps_r, mu_r, k0, dec: Decomposition, weights="pou",
                 transmission="impedance", A_global=None, beta_lf=None, mask=None):
        self.dec = dec
        self.n = topo.ndof
        self.lu = []
        for s in range(len(dec.dofs)):
            if transmission == "dirichlet":
                A = restricted_matrix(A_global, dec, s)
            else:
                A = local_matrix(topo, xyz, eps_r, mu_r, k0, dec, s, beta_lf, mask)
            self.lu.append(sla.lu_factor(A, check_finite=False))
        self.weights = weights

    def apply(self, v):
        z = np.zeros(self.n, dtype=np.complex128)
        for s, Ns in enumerate(self.dec.dofs):
            u = sla.lu_solve(self.lu[s], v[Ns], check_finite=False)
            if self.weights == "pou":
                z[Ns] += self.dec.pou[s] * u
            else:  # OAS: no partition of unity
                z[Ns] += u
        return z
