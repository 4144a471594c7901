"""Whole-chain oracle driver for one synthetic workload (test infrastructure)."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse.linalg as spla

from . import assemble, dd, fgmres, ports, topology


@dataclass
class OracleProblem:
    xyz: np.ndarray
    tets: np.ndarray
    eps_r: np.ndarray
    mu_r: np.ndarray
    k0: float
    r: int
    topo: topology.Topology
    A: object
    B: np.ndarray          # [N, k]
    dec: object = None
    oras: object = None
    mask: object = None    # degrees of freedom constrained by metallic faces (or None)


def build(xyz, tets, eps_r, mu_r, k0, r, sources, nsub=None, delta=None, part=None,
          with_oras=True, beta_face=None, face_kind=None):
    """beta_face: [T, 4] impedance coefficients on the face opposite the caller's vertex
    tets[t, q] (outer faces only), or None (derived from the materials).  face_kind: [T, 4] on
    the same faces, 1 = metallic (E x n = 0), 0 = impedance, or None.  sources: ("plane", d, p),
    ("dipole", x0, dir) or ("port", oracle.ports.Port, None)."""
    topo = topology.build(tets, xyz.shape[0], r)
    beta_lf = None if beta_face is None else assemble.face_beta_table(tets, beta_face)
    mask = None
    if face_kind is not None:
        mask = ports.constrained_dofs(topo, xyz, ports.face_kind_table(tets, face_kind))
    A = assemble.global_matrix(topo, xyz, eps_r, mu_r, k0, beta_lf, mask)
    cols = []
    for kind, a, b in sources:
        if kind == "plane":
            col = assemble.plane_wave_load(topo, xyz, eps_r, mu_r, k0, a, b, beta_lf=beta_lf)
        elif kind == "port":
            col = ports.port_load(topo, xyz, mu_r, a)
        else:
            col = assemble.dipole_load(topo, xyz, a, b)
        if mask is not None:
            col[mask] = 0.0
        cols.append(col)
    B = np.stack(cols, axis=1) if cols else np.zeros((topo.ndof, 0), dtype=np.complex128)
    prob = OracleProblem(xyz, tets, eps_r, mu_r, k0, r, topo, A, B, mask=mask)
    if with_oras and nsub is not None:
        prob.dec = dd.decompose(topo, xyz, nsub, delta, part)
        prob.oras = dd.ORAS(topo, xyz, eps_r, mu_r, k0, prob.dec, beta_lf=beta_lf, mask=mask)
    return prob


def from_workload(w, with_oras=True):
    xyz, tets = w.mesh()
    eps_r, mu_r = w.materials(xyz, tets)
    return build(xyz, tets, eps_r, mu_r, w.k0, w.r, w.sources(), w.nsub, w.overlap,
                 with_oras=with_oras)


def solve(prob: OracleProblem, tol=1e-8, m=50, max_iter=5000):
    out = []
    for j in range(prob.B.shape[1]):
        out.append(fgmres.fgmres(lambda v: prob.A @ v, prob.oras.apply, prob.B[:, j], tol, m,
                                 max_iter))
    return out


def direct(prob: OracleProblem):
    return spla.spsolve(prob.A.tocsc(), prob.B)
