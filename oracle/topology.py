"""Mesh topology and global DOF numbering (oracle; test infrastructure).

Sec. 3 numbers the unknowns by the entities (edges, faces, volumes) of the mesh
T_h.  Convention used here (shared with the CUDA library as a *convention*, not as
code):

* every tetrahedron's vertices are sorted ascending by global id, so the local
  edge (a, b) and face (a, b, c) always have a < b < c and carry the same
  orientation in every tetrahedron that contains them (no sign flips);
* edges are numbered in ascending (a, b) order, faces in ascending (a, b, c) order;
* global DOF ids: all edge DOFs (edge id * r + q), then all face DOFs
  (E*r + face id * r(r-1) + q), then the volume DOFs (E*r + F*r(r-1) + tet * nv + q),
  with q the index inside the entity as defined in `oracle.basis.local_dofs`.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import basis


@dataclass
class Topology:
    r: int
    nv: int
    st: np.ndarray          # int64[T,4] sorted vertex ids
    edges: np.ndarray       # int64[E,2]
    faces: np.ndarray       # int64[F,3]
    tet_edges: np.ndarray   # int64[T,6]  (LOCAL_EDGES order)
    tet_faces: np.ndarray   # int64[T,4]  (LOCAL_FACES order)
    face_tets: np.ndarray   # int64[F,2]  tets sharing the face (second = -1 on the boundary)
    dofmap: np.ndarray      # int64[T, n_local]
    ndof: int

    @property
    def nt(self):
        return self.st.shape[0]

    @property
    def ne(self):
        return self.edges.shape[0]

    @property
    def nf(self):
        return self.faces.shape[0]

    def boundary_faces(self):
        return np.nonzero(self.face_tets[:, 1] < 0)[0]


def build(tets, nv, r) -> Topology:
    st = np.sort(np.asarray(tets, dtype=np.int64), axis=1)
    T = st.shape[0]
    nv = int(nv)
    ekeys = np.stack([st[:, a] * nv + st[:, b] for (a, b) in basis.LOCAL_EDGES], axis=1)
    uek, einv = np.unique(ekeys.ravel(), return_inverse=True)
    edges = np.stack([uek // nv, uek % nv], axis=1)
    tet_edges = einv.reshape(T, 6)
    fkeys = np.stack([(st[:, a] * nv + st[:, b]) * nv + st[:, c] for (a, b, c) in basis.LOCAL_FACES],
                     axis=1)
    ufk, finv = np.unique(fkeys.ravel(), return_inverse=True)
    faces = np.stack([ufk // (nv * nv), (ufk // nv) % nv, ufk % nv], axis=1)
    tet_faces = finv.reshape(T, 4)
    # face -> tets (ascending tet id); interior faces have exactly two tets
    ft = np.full((len(ufk), 2), -1, dtype=np.int64)
    order = np.argsort(tet_faces.ravel(), kind="stable")
    fid_sorted = tet_faces.ravel()[order]
    tet_sorted = order // 4
    first = np.ones(len(order), dtype=bool)
    first[1:] = fid_sorted[1:] != fid_sorted[:-1]
    ft[fid_sorted[first], 0] = tet_sorted[first]
    ft[fid_sorted[~first], 1] = tet_sorted[~first]
    E, F = len(uek), len(ufk)
    ned, nfd, nvd = basis.n_edge_dofs(r), basis.n_face_dofs(r), basis.n_vol_dofs(r)
    dofs = basis.local_dofs(r)
    dofmap = np.empty((T, len(dofs)), dtype=np.int64)
    for l, (kind, ent, q, *_rest) in enumerate(dofs):
        if kind == "e":
            dofmap[:, l] = tet_edges[:, ent] * ned + q
        elif kind == "f":
            dofmap[:, l] = E * ned + tet_faces[:, ent] * nfd + q
        else:
            dofmap[:, l] = E * ned + F * nfd + np.arange(T) * nvd + q
    ndof = E * ned + F * nfd + T * nvd
    return Topology(r=r, nv=nv, st=st, edges=edges, faces=faces, tet_edges=tet_edges,
                    tet_faces=tet_faces, face_tets=ft, dofmap=dofmap, ndof=ndof)


def dof_min_tet(topo: Topology):
    """For every global DOF, the lowest-index tetrahedron whose entities carry it."""
    out = np.full(topo.ndof, np.iinfo(np.int64).max, dtype=np.int64)
    tid = np.repeat(np.arange(topo.nt), topo.dofmap.shape[1])
    np.minimum.at(out, topo.dofmap.ravel(), tid)
    return out
