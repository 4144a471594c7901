"""Nedelec generators of degree r on a tetrahedron (oracle; test infrastructure).

Sec. 3: the lowest-order (Whitney) function of the oriented edge e = {n_i, n_j} is
    w^e = lambda_i grad(lambda_j) - lambda_j grad(lambda_i),
and the degree-r generators are w^{k,e} = lambda^k w^e for every edge e and every
multi-index k of weight r-1.  Some generators are linearly dependent for r > 1;
Sec. 3 defers the choice of an independent subset to another work, so this oracle
uses the following rule (local vertices 0 < 1 < 2 < 3 sorted by global id, so every
edge and face gets the same orientation from every tetrahedron):

* edge (a, b): all k supported on {a, b}                -> r functions per edge;
* face (a, b, c): Whitney edges (a, b) and (a, c) only, k supported on the face and
  containing the face vertex opposite that edge          -> r(r-1) per face;
* volume (r = 3): Whitney edges (0,1), (0,2), (0,3), k = the two other vertices
                                                         -> 3 per tetrahedron.

Within an entity: edges order k by ascending lexicographic order of the exponents on
the entity's vertices (ascending vertex order); faces order by (edge, k); the volume
functions follow the edge order above.  Local order in a tetrahedron: the six edges
(0,1),(0,2),(0,3),(1,2),(1,3),(2,3), then the four faces (0,1,2),(0,1,3),(0,2,3),(1,2,3),
then the volume.
"""
from __future__ import annotations

import itertools
from functools import lru_cache

import numpy as np

LOCAL_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
LOCAL_FACES = ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3))
FACE_OPPOSITE = (3, 2, 1, 0)


def n_edge_dofs(r):
    return r


def n_face_dofs(r):
    return r * (r - 1)


def n_vol_dofs(r):
    return r * (r - 1) * (r - 2) // 2


def n_local(r):
    return 6 * n_edge_dofs(r) + 4 * n_face_dofs(r) + n_vol_dofs(r)


def _multi_indices(support, weight):
    """All exponent tuples on `support` (ascending vertices) of total `weight`, ascending lex."""
    out = []
    for combo in itertools.product(range(weight + 1), repeat=len(support)):
        if sum(combo) == weight:
            out.append(combo)
    out.sort()
    res = []
    for combo in out:
        k = [0, 0, 0, 0]
        for v, e in zip(support, combo):
            k[v] = e
        res.append(tuple(k))
    return res


@lru_cache(maxsize=None)
def local_dofs(r):
    """Local DOF table: tuples (kind, entity, q, i, j, k) meaning lambda^k w^{ij} (i < j)."""
    if r not in (1, 2, 3):
        raise ValueError("degree r must be 1, 2 or 3")
    dofs = []
    for e, (a, b) in enumerate(LOCAL_EDGES):
        for q, k in enumerate(_multi_indices((a, b), r - 1)):
            dofs.append(("e", e, q, a, b, k))
    if r >= 2:
        for f, (a, b, c) in enumerate(LOCAL_FACES):
            q = 0
            for (i, j, opp) in ((a, b, c), (a, c, b)):
                for k in _multi_indices((a, b, c), r - 1):
                    if k[opp] >= 1:
                        dofs.append(("f", f, q, i, j, k))
                        q += 1
    if r == 3:
        for q, (i, j) in enumerate(((0, 1), (0, 2), (0, 3))):
            rest = [v for v in range(4) if v not in (i, j)]
            k = [0, 0, 0, 0]
            for v in rest:
                k[v] = 1
            dofs.append(("v", 0, q, i, j, tuple(k)))
    assert len(dofs) == n_local(r)
    return tuple(dofs)


@lru_cache(maxsize=None)
def all_generators(r):
    """The full (dependent) generator family lambda^k w^e, |k| = r-1, of Sec. 3."""
    gens = []
    for (a, b) in LOCAL_EDGES:
        for k in _multi_indices((0, 1, 2, 3), r - 1):
            gens.append((a, b, k))
    return tuple(gens)


def barycentric_gradients(verts):
    """grad(lambda_l) for a tetrahedron with vertex coordinates verts[4,3] -> [4,3]."""
    J = np.stack([verts[1] - verts[0], verts[2] - verts[0], verts[3] - verts[0]], axis=1)
    Jinv = np.linalg.inv(J)  # rows = grad lambda_1..3
    g = np.empty((4, 3))
    g[1:] = Jinv
    g[0] = -Jinv.sum(axis=0)
    return g


def barycentrics(verts, x):
    """Barycentric coordinates of points x[P,3] in tetrahedron verts[4,3] -> [P,4]."""
    J = np.stack([verts[1] - verts[0], verts[2] - verts[0], verts[3] - verts[0]], axis=1)
    lam123 = np.linalg.solve(J, (np.atleast_2d(x) - verts[0]).T).T
    return np.concatenate([1.0 - lam123.sum(axis=1, keepdims=True), lam123], axis=1)


def eval_generator(i, j, k, lam, glam):
    """Value of lambda^k (lambda_i grad lambda_j - lambda_j grad lambda_i) at points.

    lam[P,4] barycentrics, glam[4,3] gradients -> [P,3].
    """
    lk = np.prod(lam ** np.array(k), axis=1)
    w = lam[:, i:i + 1] * glam[j] - lam[:, j:j + 1] * glam[i]
    return lk[:, None] * w


def eval_generator_curl(i, j, k, lam, glam):
    """curl(lambda^k w^{ij}) = grad(lambda^k) x w^{ij} + 2 lambda^k grad(lambda_i) x grad(lambda_j).

    This is the product formula of Sec. 3 applied to lambda^k times a Whitney function.
    """
    k = np.array(k)
    lk = np.prod(lam ** k, axis=1)
    grad_lk = np.zeros((lam.shape[0], 3))
    for m in range(4):
        if k[m] > 0:
            km = k.copy()
            km[m] -= 1
            grad_lk += (k[m] * np.prod(lam ** km, axis=1))[:, None] * glam[m]
    w = lam[:, i:i + 1] * glam[j] - lam[:, j:j + 1] * glam[i]
    return np.cross(grad_lk, w) + 2.0 * lk[:, None] * np.cross(glam[i], glam[j])[None, :]


def eval_local_basis(r, verts, x):
    """Values [P, n_local, 3] and curls [P, n_local, 3] of the local basis at points x."""
    lam = barycentrics(verts, x)
    glam = barycentric_gradients(verts)
    dofs = local_dofs(r)
    val = np.stack([eval_generator(d[3], d[4], d[5], lam, glam) for d in dofs], axis=1)
    cur = np.stack([eval_generator_curl(d[3], d[4], d[5], lam, glam) for d in dofs], axis=1)
    return val, cur


def eval_basis_batch(r, lam, glam):
    """Values and curls of the local basis of many tetrahedra at the same barycentric points.

    lam[P,4] barycentric coordinates of the points (the same in every tetrahedron), glam[T,4,3]
    barycentric gradients of each tetrahedron.  Returns values [T,P,n_local,3] and curls
    [T,P,n_local,3], evaluated from the definitions of Sec. 3 exactly as eval_generator and
    eval_generator_curl do for one tetrahedron:
        w = lambda^k (lambda_i grad lambda_j - lambda_j grad lambda_i),
        curl w = grad(lambda^k) x w^{ij} + 2 lambda^k grad lambda_i x grad lambda_j.
    """
    lam = np.asarray(lam, dtype=np.float64)
    glam = np.asarray(glam, dtype=np.float64)
    T, P = glam.shape[0], lam.shape[0]
    dofs = local_dofs(r)
    val = np.empty((T, P, len(dofs), 3))
    cur = np.empty((T, P, len(dofs), 3))
    for a, (_, _, _, i, j, k) in enumerate(dofs):
        k = np.array(k)
        lk = np.prod(lam ** k, axis=1)                                       # [P]
        w = lam[None, :, i, None] * glam[:, None, j, :] - lam[None, :, j, None] * glam[:, None, i, :]
        grad_lk = np.zeros((T, P, 3))
        for m in range(4):
            if k[m] > 0:
                km = k.copy()
                km[m] -= 1
                grad_lk += (k[m] * np.prod(lam ** km, axis=1))[None, :, None] * glam[:, None, m, :]
        val[:, :, a, :] = lk[None, :, None] * w
        cur[:, :, a, :] = (np.cross(grad_lk, w) +
                           2.0 * lk[None, :, None] * np.cross(glam[:, i, :], glam[:, j, :])[:, None, :])
    return val, cur
