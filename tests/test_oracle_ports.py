"""Pins of the metallic condition, the waveguide ports and the scattering functional of the
oracle (oracle/ports.py; Sec. 2 eqs. metallicbc, wgj, wgi; Sec. 5.1 eq. sij; Sec. 5.2 eq. errsij).

Pinned against things other than the code itself:
* closed-form counts of the constrained degrees of freedom (boundary edges and faces of the Kuhn
  cube);
* the identity-row system equals the system reduced to the free degrees of freedom;
* the tangential trace of the solution vanishes on metallic faces, evaluated pointwise (a planted
  mistake that constrains the edge degrees of freedom only fails);
* the port vector against closed forms: int |E0|^2 = |u||v|/2, and against the constant field
  v/|v| (in the edge-element space for every r), int E0 . v/|v| = 2|u||v|/pi;
* the TE10 waveguide with metallic side walls and ports at both ends, whose exact solution is the
  incident mode itself: S_11 -> 1 and S_21 -> exp(i beta) at order about 2r under refinement.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import assemble, basis, elements, ports, problem, topology

K0 = 2.5
EPS_WG = 4.0          # lossless waveguide filling: gamma = 5, beta = sqrt(25 - pi^2)
BETA = float(np.sqrt((K0 * 2.0) ** 2 - np.pi ** 2))


def wall_kinds(xyz, tets, walls):
    """Caller's face_kind table: 1 on the faces lying in one of the planes (axis, value)."""
    kind = np.zeros((len(tets), 4), dtype=np.uint8)
    for t in range(len(tets)):
        for q in range(4):
            P = xyz[[tets[t][j] for j in range(4) if j != q]]
            for ax, val in walls:
                if np.all(np.abs(P[:, ax] - val) < 1e-12):
                    kind[t, q] = 1
    return kind


SIDE_WALLS = [(0, 0.0), (0, 1.0), (1, 0.0), (1, 1.0)]
ALL_WALLS = SIDE_WALLS + [(2, 0.0), (2, 1.0)]
PORT1 = ports.Port(np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.0, 1, 0]), BETA)
PORT2 = ports.Port(np.array([0.0, 0, 1]), np.array([1.0, 0, 0]), np.array([0.0, 1, 0]), BETA)


def waveguide(n, r, face_kind=None):
    xyz, tets = synth.kuhn_cube(n)
    nt = len(tets)
    eps = np.full(nt, EPS_WG + 0j)
    mu = np.ones(nt, dtype=np.complex128)
    fk = wall_kinds(xyz, tets, SIDE_WALLS) if face_kind is None else face_kind
    bf = np.full((nt, 4), BETA)
    prob = problem.build(xyz, tets, eps, mu, K0, r, [("port", PORT1, None)], with_oras=False,
                         beta_face=bf, face_kind=fk)
    return xyz, tets, prob


@pytest.mark.parametrize("r", [1, 2, 3])
@pytest.mark.parametrize("n", [2, 3])
def test_constrained_counts_closed_form(n, r):
    """All six faces metallic: every boundary edge (18 n^2) carries r constrained degrees of
    freedom and every boundary triangle (12 n^2) r(r-1).  The four side walls: 12 n^2 + 4 n edges
    and 8 n^2 triangles."""
    xyz, tets = synth.kuhn_cube(n)
    topo = topology.build(tets, len(xyz), r)
    full = ports.constrained_dofs(topo, xyz, ports.face_kind_table(tets, wall_kinds(xyz, tets, ALL_WALLS)))
    assert full.sum() == r * 18 * n * n + r * (r - 1) * 12 * n * n
    side = ports.constrained_dofs(topo, xyz, ports.face_kind_table(tets, wall_kinds(xyz, tets, SIDE_WALLS)))
    assert side.sum() == r * (12 * n * n + 4 * n) + r * (r - 1) * 8 * n * n


def test_constrained_system_is_the_reduced_system():
    """x = 0 on the constrained degrees of freedom and the free part solves A_ff x_f = b_f."""
    xyz, tets, prob = waveguide(3, 2)
    mask = prob.mask
    A0 = assemble.global_matrix(prob.topo, xyz, prob.eps_r, prob.mu_r, K0,
                                assemble.face_beta_table(tets, np.full((len(tets), 4), BETA)))
    b = prob.B[:, 0]
    x = spla.spsolve(prob.A.tocsc(), b)
    free = ~mask
    xf = spla.spsolve(A0[free][:, free].tocsc(), b[free])
    assert np.all(x[mask] == 0.0)
    assert np.linalg.norm(x[free] - xf) <= 1e-12 * np.linalg.norm(xf)
    assert np.all(b[mask] == 0.0)


def _tangential_trace_on_walls(prob, xyz, walls, mask_override=None):
    """Largest |E x n| at random points of the faces lying in the walls, relative to max |E|."""
    topo = prob.topo
    A, B = prob.A, prob.B[:, 0]
    if mask_override is not None:
        A = ports.constrain(assemble.global_matrix(topo, xyz, prob.eps_r, prob.mu_r, K0,
                                                   assemble.face_beta_table(prob.tets, np.full((topo.nt, 4), BETA))),
                            mask_override)
        B = B.copy()
        B[mask_override] = 0.0
    x = spla.spsolve(A.tocsc(), B)
    rng = np.random.default_rng(3)
    worst = scale = 0.0
    for t in range(topo.nt):
        for lf, fv in enumerate(basis.LOCAL_FACES):
            f = topo.tet_faces[t, lf]
            if topo.face_tets[f, 1] >= 0:
                continue
            P = xyz[topo.st[t][list(fv)]]
            if not any(np.all(np.abs(P[:, ax] - val) < 1e-12) for ax, val in walls):
                continue
            lam = rng.dirichlet(np.ones(3), size=4)
            pts = lam @ P
            verts = xyz[topo.st[t]]
            val, _ = basis.eval_local_basis(topo.r, verts, pts)          # [P,n,3]
            E = np.einsum("pai,a->pi", val, x[topo.dofmap[t]])
            o = basis.FACE_OPPOSITE[lf]
            g = basis.barycentric_gradients(verts)[o]
            nrm = g / np.linalg.norm(g)
            worst = max(worst, np.abs(np.cross(E, nrm)).max())
            scale = max(scale, np.abs(E).max())
    return worst / scale


def test_tangential_trace_vanishes_on_metallic_faces():
    """E x n = 0 on the metallic side walls (evaluated from the basis at random points), and a
    planted mistake that constrains only the edge degrees of freedom (r = 2 face degrees of
    freedom left free) leaves a tangential field there."""
    xyz, tets, prob = waveguide(3, 2)
    assert _tangential_trace_on_walls(prob, xyz, SIDE_WALLS) < 1e-12
    # planted mistake: drop the face degrees of freedom from the mask
    topo = prob.topo
    nedge = topo.edges.shape[0] * topo.r
    wrong = prob.mask.copy()
    wrong[nedge:] = False
    assert _tangential_trace_on_walls(prob, xyz, SIDE_WALLS, mask_override=wrong) > 1e-3


def _constant_field_coefficients(topo, xyz, r, c):
    """Coefficients of the constant field c in the local basis (least squares per tet, shared
    coefficients agree)."""
    coef = np.zeros(topo.ndof)
    rng = np.random.default_rng(1)
    for t in range(topo.nt):
        verts = xyz[topo.st[t]]
        lam = rng.dirichlet(np.ones(4), size=3 * basis.n_local(r))
        val, _ = basis.eval_local_basis(r, verts, lam @ verts)
        M = val.transpose(0, 2, 1).reshape(-1, val.shape[1])
        rhs = np.tile(c, lam.shape[0])
        sol, *_ = np.linalg.lstsq(M, rhs, rcond=None)
        coef[topo.dofmap[t]] = sol
    return coef


@pytest.mark.parametrize("r", [1, 2, 3])
def test_port_vector_closed_forms(r):
    """int_port |E0|^2 = |u||v| / 2 and, with c the coefficients of the constant field v/|v|,
    c . p = int_port E0 . v/|v| = 2 |u||v| / pi (the port's faces tile its rectangle)."""
    xyz, tets = synth.kuhn_cube(3)
    topo = topology.build(tets, len(xyz), r)
    port = ports.Port(np.array([0.0, 0, 1]), np.array([1.0, 0, 0]), np.array([0.0, 1, 0]), BETA)
    p, norm = ports.port_vector(topo, xyz, port)
    assert abs(norm - 0.5) < 1e-13
    c = _constant_field_coefficients(topo, xyz, r, np.array([0.0, 1.0, 0.0]))
    assert abs(c @ p.real - 2.0 / np.pi) < 1e-11
    assert np.all(p.imag == 0.0)
    # a port on part of a face: the rectangle [1/3, 1] x [0, 2/3] of z = 0
    sub = ports.Port(np.array([1.0 / 3, 0, 0]), np.array([2.0 / 3, 0, 0]), np.array([0.0, 2.0 / 3, 0]), BETA)
    _, nsub = ports.port_vector(topo, xyz, sub)
    assert abs(nsub - (2.0 / 3) * (2.0 / 3) / 2) < 1e-13


@pytest.mark.parametrize("r,ns,bound", [(2, (2, 3, 4), (3e-2, 7.5e-3, 2.6e-3)), (3, (2, 3), (2.5e-3, 2.6e-4))])
def test_te10_waveguide_converges_to_the_incident_mode(r, ns, bound):
    """Metallic side walls, TE10 incident on the port z = 0, Silver-Mueller port at z = 1: the
    exact field is sin(pi x) exp(-i beta z) y, so S_11 = 1 and S_21 = exp(i beta) (the
    conjugate of the field in eq. sij).  The scattering error of eq. errsij decreases at an
    observed order of at least 2r - 1 in the mesh size (measured 3.5-3.7 for r = 2, 5.6 for
    r = 3)."""
    errs = []
    for n in ns:
        xyz, tets, prob = waveguide(n, r)
        x = spla.spsolve(prob.A.tocsc(), prob.B[:, 0])
        S = ports.s_matrix(prob.topo, xyz, [PORT1, PORT2], x)[:, 0]
        errs.append(ports.s_error(S, np.array([1.0, np.exp(1j * BETA)])))
    assert all(e <= b for e, b in zip(errs, bound)), errs
    for (n1, e1), (n2, e2) in zip(zip(ns, errs), zip(ns[1:], errs[1:])):
        order = np.log(e1 / e2) / np.log(n2 / n1)
        assert order >= 2 * r - 1, (errs, order)


def test_s_error_formula():
    rng = np.random.default_rng(2)
    S = rng.normal(size=(5, 3)) + 1j * rng.normal(size=(5, 3))
    assert ports.s_error(S, S) == 0.0
    assert abs(ports.s_error(2 * S, S) - 1.0) < 1e-15
    assert abs(ports.s_error(S + 1e-3 * S, S) - 1e-3) < 1e-12


def test_face_kind_table_brute_force():
    rng = np.random.default_rng(5)
    tets = np.array([rng.permutation(10)[:4] for _ in range(20)])
    kind = rng.integers(0, 2, size=(20, 4))
    tab = ports.face_kind_table(tets, kind)
    for t in range(20):
        st = sorted(tets[t])
        for lf, fv in enumerate(basis.LOCAL_FACES):
            opp = (set(range(4)) - set(fv)).pop()
            assert tab[t, lf] == kind[t, list(tets[t]).index(st[opp])]


def test_scattering_matrix_is_reciprocal():
    """A = A^T and ports of equal size and beta make S symmetric (S_ij = S_ji): eight ports on
    the side faces of a lossy cube with a metallic bottom, direct solves, 1e-10.  The ports' faces
    meet the metallic bottom, so constrained unknowns lie in some ports."""
    xyz, tets = synth.kuhn_cube(2)
    nt = len(tets)
    rng = np.random.default_rng(4)
    eps = rng.uniform(30, 60, nt) - 1j * rng.uniform(5, 25, nt)
    mu = np.ones(nt, dtype=np.complex128)
    beta_p = float(np.sqrt(1.85 ** 2 * 59.0 - (np.pi / 0.5) ** 2))
    P = []
    for z0 in (0.0, 0.5):
        P.append(ports.Port(np.array([0.0, 0.0, z0]), np.array([0.0, 0.5, 0.0]), np.array([0.0, 0.0, 0.5]), beta_p))
        P.append(ports.Port(np.array([1.0, 0.5, z0]), np.array([0.0, 0.5, 0.0]), np.array([0.0, 0.0, 0.5]), beta_p))
        P.append(ports.Port(np.array([0.5, 0.0, z0]), np.array([0.5, 0.0, 0.0]), np.array([0.0, 0.0, 0.5]), beta_p))
        P.append(ports.Port(np.array([0.0, 1.0, z0]), np.array([0.5, 0.0, 0.0]), np.array([0.0, 0.0, 0.5]), beta_p))
    kind = wall_kinds(xyz, tets, [(2, 0.0)])
    prob = problem.build(xyz, tets, eps, mu, 1.85, 2, [("port", q, None) for q in P], with_oras=False,
                         beta_face=np.full((nt, 4), beta_p), face_kind=kind)
    X = spla.spsolve(prob.A.tocsc(), prob.B)
    S = ports.s_matrix(prob.topo, xyz, P, X)
    assert ports.s_error(S, S.T) <= 1e-10
    assert np.linalg.norm(S - np.diag(np.diag(S))) > 1e-3 * np.linalg.norm(S)
    assert any(np.any(prob.mask[np.nonzero(ports.port_vector(prob.topo, xyz, q)[0])[0]]) for q in P)
