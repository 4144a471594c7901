"""GPU metallic walls, waveguide ports and scattering coefficients (Sec. 2 eqs. metallicbc, wgj,
wgi; Sec. 5.1 eq. sij) against the oracle (tests/test_oracle_ports.py pins it).

* TE10 waveguide (metallic side walls, ports at both ends):
  - the constrained global matrix, the port vector and its norm, and the port load all match
    the oracle to 1e-12;
  - the preconditioner apply matches the oracle's to 1e-9 with FP64 factors and to 20 * 2^-11
    with FP32 factors (the lossless filling conditions the local matrices about 4x worse than
    the lossy benchmark medium);
  - the solve reaches a true residual of 1e-8 with the oracle's A and the direct solution to
    1e-6, with zero field on the constrained unknowns;
  - the S matrix of the GPU field equals the oracle's S of the same field to 1e-12, and the
    exact S (1, exp(i beta)) within the discretisation error the oracle pins at that mesh.
* Eight ports on the side faces of a lossy cube with a metallic bottom, 8 right-hand sides
  solved together: the S matrix is symmetric (reciprocity: A = A^T and equal port norms) to the
  solver tolerance.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import assemble, dd, ports, problem
from test_oracle_ports import BETA, EPS_WG, K0, PORT1, PORT2, SIDE_WALLS, wall_kinds

pytestmark = pytest.mark.gpu

# FP32 factors: the lossless waveguide filling makes the local matrices about 4x worse
# conditioned than those of the lossy benchmark medium (cond 510-670 against 150 on 3^3, r = 2), so
# the apply takes the bar of the worse-conditioned degree-3 matrices, 20 * 2^-11 (TF32 updates).
TOL_APPLY_F32_LOSSLESS = 20 * 2.0 ** -11


@pytest.fixture(scope="module")
def O():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_04521_gb300 import build
    build.build()
    from paper_1605_04521_gb300 import oras
    return oras


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def gport(O, P):
    return O.port(P.origin, P.u, P.v, P.beta)


@pytest.mark.parametrize("n,r,bits,s_bound", [(3, 2, 32, 7.5e-3), (2, 3, 64, 2.5e-3), (3, 1, 32, 0.11)])
def test_te10_waveguide(O, n, r, bits, s_bound):
    xyz, tets = synth.kuhn_cube(n)
    rng = np.random.default_rng(n + r)
    tets = np.array([rng.permutation(t) for t in tets])       # caller's vertex order
    nt = len(tets)
    eps = np.full(nt, EPS_WG + 0j)
    mu = np.ones(nt, dtype=np.complex128)
    kind = wall_kinds(xyz, tets, SIDE_WALLS)
    beta = np.full((nt, 4), BETA)
    prob = problem.build(xyz, tets, eps, mu, K0, r, [("port", PORT1, None)], nsub=4, delta=1,
                         beta_face=beta, face_kind=kind)
    h = O.oras_setup(xyz, tets, eps, mu, K0, r, 4, 1, beta_face=beta, face_kind=kind, factor_bits=bits)
    try:
        assert np.array_equal(O.oras_constrained_dofs(h).astype(bool), prob.mask)
        # the library keeps the unconstrained pattern (explicit zeros in constrained rows and
        # columns); compare the matrices entry by entry
        rowptr, cols, vals = O.oras_global_csr(h)
        Ag = sp.csr_matrix((vals, cols, rowptr), shape=prob.A.shape)
        assert abs(Ag - prob.A).max() <= 1e-12 * abs(prob.A).max()
        p_ref, n_ref = ports.port_vector(prob.topo, xyz, PORT2)
        p, nrm = O.oras_port_vector(h, gport(O, PORT2))
        assert rel(p, p_ref) <= 1e-12 and abs(nrm - n_ref) <= 1e-13 * n_ref
        b = O.oras_rhs_port(h, gport(O, PORT1))
        assert rel(b, prob.B[:, 0]) <= 1e-12
        v = rng.normal(size=prob.topo.ndof) + 1j * rng.normal(size=prob.topo.ndof)
        z = O.oras_precond(h, v)
        assert rel(z, prob.oras.apply(v)) <= (1e-9 if bits == 64 else TOL_APPLY_F32_LOSSLESS)
        x, info, rc = O.oras_solve(h, b, 1e-8)
        assert rc == O.ORAS_OK
        assert np.linalg.norm(b - prob.A @ x) / np.linalg.norm(b) <= 1e-8
        assert np.all(x[prob.mask] == 0.0)
        xd = spla.spsolve(prob.A.tocsc(), prob.B[:, 0])
        assert rel(x, xd) <= 1e-6
        S = O.oras_s_matrix(h, [gport(O, PORT1), gport(O, PORT2)], x)[:, 0]
        S_ref = ports.s_matrix(prob.topo, xyz, [PORT1, PORT2], x)[:, 0]
        assert np.abs(S - S_ref).max() <= 1e-12 * np.abs(S_ref).max()
        exact = np.array([1.0, np.exp(1j * BETA)])
        assert O.oras_s_error(S, exact) <= s_bound
        assert abs(O.oras_s_error(S, exact) - ports.s_error(S_ref, exact)) <= 1e-10
    finally:
        O.oras_destroy(h)


def side_ports(beta):
    """Eight 0.5 x 0.5 ports on the four side faces of the unit cube (two per face, at heights
    0 and 0.5), the mode pointing up (z)."""
    out = []
    for z0 in (0.0, 0.5):
        out.append(ports.Port(np.array([0.0, 0.25, z0]), np.array([0.0, 0.5, 0.0]), np.array([0.0, 0.0, 0.5]), beta))
        out.append(ports.Port(np.array([1.0, 0.25, z0]), np.array([0.0, 0.5, 0.0]), np.array([0.0, 0.0, 0.5]), beta))
        out.append(ports.Port(np.array([0.25, 0.0, z0]), np.array([0.5, 0.0, 0.0]), np.array([0.0, 0.0, 0.5]), beta))
        out.append(ports.Port(np.array([0.25, 1.0, z0]), np.array([0.5, 0.0, 0.0]), np.array([0.0, 0.0, 0.5]), beta))
    return out


def test_eight_ports_reciprocity(O):
    """Lossy head-like cube (4^3 x 6, r = 2, 8 subdomains), metallic bottom, eight ports with the
    Silver-Mueller condition on the side faces: the 8 x 8 S matrix of the 8 solves (one
    tensor-core apply pass per iteration) equals the oracle's S of the same fields to 1e-12 and
    is symmetric to the solver tolerance."""
    w = synth.small(n=4, r=2, nsub=8, overlap=1)
    xyz, tets = w.mesh()
    eps, mu = w.materials(xyz, tets)
    nt = len(tets)
    kind = wall_kinds(xyz, tets, [(2, 0.0)])
    beta_p = float(np.sqrt(w.k0 ** 2 * 59.0 - (np.pi / 0.5) ** 2))   # ceramic-filled guide, width 0.5
    beta = np.full((nt, 4), beta_p)
    P = side_ports(beta_p)
    prob = problem.build(xyz, tets, eps, mu, w.k0, w.r, [("port", q, None) for q in P], with_oras=False,
                         beta_face=beta, face_kind=kind)
    h = O.oras_setup(xyz, tets, eps, mu, w.k0, w.r, w.nsub, w.overlap, beta_face=beta, face_kind=kind)
    try:
        gp = [gport(O, q) for q in P]
        B = np.stack([O.oras_rhs_port(h, q) for q in gp], axis=1)
        assert rel(B, prob.B) <= 1e-12
        X, info, rc = O.oras_solve(h, B, 1e-8, k=8)
        assert rc == O.ORAS_OK
        for j in range(8):
            assert np.linalg.norm(B[:, j] - prob.A @ X[:, j]) / np.linalg.norm(B[:, j]) <= 1e-8
        S = O.oras_s_matrix(h, gp, X)
        S_ref = ports.s_matrix(prob.topo, xyz, P, X)
        assert np.abs(S - S_ref).max() <= 1e-12 * np.abs(S_ref).max()
        assert O.oras_s_error(S, S.T) <= 1e-7
        off = S - np.diag(np.diag(S))
        assert np.linalg.norm(off) > 1e-3 * np.linalg.norm(S)     # the transmissions are not negligible
    finally:
        O.oras_destroy(h)
