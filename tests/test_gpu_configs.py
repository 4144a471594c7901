"""GPU parity on the paths the full-size workloads take: 32 right-hand sides solved together (eight
grouped passes of the apply, a 32-column Krylov basis), the 24^3 x 6, degree-2, 256-subdomain mesh
with 32 dipoles, degree 3 without overlap on many small subdomains, and caller-given impedance
coefficients beta on the outer faces (Sec. 2).

Bars as in test_gpu_parity.py: integer arrays bit-exact; A within 1e-12; every column's true FP64
residual <= 1e-8 measured with the oracle's own A; fields within 1e-6 of the oracle's or of a
sparse direct solve.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import assemble, dd, problem, topology

pytestmark = pytest.mark.gpu


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


def test_32_right_hand_sides_together(O):
    """Sec. 5 pseudo-block: 32 dipoles on the ring in one oras_solve (6^3 x 6, r = 2, 16
    subdomains); every column meets the FP64 bars against the oracle's A and a direct solve, and
    equals the same right-hand side solved alone to 1e-6."""
    w = synth.small(n=6, r=2, nsub=16, overlap=1, nrhs=32)
    p = problem.from_workload(w, with_oras=False)
    xyz, tets = w.mesh()
    eps, mu = w.materials(xyz, tets)
    h = O.oras_setup(xyz, tets, eps, mu, w.k0, w.r, w.nsub, w.overlap, restart=w.restart)
    try:
        X, info, rc = O.oras_solve(h, p.B, w.tol, k=32)
        assert rc == O.ORAS_OK and all(i["converged"] for i in info)
        lu = spla.splu(p.A.tocsc())
        XD = lu.solve(p.B)
        for j in range(32):
            b = p.B[:, j]
            assert np.linalg.norm(b - p.A @ X[:, j]) / np.linalg.norm(b) <= 1e-8
            assert rel(X[:, j], XD[:, j]) <= 1e-6
        for j in (0, 17, 31):
            xj, _, _ = O.oras_solve(h, p.B[:, j].copy(), w.tol)
            assert rel(X[:, j], xj) <= 1e-6
    finally:
        O.oras_destroy(h)


def test_config3_mesh_32_dipoles(O):
    """The batched multi-source workload: 24^3 x 6 tets (82,944), r = 2 (542,736 DOFs), 256
    subdomains by RCB, one vertex overlap layer, 32 z-dipoles on the ring solved together.  The
    integer set-up is bit-exact against the oracle (numbering, partition, N_s, D_s of every
    subdomain) and all 32 fields reach a true FP64 residual <= 1e-8 with the oracle's
    independently assembled A."""
    w = synth.config(2)
    xyz, tets = w.mesh()
    eps, mu = w.materials(xyz, tets)
    topo = topology.build(tets, len(xyz), w.r)
    dec = dd.decompose(topo, xyz, w.nsub, w.overlap)
    h = O.oras_setup(xyz, tets, eps, mu, w.k0, w.r, w.nsub, w.overlap, restart=w.restart)
    try:
        assert O.oras_ndof(h) == topo.ndof == 542736
        assert np.array_equal(O.oras_dofmap(h, len(tets)), topo.dofmap)
        assert np.array_equal(O.oras_partition(h, len(tets)), dec.part)
        for s in range(w.nsub):
            dofs, pou, tt = O.oras_subdomain(h, s)
            assert np.array_equal(dofs, dec.dofs[s])
            assert np.array_equal(pou, dec.pou[s].astype(np.uint8))
            assert np.array_equal(tt, dec.tets[s])
        A = assemble.global_matrix(topo, xyz, eps, mu, w.k0)
        pts = synth.dipole_ring(32)
        B = np.stack([assemble.dipole_load(topo, xyz, pts[j], [0, 0, 1.0]) for j in range(32)], axis=1)
        X, info, rc = O.oras_solve(h, B, w.tol, k=32)
        assert rc == O.ORAS_OK
        for j in range(32):
            res = np.linalg.norm(B[:, j] - A @ X[:, j]) / np.linalg.norm(B[:, j])
            assert res <= 1e-8, (j, res)
            assert abs(info[j]["relres"] - res) <= 1e-9
    finally:
        O.oras_destroy(h)


@pytest.mark.parametrize("bits", [32, 64])
def test_degree3_no_overlap_64_subdomains(O, bits):
    """Degree 3 with zero overlap on 64 subdomains of six tetrahedra each (the large degree-3
    workload's structure in small form: subdomains share interface DOFs only): the apply matches
    the oracle's ORAS and the solve reaches the oracle's field and the direct solution."""
    w = synth.small(n=4, r=3, nsub=64, overlap=0, restart=100)
    p = problem.from_workload(w)
    xyz, tets = w.mesh()
    eps, mu = w.materials(xyz, tets)
    h = O.oras_setup(xyz, tets, eps, mu, w.k0, w.r, w.nsub, w.overlap, factor_bits=bits, restart=w.restart,
                     max_iter=3000)
    try:
        rng = np.random.default_rng(64)
        v = rng.normal(size=p.topo.ndof) + 1j * rng.normal(size=p.topo.ndof)
        assert rel(O.oras_precond(h, v), p.oras.apply(v)) <= (1e-9 if bits == 64 else 20 * 2.0 ** -11)
        b = p.B[:, 0]
        x, info, rc = O.oras_solve(h, b, w.tol)
        assert rc == O.ORAS_OK
        assert np.linalg.norm(b - p.A @ x) / np.linalg.norm(b) <= 1e-8
        assert rel(x, spla.spsolve(p.A.tocsc(), b)) <= 1e-6
        if bits == 64:
            xo = problem.solve(p, tol=w.tol, m=w.restart, max_iter=3000)[0]
            assert xo.converged and rel(x, xo.x) <= 1e-6
            assert abs(info[0]["iterations"] - xo.iterations) <= 2
    finally:
        O.oras_destroy(h)


def test_caller_impedance_coefficients(O):
    """oras_problem.beta_face: a seeded beta in [4, 20] on every outer face (Sec. 2 allows one beta
    per port).  The GPU's A and plane-wave load equal the oracle's with the same table to 1e-12, a
    table equal to the derived beta reproduces the default operator bit for bit, and the solve
    meets the FP64 bars."""
    w = synth.small(n=4, r=2, nsub=8, overlap=1, head=False, source="plane")
    xyz, tets = w.mesh()
    eps, mu = w.materials(xyz, tets)
    rng = np.random.default_rng(1605)
    beta = rng.uniform(4.0, 20.0, size=(len(tets), 4))
    p = problem.build(xyz, tets, eps, mu, w.k0, w.r, w.sources(), w.nsub, w.overlap, beta_face=beta)
    h = O.oras_setup(xyz, tets, eps, mu, w.k0, w.r, w.nsub, w.overlap, beta_face=beta)
    h0 = O.oras_setup(xyz, tets, eps, mu, w.k0, w.r, w.nsub, w.overlap)
    hd = O.oras_setup(xyz, tets, eps, mu, w.k0, w.r, w.nsub, w.overlap,
                      beta_face=np.full((len(tets), 4), assemble.impedance_beta(w.k0, eps[0], mu[0])))
    try:
        A = p.A.tocsr()
        A.sort_indices()
        _, cols, vals = O.oras_global_csr(h)
        assert np.array_equal(cols, A.indices)
        assert np.abs(vals - A.data).max() <= 1e-12 * np.abs(A.data).max()
        assert not np.allclose(vals, O.oras_global_csr(h0)[2])
        assert np.array_equal(O.oras_global_csr(hd)[2], O.oras_global_csr(h0)[2])
        b = O.oras_rhs_plane_wave(h, synth.PLANE_D, synth.PLANE_P.astype(np.complex128))
        assert rel(b, p.B[:, 0]) <= 1e-12
        rngv = np.random.default_rng(2)
        v = rngv.normal(size=p.topo.ndof) + 1j * rngv.normal(size=p.topo.ndof)
        assert rel(O.oras_precond(h, v), p.oras.apply(v)) <= 10 * 2.0 ** -11
        x, info, rc = O.oras_solve(h, b, w.tol)
        assert rc == O.ORAS_OK
        assert np.linalg.norm(p.B[:, 0] - p.A @ x) / np.linalg.norm(p.B[:, 0]) <= 1e-8
        assert rel(x, spla.spsolve(p.A.tocsc(), p.B[:, 0])) <= 1e-6
    finally:
        for hh in (h, h0, hd):
            O.oras_destroy(hh)
