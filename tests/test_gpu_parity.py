"""GPU path (C ABI) against the CPU oracle on the same seeded inputs.

Bars: integer arrays bit-exact; element matrices, A, right-hand sides and A x within 1e-12
relative; true FP64 residual of the GPU field <= 1e-8 measured with the oracle's own A; GPU
field within 1e-6 (relative L2) of the oracle's field.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import assemble, dd, elements, problem, topology

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


def gpu_handle(O, w, factor_bits=32, **kw):
    xyz, tets = w.mesh()
    eps, mu = w.materials(xyz, tets)
    return O.oras_setup(xyz, tets, eps, mu, w.k0, w.r, w.nsub, w.overlap, factor_bits=factor_bits,
                        restart=w.restart, **kw)


@pytest.mark.parametrize("r", [1, 2, 3])
def test_element_matrices(O, r):
    w = synth.small(n=3, r=r, nsub=2, overlap=0)
    h = gpu_handle(O, w)
    try:
        xyz, tets = w.mesh()
        eps, mu = w.materials(xyz, tets)
        topo = topology.build(tets, len(xyz), r)
        ref = elements.element_matrices(xyz, topo.st, r, eps, mu, w.k0)
        got = O.oras_element_matrices(h, np.arange(len(tets)))
        err = np.abs(got - ref).max(axis=(1, 2)) / np.abs(ref).max(axis=(1, 2))
        assert err.max() <= 1e-12, err.max()
    finally:
        O.oras_destroy(h)


@pytest.mark.parametrize("r,n", [(1, 4), (2, 3), (3, 2)])
def test_global_matrix_and_matvec(O, r, n):
    w = synth.small(n=n, r=r, nsub=4, overlap=1)
    h = gpu_handle(O, w)
    try:
        p = problem.from_workload(w, with_oras=False)
        A = p.A.tocsr()
        A.sort_indices()
        rowptr, cols, vals = O.oras_global_csr(h)
        assert np.array_equal(rowptr, A.indptr) and np.array_equal(cols, A.indices)
        assert np.abs(vals - A.data).max() <= 1e-12 * np.abs(A.data).max()
        rng = np.random.default_rng(11)
        X = rng.normal(size=(A.shape[0], 3)) + 1j * rng.normal(size=(A.shape[0], 3))
        Y = O.oras_matvec(h, X, k=3)
        assert rel(Y, A @ X) <= 1e-13
    finally:
        O.oras_destroy(h)


@pytest.mark.parametrize("r,n,k", [(1, 4, 1), (2, 3, 3), (3, 2, 9)])
def test_fp32_input_matvec_keeps_fp64_accuracy(O, r, n, k):
    """A z for complex FP32 z on the FP32 pipes (split A, exact product and sum errors) against the
    oracle's FP64 A @ z: every column within 1e-13 relative, no worse than the FP64 kernel's bar."""
    w = synth.small(n=n, r=r, nsub=4, overlap=1)
    h = gpu_handle(O, w)
    try:
        p = problem.from_workload(w, with_oras=False)
        rng = np.random.default_rng(13)
        Z = (rng.normal(size=(p.A.shape[0], k)) + 1j * rng.normal(size=(p.A.shape[0], k))).astype(np.complex64)
        Y = np.asarray(O.oras_matvec_c64(h, Z, k=k)).reshape(-1, k)
        ref = p.A @ Z.astype(np.complex128)
        for j in range(k):
            assert rel(Y[:, j], ref[:, j]) <= 1e-13
    finally:
        O.oras_destroy(h)


def test_right_hand_sides(O):
    w = synth.config(0)
    h = gpu_handle(O, w, factor_bits=64)
    try:
        xyz, tets = w.mesh()
        eps, mu = w.materials(xyz, tets)
        topo = topology.build(tets, len(xyz), w.r)
        bp = assemble.plane_wave_load(topo, xyz, eps, mu, w.k0, synth.PLANE_D, synth.PLANE_P, nq=12)
        gp = O.oras_rhs_plane_wave(h, synth.PLANE_D, synth.PLANE_P.astype(np.complex128))
        assert rel(gp, bp) <= 1e-12
        for x0 in synth.dipole_ring(3):
            bd = assemble.dipole_load(topo, xyz, x0, [0, 0, 1.0])
            gd = O.oras_rhs_dipole(h, x0, [0, 0, 1.0])
            assert rel(gd, bd) <= 1e-12
        with pytest.raises(O.OrasError):
            O.oras_rhs_dipole(h, [2.0, 0.5, 0.5], [0, 0, 1.0])
    finally:
        O.oras_destroy(h)


# FP32 factors: the trailing updates round their operands to TF32 (unit roundoff 2^-11), so the
# apply of the FP32 factors differs from the FP64 oracle's by a small multiple of that.
TOL_APPLY_F32 = 10 * 2.0 ** -11
# Degree-3 local matrices are worse conditioned (observed up to 5.5e-3 on 4^3 x 6, 8 subdomains).
TOL_APPLY_F32_R3 = 20 * 2.0 ** -11


@pytest.mark.parametrize("bits,tol", [(64, 1e-9), (32, TOL_APPLY_F32)])
def test_preconditioner_apply(O, bits, tol):
    """z = M^-1 v against the oracle's ORAS (FP64 LU, partial pivoting)."""
    w = synth.small(n=4, r=2, nsub=8, overlap=1)
    h = gpu_handle(O, w, factor_bits=bits)
    try:
        p = problem.from_workload(w)
        rng = np.random.default_rng(12)
        v = rng.normal(size=p.topo.ndof) + 1j * rng.normal(size=p.topo.ndof)
        z = O.oras_precond(h, v)
        assert rel(z, p.oras.apply(v)) <= tol
    finally:
        O.oras_destroy(h)


@pytest.mark.parametrize("bits,tol", [(64, 1e-9), (32, TOL_APPLY_F32)])
def test_apply_many_subdomains(O, bits, tol):
    """128 subdomains without overlap: 256 CTAs (two per subdomain), more than the SMs hold at
    once, so with FP32 factors two CTAs share an SM on 3-stage rings (FP64 tiles keep one CTA
    per SM).  z = M^-1 v against the oracle's ORAS, and against the allocation-free apply of the
    same factors, which keeps its local vectors in global memory with one CTA per SM."""
    torch = pytest.importorskip("torch")
    w = synth.small(n=6, r=2, nsub=128, overlap=0)
    h = gpu_handle(O, w, factor_bits=bits)
    try:
        p = problem.from_workload(w)
        rng = np.random.default_rng(13)
        v = rng.normal(size=p.topo.ndof) + 1j * rng.normal(size=p.topo.ndof)
        z = O.oras_precond(h, v)
        assert rel(z, p.oras.apply(v)) <= tol
        vd = torch.from_numpy(v.copy()).cuda()
        zd = torch.full_like(vd, complex(np.nan, np.nan))
        O.oras_precond_noalloc(h, vd, zd, 1)
        torch.cuda.synchronize()
        assert rel(zd.cpu().numpy(), z) <= (1e-12 if bits == 64 else 1e-5)
    finally:
        O.oras_destroy(h)


@pytest.mark.parametrize("n,nsub,overlap,bits,panel", [
    (3, 1, 0, 64, 0), (3, 1, 0, 64, 2), (3, 1, 0, 32, 3), (3, 1, 0, 32, 24), (3, 1, 0, 32, 12), (3, 1, 0, 32, 20),
    (3, 1, 0, 64, 20), (4, 8, 1, 64, 0), (4, 8, 1, 32, 0), (4, 8, 1, 32, 2), (4, 8, 1, 64, 24)])
def test_preconditioner_apply_degree3(O, n, nsub, overlap, bits, panel):
    """Degree 3: the local matrices need row interchanges across panel boundaries of the batched
    LU.  With one subdomain M^-1 = A^-1 (the FGMRES converges in one step).  The single 3^3 x 6
    subdomain has 57 tile columns, so panels of 12, 20 and 24 columns leave columns beyond the
    panel: their pivot rows are solved after each sub-panel of 8 steps (12 and 20 end on a
    partial sub-panel of 4)."""
    w = synth.small(n=n, r=3, nsub=nsub, overlap=overlap)
    h = gpu_handle(O, w, factor_bits=bits, lu_panel=panel)
    try:
        p = problem.from_workload(w)
        rng = np.random.default_rng(31)
        v = rng.normal(size=p.topo.ndof) + 1j * rng.normal(size=p.topo.ndof)
        z = O.oras_precond(h, v)
        assert rel(z, p.oras.apply(v)) <= (1e-9 if bits == 64 else TOL_APPLY_F32_R3)
        if nsub == 1 and bits == 64:
            x, info, rc = O.oras_solve(h, p.B[:, 0], 1e-8)
            assert rc == O.ORAS_OK and info[0]["iterations"] == 1
    finally:
        O.oras_destroy(h)


@pytest.mark.parametrize("bits,tol", [(32, TOL_APPLY_F32), (64, 1e-9)])
def test_grouped_apply_matches_oracle(O, bits, tol):
    """Seven right-hand sides through the apply in groups (one arena pass per group)."""
    w = synth.small(n=4, r=2, nsub=8, overlap=1)
    h = gpu_handle(O, w, factor_bits=bits)
    try:
        p = problem.from_workload(w)
        rng = np.random.default_rng(21)
        k = 7
        V = rng.normal(size=(p.topo.ndof, k)) + 1j * rng.normal(size=(p.topo.ndof, k))
        Z = O.oras_precond(h, V, k=k)
        for j in range(k):
            assert rel(Z[:, j], O.oras_precond(h, V[:, j].copy())) <= 1e-5
            assert rel(Z[:, j], p.oras.apply(V[:, j])) <= tol
    finally:
        O.oras_destroy(h)


def test_grouped_apply_global_local_vectors(O):
    """One subdomain of about 21k DOFs (a cluster of four CTAs): a group of four right-hand
    sides keeps its local vectors in global memory (a CTA's quarter of the strips takes 172 KB
    for four vectors, more than fits beside two ring stages), a single vector keeps them in
    shared memory; both give the same z.  (The two-CTA kernel's global-memory path runs in the
    allocation-free apply, tests/test_zz_no_alloc.py.)"""
    w = synth.small(n=8, r=2, nsub=1, overlap=0)
    h = gpu_handle(O, w)
    try:
        n = O.oras_ndof(h)
        assert O.oras_subdomain_size(h, 0)[2] > 20000
        rng = np.random.default_rng(22)
        k = 6
        V = rng.normal(size=(n, k)) + 1j * rng.normal(size=(n, k))
        Z = O.oras_precond(h, V, k=k)
        for j in range(k):
            assert rel(Z[:, j], O.oras_precond(h, V[:, j].copy())) <= 1e-5
    finally:
        O.oras_destroy(h)


CASES = [
    dict(w=synth.config(0), bits=64),                                                   # 8^3, r=1, plane wave
    dict(w=synth.small(n=4, r=2, nsub=8, overlap=1), bits=32),                          # head, r=2
    dict(w=synth.small(n=3, r=3, nsub=4, overlap=1), bits=32),                          # r=3
    dict(w=synth.small(n=5, r=1, nsub=7, overlap=2, head=False, source="plane"), bits=32),  # nsub not 2^k
    dict(w=synth.small(n=3, r=2, nsub=1, overlap=0), bits=64),                          # one subdomain
    dict(w=synth.small(n=4, r=2, nsub=8, overlap=0), bits=32),                          # zero overlap
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_solve_matches_oracle(O, case):
    w, bits = CASES[case]["w"], CASES[case]["bits"]
    p = problem.from_workload(w)
    b = p.B[:, 0]
    h = gpu_handle(O, w, factor_bits=bits)
    try:
        x, info, rc = O.oras_solve(h, b, w.tol)
        assert rc == O.ORAS_OK and info[0]["converged"]
        true_res = np.linalg.norm(b - p.A @ x) / np.linalg.norm(b)
        assert true_res <= 1e-8
        assert abs(info[0]["relres"] - true_res) <= 1e-9
        xo = problem.solve(p, tol=w.tol, m=w.restart)[0]
        xd = spla.spsolve(p.A.tocsc(), b)
        assert rel(x, xo.x) <= 1e-6
        assert rel(x, xd) <= 1e-6
        if w.nsub == 1:
            assert info[0]["iterations"] == 1
    finally:
        O.oras_destroy(h)


def test_multi_rhs_alone_and_batched(O):
    w = synth.small(n=4, r=2, nsub=8, overlap=1, nrhs=4)
    p = problem.from_workload(w)
    h = gpu_handle(O, w)
    try:
        X, info, rc = O.oras_solve(h, p.B, w.tol, k=4)
        assert rc == O.ORAS_OK
        for j in range(4):
            b = p.B[:, j]
            assert np.linalg.norm(b - p.A @ X[:, j]) / np.linalg.norm(b) <= 1e-8
            xj, _, _ = O.oras_solve(h, b, w.tol)
            assert rel(X[:, j], xj) <= 1e-6
            assert rel(X[:, j], spla.spsolve(p.A.tocsc(), b)) <= 1e-6
    finally:
        O.oras_destroy(h)


def test_zero_rhs_and_device_pointers(O):
    import torch
    w = synth.small(n=3, r=2, nsub=4, overlap=1)
    p = problem.from_workload(w)
    h = gpu_handle(O, w)
    try:
        n = p.topo.ndof
        x, info, rc = O.oras_solve(h, np.zeros(n), 1e-8)
        assert rc == O.ORAS_OK and np.all(x == 0) and info[0]["iterations"] == 0
        xh, _, _ = O.oras_solve(h, p.B[:, 0], 1e-8)
        bt = torch.from_numpy(p.B[:, 0].copy()).cuda()
        xt = torch.empty_like(bt)
        O.oras_solve(h, bt, 1e-8, mem=O.ORAS_MEM_DEVICE, out=xt)
        torch.cuda.synchronize()
        assert np.array_equal(xt.cpu().numpy(), xh)
    finally:
        O.oras_destroy(h)


def test_refactor_equals_fresh_setup(O):
    """New materials on the same mesh handle give the same operator as a fresh set-up."""
    w = synth.small(n=4, r=2, nsub=8, overlap=1)
    xyz, tets = w.mesh()
    eps, mu = w.materials(xyz, tets)
    eps2 = eps.copy()
    eps2[::7] = 55 - 22j
    h1 = O.oras_setup(xyz, tets, eps, mu, w.k0, 2, 8, 1)
    h2 = O.oras_setup(xyz, tets, eps2, mu, w.k0, 2, 8, 1)
    try:
        O.oras_factor(h1, eps2, mu, w.k0)
        b = O.oras_rhs_dipole(h1, synth.dipole_ring(1)[0], [0, 0, 1.0])
        x1, _, _ = O.oras_solve(h1, b, 1e-8)
        x2, _, _ = O.oras_solve(h2, b, 1e-8)
        assert np.array_equal(x1, x2)
        assert np.array_equal(O.oras_global_csr(h1)[2], O.oras_global_csr(h2)[2])
    finally:
        O.oras_destroy(h1)
        O.oras_destroy(h2)


@pytest.mark.parametrize("bits,tol", [(64, 1e-9), (32, TOL_APPLY_F32)])
def test_oas_weights(O, bits, tol):
    """OAS (ORAS_WEIGHTS_NONE, Sec. 4): z = sum_s R_s^T A_s^-1 R_s v against the oracle's OAS,
    and an OAS-preconditioned solve reaching the FP64 residual bar."""
    w = synth.small(n=4, r=2, nsub=8, overlap=1)
    p = problem.from_workload(w)
    oas = dd.ORAS(p.topo, p.xyz, p.eps_r, p.mu_r, p.k0, p.dec, weights="none")
    rng = np.random.default_rng(12)
    v = rng.normal(size=p.topo.ndof) + 1j * rng.normal(size=p.topo.ndof)
    h = gpu_handle(O, w, factor_bits=bits, weights=O.ORAS_WEIGHTS_NONE)
    try:
        assert rel(O.oras_precond(h, v), oas.apply(v)) <= tol
        b = p.B[:, 0]
        x, info, rc = O.oras_solve(h, b, 1e-8)
        assert rc == O.ORAS_OK
        assert np.linalg.norm(b - p.A @ x) / np.linalg.norm(b) <= 1e-8
    finally:
        O.oras_destroy(h)


def test_pool_memory_reused_and_released(O):
    """A handle set up on memory that an earlier handle freed into the device's pool solves
    bit-identically; oras_release_memory then hands the pool's unused memory back."""
    import torch
    w = synth.small(n=5, r=2, nsub=8, overlap=1)
    xs = []
    for _ in range(2):
        h = gpu_handle(O, w)
        try:
            b = O.oras_rhs_dipole(h, synth.dipole_ring(1)[0], [0, 0, 1.0])
            x, info, rc = O.oras_solve(h, b, 1e-8)
            assert rc == O.ORAS_OK
            xs.append(x)
        finally:
            O.oras_destroy(h)
    assert np.array_equal(xs[0], xs[1])
    free0 = torch.cuda.mem_get_info(0)[0]
    O.oras_release_memory(0)
    assert torch.cuda.mem_get_info(0)[0] >= free0


def test_full_size_head16_r2_workload(O):
    """The 16^3 x 6, r = 2, 64-subdomain, 2-layer workload (163,424 DOFs): integer arrays
    bit-exact, sampled element matrices and the whole A within 1e-12, dipole load within
    1e-12, and the GPU field's true residual <= 1e-8 with the oracle's independently assembled A."""
    w = synth.config(1)
    xyz, tets = w.mesh()
    eps, mu = w.materials(xyz, tets)
    h = gpu_handle(O, w)
    try:
        topo = topology.build(tets, len(xyz), w.r)
        assert np.array_equal(O.oras_dofmap(h, len(tets)), topo.dofmap)
        part = dd.rcb(xyz, topo.st, w.nsub)
        assert np.array_equal(O.oras_partition(h, len(tets)), part)
        sample = np.random.default_rng(3).choice(len(tets), 64, replace=False)
        ref = elements.element_matrices(xyz, topo.st[sample], w.r, eps[sample], mu[sample], w.k0)
        got = O.oras_element_matrices(h, sample)
        assert (np.abs(got - ref).max(axis=(1, 2)) / np.abs(ref).max(axis=(1, 2))).max() <= 1e-12
        A = assemble.global_matrix(topo, xyz, eps, mu, w.k0)
        A.sort_indices()
        _, cols, vals = O.oras_global_csr(h)
        assert np.array_equal(cols, A.indices)
        assert np.abs(vals - A.data).max() <= 1e-12 * np.abs(A.data).max()
        x0 = synth.dipole_ring(1)[0]
        b = assemble.dipole_load(topo, xyz, x0, [0, 0, 1.0])
        assert rel(O.oras_rhs_dipole(h, x0, [0, 0, 1.0]), b) <= 1e-12
        x, info, rc = O.oras_solve(h, b, w.tol)
        assert rc == O.ORAS_OK
        assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1e-8
    finally:
        O.oras_destroy(h)


@pytest.mark.parametrize("n,r,nsub,delta", [(4, 2, 8, 1), (3, 3, 2, 1), (6, 1, 4, 2)])
def test_tensor_core_lu_matches_cuda_core_lu(O, n, r, nsub, delta):
    """The tcgen05 trailing update (TF32 operands, FP32 accumulation) gives the same
    preconditioner as the FP32 CUDA-core update up to TF32 rounding, and the solve still reaches
    the FP64 bars (true residual <= 1e-8, field within 1e-6 of the direct solution)."""
    w = synth.small(n=n, r=r, nsub=nsub, overlap=delta)
    p = problem.from_workload(w, with_oras=False)
    ht = gpu_handle(O, w, factor_bits=32, lu_engine=O.ORAS_LU_AUTO)
    hc = gpu_handle(O, w, factor_bits=32, lu_engine=O.ORAS_LU_CUDA_CORES)
    try:
        rng = np.random.default_rng(21)
        v = rng.normal(size=p.topo.ndof) + 1j * rng.normal(size=p.topo.ndof)
        zt, zc = O.oras_precond(ht, v), O.oras_precond(hc, v)
        assert np.all(np.isfinite(zt))
        # the two differ by the TF32 rounding of the tensor-core update's operands (unit
        # roundoff 2^-11), the same reading as the FP32 apply's bar against the FP64 oracle
        assert rel(zt, zc) <= (TOL_APPLY_F32_R3 if r == 3 else TOL_APPLY_F32), rel(zt, zc)
        b = p.B[:, 0]
        x, info, rc = O.oras_solve(ht, b, 1e-8)
        assert rc == O.ORAS_OK
        assert np.linalg.norm(b - p.A @ x) / np.linalg.norm(b) <= 1e-8
        assert rel(x, spla.spsolve(p.A.tocsc(), b)) <= 1e-6
    finally:
        O.oras_destroy(ht)
        O.oras_destroy(hc)


def test_autotuned_panel_width(O):
    """The autotuner times every candidate panel width once per problem shape, keeps the
    fastest, and the factors it leaves solve to the oracle's field."""
    w = synth.small(n=5, r=2, nsub=4, overlap=1)
    p = problem.from_workload(w)
    h = gpu_handle(O, w)
    try:
        panel, times = O.oras_autotune(h)
        assert {w for w, g in times if g == 8} == set(O.AUTOTUNE_WIDTHS) and len(times) == len(O.AUTOTUNE_WIDTHS) + 3
        best = min(times, key=times.get)
        assert panel == best[0] and O.oras_lu_group(h) == best[1]
        x, info, rc = O.oras_solve(h, p.B[:, 0], w.tol)
        assert rc == O.ORAS_OK
        assert np.linalg.norm(p.B[:, 0] - p.A @ x) / np.linalg.norm(p.B[:, 0]) <= 1e-8
        assert rel(x, spla.spsolve(p.A.tocsc(), p.B[:, 0])) <= 1e-6
    finally:
        O.oras_destroy(h)
    h2 = gpu_handle(O, w)      # same shape: the cached choice, no timing
    try:
        panel2, times2 = O.oras_autotune(h2)
        assert panel2 == panel and times2 == {} and O.oras_lu_group(h2) == best[1]
    finally:
        O.oras_destroy(h2)


def test_raster_group_does_not_change_factors(O):
    """The raster group only orders the tensor-core update's output blocks: every group gives
    bit-identical factors, so the same preconditioned vector."""
    w = synth.small(n=6, r=2, nsub=4, overlap=1)
    rng = np.random.default_rng(41)
    zs = []
    for group in (8, 3, 64):
        h = gpu_handle(O, w, lu_panel=4, lu_group=group)
        try:
            n = O.oras_ndof(h)
            if not zs:
                v = rng.normal(size=n) + 1j * rng.normal(size=n)
            zs.append(O.oras_precond(h, v))
        finally:
            O.oras_destroy(h)
    assert np.array_equal(zs[0], zs[1]) and np.array_equal(zs[0], zs[2])


@pytest.mark.parametrize("bits,tol", [(64, 1e-9), (32, TOL_APPLY_F32)])
def test_ras_dirichlet_transmission(O, bits, tol):
    """RAS (A_s = R_s A R_s^T) against the oracle's RAS, and the paper's comparison: the ORAS
    impedance transmission needs fewer FGMRES iterations than the Dirichlet one."""
    from oracle import dd
    w = synth.small(n=4, r=2, nsub=8, overlap=1)
    p = problem.from_workload(w)
    ras = dd.ORAS(p.topo, p.xyz, p.eps_r, p.mu_r, p.k0, p.dec, transmission="dirichlet", A_global=p.A.tocsr())
    h = gpu_handle(O, w, factor_bits=bits, transmission=O.ORAS_TRANSMISSION_DIRICHLET)
    h2 = gpu_handle(O, w, factor_bits=bits)
    try:
        rng = np.random.default_rng(51)
        v = rng.normal(size=p.topo.ndof) + 1j * rng.normal(size=p.topo.ndof)
        assert rel(O.oras_precond(h, v), ras.apply(v)) <= tol
        b = p.B[:, 0]
        x, info, rc = O.oras_solve(h, b, w.tol)
        assert rc == O.ORAS_OK
        assert np.linalg.norm(b - p.A @ x) / np.linalg.norm(b) <= 1e-8
        _, info2, _ = O.oras_solve(h2, b, w.tol)
        assert info2[0]["iterations"] < info[0]["iterations"]
    finally:
        O.oras_destroy(h)
        O.oras_destroy(h2)


@pytest.mark.parametrize("k", [1, 3])
def test_captured_arnoldi_steps_replay_identically(O, k):
    """With oras_options.graphs every Arnoldi step is captured into a CUDA graph on its second use
    and replayed afterwards (restart 4: later cycles and the second solve replay); the fields are
    bit-identical to direct launches."""
    import torch
    w = synth.small(n=4, r=2, nsub=8, overlap=1, nrhs=k, restart=4)
    p = problem.from_workload(w, with_oras=False)
    stream = torch.cuda.Stream()
    xs = {}
    for graphs in (0, 1):
        h = gpu_handle(O, w, graphs=graphs)
        try:
            O.oras_set_stream(h, stream.cuda_stream)
            l0 = O.oras_launch_count()
            x1, info1, rc1 = O.oras_solve(h, p.B, w.tol, k=k)
            x2, info2, rc2 = O.oras_solve(h, p.B, w.tol, k=k)
            assert rc1 == rc2 == O.ORAS_OK
            assert np.array_equal(x1, x2)
            assert all(i["iterations"] > 4 for i in info1)  # several restart cycles
            xs[graphs] = (x1, O.oras_launch_count() - l0)
        finally:
            O.oras_destroy(h)
    assert np.array_equal(xs[0][0], xs[1][0])
    assert xs[0][1] == xs[1][1]  # the same kernels ran, counted once each
    X = np.asarray(xs[1][0]).reshape(-1, k)
    for j in range(k):
        assert np.linalg.norm(p.B[:, j] - p.A @ X[:, j]) / np.linalg.norm(p.B[:, j]) <= 1e-8
