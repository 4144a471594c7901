"""The tensor-core preconditioner apply (8 or more right-hand sides with FP32 factors) against the
CUDA-core apply of the same factors and against the oracle's FP64 ORAS (Sec. 4), and inside the
FGMRES solve (Sec. 5 pseudo-block).

The tensor-core products round their operands to TF32 (unit roundoff 2^-11), the same rounding
the tensor-core LU applies to its trailing updates.  Bars: 10 * 2^-11 against the CUDA-core apply
of the same factors; against the FP64 oracle, the CUDA-core apply's own distance from it (the
error of the FP32 factors, which depends on the conditioning of the local matrices: up to about
1e-2 with 256 small subdomains) plus that 10 * 2^-11.  The solves meet the FP64 bars (true
residual <= 1e-8, field within 1e-6 of a direct solve).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import dd, problem

pytestmark = pytest.mark.gpu

TOL_TC_VS_CC = 10 * 2.0 ** -11


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


def handles(O, w, **kw):
    xyz, tets = w.mesh()
    eps, mu = w.materials(xyz, tets)
    ht = O.oras_setup(xyz, tets, eps, mu, w.k0, w.r, w.nsub, w.overlap, restart=w.restart, **kw)
    hc = O.oras_setup(xyz, tets, eps, mu, w.k0, w.r, w.nsub, w.overlap, restart=w.restart,
                      apply_engine=O.ORAS_APPLY_CUDA_CORES, **kw)
    return ht, hc


@pytest.mark.parametrize("n,r,nsub,delta", [(4, 2, 8, 1), (3, 3, 4, 1), (4, 1, 64, 0), (6, 2, 2, 1),
                                             (10, 2, 256, 1)])
@pytest.mark.parametrize("k", [8, 12, 16, 32])
def test_tensor_core_apply_matches_cuda_core_and_oracle(O, n, r, nsub, delta, k):
    """Subdomains from one tile (64 subdomains of 6 tets, r = 1) to 40+ tiles (2 subdomains of
    6^3 x 6 / 2 tets, r = 2), odd and even tile counts, k = 8, 12 (a pass with 4 zero columns),
    16, 32 right-hand sides: every column agrees with the CUDA-core apply of the same factors and
    with the oracle's FP64 apply.  With 256 subdomains (at least one per SM) each subdomain is one
    CTA instead of a two-CTA cluster."""
    w = synth.small(n=n, r=r, nsub=nsub, overlap=delta)
    p = problem.from_workload(w)
    ht, hc = handles(O, w)
    try:
        rng = np.random.default_rng(1000 * k + n)
        V = rng.normal(size=(p.topo.ndof, k)) + 1j * rng.normal(size=(p.topo.ndof, k))
        Zt = O.oras_precond(ht, V, k=k)
        Zc = O.oras_precond(hc, V, k=k)
        assert np.all(np.isfinite(Zt))
        for j in range(k):
            assert rel(Zt[:, j], Zc[:, j]) <= TOL_TC_VS_CC, (j, rel(Zt[:, j], Zc[:, j]))
        for j in (0, k // 2, k - 1):
            zo = p.oras.apply(V[:, j])
            assert rel(Zt[:, j], zo) <= rel(Zc[:, j], zo) + TOL_TC_VS_CC
    finally:
        O.oras_destroy(ht)
        O.oras_destroy(hc)


def test_tensor_core_apply_oas_weights(O):
    """OAS (no partition of unity): the overlapping subdomain contributions are summed."""
    w = synth.small(n=4, r=2, nsub=8, overlap=1)
    p = problem.from_workload(w)
    oas = dd.ORAS(p.topo, p.xyz, p.eps_r, p.mu_r, p.k0, p.dec, weights="none")
    ht, hc = handles(O, w, weights=O.ORAS_WEIGHTS_NONE)
    try:
        rng = np.random.default_rng(77)
        V = rng.normal(size=(p.topo.ndof, 16)) + 1j * rng.normal(size=(p.topo.ndof, 16))
        Zt = O.oras_precond(ht, V, k=16)
        Zc = O.oras_precond(hc, V, k=16)
        for j in range(16):
            assert rel(Zt[:, j], Zc[:, j]) <= TOL_TC_VS_CC
        zo = oas.apply(V[:, 3])
        assert rel(Zt[:, 3], zo) <= rel(Zc[:, 3], zo) + TOL_TC_VS_CC
    finally:
        O.oras_destroy(ht)
        O.oras_destroy(hc)


def test_tensor_core_apply_in_the_solve(O):
    """32 right-hand sides through FGMRES with the tensor-core apply (one arena pass per
    iteration) and with the CUDA-core apply (eight passes): both reach the FP64 bars, and the
    iteration counts differ by at most one per column."""
    w = synth.small(n=6, r=2, nsub=16, overlap=1, nrhs=32)
    p = problem.from_workload(w, with_oras=False)
    ht, hc = handles(O, w)
    try:
        Xt, it_t, rc_t = O.oras_solve(ht, p.B, w.tol, k=32)
        Xc, it_c, rc_c = O.oras_solve(hc, p.B, w.tol, k=32)
        assert rc_t == rc_c == O.ORAS_OK
        XD = spla.splu(p.A.tocsc()).solve(p.B)
        for j in range(32):
            b = p.B[:, j]
            assert np.linalg.norm(b - p.A @ Xt[:, j]) / np.linalg.norm(b) <= 1e-8
            assert rel(Xt[:, j], XD[:, j]) <= 1e-6
            assert abs(it_t[j]["iterations"] - it_c[j]["iterations"]) <= 1
    finally:
        O.oras_destroy(ht)
        O.oras_destroy(hc)
