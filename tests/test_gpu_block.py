"""GPU block flexible GMRES (oras_options.block, Sec. 6 Block GMRES for the several right-hand
sides of one system) against the oracle's block_fgmres (tests/test_oracle_block.py pins it) and a
sparse direct solve.

With FP64 factors the two preconditioners agree to 1e-9, so the GPU takes the same number of block
steps as the oracle; with FP32 factors every column still meets the FP64 bars (true residual <=
1e-8, field within 1e-6 of the direct solution), and the block method needs no more block steps
than the slowest column of the pseudo-block solve (its block Krylov space contains every column's
own space).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import fgmres, problem

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


def setup(O, w, **kw):
    xyz, tets = w.mesh()
    eps, mu = w.materials(xyz, tets)
    return O.oras_setup(xyz, tets, eps, mu, w.k0, w.r, w.nsub, w.overlap, restart=w.restart, **kw)


@pytest.mark.parametrize("restart", [50, 3])
def test_block_fgmres_matches_the_oracle_fp64_factors(O, restart):
    """8 dipoles as one block, FP64 factors: the same block steps as the oracle's block FGMRES
    (unrestarted, and restarted every 3 block steps), the oracle's fields to 1e-6, the direct
    solution to 1e-6 and true residuals <= 1e-8."""
    w = synth.small(n=4, r=2, nsub=8, overlap=1, nrhs=8, restart=restart, factor_bits=64)
    p = problem.from_workload(w)
    h = setup(O, w, factor_bits=64, block=1)
    try:
        X, info, rc = O.oras_solve(h, p.B, w.tol, k=8)
        assert rc == O.ORAS_OK
        ref = fgmres.block_fgmres(lambda v: p.A @ v, p.oras.apply, p.B, w.tol, restart)
        assert ref.converged
        assert all(i["iterations"] == ref.iterations for i in info), ([i["iterations"] for i in info], ref.iterations)
        XD = spla.splu(p.A.tocsc()).solve(p.B)
        for j in range(8):
            b = p.B[:, j]
            res = np.linalg.norm(b - p.A @ X[:, j]) / np.linalg.norm(b)
            assert res <= 1e-8 and abs(info[j]["relres"] - res) <= 1e-9
            assert rel(X[:, j], ref.x[:, j]) <= 1e-6
            assert rel(X[:, j], XD[:, j]) <= 1e-6
    finally:
        O.oras_destroy(h)


def test_block_fgmres_32_columns_fp32_factors(O):
    """32 dipoles on the ring (6^3 x 6, r = 2, 16 subdomains), FP32 factors, the tensor-core apply
    of all 32 block columns together: every column meets the FP64 bars, and the block steps are
    at most the iterations of the slowest pseudo-block column."""
    w = synth.small(n=6, r=2, nsub=16, overlap=1, nrhs=32)
    p = problem.from_workload(w, with_oras=False)
    hb = setup(O, w, block=1)
    hp = setup(O, w)
    try:
        Xb, ib, rc = O.oras_solve(hb, p.B, w.tol, k=32)
        assert rc == O.ORAS_OK
        _, ip, rcp = O.oras_solve(hp, p.B, w.tol, k=32)
        assert rcp == O.ORAS_OK
        assert ib[0]["iterations"] <= max(i["iterations"] for i in ip)
        XD = spla.splu(p.A.tocsc()).solve(p.B)
        for j in range(32):
            b = p.B[:, j]
            assert np.linalg.norm(b - p.A @ Xb[:, j]) / np.linalg.norm(b) <= 1e-8
            assert rel(Xb[:, j], XD[:, j]) <= 1e-6
    finally:
        O.oras_destroy(hb)
        O.oras_destroy(hp)


def test_block_fgmres_one_column_is_fgmres(O):
    """k = 1 with the block option is the single-vector FGMRES (bit-identical)."""
    w = synth.small(n=4, r=2, nsub=8, overlap=1)
    p = problem.from_workload(w, with_oras=False)
    hb = setup(O, w, block=1)
    hs = setup(O, w)
    try:
        xb, ib, _ = O.oras_solve(hb, p.B[:, 0], w.tol)
        xs, is_, _ = O.oras_solve(hs, p.B[:, 0], w.tol)
        assert np.array_equal(xb, xs) and ib[0]["iterations"] == is_[0]["iterations"]
    finally:
        O.oras_destroy(hb)
        O.oras_destroy(hs)
