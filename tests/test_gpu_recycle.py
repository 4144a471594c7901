"""GPU GCRO-DR (oras_options.recycle; Sec. 6 subspace recycling for the imaging loop's sequence
of slowly varying systems) against the oracle's gcrodr (tests/test_oracle_gcrodr.py pins it) and
a sparse direct solve.

With FP64 factors the two operators A M^{-1} agree to rounding, so the GPU solver takes the
oracle's products to within 3 per solve: the GPU projects with classical Gram-Schmidt
reorthogonalised, the oracle with modified Gram-Schmidt, and both re-solve the small
least-squares problem after every step.  Over a sequence of three systems whose permittivity
changes slightly, the subspace the handle keeps is recycled as the oracle's is.  Every solve
meets the FP64 bars (true residual <= 1e-8, field within 1e-6 of the direct solution).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import gcrodr, problem

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


def sequence(w, n_sys=3, seed=11):
    """Materials of a slowly varying sequence: eps_t = eps (1 + 2e-3 t xi), xi ~ U(-1, 1) per tet."""
    xyz, tets = w.mesh()
    eps, mu = w.materials(xyz, tets)
    rng = np.random.default_rng(seed)
    xi = rng.uniform(-1.0, 1.0, len(tets))
    return xyz, tets, [(eps * (1.0 + 2e-3 * t * xi), mu) for t in range(n_sys)]


@pytest.mark.parametrize("m,k", [(30, 8), (20, 5)])
def test_gcrodr_matches_the_oracle_fp64_factors(O, m, k):
    w = synth.small(n=6, r=2, nsub=64, overlap=0)
    xyz, tets, mats = sequence(w)
    b = None
    U_ref = None
    h = O.oras_create(xyz, tets, w.r, w.nsub, w.overlap, factor_bits=64, restart=m, recycle=k)
    try:
        for t, (eps, mu) in enumerate(mats):
            p = problem.build(xyz, tets, eps, mu, w.k0, w.r, w.sources(), w.nsub, w.overlap)
            if b is None:
                b = p.B[:, 0]
            O.oras_factor(h, eps, mu, w.k0)
            x, info, rc = O.oras_solve(h, b, 1e-8)
            assert rc == O.ORAS_OK
            ref = gcrodr.gcrodr(lambda v: p.A @ p.oras.apply(v), b, m=m, k=k, tol=1e-8, U=U_ref)
            U_ref = ref.U
            assert ref.converged
            assert abs(info[0]["iterations"] - ref.matvecs) <= 3, (t, info[0]["iterations"], ref.matvecs)
            x_ref = p.oras.apply(ref.y)
            xd = spla.spsolve(p.A.tocsc(), b)
            res = np.linalg.norm(b - p.A @ x) / np.linalg.norm(b)
            assert res <= 1e-8 and abs(info[0]["relres"] - res) <= 1e-9
            assert rel(x, xd) <= 1e-6 and rel(x, x_ref) <= 1e-6
    finally:
        O.oras_destroy(h)


def test_gcrodr_fp32_factors_and_reset(O):
    """FP32 factors (the tensor-core LU): every solve of the sequence reaches the FP64 bars; after
    oras_recycle_reset the next solve takes as many products as a fresh handle's first solve."""
    w = synth.small(n=6, r=2, nsub=64, overlap=0)
    xyz, tets, mats = sequence(w, n_sys=2)
    h = O.oras_create(xyz, tets, w.r, w.nsub, w.overlap, restart=30, recycle=8)
    try:
        its = []
        for eps, mu in mats:
            p = problem.build(xyz, tets, eps, mu, w.k0, w.r, w.sources(), with_oras=False)
            O.oras_factor(h, eps, mu, w.k0)
            b = p.B[:, 0]
            x, info, rc = O.oras_solve(h, b, 1e-8)
            assert rc == O.ORAS_OK
            assert np.linalg.norm(b - p.A @ x) / np.linalg.norm(b) <= 1e-8
            assert rel(x, spla.spsolve(p.A.tocsc(), b)) <= 1e-6
            its.append(info[0]["iterations"])
        first = its[0]
        O.oras_recycle_reset(h)
        _, info, rc = O.oras_solve(h, b, 1e-8)
        h2 = O.oras_create(xyz, tets, w.r, w.nsub, w.overlap, restart=30, recycle=8)
        try:
            O.oras_factor(h2, mats[-1][0], mats[-1][1], w.k0)
            _, info2, rc2 = O.oras_solve(h2, b, 1e-8)
            assert rc == rc2 == O.ORAS_OK and info[0]["iterations"] == info2[0]["iterations"]
        finally:
            O.oras_destroy(h2)
        assert first > 0
    finally:
        O.oras_destroy(h)
