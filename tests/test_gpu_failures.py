"""Failure detection of the GPU path, tested without faulting or hanging the GPU.

* Bounded device waits: a self-test kernel runs every wait primitive of the library's kernels on a
  condition nothing satisfies (a barrier nobody arrives on, a counter nobody increments) with a
  short limit; each gives up, the kernel returns, the call reports ORAS_ERR_DEVICE_TIMEOUT, and
  the handle keeps working afterwards.
* Non-convergence: max_iter reached -> ORAS_NOT_CONVERGED with the best iterate of the last cycle
  (the same x the oracle's FGMRES holds after the same number of steps) and its true residual.
* An exactly singular local matrix (every entry zero) -> ORAS_ERR_SINGULAR_LOCAL from oras_factor.
"""
import time

import numpy as np
import pytest

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


def test_bounded_waits_give_up_and_are_reported(O):
    w = synth.small(n=3, r=2, nsub=4, overlap=1)
    xyz, tets = w.mesh()
    eps, mu = w.materials(xyz, tets)
    h = O.oras_setup(xyz, tets, eps, mu, w.k0, w.r, w.nsub, w.overlap, wait_ms=200)
    try:
        n = O.oras_ndof(h)
        rng = np.random.default_rng(3)
        v = rng.normal(size=n) + 1j * rng.normal(size=n)
        z0 = O.oras_precond(h, v)
        t0 = time.perf_counter()
        rc, detail = O.oras_wait_selftest(h)
        dt = time.perf_counter() - t0
        assert rc == O.ORAS_ERR_DEVICE_TIMEOUT
        assert detail == 7                      # all three primitives gave up
        assert 0.55 <= dt < 5.0                 # three waits of 200 ms each, then the kernel returned
        assert "bounded device wait" in O.lib.oras_last_error(h).decode()
        # the context and the handle still work, and give the same result as before
        z1 = O.oras_precond(h, v)
        assert np.array_equal(z0, z1)
        x, info, rc = O.oras_solve(h, O.oras_rhs_dipole(h, synth.dipole_ring(1)[0], [0, 0, 1.0]), 1e-8)
        assert rc == O.ORAS_OK and info[0]["converged"]
    finally:
        O.oras_destroy(h)


def test_not_converged_returns_best_iterate(O):
    """max_iter = 2 (FP64 factors): the solve stops after two Arnoldi steps, reports
    ORAS_NOT_CONVERGED, and returns the iterate of that cycle with its true FP64 residual; the
    oracle's FGMRES with the same cap holds the same iterate."""
    w = synth.small(n=4, r=2, nsub=8, overlap=1, factor_bits=64)
    p = problem.from_workload(w)
    b = p.B[:, 0]
    xyz, tets = w.mesh()
    eps, mu = w.materials(xyz, tets)
    h = O.oras_setup(xyz, tets, eps, mu, w.k0, w.r, w.nsub, w.overlap, factor_bits=64, max_iter=2)
    try:
        x, info, rc = O.oras_solve(h, b, 1e-8)
        assert rc == O.ORAS_NOT_CONVERGED
        assert info[0]["iterations"] == 2 and not info[0]["converged"] and info[0]["restarts"] == 1
        true_res = np.linalg.norm(b - p.A @ x) / np.linalg.norm(b)
        assert true_res > 1e-8
        assert abs(info[0]["relres"] - true_res) <= 1e-9 * max(1.0, true_res)
        ref = fgmres.fgmres(lambda v: p.A @ v, p.oras.apply, b, 1e-8, 50, max_iter=2)
        assert ref.iterations == 2 and not ref.converged
        assert rel(x, ref.x) <= 1e-8
        assert abs(ref.relres - true_res) <= 1e-8 * true_res
    finally:
        O.oras_destroy(h)


@pytest.mark.parametrize("bits", [32, 64])
def test_zero_local_matrix_is_reported_singular(O, bits):
    """eps_r = 0 and 1/mu_r = 0 (mu_r = 1e300, whose inverse underflows to exactly zero) make every
    element matrix, every impedance coefficient and so every local matrix A_s exactly zero: the
    batched LU finds a zero pivot column and oras_factor reports ORAS_ERR_SINGULAR_LOCAL."""
    xyz, tets = synth.kuhn_cube(3)
    eps = np.zeros(len(tets), dtype=np.complex128)
    mu = np.full(len(tets), 1e300, dtype=np.complex128)
    with pytest.raises(O.OrasError) as e:
        O.oras_setup(xyz, tets, eps, mu, synth.K0, 2, 4, 1, factor_bits=bits)
    assert e.value.code == O.ORAS_ERR_SINGULAR_LOCAL
    assert "zero pivot" in str(e.value)
