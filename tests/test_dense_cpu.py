"""The library's host QR algorithm (the harmonic Ritz eigenproblems of its GCRO-DR, Sec. 6)
against LAPACK (numpy.linalg.eig): eigenvalues as a multiset and A v = lambda v for every unit
eigenvector, on random, non-normal, Hessenberg and clustered-spectrum matrices.  CPU only."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def O():
    from paper_1605_04521_gb300 import build
    build.build()
    from paper_1605_04521_gb300 import oras
    return oras


def _check(O, A):
    w, V = O.oras_dense_eig(A)
    ref = np.linalg.eigvals(A)
    scale = max(1.0, np.abs(A).max())
    # match every eigenvalue to a distinct reference one
    left = list(ref)
    for lam in w:
        i = int(np.argmin([abs(lam - x) for x in left]))
        assert abs(lam - left[i]) <= 1e-10 * scale * len(w), (lam, left[i])
        left.pop(i)
    assert np.allclose(np.linalg.norm(V, axis=0), 1.0)
    R = A @ V - V * w[None, :]
    assert np.abs(R).max() <= 1e-10 * scale * len(w)


@pytest.mark.parametrize("n", [1, 2, 5, 17, 60])
def test_random_complex(O, n):
    rng = np.random.default_rng(n)
    _check(O, rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))


def test_nonnormal_and_hessenberg(O):
    rng = np.random.default_rng(3)
    n = 40
    lam = np.concatenate([np.linspace(0.01, 0.05, 6), rng.uniform(1, 3, n - 6)]) * np.exp(1j * rng.uniform(-0.3, 0.3, n))
    S = np.eye(n) + 0.3 * rng.normal(size=(n, n)) / np.sqrt(n)
    _check(O, S @ np.diag(lam) @ np.linalg.inv(S))
    H = np.triu(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)), -1)
    _check(O, H)
    _check(O, np.diag(np.arange(1, 9, dtype=float)) + np.diag(np.ones(7), 1))   # real, upper triangular


def test_rejects_bad_input(O):
    import ctypes as C
    assert O.lib.oras_dense_eig(0, None, None, None) == O.ORAS_ERR_INVALID_ARG
