"""The host eigensolver of the build's Rayleigh-Ritz step (Householder +
implicit QL) against the eigen-equation, orthonormality and numpy's eigvalsh, on
Rayleigh matrices like the build's (graded spectra) and on hard cases."""
import numpy as np
import pytest

from paper_2510_26611_gb300 import lib


def _check(A, lam, W, tol=1e-12):
    n = A.shape[0]
    S = 0.5 * (A + A.T)
    scale = max(np.abs(np.linalg.eigvalsh(S)).max(), 1e-300)
    assert np.all(np.diff(lam) <= 0)
    assert np.allclose(W.T @ W, np.eye(n), atol=1e-13)
    assert np.abs(S @ W - W * lam[None, :]).max() <= tol * scale
    assert np.abs(np.sort(lam) - np.linalg.eigvalsh(S)).max() <= tol * scale


@pytest.mark.parametrize("n", [1, 2, 3, 7, 32, 48])
def test_random_graded_spectra(n):
    rng = np.random.default_rng(n)
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    lam = 0.5 ** np.arange(n) * rng.uniform(0.5, 1.5, n)   # geometric decay like a Gram's
    A = (Q * lam) @ Q.T
    A += 1e-18 * rng.normal(size=(n, n))                    # not exactly symmetric
    l, W = lib.rs_symeig_host(A)
    _check(A, l, W)


def test_hard_cases():
    # repeated eigenvalues, zero matrix, diagonal with mixed signs, tiny and huge scales
    n = 16
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    for lam in [np.ones(n), np.r_[np.ones(8), np.zeros(8)], np.linspace(-3, 3, n),
                1e-200 * np.arange(1, n + 1), 1e200 * np.arange(1, n + 1)]:
        A = (Q * lam) @ Q.T
        l, W = lib.rs_symeig_host(A)
        _check(A, l, W)
    l, W = lib.rs_symeig_host(np.zeros((5, 5)))
    assert np.all(l == 0) and np.allclose(W.T @ W, np.eye(5))
    D = np.diag([3.0, -1.0, 2.0])
    l, W = lib.rs_symeig_host(D)
    assert np.allclose(l, [3.0, 2.0, -1.0])


@pytest.mark.parametrize("n,r", [(73, 12), (144, 12), (40, 1)])
def test_rank_deficient_gram(n, r):
    # a Gram of rank r << n: most eigenvalues are (near) zero and the couplings between
    # them shrink toward rounding level, where only an absolute deflation test ends QL
    rng = np.random.default_rng(n + r)
    X = rng.normal(size=(n, r)) * (10.0 ** rng.uniform(-3, 3, size=(1, r)))
    A = X @ X.T
    l, W = lib.rs_symeig_host(A)
    _check(A, l, W)
    assert np.all(np.abs(l[r:]) <= 1e-12 * l[0])
