"""The host thin QR of add-and-compress (stacked factor matrices of several
molecules, Algorithm TEP step 4), through the C ABI on the CPU: A = Q R with R upper
triangular, Q orthonormal on its kept columns, the diagonal of R equal in magnitude to
a Householder QR's, and exactly or nearly dependent columns (a molecule given twice)
taken out with a zero column of Q instead of normalised rounding noise."""
import numpy as np
import pytest

from paper_2510_26611_gb300 import lib


def _check(A, Q, R, tol=1e-13):
    assert np.allclose(np.tril(R, -1), 0.0)
    assert np.linalg.norm(Q @ R - A) <= tol * np.linalg.norm(A)
    keep = np.abs(np.diag(R)) > 0
    Qk = Q[:, keep]
    assert np.abs(Qk.T @ Qk - np.eye(keep.sum())).max() <= 1e-13
    assert np.all(Q[:, ~keep] == 0.0)
    return keep


@pytest.mark.parametrize("n,k", [(33, 8), (257, 24), (1025, 40)])
def test_random_matrix_matches_householder(n, k):
    rng = np.random.default_rng(n + k)
    A = rng.normal(size=(n, k)) * np.logspace(0, -6, k)  # graded columns
    Q, R = lib.rs_qr_host(A)
    keep = _check(A, Q, R)
    assert keep.all()
    Rh = np.linalg.qr(A, mode="r")
    assert np.allclose(np.abs(np.diag(R)), np.abs(np.diag(Rh)), rtol=1e-10)


def test_repeated_block_gives_zero_columns():
    # three molecules' factors side by side, the first given twice (bit-identical
    # columns): the repeat adds no direction
    rng = np.random.default_rng(7)
    V1, V2 = rng.normal(size=(257, 8)), rng.normal(size=(257, 8))
    A = np.concatenate([V1, V2, V1], axis=1)
    Q, R = lib.rs_qr_host(A)
    keep = _check(A, Q, R)
    assert keep.tolist() == [True] * 16 + [False] * 8
    # R's block of the repeat reproduces the first block's coefficients
    assert np.allclose(R[:, 16:24], R[:, 0:8], atol=1e-12 * np.abs(R).max())


def test_nearly_dependent_columns_are_kept_above_the_threshold():
    rng = np.random.default_rng(11)
    B = rng.normal(size=(129, 4))
    d = rng.normal(size=129)
    d -= B @ np.linalg.lstsq(B, d, rcond=None)[0]
    d /= np.linalg.norm(d)
    c = B @ rng.normal(size=4)
    A = np.column_stack([B, c + 1e-9 * np.linalg.norm(c) * d, c + 1e-14 * np.linalg.norm(c) * d])
    Q, R = lib.rs_qr_host(A)
    keep = _check(A, Q, R, tol=1e-12)
    # 1e-9 of the column's norm outside the span is a direction; 1e-14 is rounding level
    assert keep.tolist() == [True] * 5 + [False]
    assert abs(abs(Q[:, 4] @ d) - 1.0) <= 1e-6


def test_zero_column_and_argument_checks():
    A = np.zeros((16, 3))
    A[:, 0] = 1.0
    A[:, 2] = np.arange(16.0)
    Q, R = lib.rs_qr_host(A)
    keep = _check(A, Q, R)
    assert keep.tolist() == [True, False, True]
    buf = np.zeros(4)
    assert lib._lib.rs_qr_host(0, 1, buf.ctypes.data, buf.ctypes.data) == lib.RS_ERR_INVALID
    assert lib._lib.rs_qr_host(4, 1, None, buf.ctypes.data) == lib.RS_ERR_INVALID
