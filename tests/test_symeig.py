"""The host eigensolver behind the spectral step (b) of a symmetric Riesz operator
(aao_sym_eig: Householder tridiagonalisation + symmetric QR with the Wilkinson shift), checked through the C ABI
against the defining identities and numpy's LAPACK eigenvalues. CPU only."""
import numpy as np
import pytest

from oracle import aao_oracle as O
from paper_2401_16113_gb300 import aao, build, workloads as W


@pytest.fixture(scope="module")
def lib():
    build.build()
    return aao.load()


def check(A, w, Qt, tol):
    n = A.shape[0]
    scale = max(np.abs(A).max(), 1e-300)
    # A Q = Q diag(w), Q^T Q = I, and the same spectrum as LAPACK
    assert np.abs(A @ Qt.T - Qt.T * w).max() <= tol * n * scale
    assert np.abs(Qt @ Qt.T - np.eye(n)).max() <= tol * n
    assert np.allclose(np.sort(w), np.linalg.eigvalsh(A), rtol=0, atol=tol * n * scale)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 64, 129])
def test_random_symmetric(lib, n):
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n, n))
    A = B + B.T
    w, Qt = aao.sym_eig(A)
    check(A, w, Qt, 1e-14)


def test_special_structures(lib):
    for A in (np.zeros((6, 6)), np.eye(7), np.diag(np.arange(9.0)), np.ones((8, 8)),
              np.diag(np.full(10, 2.0)) - np.diag(np.ones(9), 1) - np.diag(np.ones(9), -1)):
        w, Qt = aao.sym_eig(A)
        check(A, w, Qt, 1e-14)
    # the second-difference matrix has the closed-form spectrum 2 - 2 cos(k pi / (n + 1))
    n = 10
    T = np.diag(np.full(n, 2.0)) - np.diag(np.ones(n - 1), 1) - np.diag(np.ones(n - 1), -1)
    w, _ = aao.sym_eig(T)
    k = np.arange(1, n + 1)
    assert np.allclose(np.sort(w), np.sort(2 - 2 * np.cos(k * np.pi / (n + 1))), rtol=0, atol=1e-13)


def test_riesz_operator_without_drift_is_symmetric_and_decomposes(lib):
    p = W.with_(W.riesz_sym_1023x512(), nx=200)
    A, _, _ = O.riesz_matrix(p)
    assert np.array_equal(A, A.T)
    w, Qt = aao.sym_eig(A)
    check(A, w, Qt, 1e-14)
    # with drift the matrix is not symmetric (the spectral step (b) is not used)
    Ad, _, _ = O.riesz_matrix(W.with_(W.riesz_1023x512(), nx=200))
    assert not np.array_equal(Ad, Ad.T)


def test_rejects_bad_arguments(lib):
    assert lib.aao_sym_eig(0, None, None) == aao.AAO_EINVAL
