"""The host eigensolver behind the optimized-sampling iteration (Householder
tridiagonalisation + implicit QL), against numpy.linalg.eigh.  Host code only."""
import numpy as np
import pytest

from paper_1706_05586_gb300 import build as B
from paper_1706_05586_gb300 import dot as D


@pytest.fixture(scope="module", autouse=True)
def lib():
    import os
    if not os.path.exists(B.LIB):
        B.build()
    D.load()


@pytest.mark.parametrize("n", [1, 2, 5, 33, 128])
def test_matches_numpy(n):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, n))
    A = X + X.T
    w, Q = D.dot_symeig(A)
    ref = np.linalg.eigvalsh(A)
    assert np.allclose(w, ref, rtol=0, atol=1e-13 * max(1.0, np.abs(ref).max()))
    assert np.allclose(Q.T @ Q, np.eye(n), atol=1e-13)
    assert np.allclose(A @ Q, Q * w, atol=1e-12 * max(1.0, np.abs(ref).max()))


def test_degenerate_and_gram_like():
    w, Q = D.dot_symeig(np.diag([3.0, 1.0, 2.0, 2.0]))
    assert np.array_equal(w, [1.0, 2.0, 2.0, 3.0])
    rng = np.random.default_rng(9)
    Xr = rng.standard_normal((40, 6)) @ np.diag(10.0 ** -np.arange(6)) @ rng.standard_normal((6, 500))
    G = Xr @ Xr.T                    # rank 6, spread over 10 orders of magnitude
    w, Q = D.dot_symeig(G)
    ref = np.linalg.eigvalsh(G)
    assert np.allclose(w, ref, rtol=0, atol=1e-12 * ref.max())
    U, s, _ = np.linalg.svd(Xr)
    for c in range(3):               # leading eigenvectors = leading left singular vectors
        assert abs(abs(Q[:, -1 - c] @ U[:, c]) - 1.0) < 1e-10


@pytest.mark.parametrize("n,rank", [(128, 20), (256, 12), (512, 40)])
def test_gram_with_many_null_eigenvalues(n, rank):
    """Gram matrices of low-rank unfoldings (the Jacobian tensors of Algorithm 1): a few
    eigenvalues spread over decades and n - rank that are zero up to rounding.  The QL
    sweeps must deflate the rounding-level off-diagonals of that null cluster against
    the matrix's scale, and the leading eigenpairs must match numpy."""
    rng = np.random.default_rng(n + rank)
    X = rng.standard_normal((n, rank)) @ np.diag(10.0 ** -np.linspace(0, 8, rank)) @ rng.standard_normal((rank, 3 * n))
    G = X @ X.T
    w, Q = D.dot_symeig(G)
    ref, V = np.linalg.eigh(G)
    assert np.allclose(w, ref, rtol=0, atol=1e-12 * ref.max())
    assert np.allclose(Q.T @ Q, np.eye(n), atol=1e-12)
    for c in range(4):
        assert abs(abs(Q[:, -1 - c] @ V[:, -1 - c]) - 1.0) < 1e-10
