"""Pins for the oracle's optimized simultaneous sources and detectors (Sec. 3.2,
Algorithm 1) and the complementary random ones (Eqs. (newW), (newV), Theorem 2)."""
import itertools
import math

import numpy as np
import pytest

from oracle import dot_oracle as orc


def _kron_rank_tensor(rng, nd, ns, npar, qd, qs, terms=4):
    """J with every slice in span(A) (x) span(Bs): ||(Bs^T (x) A^T) J|| = ||J||."""
    A, _ = np.linalg.qr(rng.standard_normal((nd, qd)))
    Bs, _ = np.linalg.qr(rng.standard_normal((ns, qs)))
    J = np.zeros((nd, ns, npar))
    for _ in range(terms):
        a = A @ rng.standard_normal(qd)
        b = Bs @ rng.standard_normal(qs)
        c = rng.standard_normal(npar)
        J += np.einsum("i,j,k->ijk", a, b, c)
    return J, A, Bs


def test_theorem3_exact_in_one_iteration():
    """If isometric W, V preserve ||J||_F exactly, steps (1)-(3) find such W, V in one sweep."""
    rng = np.random.default_rng(70)
    J, A, Bs = _kron_rank_tensor(rng, 7, 6, 9, 2, 2)
    W, V, sweeps = orc.optimized_sources_detectors(J, 2, 2, maxit=1)
    assert orc.sampled_jacobian_norm2(J, W, V) == pytest.approx(np.sum(J ** 2), rel=1e-12)
    assert np.allclose(W @ W.T, Bs @ Bs.T, atol=1e-10)
    assert np.allclose(V @ V.T, A @ A.T, atol=1e-10)


def test_brute_force_maximum_q1():
    """n_s = n_d = 3, q = 1: the alternating iteration reaches the global maximum of
    ||(w^T (x) v^T) J||^2 over unit w, v found by a dense search over v on the sphere
    with the exact best w for each v."""
    rng = np.random.default_rng(71)
    J = rng.standard_normal((3, 3, 5))
    W, V, _ = orc.optimized_sources_detectors(J, 1, 1, maxit=500, tol=1e-14)
    best = 0.0
    n_t, n_p = 181, 361
    for th in np.linspace(0, math.pi, n_t):
        for ph in np.linspace(0, 2 * math.pi, n_p):
            v = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
            K = np.einsum("m,mjk->jk", v, J)
            best = max(best, np.linalg.svd(K, compute_uv=False)[0] ** 2)
    val = orc.sampled_jacobian_norm2(J, W, V)
    assert val >= best * (1 - 1e-9)
    # and nothing on the grid beats it by more than the grid resolution allows
    assert val <= best * (1 + 1e-3)


def test_objective_monotone_and_bounded():
    rng = np.random.default_rng(72)
    J = rng.standard_normal((8, 6, 11)) + 1j * rng.standard_normal((8, 6, 11))
    vals = [orc.sampled_jacobian_norm2(J, *orc.optimized_sources_detectors(J, 2, 3, maxit=m)[:2])
            for m in (1, 2, 4, 8, 16)]
    assert all(b >= a * (1 - 1e-12) for a, b in zip(vals, vals[1:]))
    assert vals[-1] <= np.sum(np.abs(J) ** 2) * (1 + 1e-12)


def test_isometric_outputs():
    rng = np.random.default_rng(73)
    J = rng.standard_normal((9, 7, 4))
    W, V, _ = orc.optimized_sources_detectors(J, 3, 2)
    assert np.allclose(W.T @ W, np.eye(3), atol=1e-12)
    assert np.allclose(V.T @ V, np.eye(2), atol=1e-12)


def test_theorem3_exact_complex_tensor():
    """Theorem 3 for a complex Jacobian (omega != 0): when the real and the imaginary
    slices both lie in span(A) (x) span(Bs), real isometric W, V keep all of
    ||J||_F^2 = sum |J_ijk|^2, and steps (1)-(3) find them in one sweep."""
    rng = np.random.default_rng(76)
    nd, ns, npar, qd, qs = 7, 6, 5, 2, 3
    Jr, A, Bs = _kron_rank_tensor(rng, nd, ns, npar, qd, qs)
    Ji = np.zeros_like(Jr)
    for _ in range(3):        # a second tensor in the same subspaces, independent of the first
        a = A @ rng.standard_normal(qd)
        b = Bs @ rng.standard_normal(qs)
        Ji += np.einsum("i,j,k->ijk", a, b, rng.standard_normal(npar))
    J = Jr + 1j * Ji
    W, V, _ = orc.optimized_sources_detectors(J, qs, qd, maxit=1)
    assert orc.sampled_jacobian_norm2(J, W, V) == pytest.approx(np.sum(np.abs(J) ** 2), rel=1e-12)
    assert np.allclose(W @ W.T, Bs @ Bs.T, atol=1e-10)
    assert np.allclose(V @ V.T, A @ A.T, atol=1e-10)


def test_brute_force_maximum_q1_complex():
    """q = 1 on a complex 3 x 3 x 4 tensor: the objective over real unit w, v is
    sum_k |v^T J_k w|^2.  For a fixed v it is w^T Re(K K^H) w with K = sum_m v_m J_m, so
    the best w is the top eigenvector of that real symmetric matrix; a dense search of v
    over the sphere gives the global maximum, which Algorithm 1 must reach."""
    rng = np.random.default_rng(77)
    J = rng.standard_normal((3, 3, 4)) + 1j * rng.standard_normal((3, 3, 4))
    W, V, _ = orc.optimized_sources_detectors(J, 1, 1, maxit=500, tol=1e-14)
    best = 0.0
    for th in np.linspace(0, math.pi, 181):
        for ph in np.linspace(0, 2 * math.pi, 361):
            v = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
            K = np.einsum("m,mjk->jk", v, J)
            best = max(best, np.linalg.eigvalsh(np.real(K @ K.conj().T))[-1])
    val = orc.sampled_jacobian_norm2(J, W, V)
    # the objective at (W, V) written out as the sum over parameters of |v^T J_k w|^2
    direct = sum(abs(V[:, 0] @ J[:, :, k] @ W[:, 0]) ** 2 for k in range(J.shape[2]))
    assert val == pytest.approx(direct, rel=1e-12)
    assert val >= best * (1 - 1e-9)
    assert val <= best * (1 + 1e-3)


def test_theorem2_complement_unbiased_enumeration():
    """E[W W^T] = I for W = [W^, (I - W^W^T) Y~] over every Rademacher Y~ (Eq. (covW))."""
    rng = np.random.default_rng(75)
    n, q, m = 4, 1, 2
    What, _ = np.linalg.qr(rng.standard_normal((n, q)))
    acc = np.zeros((n, n))
    count = 0
    for signs in itertools.product((-1.0, 1.0), repeat=n * m):
        Y = np.array(signs).reshape(n, m) / math.sqrt(m)
        W = orc.complement_sampling(What, Y)
        acc += W @ W.T
        count += 1
    assert np.allclose(acc / count, np.eye(n), atol=1e-14)
    # the random columns lie in the complement of W^
    W = orc.complement_sampling(What, rng.standard_normal((n, m)))
    assert np.allclose(What.T @ W[:, q:], 0.0, atol=1e-14)
