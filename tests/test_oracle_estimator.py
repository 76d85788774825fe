"""Pins for the randomized estimator (Sec. 3.1: Theorem 1, Eqs. (EWWT=I), (UnbiasedGrad),
(UnbiasedHess)) and for the oracle's sampled misfit and sampled Jacobian.

Unbiasedness is checked exactly by enumerating every Rademacher draw, so a
transposed W/V, a dropped 1/sqrt(l) or a wrong Kronecker row order fails.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import dot_oracle as orc
from paper_1706_05586_gb300 import synth
from tests import problem


def _all_rademacher(n, l):
    """Every n x l Rademacher matrix scaled by l^{-1/2}, Eq. (defW)."""
    cols = [np.array(s, dtype=float) for s in itertools.product((-1.0, 1.0), repeat=n)]
    for combo in itertools.product(range(len(cols)), repeat=l):
        yield np.stack([cols[c] for c in combo], axis=1) / math.sqrt(l)


@pytest.mark.parametrize("l", [1, 2])
def test_theorem1_exact_enumeration(l):
    rng = np.random.default_rng(7)
    n = 3 if l == 2 else 4
    R = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Ws = list(_all_rademacher(n, l))
    tot = 0.0
    for W in Ws:
        for V in Ws:
            tot += orc.sampled_misfit(R, W, V)
    mean = tot / len(Ws) ** 2
    assert mean == pytest.approx(np.sum(np.abs(R) ** 2), rel=1e-13)


def test_eq_EWWT_identity_enumeration():
    n, l = 4, 2
    Ws = list(_all_rademacher(n, l))
    E = sum(W @ W.T for W in Ws) / len(Ws)
    assert np.allclose(E, np.eye(n), atol=1e-14)


def test_generator_scaling_monte_carlo():
    rng = np.random.default_rng(8)
    for kind in ("rademacher", "gaussian"):
        acc = np.zeros((5, 5))
        T = 20000
        for _ in range(T):
            W = synth.sampling_matrix(rng, 5, 3, kind)
            acc += W @ W.T
        assert np.allclose(acc / T, np.eye(5), atol=0.04), kind


def test_identity_and_orthogonal_sampling_give_frobenius():
    rng = np.random.default_rng(9)
    R = rng.standard_normal((6, 5))
    fro = np.sum(R ** 2)
    assert orc.sampled_misfit(R, np.eye(5), np.eye(6)) == pytest.approx(fro, rel=1e-14)
    Wf, _ = np.linalg.qr(rng.standard_normal((5, 5)))
    Vf, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    assert orc.sampled_misfit(R, Wf, Vf) == pytest.approx(fro, rel=1e-13)


def test_sampled_residual_is_kron_times_vec():
    """vec(V^T R W) = (W^T (x) V^T) vec(R) (Horn and Johnson, used in Sec. 3.1)."""
    rng = np.random.default_rng(10)
    R = rng.standard_normal((4, 3))
    W = rng.standard_normal((3, 2))
    V = rng.standard_normal((4, 2))
    lhs = orc.sampled_residual(R, W, V).reshape(-1, order="F")
    rhs = np.kron(W.T, V.T) @ R.reshape(-1, order="F")
    assert np.allclose(lhs, rhs, rtol=1e-14, atol=1e-14)


def _tiny():
    wl = synth.small_workload(4, 4, 3, 0.5, src_grid=(3, 1), det_grid=(3, 1), ls=1, ld=1, m0=3,
                              seed_index=21)
    return problem.build(wl)


def test_unbiased_gradient_and_gn_hessian_enumeration():
    """E[(S J)^T S r] = J^T r and E[(S J)^T (S J)] = J^T J with S = W^T (x) V^T,
    Eqs. (UnbiasedGrad), (UnbiasedHess), by enumerating all Rademacher W, V."""
    pb = _tiny()
    p = pb.inp.p0
    mu = pb.mu_of(p)
    A = pb.A_of(mu)
    Uf, Zf = orc.fields_full(A, pb.Bd, pb.Cd)
    J3 = orc.jacobian_tensor(Uf, Zf, pb.dmu_of(p))
    R = pb.Cd.T @ Uf - pb.M
    ns, nd = pb.wl.ns, pb.wl.nd
    Jfull = orc.sampled_jacobian(J3, np.eye(ns), np.eye(nd))
    r = R.reshape(-1, order="F")
    g_true = Jfull.T @ r
    H_true = Jfull.T @ Jfull
    Ws = list(_all_rademacher(ns, 1))
    Vs = list(_all_rademacher(nd, 1))
    g = np.zeros_like(g_true)
    H = np.zeros_like(H_true)
    for W in Ws:
        for V in Vs:
            Js = orc.sampled_jacobian(J3, W, V)
            rs = orc.sampled_residual(R, W, V).reshape(-1, order="F")
            g += Js.T @ rs
            H += Js.T @ Js
    n = len(Ws) * len(Vs)
    assert np.allclose(g / n, g_true, rtol=1e-12, atol=1e-12 * np.abs(g_true).max())
    assert np.allclose(H / n, H_true, rtol=1e-12, atol=1e-12 * np.abs(H_true).max())
    # and the full Jacobian row order is vec(R): row d + nd * s
    assert np.allclose(Jfull.reshape(ns, nd, -1).transpose(1, 0, 2), J3, rtol=0, atol=0)


@pytest.mark.slow
def test_monte_carlo_unbiased_at_32x32x16():
    """10^4 Rademacher samples (l_s = l_d = 2) of ||V^T R W||^2 at the 32x32x16 workload
    average to ||R||_F^2 within 4 standard errors (Theorem 1)."""
    pb = problem.build(synth.WORKLOADS["dot32x32x16"])
    A = pb.A_of(pb.mu_of(pb.inp.p0))
    R = orc.residual_matrix(A, pb.Bd, pb.Cd, pb.M)
    rng = np.random.default_rng(12)
    vals = np.array([orc.sampled_misfit(R, synth.sampling_matrix(rng, pb.wl.ns, 2, "rademacher"),
                                        synth.sampling_matrix(rng, pb.wl.nd, 2, "rademacher"))
                     for _ in range(10000)])
    se = vals.std(ddof=1) / math.sqrt(vals.size)
    assert abs(vals.mean() - np.sum(np.abs(R) ** 2)) < 4 * se
