"""Pins for the oracle's solves (dense brute force, reciprocity, linearity) and for its
PaLS map (closed forms of the Wendland function, the smoothed Heaviside, finite
differences of phi and mu), Sec. 2 and Sec. 3."""
import math

import numpy as np
import pytest

from oracle import dot_oracle as orc
from paper_1706_05586_gb300 import synth
from tests import problem

ROB, DIR = orc.ROBIN, orc.DIRICHLET


@pytest.mark.parametrize("omega_nu", [0.0, 0.29])
def test_solve_matches_dense_numpy(omega_nu):
    rng = np.random.default_rng(31)
    nx, ny, nz = 6, 5, 4          # 120 unknowns
    D = 0.03 + 0.02 * rng.random(nx * ny * nz)
    mu = 0.05 + 0.15 * rng.random(nx * ny * nz)
    A = orc.assemble(D, mu, nx, ny, nz, 0.25, (ROB, DIR, ROB, ROB, ROB, DIR), omega_nu)
    b = rng.standard_normal((nx * ny * nz, 3))
    ref = np.linalg.solve(A.toarray(), b.astype(A.dtype))
    assert np.allclose(orc.solve(A, b), ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())
    for c in range(3):
        x, _ = orc.krylov_solve(A, b[:, c], rtol=1e-14)
        assert np.allclose(x, ref[:, c], rtol=1e-10, atol=1e-11 * np.abs(ref[:, c]).max())


def test_krylov_matches_direct_at_32x32x16():
    pb = problem.build(synth.WORKLOADS["dot32x32x16"])
    A = pb.A_of(pb.mu_true)
    b = pb.Bd[:, 5]
    x_direct = orc.solve(A, b)
    x_cg, it = orc.krylov_solve(A, b, rtol=1e-13)
    assert it > 10
    assert np.linalg.norm(x_cg - x_direct) <= 1e-11 * np.linalg.norm(x_direct)


@pytest.mark.parametrize("omega_nu", [0.0, synth.OMEGA_NU_100MHZ * 20])
def test_reciprocity_source_detector_swap(omega_nu):
    """C^T A^{-1} B = (B^T A^{-1} C)^T because the discretized A is (complex) symmetric."""
    wl = synth.small_workload(8, 7, 6, 0.3, omega_nu=omega_nu, src_grid=(2, 2), det_grid=(3, 1),
                              seed_index=32)
    pb = problem.build(wl)
    A = pb.A_of(pb.mu_true)
    m_fwd = pb.Cd.T @ orc.solve(A, pb.Bd)
    m_rev = pb.Bd.T @ orc.solve(A, pb.Cd)
    assert np.allclose(m_fwd, m_rev.T, rtol=1e-11, atol=1e-13 * np.abs(m_fwd).max())


def test_linearity_simultaneous_sources():
    """A^{-1}(B W) = (A^{-1} B) W, the identity behind Eq. (Rw)."""
    pb = problem.build(synth.small_workload(7, 6, 5, 0.3, src_grid=(3, 2), ls=3, seed_index=33))
    A = pb.A_of(pb.mu_true)
    lhs = orc.solve(A, pb.Bd @ pb.inp.W)
    rhs = orc.solve(A, pb.Bd) @ pb.inp.W
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(rhs)


# ------------------------------------------------------------------------ PaLS

def test_wendland_closed_forms():
    assert orc.wendland(0.0) == 1.0
    assert orc.wendland(1.0) == 0.0
    assert orc.wendland(1.5) == 0.0
    assert orc.wendland(0.5) == pytest.approx(0.5 ** 4 * 3.0, rel=1e-15)
    assert orc.wendland_prime(1.0) == 0.0
    assert orc.wendland_prime(0.0) == 0.0
    r = np.linspace(0.05, 0.95, 19)
    fd = (orc.wendland(r + 1e-6) - orc.wendland(r - 1e-6)) / 2e-6
    assert np.allclose(orc.wendland_prime(r), fd, rtol=1e-8, atol=1e-9)


def test_heaviside_is_c1_ramp():
    eps = 0.3
    assert orc.heaviside(-eps, eps) == pytest.approx(0.0, abs=1e-16)
    assert orc.heaviside(eps, eps) == pytest.approx(1.0, abs=1e-15)
    assert orc.heaviside(0.0, eps) == 0.5
    assert orc.heaviside_prime(eps, eps) == pytest.approx(0.0, abs=1e-15)
    assert orc.heaviside_prime(-eps, eps) == pytest.approx(0.0, abs=1e-15)
    t = np.linspace(-0.99 * eps, 0.99 * eps, 41)
    fd = (orc.heaviside(t + 1e-7, eps) - orc.heaviside(t - 1e-7, eps)) / 2e-7
    assert np.allclose(orc.heaviside_prime(t, eps), fd, rtol=1e-6, atol=1e-7)
    tt = np.linspace(-eps, eps, 200001)
    assert np.trapezoid(orc.heaviside_prime(tt, eps), tt) == pytest.approx(1.0, rel=1e-9)
    # monotone
    assert np.all(np.diff(orc.heaviside(np.linspace(-2 * eps, 2 * eps, 1001), eps)) >= -1e-15)


def test_pals_phi_single_rbf_closed_form():
    gamma = 0.01
    p = np.array([1.7, 2.0, 0.5, 0.4, 0.3])
    X = np.array([[0.5, 0.4, 0.3], [0.7, 0.4, 0.3], [0.5, 0.4, 1.0]])
    r = np.sqrt(4.0 * np.array([0.0, 0.04, 0.49]) + gamma ** 2)
    expect = 1.7 * np.where(r < 1, (1 - r) ** 4 * (4 * r + 1), 0.0)
    assert np.allclose(orc.pals_phi(p, X, gamma), expect, rtol=1e-15, atol=1e-16)
    assert orc.pals_phi(p, X, gamma)[2] == 0.0


def test_pals_derivatives_finite_difference():
    rng = np.random.default_rng(41)
    wl = synth.small_workload(9, 8, 7, 0.25, m0=5, seed_index=41)
    inp = synth.draw(wl)
    X = orc.cell_centres(wl.nx, wl.ny, wl.nz, wl.h)
    p = inp.p0
    J = orc.pals_dphi_dp(p, X, wl.gamma).toarray()
    step = 1e-6
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = step
        fd = (orc.pals_phi(p + e, X, wl.gamma) - orc.pals_phi(p - e, X, wl.gamma)) / (2 * step)
        assert np.allclose(J[:, k], fd, rtol=1e-5, atol=1e-7 * max(1.0, np.abs(fd).max())), k
    kw = dict(mu_in=synth.MU_IN, mu_out=synth.MU_OUT, c=0.0, eps=0.05, gamma=wl.gamma)
    Jm = orc.pals_dmu_dp(p, X, **kw).toarray()
    for k in rng.choice(p.size, 8, replace=False):
        e = np.zeros_like(p)
        e[k] = 1e-7
        fd = (orc.pals_mu(p + e, X, **kw) - orc.pals_mu(p - e, X, **kw)) / 2e-7
        assert np.allclose(Jm[:, k], fd, rtol=1e-4, atol=1e-6 * max(1.0, np.abs(fd).max())), k


def test_pals_mu_levels():
    wl = synth.small_workload(10, 10, 8, 0.25, m0=6, seed_index=42)
    inp = synth.draw(wl)
    X = orc.cell_centres(wl.nx, wl.ny, wl.nz, wl.h)
    mu = orc.pals_mu(inp.p_true, X, 0.2, 0.05, 0.0, wl.eps, wl.gamma)
    phi = orc.pals_phi(inp.p_true, X, wl.gamma)
    assert np.all(mu[phi > wl.eps] == 0.2)
    assert np.all(mu[phi < -wl.eps] == 0.05)
    assert np.all((mu >= 0.05) & (mu <= 0.2))
