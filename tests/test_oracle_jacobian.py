"""Pins for the oracle's sampled Jacobians and gradient (Eq. (Jacobiancomp),
Eq. (Jacobian kth column), Eq. (UnbiasedGrad)): a complex step on mu (exact to
rounding at omega = 0), central finite differences on p and on the misfit, and
agreement of the two gradient routes."""
import numpy as np
import pytest

from oracle import dot_oracle as orc
from paper_1706_05586_gb300 import synth
from tests import problem


def _sampled_S(pb, mu):
    A = orc.assemble(pb.D, mu, *pb.grid, pb.wl.bc, pb.wl.omega_nu)
    U = orc.solve(A, pb.Bd @ pb.inp.W)
    return pb.inp.V.T @ pb.Cd.T @ U


@pytest.fixture(scope="module")
def pb_real():
    return problem.build(synth.small_workload(7, 6, 5, 0.4, src_grid=(2, 2), det_grid=(2, 2),
                                              ls=2, ld=2, m0=4, seed_index=51))


@pytest.fixture(scope="module")
def pb_cplx():
    return problem.build(synth.small_workload(6, 6, 5, 0.4, omega_nu=0.6, src_grid=(2, 2),
                                              det_grid=(2, 1), ls=2, ld=1, m0=4, seed_index=52,
                                              sampling="gaussian"))


def test_jacobian_mu_complex_step(pb_real):
    """At omega = 0 the map mu -> S is real-analytic, so Im S(mu + i t e_v)/t with t = 1e-30
    is dS/dmu_v to rounding: an exact pin for J_mu[(l,i), v] = -Z_l[v] U_i[v]."""
    pb = pb_real
    mu = pb.mu_of(pb.inp.p0)
    out = pb.evaluate(pb.inp.p0, with_p=False)
    ld, ls = pb.wl.ld, pb.wl.ls
    rng = np.random.default_rng(53)
    for v in rng.choice(pb.wl.n, 12, replace=False):
        t = 1e-30
        mc = mu.astype(complex)
        mc[v] += 1j * t
        A = orc.assemble(pb.D, np.zeros(pb.wl.n), *pb.grid, pb.wl.bc, 0.0).astype(complex)
        A = A + __import__("scipy.sparse", fromlist=["diags"]).diags(mc)
        U = orc.solve(A, pb.Bd @ pb.inp.W)
        dS = (pb.inp.V.T @ pb.Cd.T @ U).imag / t
        col = out["J_mu"][:, v].reshape(ld, ls, order="F")
        assert np.allclose(col, dS, rtol=1e-12, atol=1e-14 * np.abs(dS).max() + 1e-300), v


def test_jacobian_mu_central_difference_complex(pb_cplx):
    pb = pb_cplx
    mu = pb.mu_of(pb.inp.p0)
    out = pb.evaluate(pb.inp.p0, with_p=False)
    ld, ls = pb.wl.ld, pb.wl.ls
    for v in (0, 17, 63, pb.wl.n - 1):
        t = 1e-5
        e = np.zeros(pb.wl.n)
        e[v] = t
        dS = (_sampled_S(pb, mu + e) - _sampled_S(pb, mu - e)) / (2 * t)
        col = out["J_mu"][:, v].reshape(ld, ls, order="F")
        assert np.allclose(col, dS, rtol=1e-7, atol=1e-9 * np.abs(dS).max()), v


@pytest.mark.parametrize("which", ["real", "cplx"])
def test_jacobian_p_central_difference(which, pb_real, pb_cplx):
    pb = pb_real if which == "real" else pb_cplx
    p = pb.inp.p0
    out = pb.evaluate(p)
    ld, ls = pb.wl.ld, pb.wl.ls
    scale = np.abs(out["J_p"]).max()
    for k in range(p.size):
        step = 1e-6
        e = np.zeros_like(p)
        e[k] = step
        dS = (_sampled_S(pb, pb.mu_of(p + e)) - _sampled_S(pb, pb.mu_of(p - e))) / (2 * step)
        col = out["J_p"][:, k].reshape(ld, ls, order="F")
        assert np.allclose(col, dS, rtol=1e-5, atol=1e-6 * scale), k


@pytest.mark.parametrize("which", ["real", "cplx"])
def test_gradient_routes_and_finite_difference(which, pb_real, pb_cplx):
    pb = pb_real if which == "real" else pb_cplx
    p = pb.inp.p0
    out = pb.evaluate(p)
    g_chain = pb.dmu_of(p).T @ out["g_mu"]
    assert np.allclose(out["g_p"], g_chain, rtol=1e-12, atol=1e-13 * np.abs(g_chain).max())

    def f_of(pp):
        S = _sampled_S(pb, pb.mu_of(pp)) - pb.inp.V.T @ pb.M @ pb.inp.W
        return float(np.sum(np.abs(S) ** 2))

    scale = np.abs(out["g_p"]).max()
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = 1e-6
        fd = (f_of(p + e) - f_of(p - e)) / 2e-6
        assert abs(fd - out["g_p"][k]) <= 1e-5 * scale, (k, fd, out["g_p"][k])
    assert out["f"] == pytest.approx(f_of(p), rel=1e-12)


def test_full_tensor_matches_mu_jacobian_with_identity_dmu(pb_real):
    """With dmu/dp = I the tensor route and the voxelwise-product route coincide."""
    pb = pb_real
    mu = pb.mu_of(pb.inp.p0)
    A = pb.A_of(mu)
    Uf, Zf = orc.fields_full(A, pb.Bd, pb.Cd)
    J3 = orc.jacobian_tensor(Uf, Zf, np.eye(pb.wl.n))
    Js = orc.sampled_jacobian(J3, pb.inp.W, pb.inp.V)
    Jmu = orc.sampled_jacobian_mua(Uf, Zf, pb.inp.W, pb.inp.V)
    assert np.allclose(Js, Jmu, rtol=1e-13, atol=1e-15 * np.abs(Jmu).max())
