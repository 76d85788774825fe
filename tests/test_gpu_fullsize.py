"""Parity at the full 1,048,576-cell frequency-domain workload, in the launch
configuration the benchmark times (complex64 COCG with FP64 reliable updates to
relative residual 1e-10, 32 + 32 columns).  The oracle cannot evaluate the whole
workload here, so it checks what it can compute one by one, and properties that
hold at any size:
  * the true FP64 residual ||BW - A U|| / ||BW|| of every column, with A assembled
    by the oracle;
  * one forward column solved by the oracle's own COCG (rtol 1e-14), against U_0 and
    the measurements S[:, 0] = (CV)^T U_0 it implies, at the benchmark's rtol 1e-10
    (S is a far-field functional, so its error is ~1e3 x the residual) and at rtol
    1e-13, where every output must meet 1e-8;
  * the gradient against a central difference of the GPU misfit along a random
    direction (a property of any correct gradient);
  * the whole post-processing chain at this size: the oracle's own restriction,
    residual, sensitivity loops and PaLS derivative applied to the GPU's fields
    against the library's S, f, g_mu and g_p, in the benchmark's mixed path and in
    the plain FP64 path.
"""
import numpy as np
import pytest

from oracle import dot_oracle as orc
from paper_1706_05586_gb300 import dot as D
from paper_1706_05586_gb300 import synth

pytestmark = pytest.mark.gpu

WL = synth.WORKLOADS["dot128x128x64_w100MHz"]


@pytest.fixture(scope="module")
def setup():
    inp = synth.draw(WL)
    X = orc.cell_centres(WL.nx, WL.ny, WL.nz, WL.h)
    kw = dict(mu_in=synth.MU_IN, mu_out=synth.MU_OUT, c=WL.cutoff, eps=WL.eps, gamma=WL.gamma)
    Dfield = synth.diffusion_from_mua(orc.pals_mu(inp.p_true, X, **kw))
    mu0 = orc.pals_mu(inp.p0, X, **kw)
    A = orc.assemble(Dfield, mu0, WL.nx, WL.ny, WL.nz, WL.h, WL.bc, WL.omega_nu)
    B = orc.sparse_of_csc(WL.n, inp.B)
    C = orc.sparse_of_csc(WL.n, inp.C)
    rng = np.random.default_rng(3)
    M = (rng.standard_normal((WL.nd, WL.ns)) + 1j * rng.standard_normal((WL.nd, WL.ns))) * 1e-6
    h = D.dot_create(0)
    D.dot_set_grid(h, WL.nx, WL.ny, WL.nz, WL.h, WL.bc)
    D.dot_set_omega(h, WL.omega_nu)
    D.dot_set_diffusion(h, Dfield)
    D.dot_set_pals(h, inp.p0, synth.MU_IN, synth.MU_OUT, WL.cutoff, WL.eps, WL.gamma)
    D.dot_set_sources(h, inp.B)
    D.dot_set_detectors(h, inp.C)
    D.dot_set_data(h, M)
    D.dot_set_sampling(h, inp.W, inp.V)
    D.dot_set_solver(h, D.PREC_MIXED, 1e-10, 0)
    f, g, rc = D.dot_gradient(h, WL.np_)
    assert rc == D.DOT_OK
    yield dict(h=h, inp=inp, A=A, B=B, C=C, mu0=mu0, M=M, f=f, g=g, st=D.dot_get_stats(h))
    D.dot_destroy(h)


def test_absorption_matches(setup):
    mu = D.dot_get_mua(setup["h"], WL.n)
    assert np.max(np.abs(mu - setup["mu0"])) <= 1e-12


def test_true_residual_every_column(setup):
    h, inp, A = setup["h"], setup["inp"], setup["A"]
    U, Z = D.dot_get_fields(h, WL.n, WL.ls, WL.ld, True)
    for X, R in ((U, setup["B"] @ inp.W), (Z, setup["C"] @ inp.V)):
        res = np.linalg.norm(R - A @ X, axis=0) / np.linalg.norm(R, axis=0)
        assert np.all(res <= 1.5e-10), res.max()
    assert setup["st"]["relres_max"] <= 1e-10


@pytest.fixture(scope="module")
def oracle_column(setup):
    b0 = setup["B"] @ setup["inp"].W[:, 0]
    u0, _ = orc.krylov_solve(setup["A"], b0.astype(complex), rtol=1e-14)
    return u0, (setup["C"] @ setup["inp"].V).T @ u0


def test_one_column_against_oracle_solve(setup, oracle_column):
    h = setup["h"]
    u0, s_ref = oracle_column
    U, _ = D.dot_get_fields(h, WL.n, WL.ls, WL.ld, True)
    assert np.linalg.norm(U[:, 0] - u0) <= 1e-7 * np.linalg.norm(u0)
    S, _ = D.dot_measurements(h, WL.ls, WL.ld, True)
    assert np.linalg.norm(S[:, 0] - s_ref) <= 1e-5 * np.linalg.norm(s_ref)


def test_one_column_tight_tolerance(setup, oracle_column):
    h = setup["h"]
    u0, s_ref = oracle_column
    D.dot_set_solver(h, D.PREC_MIXED, 1e-13, 0)
    try:
        f, g, rc = D.dot_gradient(h, WL.np_)
        assert rc == D.DOT_OK and D.dot_get_stats(h)["relres_max"] <= 1e-13
        U, _ = D.dot_get_fields(h, WL.n, WL.ls, WL.ld, True)
        assert np.linalg.norm(U[:, 0] - u0) <= 1e-10 * np.linalg.norm(u0)
        S, _ = D.dot_measurements(h, WL.ls, WL.ld, True)
        assert np.linalg.norm(S[:, 0] - s_ref) <= 1e-8 * np.linalg.norm(s_ref)
        # the benchmark-tolerance gradient agrees with the tight one to its own accuracy
        assert np.linalg.norm(setup["g"] - g) <= 1e-4 * np.linalg.norm(g)
    finally:
        D.dot_set_solver(h, D.PREC_MIXED, 1e-10, 0)


def test_gradient_directional_difference(setup):
    h, inp = setup["h"], setup["inp"]
    rng = np.random.default_rng(11)
    d = rng.standard_normal(WL.np_)
    d[1::5] = 0.0
    d /= np.linalg.norm(d)
    eps = 1e-3
    D.dot_set_solver(h, D.PREC_MIXED, 1e-13, 0)
    try:
        D.dot_set_pals(h, inp.p0, synth.MU_IN, synth.MU_OUT, WL.cutoff, WL.eps, WL.gamma)
        _, g, _ = D.dot_gradient(h, WL.np_)
        fs = []
        for s in (+1, -1):
            D.dot_set_pals(h, inp.p0 + s * eps * d, synth.MU_IN, synth.MU_OUT, WL.cutoff, WL.eps, WL.gamma)
            fs.append(D.dot_misfit(h)[0])
    finally:
        D.dot_set_pals(h, inp.p0, synth.MU_IN, synth.MU_OUT, WL.cutoff, WL.eps, WL.gamma)
        D.dot_set_solver(h, D.PREC_MIXED, 1e-10, 0)
    fd = (fs[0] - fs[1]) / (2 * eps)
    gd = float(g @ d)
    assert abs(fd - gd) <= 1e-4 * np.linalg.norm(g), (fd, gd)


def _oracle_post(setup, U, Z, M):
    """S, R_s, f, g_mu and g_p of the oracle's definitions (Sec. 3.3, Eq. (EsTResidual),
    Eq. (Jacobian kth column), Eq. (UnbiasedGrad); Sec. 2 for dmu/dp) from given fields,
    with the rounding scale of each entry (the sum of the absolute values of its terms)."""
    inp = setup["inp"]
    W, V = inp.W, inp.V
    CV = setup["C"] @ V
    S = CV.T @ U
    S_scale = np.abs(CV).T @ np.abs(U)
    R_s = S - V.T @ M @ W
    ls, ld = W.shape[1], V.shape[1]
    r_abs = np.abs(R_s).ravel(order="F")
    g_mu = np.empty(WL.n)
    g_scale = np.empty(WL.n)
    chunk = 8192
    for v0 in range(0, WL.n, chunk):
        v1 = min(WL.n, v0 + chunk)
        J = orc.sampled_jacobian_mua(U[v0:v1], Z[v0:v1], np.eye(ls), np.eye(ld))   # -Z_l (.) U_i, row l + ld i
        g_mu[v0:v1] = orc.misfit_gradient(R_s, J)
        g_scale[v0:v1] = 2.0 * (np.abs(J).T @ r_abs)
    X = orc.cell_centres(WL.nx, WL.ny, WL.nz, WL.h)
    dmu = orc.pals_dmu_dp(inp.p0, X, synth.MU_IN, synth.MU_OUT, WL.cutoff, WL.eps, WL.gamma)
    g_p = dmu.T @ g_mu
    gp_scale = abs(dmu).T @ g_scale
    return dict(S=S, S_scale=S_scale, R_s=R_s, f=float(np.sum(np.abs(R_s) ** 2)), g_mu=g_mu, g_mu_scale=g_scale,
                g_p=g_p, g_p_scale=gp_scale)


@pytest.mark.parametrize("prec", [D.PREC_MIXED, D.PREC_FP64])
def test_gradient_chain_against_oracle(setup, prec):
    """The library's restriction (k_restrict_T, k_vt), misfit, double-float sensitivity sums
    (k_gmu: l_s l_d = 1,024 complex products per cell), tile-culled PaLS (k_pals_eval) and
    chain rule (k_chain_gp, 125 RBFs) at 1M cells against the oracle's plain loops applied
    to the same fields: agreement to rounding, 1e-10 relative and every entry within 1e-10
    of the absolute sum of its terms.  g_mu comes from the same context switched to
    dot_set_mua with the GPU's own absorption (the same coefficients, hence the same
    deterministic solve: f agrees bitwise)."""
    h, inp = setup["h"], setup["inp"]
    M = setup["M"]
    D.dot_set_pals(h, inp.p0, synth.MU_IN, synth.MU_OUT, WL.cutoff, WL.eps, WL.gamma)
    D.dot_set_solver(h, prec, 1e-10, 0)
    try:
        f, g_p, rc = D.dot_gradient(h, WL.np_)
        assert rc == D.DOT_OK
        S, _ = D.dot_measurements(h, WL.ls, WL.ld, True)
        U, Z = D.dot_get_fields(h, WL.n, WL.ls, WL.ld, True)
        mu = D.dot_get_mua(h, WL.n)
        D.dot_set_mua(h, mu)
        f_mu, g_mu, rc = D.dot_gradient(h, WL.n)
        assert rc == D.DOT_OK
        assert f_mu == f
        ref = _oracle_post(setup, U, Z, M)
        del U, Z
        for name in ("S", "g_mu", "g_p"):
            got = {"S": S, "g_mu": g_mu, "g_p": g_p}[name]
            d = np.abs(got - ref[name])
            assert np.linalg.norm(d) <= 1e-10 * np.linalg.norm(ref[name]), name
            assert np.all(d <= 1e-10 * ref[name + "_scale"]), name
        assert abs(f - ref["f"]) <= 1e-10 * ref["f"]
    finally:
        D.dot_set_pals(h, inp.p0, synth.MU_IN, synth.MU_OUT, WL.cutoff, WL.eps, WL.gamma)
        D.dot_set_solver(h, D.PREC_MIXED, 1e-10, 0)
