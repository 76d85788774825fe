"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same
seeded inputs, entry by entry.

FP64 path: the GPU solves until the FP64 true residual ||b - A x|| <= 2e-15 ||b|| in
every column (the oracle solves by sparse LU, whose own true residual is 0.5-1.7e-15
on these cases) and every output must agree to 1e-10.  Mixed precision (FP32 /
complex64 recurrence with FP64 reliable updates, true residual to 1e-13): 1e-8.  What
is asserted, with tol the bar of the path:
  * true relative errors |df| / f and ||dg|| / ||g|| at p0 (where R_s is 1-13% of S);
  * every column of U, Z and S and every row of J_mu and J_p: relative 2-norm error;
  * every solved column u: max |du| <= tol max |u| (pointwise field accuracy);
  * every entry of S, J_mu, J_p, g_mu, g_p and f: |d| <= tol E, where E is the entry's
    first-order error size under that pointwise field error (gpu_setup.oracle_scales:
    propagation through the definitions of Sec. 3.3, no tuned floor).
A residual stop at 1e-14 is not enough for the true relative f and g at 1e-10: S is
a far-field functional whose relative error is 1e2-1e3 x the residual, and near the
data f and g amplify it by ||S|| / ||R_s|| (a plain CG at 1e-14 gives 2e-10 in g on the
32x32x16 workload, 3e-11 at 2e-15).
"""
import numpy as np
import pytest

from oracle import dot_oracle as orc
from paper_1706_05586_gb300 import dot as D
from paper_1706_05586_gb300 import synth
from tests import problem
from tests.gpu_setup import (col_max_rel, col_rel, configure, entry_ratio, grad_err, misfit_err,
                             oracle_scales, rel)

pytestmark = pytest.mark.gpu

FP64_RTOL = 2e-15

ROB, DIR = synth.ROBIN, synth.DIRICHLET

CASES = {
    # odd shape, the paper's boundary setting (Dirichlet laterally, Robin top and bottom)
    "real_9x7x5_mixedbc": synth.small_workload(9, 7, 5, 0.4, src_grid=(2, 2), det_grid=(2, 1), ls=2, ld=1, m0=4,
                                               bc=(DIR, DIR, DIR, DIR, ROB, ROB), seed_index=61),
    # complex (COCG), ragged sizes, Gaussian sampling
    "cplx_11x6x7": synth.small_workload(11, 6, 7, 0.35, omega_nu=0.3, src_grid=(3, 1), det_grid=(2, 2), ls=3, ld=2,
                                        m0=5, sampling="gaussian", seed_index=62),
    # single simultaneous source and detector
    "real_13x10x6_l1": synth.small_workload(13, 10, 6, 0.3, src_grid=(3, 2), det_grid=(2, 3), ls=1, ld=1, m0=3,
                                            seed_index=63),
    # the 32x32x16 workload (16,384 cells, 27 RBFs, 2 + 2 Rademacher columns)
    "dot32x32x16": synth.WORKLOADS["dot32x32x16"],
    # a block of 16 + 16 columns on 8-aligned x, y: the mixed path takes the TMA-staged stencil
    "cplx_24x16x10_k32": synth.small_workload(24, 16, 10, 0.3, omega_nu=0.4, src_grid=(4, 4), det_grid=(4, 4),
                                              ls=16, ld=16, m0=5, sampling="gaussian", seed_index=65),
    "real_16x16x9_k32": synth.small_workload(16, 16, 9, 0.3, src_grid=(4, 4), det_grid=(4, 4), ls=16, ld=16,
                                             m0=4, sampling="gaussian", seed_index=66),
    # block widths 48 and 16 (odd multiples of 16): the TMA stencil with 16-column tiles
    "cplx_16x24x8_k48": synth.small_workload(16, 24, 8, 0.3, omega_nu=0.4, src_grid=(5, 5), det_grid=(5, 5),
                                             ls=24, ld=24, m0=5, sampling="gaussian", seed_index=67),
    "real_24x8x7_k16": synth.small_workload(24, 8, 7, 0.3, src_grid=(3, 3), det_grid=(3, 3), ls=8, ld=8,
                                            m0=4, sampling="gaussian", seed_index=68),
    # real block of 64 columns: the FP32 TMA stencil with 64-column tiles, two columns per lane
    "real_16x8x5_k64": synth.small_workload(16, 8, 5, 0.3, src_grid=(6, 6), det_grid=(6, 6), ls=32, ld=32, m0=4,
                                            sampling="gaussian", seed_index=74),
    # degenerate depth: a single layer of cells (no z neighbours), TMA path
    "real_16x16x1_k32": synth.small_workload(16, 16, 1, 0.3, src_grid=(4, 4), det_grid=(4, 4), ls=16, ld=16,
                                             m0=4, sampling="gaussian", seed_index=69),
    # a wide block: 128 + 128 columns (eight 32-column tiles, 256 column accumulators per block)
    "cplx_8x8x6_k256": synth.small_workload(8, 8, 6, 0.3, omega_nu=0.4, src_grid=(4, 4), det_grid=(4, 4), ls=128,
                                            ld=128, m0=3, sampling="gaussian", seed_index=70),
    # the 100 MHz frequency on a 24x20x12 grid
    "cplx_24x20x12_100MHz": synth.small_workload(24, 20, 12, 0.25, omega_nu=synth.OMEGA_NU_100MHZ, src_grid=(3, 3),
                                                 det_grid=(3, 3), ls=4, ld=4, m0=8, sampling="gaussian",
                                                 seed_index=64, rbf_radius=1.0),
}


@pytest.fixture(scope="module")
def ctx():
    h = D.dot_create(0)
    yield h
    D.dot_destroy(h)


_cache = {}


def _case(name):
    if name not in _cache:
        pb = problem.build(CASES[name])
        _cache[name] = (pb, pb.evaluate(pb.inp.p0))
    return _cache[name]


def _cplx(pb):
    return pb.wl.omega_nu != 0.0


@pytest.mark.parametrize("name", list(CASES))
def test_stencil_apply(name, ctx):
    pb, _ = _case(name)
    mu = pb.mu_of(pb.inp.p0)
    configure(ctx, pb, mua=mu)
    A = pb.A_of(mu)
    rng = np.random.default_rng(5)
    for k in (1, 3):
        X = rng.standard_normal((pb.wl.n, k))
        if _cplx(pb):
            X = X + 1j * rng.standard_normal((pb.wl.n, k))
        Y = D.dot_apply(ctx, X, _cplx(pb))
        ref = A @ X
        assert np.max(np.abs(Y - ref)) <= 1e-14 * np.max(np.abs(ref)), name


@pytest.mark.parametrize("name", list(CASES))
def test_pals_absorption(name, ctx):
    pb, _ = _case(name)
    configure(ctx, pb, p=pb.inp.p0)
    mu = D.dot_get_mua(ctx, pb.wl.n)
    assert np.max(np.abs(mu - pb.mu_of(pb.inp.p0))) <= 1e-12


_scales = {}


def _oracle_scales(name):
    if name not in _scales:
        pb, ref = _case(name)
        _scales[name] = oracle_scales(pb, ref, pb.dmu_of(pb.inp.p0))
    return _scales[name]


def _check_misfit_gradient(ctx, name, prec, rtol, tol):
    """f, g_p and S of one evaluation at p0 against the oracle, entry by entry."""
    pb, ref = _case(name)
    E = _oracle_scales(name)
    configure(ctx, pb, p=pb.inp.p0, prec=prec, rtol=rtol)
    f, g, rc = D.dot_gradient(ctx, pb.wl.np_)
    assert rc == D.DOT_OK
    st = D.dot_get_stats(ctx)
    assert st["k"] == pb.wl.ls + pb.wl.ld and st["relres_max"] <= rtol
    assert abs(f - ref["f"]) <= tol * ref["f"]
    assert rel(g, ref["g_p"]) <= tol
    assert abs(f - ref["f"]) <= tol * E["f"]
    assert entry_ratio(g, ref["g_p"], E["g_p"]) <= tol
    S, _ = D.dot_measurements(ctx, pb.wl.ls, pb.wl.ld, _cplx(pb))
    assert col_rel(S, ref["S"]) <= tol
    assert entry_ratio(S, ref["S"], E["S"]) <= tol
    return st


@pytest.mark.parametrize("name", list(CASES))
def test_misfit_gradient_fp64(name, ctx):
    _check_misfit_gradient(ctx, name, D.PREC_FP64, FP64_RTOL, 1e-10)


def _check_fields_jacobians(ctx, name, prec, rtol, tol):
    pb, ref = _case(name)
    E = _oracle_scales(name)
    configure(ctx, pb, p=pb.inp.p0, prec=prec, rtol=rtol)
    U, Z = D.dot_get_fields(ctx, pb.wl.n, pb.wl.ls, pb.wl.ld, _cplx(pb))
    for X, Xr in ((U, E["U"]), (Z, E["Z"])):
        assert col_rel(X, Xr) <= tol
        assert col_max_rel(X, Xr) <= tol
    Jmu, _ = D.dot_jacobian_mua(ctx, pb.wl.ls, pb.wl.ld, pb.wl.n, _cplx(pb))
    assert col_rel(Jmu.T, ref["J_mu"].T) <= tol          # every row
    assert entry_ratio(Jmu, ref["J_mu"], E["J_mu"]) <= tol
    Jp, _ = D.dot_jacobian_p(ctx, pb.wl.ls, pb.wl.ld, pb.wl.np_, _cplx(pb))
    assert col_rel(Jp.T, ref["J_p"].T) <= tol
    assert entry_ratio(Jp, ref["J_p"], E["J_p"]) <= tol


@pytest.mark.parametrize("name", list(CASES))
def test_fields_and_jacobians_fp64(name, ctx):
    _check_fields_jacobians(ctx, name, D.PREC_FP64, FP64_RTOL, 1e-10)


@pytest.mark.parametrize("name", list(CASES))
def test_gradient_wrt_mua(name, ctx):
    pb, ref = _case(name)
    E = _oracle_scales(name)
    mu = pb.mu_of(pb.inp.p0)
    configure(ctx, pb, mua=mu, rtol=FP64_RTOL)
    f, g, rc = D.dot_gradient(ctx, pb.wl.n)
    assert rc == D.DOT_OK
    assert rel(g, ref["g_mu"]) <= 1e-10
    assert entry_ratio(g, ref["g_mu"], E["g_mu"]) <= 1e-10
    assert abs(f - ref["f"]) <= 1e-10 * ref["f"]


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_precision(name, ctx):
    st = _check_misfit_gradient(ctx, name, D.PREC_MIXED, 1e-13, 1e-8)
    assert st["outer_steps"] >= 2


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_precision_fields_and_jacobians(name, ctx):
    _check_fields_jacobians(ctx, name, D.PREC_MIXED, 1e-13, 1e-8)


def test_gradient_at_true_parameters(ctx):
    """Near p_true the residual is noise-sized (1% of S), the case the scaled error is for."""
    pb, _ = _case("dot32x32x16")
    ref = pb.evaluate(pb.inp.p_true)
    configure(ctx, pb, p=pb.inp.p_true, rtol=FP64_RTOL)
    f, g, _ = D.dot_gradient(ctx, pb.wl.np_)
    assert grad_err(g, ref["g_p"], ref["J_p"], ref["R_s"], ref["S"]) <= 1e-10
    assert misfit_err(f, ref) <= 1e-10
    # entry by entry against each entry's first-order error size (at p_true that size
    # is set by S, not by the noise-sized R_s)
    E = oracle_scales(pb, ref, pb.dmu_of(pb.inp.p_true))
    assert entry_ratio(g, ref["g_p"], E["g_p"]) <= 1e-10
    assert abs(f - ref["f"]) <= 1e-10 * E["f"]


# ------------------------------------------------------------------ edge cases

def test_zero_column_and_determinism(ctx):
    pb, ref = _case("cplx_11x6x7")
    W = pb.inp.W.copy()
    W[:, 1] = 0.0                       # a simultaneous source with no light
    configure(ctx, pb, p=pb.inp.p0, W=W)
    f1, g1, rc = D.dot_gradient(ctx, pb.wl.np_)
    assert rc == D.DOT_OK
    S, _ = D.dot_measurements(ctx, pb.wl.ls, pb.wl.ld, True)
    assert np.all(S[:, 1] == 0)
    D.dot_set_solver(ctx, D.PREC_FP64, 1e-13, 0)   # invalidates the solve
    f2, g2, _ = D.dot_gradient(ctx, pb.wl.np_)
    assert f1 == f2 and np.array_equal(g1, g2)


def test_cache_reuse_and_invalidation(ctx):
    pb, _ = _case("real_9x7x5_mixedbc")
    configure(ctx, pb, p=pb.inp.p0)
    D.dot_gradient(ctx, pb.wl.np_)
    n0 = D.dot_get_stats(ctx)["block_solves"]
    D.dot_misfit(ctx)
    D.dot_gradient(ctx, pb.wl.np_)
    assert D.dot_get_stats(ctx)["block_solves"] == n0
    D.dot_set_pals(ctx, pb.inp.p_true, synth.MU_IN, synth.MU_OUT, pb.wl.cutoff, pb.wl.eps, pb.wl.gamma)
    D.dot_gradient(ctx, pb.wl.np_)
    assert D.dot_get_stats(ctx)["block_solves"] == n0 + 1


def test_not_converged_reports_status(ctx):
    pb, _ = _case("dot32x32x16")
    configure(ctx, pb, p=pb.inp.p0, maxit=3)
    f, rc = D.dot_misfit(ctx, allow=(D.DOT_ENOTCONV,))
    assert rc == D.DOT_ENOTCONV and np.isfinite(f)
    assert D.dot_get_stats(ctx)["iters_max"] == 3
    D.dot_set_solver(ctx, D.PREC_FP64, 1e-10, 0)
    f, rc = D.dot_misfit(ctx)
    assert rc == D.DOT_OK


def test_argument_and_state_errors(ctx):
    h = D.dot_create(0)
    try:
        with pytest.raises(D.DotError) as e:
            D.dot_misfit(h)
        assert e.value.code == D.DOT_ESTATE
        with pytest.raises(D.DotError) as e:
            D.dot_set_grid(h, 4, 4, 0, 0.1, (0,) * 6)
        assert e.value.code == D.DOT_EINVAL
        with pytest.raises(D.DotError) as e:
            D.dot_set_grid(h, 4, 4, 4, 0.1, (0, 0, 7, 0, 0, 0))
        assert e.value.code == D.DOT_EINVAL
        D.dot_set_grid(h, 4, 4, 4, 0.1, (0,) * 6)
        with pytest.raises(D.DotError) as e:
            D.dot_set_diffusion(h, -np.ones(64))
        assert e.value.code == D.DOT_EINVAL
        with pytest.raises(D.DotError) as e:
            D.dot_set_sources(h, (np.array([0, 1]), np.array([64]), np.array([1.0])))
        assert e.value.code == D.DOT_EINVAL
        D.dot_set_sources(h, (np.array([0, 1]), np.array([3]), np.array([1.0])))
        D.dot_set_detectors(h, (np.array([0, 1]), np.array([60]), np.array([1.0])))
        with pytest.raises(D.DotError) as e:
            D.dot_set_sampling(h, np.ones((1, 600)), np.ones((1, 600)))
        assert e.value.code == D.DOT_EINVAL
        with pytest.raises(D.DotError) as e:
            D.dot_misfit(h)
        assert e.value.code == D.DOT_ESTATE
    finally:
        D.dot_destroy(h)


@pytest.mark.parametrize("name", ["cplx_11x6x7", "real_13x10x6_l1"])
def test_forward_model_all_sources(name, ctx):
    """dot_forward_model returns C^T A^{-1} B for every physical source (Eq. (Eq:compmeas))."""
    pb, _ = _case(name)
    mu = pb.mu_of(pb.inp.p0)
    configure(ctx, pb, mua=mu, rtol=FP64_RTOL)
    M, rc = D.dot_forward_model(ctx, pb.wl.ns, pb.wl.nd, _cplx(pb))
    assert rc == D.DOT_OK
    ref = pb.Cd.T @ orc.solve(pb.A_of(mu), pb.Bd)
    assert rel(M, ref) <= 1e-10
    # the sampled state is untouched: the next misfit uses W, V again
    f, _ = D.dot_misfit(ctx)
    out = orc.evaluate(pb.D, mu, pb.grid, pb.wl.bc, pb.wl.omega_nu, pb.Bd, pb.Cd, pb.M, pb.inp.W, pb.inp.V)
    assert abs(f - out["f"]) <= 1e-10 * out["f"]


@pytest.mark.parametrize("name", ["cplx_24x16x10_k32", "real_16x16x9_k32", "cplx_16x24x8_k48", "real_24x8x7_k16",
                                  "real_16x16x1_k32", "cplx_8x8x6_k256", "real_16x8x5_k64"])
def test_tma_stencil_matches_direct_load_kernel(name, ctx):
    """The three stencil paths (direction update fused into the TMA stencil, TMA stencil
    after a separate direction pass, direct loads) give the same solve to rounding (their
    column sums p^T q add in different orders); the fused path runs on every case whose
    padded width is a multiple of 16 (complex) or 32 (real) columns."""
    pb, ref = _case(name)
    out = {}
    try:
        for mode in (2, 1, 0):
            configure(ctx, pb, p=pb.inp.p0, prec=D.PREC_MIXED, rtol=1e-13)
            D.dot_set_stencil_path(ctx, mode)
            f, g, rc = D.dot_gradient(ctx, pb.wl.np_)
            assert rc == D.DOT_OK
            st = D.dot_get_stats(ctx)
            out[mode] = (f, g, st["iters_max"], st["fused_direction"], st["tuned_tma"])
    finally:
        D.dot_set_stencil_path(ctx, 2)
    kp = -(-(pb.wl.ls + pb.wl.ld) // 4) * 4
    fused_ok = kp % (16 if _cplx(pb) else 32) == 0
    assert out[2][3] == (1 if fused_ok else 0) and out[1][3] == 0 and out[0][3] == 0
    assert out[2][4] == 1 and out[1][4] == 1 and out[0][4] == 0
    for m in (2, 1):
        assert abs(out[m][0] - out[0][0]) <= 1e-10 * abs(out[0][0])
        assert rel(out[m][1], out[0][1]) <= 1e-9
        assert abs(out[m][2] - out[0][2]) <= 3
        assert abs(out[m][0] - ref["f"]) <= 1e-8 * ref["f"]


@pytest.mark.parametrize("prec", [D.PREC_FP64, D.PREC_MIXED])
def test_widest_block_fields(prec, ctx):
    """The widest block the library accepts, 512 + 512 columns (32-column TMA tiles in
    the mixed path, one column per thread in the FP64 path), against the oracle's
    solves of the same right-hand sides; the misfit from those fields."""
    wl = synth.small_workload(8, 8, 4, 0.3, omega_nu=0.4, src_grid=(4, 4), det_grid=(4, 4), ls=512, ld=512, m0=3,
                              sampling="gaussian", seed_index=72)
    pb = problem.build(wl)
    configure(ctx, pb, p=pb.inp.p0, prec=prec, rtol=1e-13)
    f, rc = D.dot_misfit(ctx)
    assert rc == D.DOT_OK
    st = D.dot_get_stats(ctx)
    assert st["k"] == 1024 and st["relres_max"] <= 1e-13
    if prec == D.PREC_MIXED:
        assert st["tuned_tma"] == 1
    U, Z = D.dot_get_fields(ctx, wl.n, wl.ls, wl.ld, True)
    mu = pb.mu_of(pb.inp.p0)
    A = orc.assemble(pb.D, mu, wl.nx, wl.ny, wl.nz, wl.h, wl.bc, wl.omega_nu)
    U_ref = orc.solve(A, pb.Bd @ pb.inp.W)
    Z_ref = orc.solve(A, pb.Cd @ pb.inp.V)
    assert rel(U, U_ref) <= 1e-10 and rel(Z, Z_ref) <= 1e-10
    S = (pb.Cd @ pb.inp.V).T @ U_ref
    R_s = S - pb.inp.V.T @ pb.M @ pb.inp.W
    f_ref = float(np.sum(np.abs(R_s) ** 2))
    assert abs(f - f_ref) <= 1e-8 * max(f_ref, 2.0 * np.linalg.norm(R_s) * np.linalg.norm(S))
