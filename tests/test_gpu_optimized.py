"""Optimized + complementary simultaneous sources and detectors on the GPU
(dot_optimized_sampling) against the oracle's Algorithm 1 on the same Jacobian
tensor (Sec. 3.2; Eqs. (Jtilde), (Ktilde), (Ltilde), (newW), (newV)).  The optimized
columns are unique only up to a rotation inside their span, so their projectors are
compared; the complementary columns (I - W^W^T) Y~ are unique given the projector."""
import numpy as np
import pytest

from oracle import dot_oracle as orc
from paper_1706_05586_gb300 import dot as D
from paper_1706_05586_gb300 import synth
from tests import problem
from tests.gpu_setup import configure

pytestmark = pytest.mark.gpu

CASES = {
    "real_14x12x8": synth.small_workload(14, 12, 8, 0.3, src_grid=(3, 3), det_grid=(3, 3), ls=4, ld=4, m0=4,
                                         sampling="gaussian", seed_index=81),
    "cplx_12x12x9": synth.small_workload(12, 12, 9, 0.3, omega_nu=0.4, src_grid=(4, 2), det_grid=(3, 3), ls=5, ld=4,
                                         m0=5, sampling="gaussian", seed_index=82),
    # 128 x 128 physical sources and detectors: the Gram products of the unfoldings take
    # the 64 x 64 register-tiled kernel (n >= 128)
    "real_16x16x8_n128": synth.small_workload(16, 16, 8, 0.3, src_grid=(16, 8), det_grid=(16, 8), ls=4, ld=4,
                                              m0=4, sampling="gaussian", seed_index=83),
    "cplx_16x16x8_n128": synth.small_workload(16, 16, 8, 0.3, omega_nu=0.4, src_grid=(8, 16), det_grid=(16, 8),
                                              ls=4, ld=4, m0=4, sampling="gaussian", seed_index=84),
}


@pytest.mark.parametrize("name", list(CASES))
def test_optimized_sampling_matches_oracle(name):
    pb = problem.build(CASES[name])
    wl = pb.wl
    qs, qd = 2, 2
    mu = pb.mu_of(pb.inp.p0)
    A = pb.A_of(mu)
    Uf, Zf = orc.fields_full(A, pb.Bd, pb.Cd)
    J3 = orc.jacobian_tensor(Uf, Zf, pb.dmu_of(pb.inp.p0))
    Wo, Vo, sweeps_o = orc.optimized_sources_detectors(J3, qs, qd)
    rng = np.random.default_rng(5)
    Yt = rng.standard_normal((wl.ns, wl.ls - qs)) / np.sqrt(wl.ls - qs)
    Zt = rng.standard_normal((wl.nd, wl.ld - qd)) / np.sqrt(wl.ld - qd)
    h = D.dot_create(0)
    try:
        configure(h, pb, p=pb.inp.p0, rtol=1e-14)
        f_before, _ = D.dot_misfit(h)
        W, V, sweeps, obj = D.dot_optimized_sampling(h, qs, qd, wl.ns, wl.nd, wl.ls, wl.ld, Yt, Zt)
        f_after, _ = D.dot_misfit(h)
    finally:
        D.dot_destroy(h)
    assert f_after == f_before                      # the context's own sampling is untouched
    Wh, Vh = W[:, :qs], V[:, :qd]
    assert np.allclose(Wh.T @ Wh, np.eye(qs), atol=1e-12)
    assert np.allclose(Vh.T @ Vh, np.eye(qd), atol=1e-12)
    assert np.linalg.norm(Wh @ Wh.T - Wo @ Wo.T) <= 1e-8
    assert np.linalg.norm(Vh @ Vh.T - Vo @ Vo.T) <= 1e-8
    assert np.allclose(W[:, qs:], orc.complement_sampling(Wo, Yt)[:, qs:], atol=1e-8)
    assert np.allclose(V[:, qd:], orc.complement_sampling(Vo, Zt)[:, qd:], atol=1e-8)
    ref_obj = orc.sampled_jacobian_norm2(J3, Wo, Vo)
    assert obj == pytest.approx(ref_obj, rel=1e-9)
    assert abs(sweeps - sweeps_o) <= 2
    assert obj <= np.sum(np.abs(J3) ** 2) * (1 + 1e-12)


def test_optimized_sampling_argument_errors():
    pb = problem.build(CASES["real_14x12x8"])
    h = D.dot_create(0)
    try:
        configure(h, pb, p=pb.inp.p0, rtol=1e-12)
        with pytest.raises(D.DotError) as e:
            D.dot_optimized_sampling(h, 9, 1, pb.wl.ns, pb.wl.nd, 10, 2, np.zeros((9, 1)), np.zeros((9, 1)))
        assert e.value.code == D.DOT_EINVAL
        D.dot_set_mua(h, pb.mu_true)
        with pytest.raises(D.DotError) as e:
            D.dot_optimized_sampling(h, 1, 1, pb.wl.ns, pb.wl.nd, 1, 1)
        assert e.value.code == D.DOT_ESTATE
    finally:
        D.dot_destroy(h)


def test_optimized_sampling_64x64x32_properties():
    """The 64x64x32 workload (131,072 cells, 64 x 64 physical, 125 RBFs): 4 optimized +
    8 complementary columns per side; isometry, complement orthogonality, and the
    optimized sampling captures more of ||J||_F^2 than the random columns alone."""
    wl = synth.WORKLOADS["dot64x64x32"]
    inp = synth.draw(wl)
    h = D.dot_create(0)
    try:
        D.dot_set_grid(h, wl.nx, wl.ny, wl.nz, wl.h, wl.bc)
        D.dot_set_omega(h, wl.omega_nu)
        D.dot_set_diffusion(h, np.full(wl.n, 1.0 / 30.0))
        D.dot_set_pals(h, inp.p_true, synth.MU_IN, synth.MU_OUT, wl.cutoff, wl.eps, wl.gamma)
        D.dot_set_diffusion(h, synth.diffusion_from_mua(D.dot_get_mua(h, wl.n)))
        D.dot_set_pals(h, inp.p0, synth.MU_IN, synth.MU_OUT, wl.cutoff, wl.eps, wl.gamma)
        D.dot_set_sources(h, inp.B)
        D.dot_set_detectors(h, inp.C)
        D.dot_set_solver(h, D.PREC_MIXED, 1e-10, 0)
        rng = np.random.default_rng(6)
        q, l = 4, 12
        Yt = rng.standard_normal((wl.ns, l - q)) / np.sqrt(l - q)
        Zt = rng.standard_normal((wl.nd, l - q)) / np.sqrt(l - q)
        W, V, sweeps, obj = D.dot_optimized_sampling(h, q, q, wl.ns, wl.nd, l, l, Yt, Zt)
    finally:
        D.dot_destroy(h)
    assert np.allclose(W[:, :q].T @ W[:, :q], np.eye(q), atol=1e-10)
    assert np.allclose(V[:, :q].T @ V[:, :q], np.eye(q), atol=1e-10)
    assert np.abs(W[:, :q].T @ W[:, q:]).max() < 1e-10
    assert np.abs(V[:, :q].T @ V[:, q:]).max() < 1e-10
    assert 1 <= sweeps <= 100 and obj > 0
