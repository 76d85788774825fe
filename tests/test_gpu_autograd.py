"""The misfit as a torch.autograd.Function: gradient against the FP64 oracle and
against central differences of the library's own misfit, in checkpoint and recompute
modes, plus a forward/backward at the 128^3 workload (2,097,152 cells, 1,000 RBFs,
5,000 parameters) checked along a random direction."""
import time

import numpy as np
import pytest

from paper_1706_05586_gb300 import dot as D
from paper_1706_05586_gb300 import synth
from tests import problem
from tests.gpu_setup import configure, grad_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _consts(wl):
    from paper_1706_05586_gb300.autograd import PalsConstants
    return PalsConstants(synth.MU_IN, synth.MU_OUT, wl.cutoff, wl.eps, wl.gamma)


@pytest.mark.parametrize("recompute", [False, True])
@pytest.mark.parametrize("device", ["cuda", "cpu"])
def test_autograd_matches_oracle(recompute, device):
    from paper_1706_05586_gb300.autograd import misfit
    wl = synth.small_workload(11, 6, 7, 0.35, omega_nu=0.3, src_grid=(3, 1), det_grid=(2, 2), ls=3, ld=2, m0=5,
                              sampling="gaussian", seed_index=62)
    pb = problem.build(wl)
    ref = pb.evaluate(pb.inp.p0)
    h = D.dot_create(0)
    try:
        configure(h, pb, p=pb.inp.p0, prec=D.PREC_MIXED, rtol=1e-13)
        p = torch.tensor(pb.inp.p0, dtype=torch.float64, device=device, requires_grad=True)
        f = misfit(p, h, _consts(wl), recompute=recompute)
        (3.0 * f).backward()
        assert abs(f.item() - ref["f"]) <= 1e-8 * ref["f"]
        g = p.grad.cpu().numpy() / 3.0
        assert grad_err(g, ref["g_p"], ref["J_p"], ref["R_s"], ref["S"]) <= 1e-8
    finally:
        D.dot_destroy(h)


def test_backward_after_a_second_forward_uses_its_own_point():
    from paper_1706_05586_gb300.autograd import misfit
    wl = synth.small_workload(9, 7, 5, 0.4, src_grid=(2, 2), det_grid=(2, 1), ls=2, ld=1, m0=4, seed_index=61)
    pb = problem.build(wl)
    ref0 = pb.evaluate(pb.inp.p0)
    h = D.dot_create(0)
    try:
        configure(h, pb, p=pb.inp.p0, prec=D.PREC_FP64, rtol=1e-14)
        p0 = torch.tensor(pb.inp.p0, dtype=torch.float64, requires_grad=True)
        p1 = torch.tensor(pb.inp.p_true, dtype=torch.float64, requires_grad=True)
        f0 = misfit(p0, h, _consts(wl))
        f1 = misfit(p1, h, _consts(wl))
        f0.backward()
        assert grad_err(p0.grad.numpy(), ref0["g_p"], ref0["J_p"], ref0["R_s"], ref0["S"]) <= 1e-10
        f1.backward()
        assert np.all(np.isfinite(p1.grad.numpy()))
    finally:
        D.dot_destroy(h)


def test_autograd_128cubed_against_oracle_and_central_differences():
    """The 128^3 workload (2,097,152 cells, omega = 0, 1,000 RBFs, 5,000 parameters) sampled
    as its configuration asks: 24 random + 8 optimized simultaneous sources and detectors
    from the 512 x 512 physical ones (Algorithm 1 on the full Jacobian tensor at p0,
    dot_optimized_sampling: a 1,024-column solve and a 512 x 512 x 5,000 tensor), then
    through the autograd wrapper in the plain FP64 path:
      * the backward pass against the oracle's gradient chain applied to the fields the
        forward pass checkpointed (restriction, the explicit (i, l) sensitivity loops in
        cell chunks, the oracle's PaLS derivative): agreement to rounding, 1e-10
        relative, every entry within 1e-10 of the absolute sum of its terms;
      * the directional derivative g.d against a central difference of the misfit with
        step 1e-6 along the unit gradient direction d = g / ||g||.  The difference's error
        is the misfit's solve-level error over the step (f is accurate to about 1e-12
        relative with the solves at a true residual of 1e-13); along d the misfit changes
        most, so that error stays below 1e-3 |g.d|.  (Along a random direction of the
        5,000 parameters the change of f over the step is 2.6e-10 relative, at the
        solves' accuracy, and the difference is off by 1%.)"""
    from oracle import dot_oracle as orc
    from paper_1706_05586_gb300.autograd import misfit
    wl = synth.WORKLOADS["dot128x128x128"]
    inp = synth.draw(wl)
    X = orc.cell_centres(wl.nx, wl.ny, wl.nz, wl.h)
    kw = dict(mu_in=synth.MU_IN, mu_out=synth.MU_OUT, c=wl.cutoff, eps=wl.eps, gamma=wl.gamma)
    rng = np.random.default_rng(4)
    M = 1e-6 * rng.standard_normal((wl.nd, wl.ns))
    h = D.dot_create(0)
    try:
        D.dot_set_grid(h, wl.nx, wl.ny, wl.nz, wl.h, wl.bc)
        D.dot_set_omega(h, wl.omega_nu)
        # D enters only the GPU solve (the oracle's chain below starts from its fields), so
        # it comes from the library's absorption at p_true, as in the benchmark
        D.dot_set_diffusion(h, np.full(wl.n, 1.0 / 30.0))
        D.dot_set_pals(h, inp.p_true, synth.MU_IN, synth.MU_OUT, wl.cutoff, wl.eps, wl.gamma)
        D.dot_set_diffusion(h, synth.diffusion_from_mua(D.dot_get_mua(h, wl.n)))
        D.dot_set_pals(h, inp.p0, synth.MU_IN, synth.MU_OUT, wl.cutoff, wl.eps, wl.gamma)
        D.dot_set_sources(h, inp.B)
        D.dot_set_detectors(h, inp.C)
        D.dot_set_data(h, M)
        # 8 optimized + 24 complementary random columns per side (mixed-precision solves)
        D.dot_set_solver(h, D.PREC_MIXED, 1e-10, 0)
        q, l = 8, 32
        Yt = rng.standard_normal((wl.ns, l - q)) / np.sqrt(l - q)
        Zt = rng.standard_normal((wl.nd, l - q)) / np.sqrt(l - q)
        t0 = time.perf_counter()
        W, V, sweeps, obj = D.dot_optimized_sampling(h, q, q, wl.ns, wl.nd, l, l, Yt, Zt)
        print(f"optimized sampling at 128^3: {time.perf_counter() - t0:.1f} s, {sweeps} sweeps, objective {obj:.3e}")
        assert np.allclose(W[:, :q].T @ W[:, :q], np.eye(q), atol=1e-10)
        assert np.allclose(V[:, :q].T @ V[:, :q], np.eye(q), atol=1e-10)
        assert np.abs(W[:, :q].T @ W[:, q:]).max() < 1e-10 and np.abs(V[:, :q].T @ V[:, q:]).max() < 1e-10
        assert 1 <= sweeps <= 100 and obj > 0
        D.dot_set_sampling(h, W, V)
        D.dot_set_solver(h, D.PREC_FP64, 1e-13, 0)
        p = torch.tensor(inp.p0, dtype=torch.float64, device="cuda", requires_grad=True)
        f = misfit(p, h, _consts(wl))
        f.backward()
        g = p.grad.cpu().numpy()
        U, Z = D.dot_get_fields(h, wl.n, wl.ls, wl.ld, False)
        # the oracle's chain on these fields
        C = orc.sparse_of_csc(wl.n, inp.C)
        CV = C @ V
        R_s = CV.T @ U - V.T @ M @ W
        assert abs(f.item() - float(np.sum(R_s ** 2))) <= 1e-10 * f.item()
        r_abs = np.abs(R_s).ravel(order="F")
        g_mu = np.empty(wl.n)
        g_scale = np.empty(wl.n)
        for v0 in range(0, wl.n, 8192):
            v1 = min(wl.n, v0 + 8192)
            J = orc.sampled_jacobian_mua(U[v0:v1], Z[v0:v1], np.eye(wl.ls), np.eye(wl.ld))
            g_mu[v0:v1] = orc.misfit_gradient(R_s, J)
            g_scale[v0:v1] = 2.0 * (np.abs(J).T @ r_abs)
        del U, Z
        dmu = orc.pals_dmu_dp(inp.p0, X, **kw)
        g_ref = dmu.T @ g_mu
        assert np.linalg.norm(g - g_ref) <= 1e-10 * np.linalg.norm(g_ref)
        assert np.all(np.abs(g - g_ref) <= 1e-10 * (abs(dmu).T @ g_scale))
        # central difference with step 1e-6 along the gradient direction
        d = g / np.linalg.norm(g)
        eps = 1e-6
        dd = torch.tensor(d, device="cuda")
        fp = misfit(p.detach() + eps * dd, h, _consts(wl)).item()
        fm = misfit(p.detach() - eps * dd, h, _consts(wl)).item()
        fd = (fp - fm) / (2 * eps)
        gd = float(g @ d)
        assert abs(fd - gd) <= 1e-3 * abs(gd), (fd, gd)
    finally:
        D.dot_destroy(h)


def test_gradient_dev_equals_host_outputs():
    wl = synth.small_workload(16, 16, 9, 0.3, src_grid=(4, 4), det_grid=(4, 4), ls=16, ld=16, m0=4,
                              sampling="gaussian", seed_index=66)
    pb = problem.build(wl)
    h = D.dot_create(0)
    try:
        configure(h, pb, p=pb.inp.p0, prec=D.PREC_MIXED, rtol=1e-12)
        f, g, _ = D.dot_gradient(h, wl.np_)
        f_d = torch.empty(1, dtype=torch.float64, device="cuda")
        g_d = torch.empty(wl.np_, dtype=torch.float64, device="cuda")
        assert D.dot_gradient_dev(h, f_d.data_ptr(), g_d.data_ptr()) == D.DOT_OK
        assert f_d.item() == f and np.array_equal(g_d.cpu().numpy(), g)
        with pytest.raises(D.DotError) as e:
            D.dot_gradient_dev(h, 0, g_d.data_ptr())
        assert e.value.code == D.DOT_EINVAL
    finally:
        D.dot_destroy(h)
