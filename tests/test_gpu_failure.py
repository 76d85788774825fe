"""Failure detection on the device without a fault: every device-side wait of the
library is bounded by a clock budget, after which the kernel gives up, records an
error word and returns, so that the host reports DOT_ETIMEOUT and the context stays
usable.  dot_probe_wait makes such a wait run out on purpose (an mbarrier that
nothing arrives at, no copy in flight) and the context then solves as before."""
import time

import numpy as np
import pytest

from paper_1706_05586_gb300 import dot as D
from paper_1706_05586_gb300 import synth
from tests import problem
from tests.gpu_setup import configure, misfit_err

pytestmark = pytest.mark.gpu

WL = synth.small_workload(16, 16, 9, 0.3, src_grid=(4, 4), det_grid=(4, 4), ls=16, ld=16, m0=4, sampling="gaussian",
                          seed_index=73)


def test_bounded_wait_gives_up_and_context_survives():
    pb = problem.build(WL)
    ref = pb.evaluate(pb.inp.p0)
    h = D.dot_create(0)
    try:
        configure(h, pb, p=pb.inp.p0, prec=D.PREC_MIXED, rtol=1e-13)
        f0, _ = D.dot_misfit(h)
        for budget in (0, 2_000_000):  # no wait at all, then about 1 ms
            t0 = time.perf_counter()
            assert D.dot_probe_wait(h, budget) == D.DOT_ETIMEOUT
            assert time.perf_counter() - t0 < 5.0
        # the same context still evaluates, through the TMA stencil's bounded waits
        D.dot_set_pals(h, pb.inp.p0 * (1.0 + 1e-12), synth.MU_IN, synth.MU_OUT, WL.cutoff, WL.eps, WL.gamma)
        f1, rc = D.dot_misfit(h)
        assert rc == D.DOT_OK
        assert D.dot_get_stats(h)["tuned_tma"] == 1
        assert misfit_err(f0, ref) <= 1e-8 and abs(f1 - f0) <= 1e-6 * abs(f0)
    finally:
        D.dot_destroy(h)


def test_probe_rejects_bad_budget():
    h = D.dot_create(0)
    try:
        with pytest.raises(D.DotError) as e:
            D.dot_probe_wait(h, -1)
        assert e.value.code == D.DOT_EINVAL
    finally:
        D.dot_destroy(h)


@pytest.mark.parametrize("prec", [D.PREC_FP64, D.PREC_MIXED])
def test_breakdown_is_reported_and_outputs_written(prec):
    """A zero Jacobi diagonal breaks CG down at its first step (z = M^{-1} r is not finite):
    a single cell with six Dirichlet faces, D = 1/2 and h = 1 gives each face exactly
    2 D / h^2 = 1, so mu = -6 makes the diagonal exactly zero.  The solve stops the
    column with DOT_EBREAKDOWN, the misfit is still written, and the same context then
    evaluates a well-posed problem as before."""
    h = D.dot_create(0)
    try:
        D.dot_set_grid(h, 1, 1, 1, 1.0, (synth.DIRICHLET,) * 6)
        D.dot_set_omega(h, 0.0)
        D.dot_set_diffusion(h, np.array([0.5]))
        D.dot_set_mua(h, np.array([-6.0]))
        one = (np.array([0, 1], dtype=np.int64), np.array([0], dtype=np.int32), np.array([1.0]))
        D.dot_set_sources(h, one)
        D.dot_set_detectors(h, one)
        D.dot_set_data(h, np.array([[0.25]]))
        D.dot_set_sampling(h, np.ones((1, 1)), np.ones((1, 1)))
        D.dot_set_solver(h, prec, 1e-10, 0)
        f, rc = D.dot_misfit(h, allow=(D.DOT_EBREAKDOWN,))
        assert rc == D.DOT_EBREAKDOWN
        assert f == pytest.approx(0.0625)          # S = C^T U = 0 with U = 0, R_s = -0.25
        st = D.dot_get_stats(h)
        assert st["status"] == D.DOT_EBREAKDOWN and st["iters_max"] == 0
        # a positive diagonal: A = [1] (mu = -5), so U = 1, S = 1, f = (1 - 0.25)^2
        D.dot_set_mua(h, np.array([-5.0]))
        f, rc = D.dot_misfit(h)
        assert rc == D.DOT_OK and f == pytest.approx(0.5625, rel=1e-12)
    finally:
        D.dot_destroy(h)


def test_allocation_failure_is_reported_and_context_survives():
    """Block vectors that cannot fit: 256 x 256 x 512 cells x 1,024 complex columns need
    550 GB for the right-hand sides alone, more than the device holds.  The evaluation
    fails at that allocation with DOT_ENOMEM before any solve, and the same context then
    evaluates a small problem against the oracle."""
    nx, ny, nz = 256, 256, 512
    n = nx * ny * nz
    big = synth.small_workload(nx, ny, nz, 8.0 / nx, omega_nu=synth.OMEGA_NU_100MHZ, src_grid=(4, 4),
                               det_grid=(4, 4), ls=512, ld=512, m0=1, sampling="gaussian", seed_index=75)
    inp = synth.draw(big)
    h = D.dot_create(0)
    try:
        D.dot_set_grid(h, nx, ny, nz, big.h, big.bc)
        D.dot_set_omega(h, big.omega_nu)
        D.dot_set_diffusion(h, np.full(n, 1.0 / 30.0))
        D.dot_set_mua(h, np.full(n, synth.MU_OUT))
        D.dot_set_sources(h, inp.B)
        D.dot_set_detectors(h, inp.C)
        D.dot_set_data(h, np.zeros((big.nd, big.ns), dtype=complex))
        D.dot_set_sampling(h, inp.W, inp.V)
        D.dot_set_solver(h, D.PREC_MIXED, 1e-10, 0)
        with pytest.raises(D.DotError) as e:
            D.dot_misfit(h)
        assert e.value.code == D.DOT_ENOMEM
        assert "cudaMalloc" in D.dot_last_error()
        assert D.dot_get_stats(h)["block_solves"] == 0
        # the same context, now sized for a small problem
        pb = problem.build(synth.small_workload(11, 6, 7, 0.35, omega_nu=0.3, src_grid=(3, 1), det_grid=(2, 2),
                                                ls=3, ld=2, m0=5, sampling="gaussian", seed_index=62))
        ref = pb.evaluate(pb.inp.p0)
        configure(h, pb, p=pb.inp.p0, prec=D.PREC_FP64, rtol=2e-15)
        f, rc = D.dot_misfit(h)
        assert rc == D.DOT_OK and abs(f - ref["f"]) <= 1e-10 * ref["f"]
    finally:
        D.dot_destroy(h)
