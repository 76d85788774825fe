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
