"""The fused direction + stencil kernel when whole column tiles have stopped.

A CTA of the fused kernel skips a work item whose column tile has no active column and
loads the first planes of its next item while the current one ends, but only when that
item has an active column.  With three column tiles and more items than CTAs, a CTA's
consecutive items cycle through the tiles, so it meets every sequence: running ->
running (planes loaded ahead), running -> stopped (nothing loaded ahead), stopped ->
running (nothing was loaded ahead).  The first tile's sources are zero (its columns are
inactive from the start, Sec. 3.1's block of simultaneous sources with some weights
zero); the solve must match the direct-load path to rounding and leave those columns
exactly zero."""
import numpy as np
import pytest

from paper_1706_05586_gb300 import dot as D
from paper_1706_05586_gb300 import synth
from tests.gpu_setup import rel

pytestmark = pytest.mark.gpu


def _setup(ctx, wl, inp, W):
    D.dot_set_grid(ctx, wl.nx, wl.ny, wl.nz, wl.h, wl.bc)
    D.dot_set_omega(ctx, wl.omega_nu)
    D.dot_set_diffusion(ctx, np.full(wl.n, 1.0 / 30.0))
    D.dot_set_pals(ctx, inp.p_true, synth.MU_IN, synth.MU_OUT, wl.cutoff, wl.eps, wl.gamma)
    D.dot_set_diffusion(ctx, synth.diffusion_from_mua(D.dot_get_mua(ctx, wl.n)))
    D.dot_set_pals(ctx, inp.p0, synth.MU_IN, synth.MU_OUT, wl.cutoff, wl.eps, wl.gamma)
    D.dot_set_sources(ctx, inp.B)
    D.dot_set_detectors(ctx, inp.C)
    D.dot_set_data(ctx, np.zeros((wl.nd, wl.ns)))
    D.dot_set_sampling(ctx, W, inp.V)
    D.dot_set_solver(ctx, D.PREC_MIXED, 1e-12, 0)


@pytest.mark.parametrize("cplx", [True, False], ids=["complex64_kc16", "fp32_kc32"])
def test_fused_kernel_with_a_stopped_column_tile(cplx):
    kc = 16 if cplx else 32
    ls = ld = 3 * kc // 2                       # 3 column tiles of kc
    wl = synth.small_workload(64, 64, 32, 0.1, omega_nu=0.4 if cplx else 0.0, src_grid=(4, 4), det_grid=(4, 4),
                              ls=ls, ld=ld, m0=8, sampling="gaussian", seed_index=91)
    inp = synth.draw(wl)
    W = np.array(inp.W, copy=True)
    W[:, :kc] = 0.0                             # block columns 0 .. kc-1: the first tile
    h = D.dot_create(0)
    out = {}
    try:
        _setup(h, wl, inp, W)
        for mode in (2, 0):
            D.dot_set_stencil_path(h, mode)
            f, g, rc = D.dot_gradient(h, wl.np_)
            assert rc == D.DOT_OK
            st = D.dot_get_stats(h)
            U, Z = D.dot_get_fields(h, wl.n, wl.ls, wl.ld, cplx)
            out[mode] = (f, g, U, Z, st)
    finally:
        D.dot_destroy(h)
    f2, g2, U2, Z2, st2 = out[2]
    f0, g0, U0, Z0, st0 = out[0]
    assert st2["fused_direction"] == 1 and st0["fused_direction"] == 0
    assert st2["k"] == 3 * kc
    assert st2["relres_max"] <= 1e-12 and st0["relres_max"] <= 1e-12
    # the stopped tile: zero right-hand sides give exactly zero fields on both paths
    assert not np.any(U2[:, :kc]) and not np.any(U0[:, :kc])
    assert np.all(np.linalg.norm(U2[:, kc:], axis=0) > 0)
    # the running tiles agree with the direct-load path to the solver's rounding
    assert rel(U2, U0) <= 1e-10 and rel(Z2, Z0) <= 1e-10
    assert abs(f2 - f0) <= 1e-9 * abs(f0)
    assert rel(g2, g0) <= 1e-8
    assert abs(st2["iters_max"] - st0["iters_max"]) <= 3
