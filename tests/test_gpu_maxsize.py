"""The largest grid the batch workload uses (256 x 256 x 128 = 8,388,608 cells,
omega = 2 pi 100 MHz), through the same mixed-precision block solve, with 8 + 8
columns (block width 16: the TMA stencil with 16-column tiles).  The oracle cannot
solve this size, so the checks are mu on 20,000 sampled cells against the oracle's
PaLS, and properties that hold at any size: the FP64 true residual ||R - A X|| / ||R||
of every forward and adjoint column with A assembled by the oracle from that mu, and
the misfit recomputed from the returned fields and the data
(S = (CV)^T U, R_s = S - V^T M W, f = ||R_s||^2)."""
import dataclasses

import numpy as np
import pytest

from oracle import dot_oracle as orc
from paper_1706_05586_gb300 import dot as D
from paper_1706_05586_gb300 import synth

pytestmark = pytest.mark.gpu

WL = dataclasses.replace(synth.BATCH8[7], name="max256x256x128_l8", ls=8, ld=8, m0=27, seed_index=71)
RTOL = 1e-8


@pytest.fixture(scope="module")
def setup():
    inp = synth.draw(WL)
    kw = dict(mu_in=synth.MU_IN, mu_out=synth.MU_OUT, c=WL.cutoff, eps=WL.eps, gamma=WL.gamma)
    pals = (synth.MU_IN, synth.MU_OUT, WL.cutoff, WL.eps, WL.gamma)
    rng = np.random.default_rng(5)
    M = (rng.standard_normal((WL.nd, WL.ns)) + 1j * rng.standard_normal((WL.nd, WL.ns))) * 1e-7
    h = D.dot_create(0)
    D.dot_set_grid(h, WL.nx, WL.ny, WL.nz, WL.h, WL.bc)
    D.dot_set_omega(h, WL.omega_nu)
    D.dot_set_diffusion(h, np.full(WL.n, 1.0 / 30.0))
    # the oracle's PaLS at every cell takes minutes at this size: D comes from the
    # library's mu at p_true, and mu at p0 is checked against the oracle on sampled cells
    D.dot_set_pals(h, inp.p_true, *pals)
    Dfield = synth.diffusion_from_mua(D.dot_get_mua(h, WL.n))
    D.dot_set_diffusion(h, Dfield)
    D.dot_set_pals(h, inp.p0, *pals)
    mu0 = D.dot_get_mua(h, WL.n)
    cells = rng.choice(WL.n, 20000, replace=False)
    Xs = orc.cell_centres(WL.nx, WL.ny, WL.nz, WL.h)[cells]
    mu_err = np.max(np.abs(mu0[cells] - orc.pals_mu(inp.p0, Xs, **kw)))
    D.dot_set_sources(h, inp.B)
    D.dot_set_detectors(h, inp.C)
    D.dot_set_data(h, M)
    D.dot_set_sampling(h, inp.W, inp.V)
    D.dot_set_solver(h, D.PREC_MIXED, RTOL, 0)
    f, rc = D.dot_misfit(h)
    assert rc == D.DOT_OK
    st = D.dot_get_stats(h)
    U, Z = D.dot_get_fields(h, WL.n, WL.ls, WL.ld, True)
    yield dict(h=h, inp=inp, Dfield=Dfield, mu0=mu0, mu_err=mu_err, M=M, f=f, st=st, U=U, Z=Z)
    D.dot_destroy(h)


def test_absorption_on_sampled_cells(setup):
    assert setup["mu_err"] <= 1e-12


def test_launch_configuration(setup):
    st = setup["st"]
    assert st["tuned_tma"] == 1 and st["fused_direction"] == 1 and st["k"] == 16
    assert st["relres_max"] <= RTOL


def test_true_residual_every_column(setup):
    inp = setup["inp"]
    A = orc.assemble(setup["Dfield"], setup["mu0"], WL.nx, WL.ny, WL.nz, WL.h, WL.bc, WL.omega_nu)
    B = orc.sparse_of_csc(WL.n, inp.B)
    C = orc.sparse_of_csc(WL.n, inp.C)
    for X, R in ((setup["U"], B @ inp.W), (setup["Z"], C @ inp.V)):
        res = np.linalg.norm(R - A @ X, axis=0) / np.linalg.norm(R, axis=0)
        assert np.all(res <= 1.5 * RTOL), res.max()


def test_misfit_consistent_with_fields(setup):
    inp = setup["inp"]
    C = orc.sparse_of_csc(WL.n, inp.C)
    S = (C @ inp.V).T @ setup["U"]
    Rs = S - inp.V.T @ setup["M"] @ inp.W
    f = float(np.sum(np.abs(Rs) ** 2))
    assert abs(setup["f"] - f) <= 1e-10 * max(f, 2.0 * np.linalg.norm(Rs) * np.linalg.norm(S))
