"""Test helper: a complete DOT problem (inputs plus oracle data) for a workload.

Inputs come from the seeded generator; the true absorption (which sets D) and the
measured data M come from the oracle's FP64 forward model, never from the CUDA path.
"""
import dataclasses

import numpy as np

from oracle import dot_oracle as orc
from paper_1706_05586_gb300 import synth


@dataclasses.dataclass
class Problem:
    wl: synth.Workload
    inp: synth.Inputs
    X: np.ndarray        # cell centres (N, 3)
    mu_true: np.ndarray
    D: np.ndarray
    Bd: np.ndarray       # dense B (N, ns)
    Cd: np.ndarray       # dense C (N, nd)
    M: np.ndarray        # data (nd, ns), real or complex

    @property
    def grid(self):
        return (self.wl.nx, self.wl.ny, self.wl.nz, self.wl.h)

    def pals(self):
        wl = self.wl
        return dict(mu_in=synth.MU_IN, mu_out=synth.MU_OUT, c=wl.cutoff, eps=wl.eps, gamma=wl.gamma)

    def mu_of(self, p):
        k = self.pals()
        return orc.pals_mu(p, self.X, k["mu_in"], k["mu_out"], k["c"], k["eps"], k["gamma"])

    def dmu_of(self, p):
        k = self.pals()
        return orc.pals_dmu_dp(p, self.X, k["mu_in"], k["mu_out"], k["c"], k["eps"], k["gamma"])

    def A_of(self, mu):
        return orc.assemble(self.D, mu, *self.grid, self.wl.bc, self.wl.omega_nu)

    def evaluate(self, p, with_p=True):
        mu = self.mu_of(p)
        return orc.evaluate(self.D, mu, self.grid, self.wl.bc, self.wl.omega_nu, self.Bd, self.Cd,
                            self.M, self.inp.W, self.inp.V, dmu=self.dmu_of(p) if with_p else None)


def build(wl: synth.Workload) -> Problem:
    inp = synth.draw(wl)
    X = orc.cell_centres(wl.nx, wl.ny, wl.nz, wl.h)
    mu_true = orc.pals_mu(inp.p_true, X, synth.MU_IN, synth.MU_OUT, wl.cutoff, wl.eps, wl.gamma)
    D = synth.diffusion_from_mua(mu_true)
    Bd = orc.dense_of_csc(wl.n, inp.B)
    Cd = orc.dense_of_csc(wl.n, inp.C)
    A = orc.assemble(D, mu_true, wl.nx, wl.ny, wl.nz, wl.h, wl.bc, wl.omega_nu)
    M = synth.add_noise(Cd.T @ orc.solve(A, Bd), inp)
    return Problem(wl, inp, X, mu_true, D, Bd, Cd, M)
