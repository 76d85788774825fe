"""Test helper: configure a library context from a synthetic problem (C ABI calls only)."""
import numpy as np

from paper_1706_05586_gb300 import dot as D
from paper_1706_05586_gb300 import synth


def configure(ctx, pb, *, p=None, mua=None, prec=D.PREC_FP64, rtol=1e-13, maxit=0, W=None, V=None,
              data=True):
    wl = pb.wl
    D.dot_set_grid(ctx, wl.nx, wl.ny, wl.nz, wl.h, wl.bc)
    D.dot_set_omega(ctx, wl.omega_nu)
    D.dot_set_diffusion(ctx, pb.D)
    if mua is not None:
        D.dot_set_mua(ctx, mua)
    else:
        D.dot_set_pals(ctx, pb.inp.p0 if p is None else p, synth.MU_IN, synth.MU_OUT, wl.cutoff, wl.eps,
                       wl.gamma)
    D.dot_set_sources(ctx, pb.inp.B)
    D.dot_set_detectors(ctx, pb.inp.C)
    if data:
        D.dot_set_data(ctx, pb.M)
    D.dot_set_sampling(ctx, pb.inp.W if W is None else W, pb.inp.V if V is None else V)
    D.dot_set_solver(ctx, prec, rtol, maxit)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    den = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0)


def grad_err(g, ref_g, J, R_s, S):
    """Gradient error over 2 ||J|| (||R_s|| + ||S||): the first-order size of the change of
    g = 2 Re J^T conj(R_s) under relative perturbations of J and of S (R_s = S - V^T M W, so
    near the data R_s is a difference of nearly equal terms and its own relative error is
    amplified by ||S|| / ||R_s||)."""
    scale = 2.0 * np.linalg.norm(J) * (np.linalg.norm(R_s) + np.linalg.norm(S))
    return float(np.linalg.norm(np.asarray(g) - np.asarray(ref_g)) / scale)


def misfit_err(f, ref):
    """Misfit error over max(f, 2 ||R_s|| ||S||): f = ||R_s||^2 with R_s = S - V^T M W moves by
    at most 2 ||R_s|| ||dS|| under a perturbation dS, so near the data (R_s ~ 1% of S) the
    relative error of f is the relative error of S amplified by ||S|| / ||R_s||."""
    scale = max(ref["f"], 2.0 * np.linalg.norm(ref["R_s"]) * np.linalg.norm(ref["S"]))
    return abs(f - ref["f"]) / scale
