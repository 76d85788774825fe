"""Test helper: configure a library context from a synthetic problem (C ABI calls only),
and the error measures the GPU parity tests assert."""
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
    """Relative error in the Frobenius (2-) norm of the whole array."""
    a, b = np.asarray(a), np.asarray(b)
    den = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0)


def col_rel(a, b):
    """Largest relative 2-norm error over the columns of 2-D arrays (an all-zero
    reference column must be matched exactly)."""
    a, b = np.atleast_2d(np.asarray(a)), np.atleast_2d(np.asarray(b))
    num = np.linalg.norm(a - b, axis=0)
    den = np.linalg.norm(b, axis=0)
    return float(np.max(np.where(den > 0, num / np.where(den > 0, den, 1.0), np.where(num > 0, np.inf, 0.0))))


def col_max_rel(a, b):
    """Largest entry error of each column over that column's largest reference entry,
    maximised over the columns: the pointwise accuracy of a solved field."""
    a, b = np.atleast_2d(np.asarray(a)), np.atleast_2d(np.asarray(b))
    num = np.max(np.abs(a - b), axis=0)
    den = np.max(np.abs(b), axis=0)
    return float(np.max(np.where(den > 0, num / np.where(den > 0, den, 1.0), np.where(num > 0, np.inf, 0.0))))


def entry_ratio(a, b, scale):
    """max over entries of |a - b| / scale (scale: the entry's first-order error size
    per unit relative field error, from oracle_scales).  An entry with scale 0 must be
    matched exactly."""
    a, b, s = np.asarray(a), np.asarray(b), np.asarray(scale, dtype=np.float64)
    d = np.abs(a - b)
    out = np.where(s > 0, d / np.where(s > 0, s, 1.0), np.where(d > 0, np.inf, 0.0))
    return float(np.max(out))


def oracle_scales(pb, ref, dmu=None):
    """First-order error size of every output entry per unit pointwise field error.

    Premise (checked separately with col_max_rel): each solved column u of U = A^{-1} B W
    and Z = A^{-T} C V is accurate to tau * max|u| at every cell.  Propagating that
    through the definitions (Sec. 3.3, Eq. (EsTResidual), Eq. (Jacobian kth column),
    Eq. (UnbiasedGrad)) bounds each entry's error by tau times:
      S[l, i] = (C v_l)^T U_i             ->  ||C v_l||_1 max|U_i|
      J_mu[(l, i), v] = -Z_l[v] U_i[v]     ->  max|Z_l| |U_i[v]| + |Z_l[v]| max|U_i|
      J_p = J_mu dmu/dp                    ->  E_Jmu |dmu/dp|
      g = 2 Re J^T conj(vec R_s)           ->  2 sum_r (E_J[r] |R_s[r]| + |J[r]| E_S[r])
      f = ||R_s||^2                        ->  2 sum_r |R_s[r]| E_S[r]
    Rows r = l + l_d i (column-major vec of the l_d x l_s matrices)."""
    W, V = pb.inp.W, pb.inp.V
    U = ref["Uf"] @ W
    Z = ref["Zf"] @ V
    CV = pb.Cd @ V
    mU = np.max(np.abs(U), axis=0)
    mZ = np.max(np.abs(Z), axis=0)
    aU, aZ = np.abs(U), np.abs(Z)
    ls, ld = W.shape[1], V.shape[1]
    E_S = np.outer(np.sum(np.abs(CV), axis=0), mU)            # (ld, ls)
    E_Jmu = np.empty((ls * ld, U.shape[0]))
    for i in range(ls):
        for l in range(ld):
            E_Jmu[l + ld * i] = mZ[l] * aU[:, i] + aZ[:, l] * mU[i]
    Rs = np.abs(np.asarray(ref["R_s"])).ravel(order="F")
    eS = E_S.ravel(order="F")
    out = {"U": U, "Z": Z, "S": E_S, "J_mu": E_Jmu,
           "g_mu": 2.0 * (E_Jmu.T @ Rs + np.abs(ref["J_mu"]).T @ eS),
           "f": 2.0 * float(Rs @ eS)}
    if dmu is not None:
        adm = abs(dmu.tocsc()) if hasattr(dmu, "tocsc") else np.abs(dmu)
        E_Jp = np.asarray((adm.T @ E_Jmu.T).T)
        out["J_p"] = E_Jp
        out["g_p"] = 2.0 * (E_Jp.T @ Rs + np.abs(ref["J_p"]).T @ eS)
    return out


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
