"""Plain FP64 CPU oracle for the randomized DOT hot path.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg may import this module.  It shares no code with the
CUDA path and imports nothing from the package: its inputs are plain numpy
arrays (the seeded generator lives in a module of its own).

What it computes (Aslan, de Sturler, Kilmer, "Randomized approach to nonlinear
inversion combining random and optimized simultaneous sources and detectors"):

  * the frequency-domain diffusion operator A(mu) + i(omega/nu) E of Sec. 2,
    Eq. (PDE) and Eq. (Eq:compmeas), assembled as a sparse matrix by a
    cell-centred finite-volume discretization (readings below);
  * the PaLS absorption mu(x; p) of Sec. 2, Eq. (absorption const), with the
    Wendland CSRBF psi_{2,1} and the regularized norm ||x||^dagger;
  * the residual matrix R = C^T A^{-1} B - M of Eq. (MartixR), by solving every
    physical source and detector column explicitly;
  * the sampled misfit ||V^T R W||_F^2 (Theorem 1, Eq. (EsTResidual));
  * the Jacobian tensor J_ijk = -c_i^T A^{-1} dA/dp_k A^{-1} b_j of
    Eq. (Jacobiancomp) / Eq. (Jtensor), its sampled form (W^T (x) V^T) J of
    Eq. (TREGS J) / Eq. (Jacobian kth column), and the gradient
    2 Re J^T conj(r) of the misfit (Eq. (UnbiasedGrad) at W = I, V = I).

Readings where the paper is silent (the same ones the CUDA path implements):
  * cell-centred grid, so the frequency mass E is the identity;
  * interior faces use the harmonic mean D_f = 2 D_a D_b / (D_a + D_b), coupling
    D_f / h^2 per unit volume;
  * a Robin face (0.25 eta + (D/2) d eta/d xi = 0, i.e. eta + 2 D d eta/dn = 0)
    eliminates the boundary value from the cell centre and adds
    2 D_c / (h (h + 4 D_c)) to the diagonal; a Dirichlet face adds 2 D_c / h^2;
  * D is a known, fixed field (Sec. 2 assumes D known), so dA/dmu_v = e_v e_v^T;
  * smoothed Heaviside H_eps(t) = 1/2 (1 + t/eps + sin(pi t/eps)/pi) on |t| <= eps,
    0 below and 1 above; delta_eps = H_eps' = (1 + cos(pi t/eps)) / (2 eps);
  * misfit with no factor 1/2 (Sec. 4 drops it); complex data enter through
    sum |R|^2, i.e. the real/imaginary split of the Eq. (Eq:compmeas) footnote;
  * the sampled Jacobian row index is l + l_d * i (vec order of V^T R W).

Parity pins: every function here is checked by tests/test_oracle_*.py against
closed forms, brute force, invariants and finite differences (see those tests).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

ROBIN = 0
DIRICHLET = 1

# Direct sparse LU below this many unknowns, Jacobi CG / COCG above.
DIRECT_MAX = 200_000


# --------------------------------------------------------------------------- grid

def cell_centres(nx, ny, nz, h):
    """Cell centres ((i+1/2)h, (j+1/2)h, (k+1/2)h), voxel order v = i + nx (j + ny k)."""
    xs = (np.arange(nx) + 0.5) * h
    ys = (np.arange(ny) + 0.5) * h
    zs = (np.arange(nz) + 0.5) * h
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


# ---------------------------------------------------------------- operator (Sec. 2)

def assemble(D, mu, nx, ny, nz, h, bc, omega_nu=0.0):
    """Sparse A(mu) + i (omega/nu) I of Eq. (Eq:compmeas), per unit volume.

    -div(D grad eta) + mu eta + i(omega/nu) eta, Eq. (PDE), discretized with the
    readings in the module header.  bc: six flags (-x, +x, -y, +y, -z, +z).
    Returns CSR, float64 when omega_nu == 0 else complex128.
    """
    N = nx * ny * nz
    D3 = np.asarray(D, dtype=np.float64).reshape(nz, ny, nx)
    idx = np.arange(N).reshape(nz, ny, nx)
    dtype = np.complex128 if omega_nu != 0.0 else np.float64
    diag = np.asarray(mu, dtype=np.float64).reshape(nz, ny, nx).astype(dtype)
    if omega_nu != 0.0:
        diag = diag + 1j * omega_nu
    rows, cols, vals = [], [], []
    # axis 2 = x, 1 = y, 0 = z in the (z, y, x) array; faces (-x,+x) (-y,+y) (-z,+z)
    for axis, (f_lo, f_hi) in ((2, (0, 1)), (1, (2, 3)), (0, (4, 5))):
        n_ax = D3.shape[axis]
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[axis] = slice(0, n_ax - 1)
        hi[axis] = slice(1, n_ax)
        lo, hi = tuple(lo), tuple(hi)
        Da, Db = D3[lo], D3[hi]
        coef = (2.0 * Da * Db / (Da + Db)) / h ** 2
        rows += [idx[lo].ravel(), idx[hi].ravel()]
        cols += [idx[hi].ravel(), idx[lo].ravel()]
        vals += [-coef.ravel(), -coef.ravel()]
        diag[lo] += coef
        diag[hi] += coef
        for face, layer in ((f_lo, 0), (f_hi, n_ax - 1)):
            sl = [slice(None)] * 3
            sl[axis] = slice(layer, layer + 1)
            sl = tuple(sl)
            Dc = D3[sl]
            if bc[face] == ROBIN:
                diag[sl] += 2.0 * Dc / (h * (h + 4.0 * Dc))
            elif bc[face] == DIRICHLET:
                diag[sl] += 2.0 * Dc / h ** 2
            else:
                raise ValueError(f"bad bc flag {bc[face]}")
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    A = sp.coo_matrix((np.concatenate(vals).astype(dtype),
                       (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    return A.tocsr()


# ----------------------------------------------------------------------- solves

def krylov_solve(A, b, rtol=1e-13, maxit=None):
    """Jacobi-preconditioned CG (real SPD) or COCG (complex symmetric), zero start.

    COCG is CG with the bilinear form x^T y in place of x^H y.  Stops when
    ||r||_2 <= rtol ||b||_2.  One column at a time.
    """
    b = np.asarray(b)
    dtype = np.result_type(A.dtype, b.dtype)
    n = b.shape[0]
    maxit = maxit or 20 * n
    d = A.diagonal().astype(dtype)
    x = np.zeros(n, dtype=dtype)
    r = b.astype(dtype).copy()
    bn = np.linalg.norm(r)
    if bn == 0.0:
        return x, 0
    z = r / d
    p = z.copy()
    rho = np.dot(r, z)
    for it in range(1, maxit + 1):
        q = A @ p
        alpha = rho / np.dot(p, q)
        x += alpha * p
        r -= alpha * q
        if np.linalg.norm(r) <= rtol * bn:
            return x, it
        z = r / d
        rho_new = np.dot(r, z)
        p = z + (rho_new / rho) * p
        rho = rho_new
    raise RuntimeError(f"oracle Krylov solve did not reach rtol={rtol} in {maxit} iterations")


def solve(A, RHS, rtol=1e-13):
    """X = A^{-1} RHS column by column: sparse LU when small, Jacobi CG/COCG otherwise."""
    RHS = np.asarray(RHS)
    one = RHS.ndim == 1
    R2 = RHS.reshape(RHS.shape[0], -1)
    dtype = np.result_type(A.dtype, R2.dtype)
    if A.shape[0] <= DIRECT_MAX:
        lu = spla.splu(A.astype(dtype).tocsc())
        X = lu.solve(np.ascontiguousarray(R2.astype(dtype)))
    else:
        X = np.empty(R2.shape, dtype=dtype)
        for c in range(R2.shape[1]):
            X[:, c], _ = krylov_solve(A, R2[:, c], rtol=rtol)
    return X[:, 0] if one else X


def dense_of_csc(n, csc):
    colptr, rows, vals = csc
    ncol = len(colptr) - 1
    out = np.zeros((n, ncol))
    for c in range(ncol):
        out[rows[colptr[c]:colptr[c + 1]], c] = vals[colptr[c]:colptr[c + 1]]
    return out


def sparse_of_csc(n, csc):
    colptr, rows, vals = csc
    return sp.csc_matrix((vals, rows, colptr), shape=(n, len(colptr) - 1))


# ------------------------------------------------------------------ PaLS (Sec. 2)

def wendland(r):
    """psi_{2,1}(r) = (1 - r)^4 (4 r + 1) for 0 <= r < 1, else 0 (Sec. 2 footnote)."""
    r = np.asarray(r, dtype=np.float64)
    return np.where(r < 1.0, (1.0 - r) ** 4 * (4.0 * r + 1.0), 0.0)


def wendland_prime(r):
    """d psi_{2,1} / dr = -20 r (1 - r)^3 for r < 1, else 0."""
    r = np.asarray(r, dtype=np.float64)
    return np.where(r < 1.0, -20.0 * r * (1.0 - r) ** 3, 0.0)


def heaviside(t, eps):
    """Smoothed Heaviside H_eps(t) (reading: compact C^1 sine ramp of half width eps)."""
    t = np.asarray(t, dtype=np.float64)
    mid = 0.5 * (1.0 + t / eps + np.sin(math.pi * t / eps) / math.pi)
    return np.where(t < -eps, 0.0, np.where(t > eps, 1.0, mid))


def heaviside_prime(t, eps):
    """delta_eps(t) = dH_eps/dt = (1 + cos(pi t / eps)) / (2 eps) on |t| <= eps, else 0."""
    t = np.asarray(t, dtype=np.float64)
    return np.where(np.abs(t) <= eps, (1.0 + np.cos(math.pi * t / eps)) / (2.0 * eps), 0.0)


def pals_phi(p, X, gamma):
    """phi(x, p) = sum_j alpha_j psi(||beta_j (x - chi_j)||^dagger), Sec. 2.

    ||y||^dagger = sqrt(||y||^2 + gamma^2).  p per RBF: (alpha, beta, chi_x, chi_y, chi_z).
    """
    p = np.asarray(p, dtype=np.float64)
    m0 = p.size // 5
    phi = np.zeros(X.shape[0])
    for j in range(m0):
        a, be = p[5 * j], p[5 * j + 1]
        chi = p[5 * j + 2:5 * j + 5]
        d2 = np.sum((X - chi) ** 2, axis=1)
        r = np.sqrt(be * be * d2 + gamma * gamma)
        phi += a * wendland(r)
    return phi


def pals_dphi_dp(p, X, gamma):
    """d phi / d p as a sparse (N x 5 m0) matrix, differentiating Sec. 2's phi term by term.

    d/d alpha_j = psi(r_j); d/d beta_j = alpha_j psi'(r_j) beta_j |x - chi_j|^2 / r_j;
    d/d chi_j = -alpha_j psi'(r_j) beta_j^2 (x - chi_j) / r_j.
    """
    p = np.asarray(p, dtype=np.float64)
    m0 = p.size // 5
    N = X.shape[0]
    rows, cols, vals = [], [], []
    for j in range(m0):
        a, be = p[5 * j], p[5 * j + 1]
        chi = p[5 * j + 2:5 * j + 5]
        diff = X - chi
        d2 = np.sum(diff ** 2, axis=1)
        r = np.sqrt(be * be * d2 + gamma * gamma)
        sel = np.nonzero(r < 1.0)[0]
        if sel.size == 0:
            continue
        rs, ds = r[sel], diff[sel]
        psi = wendland(rs)
        dpsi = wendland_prime(rs)
        cols_j = [psi,
                  a * dpsi * be * d2[sel] / rs,
                  -a * dpsi * be * be * ds[:, 0] / rs,
                  -a * dpsi * be * be * ds[:, 1] / rs,
                  -a * dpsi * be * be * ds[:, 2] / rs]
        for q in range(5):
            rows.append(sel)
            cols.append(np.full(sel.size, 5 * j + q))
            vals.append(cols_j[q])
    if not rows:
        return sp.csr_matrix((N, 5 * m0))
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, 5 * m0)).tocsr()


def pals_mu(p, X, mu_in, mu_out, c, eps, gamma):
    """mu(x, p) = mu_in H_eps(phi - c) + mu_out (1 - H_eps(phi - c)), Eq. (absorption const)."""
    H = heaviside(pals_phi(p, X, gamma) - c, eps)
    return mu_in * H + mu_out * (1.0 - H)


def pals_dmu_dp(p, X, mu_in, mu_out, c, eps, gamma):
    """d mu / d p = (mu_in - mu_out) delta_eps(phi - c) d phi / d p (chain rule of Eq. (absorption const))."""
    phi = pals_phi(p, X, gamma)
    w = (mu_in - mu_out) * heaviside_prime(phi - c, eps)
    return sp.diags(w) @ pals_dphi_dp(p, X, gamma)


# -------------------------------------------------------- residual and misfit (Sec. 3)

def fields_full(A, B, C):
    """All physical forward fields A^{-1} B and adjoint fields A^{-T} C (n_s + n_d solves)."""
    Uf = solve(A, B)
    Zf = solve(A.T.tocsr(), C)
    return Uf, Zf


def residual_matrix(A, B, C, M):
    """R = C^T A^{-1} B - M, Eq. (MartixR); M is the data matrix (called D in the paper)."""
    return C.T @ solve(A, B) - M


def sampled_residual(R, W, V):
    """V^T R W, the sampled residual whose vec is (W^T (x) V^T) r, Eq. (EsTResidual)."""
    return V.T @ R @ W


def sampled_misfit(R, W, V):
    """||V^T R W||_F^2 (Theorem 1); the sum of |.|^2 over real and imaginary parts."""
    S = sampled_residual(R, W, V)
    return float(np.sum(np.abs(S) ** 2))


# ---------------------------------------------------------------- Jacobians (Sec. 2, 3.3)

def jacobian_tensor(Uf, Zf, dmu):
    """J_ijk = -c_i^T A^{-1} (dA/dp_k) A^{-1} b_j, Eq. (Jacobiancomp) / Eq. (Jtensor).

    With D known, dA/dp_k = diag(dmu/dp_k), so J_ijk = -sum_v Zf[v, i] dmu[v, k] Uf[v, j]
    where Zf = A^{-T} C.  dmu: (N x n_p) sparse or dense.  Returns (n_d, n_s, n_p).
    """
    nd, ns = Zf.shape[1], Uf.shape[1]
    dmu = sp.csr_matrix(dmu)
    npar = dmu.shape[1]
    dt = np.result_type(Uf.dtype, Zf.dtype)
    J = np.zeros((nd, ns, npar), dtype=dt)
    for j in range(ns):
        # rows i, cols k: -(Zf * Uf[:, j])^T dmu
        J[:, j, :] = -(dmu.T @ (Zf * Uf[:, j:j + 1])).T
    return J


def sampled_jacobian(J3, W, V):
    """(W^T (x) V^T) J with rows ordered l + l_d i, Eq. (TREGS J) and Eq. (Jacobian kth column)."""
    nd, ns, npar = J3.shape
    ls, ld = W.shape[1], V.shape[1]
    out = np.zeros((ld * ls, npar), dtype=J3.dtype)
    for i in range(ls):
        for l in range(ld):
            out[l + ld * i, :] = np.einsum("d,s,dsk->k", V[:, l], W[:, i], J3)
    return out


def sampled_jacobian_mua(Uf, Zf, W, V):
    """Sampled mu-Jacobian rows -(A^{-T} C V)_l (.) (A^{-1} B W)_i over all voxels.

    Eq. (Jacobian kth column) with dA/dmu_v = e_v e_v^T and the sign of Eq. (Jacobiancomp);
    row l + l_d i.  Returns (l_s l_d, N).
    """
    U = Uf @ W
    Z = Zf @ V
    ls, ld = W.shape[1], V.shape[1]
    out = np.zeros((ld * ls, Uf.shape[0]), dtype=np.result_type(U.dtype, Z.dtype))
    for i in range(ls):
        for l in range(ld):
            out[l + ld * i, :] = -Z[:, l] * U[:, i]
    return out


def misfit_gradient(S_res, Js):
    """d/dp ||S_res||^2 = 2 Re( J_s^T conj(vec S_res) ), vec in column-major order."""
    r = np.asarray(S_res).reshape(-1, order="F")
    return 2.0 * np.real(Js.T @ np.conj(r))


# ------------------------------------------------------------ one whole evaluation

def evaluate(D, mu, grid, bc, omega_nu, B, C, M, W, V, dmu=None):
    """The hot path's outputs for fixed W, V, computed the plain way.

    grid = (nx, ny, nz, h); B, C dense (N x n_s), (N x n_d); M (n_d x n_s).
    Returns dict with S = V^T C^T A^{-1} B W, R_s = V^T R W, f, J_mu, g_mu and,
    when dmu (N x n_p) is given, J_p and g_p.
    """
    nx, ny, nz, h = grid
    A = assemble(D, mu, nx, ny, nz, h, bc, omega_nu)
    Uf, Zf = fields_full(A, B, C)
    meas = C.T @ Uf
    R = meas - M
    out = {"S": V.T @ meas @ W, "R_s": sampled_residual(R, W, V)}
    out["f"] = float(np.sum(np.abs(out["R_s"]) ** 2))
    Jmu = sampled_jacobian_mua(Uf, Zf, W, V)
    out["J_mu"] = Jmu
    out["g_mu"] = misfit_gradient(out["R_s"], Jmu)
    if dmu is not None:
        J3 = jacobian_tensor(Uf, Zf, dmu)
        Jp = sampled_jacobian(J3, W, V)
        out["J_p"] = Jp
        out["g_p"] = misfit_gradient(out["R_s"], Jp)
    out["Uf"], out["Zf"] = Uf, Zf
    return out


# --------------------------------------------- optimized sources and detectors (Sec. 3.2)

def _real_stack(J3):
    """A complex tensor enters ||(W^T (x) V^T) J||_F with real W, V through its real and
    imaginary parts, which act as separate parameter columns."""
    J3 = np.asarray(J3)
    if np.iscomplexobj(J3):
        return np.concatenate([J3.real, J3.imag], axis=2)
    return J3


def _leading_left(Mat, q):
    """The q leading left singular vectors of a real matrix (numpy SVD)."""
    U, _, _ = np.linalg.svd(Mat, full_matrices=False)
    return U[:, :q]


def unfold_lateral(J3):
    """J~ = [J_{:,1,:} J_{:,2,:} ... J_{:,n_s,:}] (n_d x n_s n_p), Eq. (Jtilde)."""
    nd, ns, npar = J3.shape
    return np.concatenate([J3[:, j, :] for j in range(ns)], axis=1)


def contract_detectors(J3, Vt):
    """K~ = [K_1 ... K_qd] with (K_l)_{jk} = sum_m (v_l)_m J_{mjk} (n_s x n_p q_d), Eq. (Ktilde)."""
    return np.concatenate([np.einsum("m,mjk->jk", Vt[:, l], J3) for l in range(Vt.shape[1])], axis=1)


def contract_sources(J3, Wt):
    """L~ = [L_1 ... L_qs] with (L_l)_{ik} = sum_m (w_l)_m J_{imk} (n_d x n_p q_s), Eq. (Ltilde)."""
    return np.concatenate([np.einsum("m,imk->ik", Wt[:, l], J3) for l in range(Wt.shape[1])], axis=1)


def optimized_sources_detectors(J3, qs, qd, maxit=100, tol=1e-10):
    """Algorithm 1 (Sec. 3.3): Tucker2 alternating iteration for isometric W^, V^ maximizing
    ||(W^T (x) V^T) J||_F^2 (Eq. (maxprob)).

    Start from the q_d leading left singular vectors of J~; then alternate W~ from K~ and
    V~ from L~ until the change of the projectors W~W~^T, V~V~^T is below tol (reading:
    the paper leaves the test open) or maxit sweeps.  Returns (W^, V^, sweeps).
    """
    J = _real_stack(J3)
    Vt = _leading_left(unfold_lateral(J), qd)
    Wt = None
    for it in range(1, maxit + 1):
        W_new = _leading_left(contract_detectors(J, Vt), qs)
        V_new = _leading_left(contract_sources(J, W_new), qd)
        change = np.linalg.norm(V_new @ V_new.T - Vt @ Vt.T)
        if Wt is not None:
            change += np.linalg.norm(W_new @ W_new.T - Wt @ Wt.T)
        Wt, Vt = W_new, V_new
        if it > 1 and change < tol:
            return Wt, Vt, it
    return Wt, Vt, maxit


def sampled_jacobian_norm2(J3, W, V):
    """||(W^T (x) V^T) J||_F^2 (Eq. (maxprob)), complex entries counted as |.|^2."""
    out = np.einsum("ml,jq,mjk->lqk", V, W, np.asarray(J3))
    return float(np.sum(np.abs(out) ** 2))


def complement_sampling(What, Ytil):
    """W = [W^, W_c Y] of Eq. (newW) with W_c Y read as (I - W^ W^T) Y~: Y~ has n rows and
    i.i.d. zero-mean, covariance-(ell - q)^{-1} entries, so W_c Y has covariance I - W^W^T
    for any orthonormal basis W_c of the complement (Theorem 2 needs only that)."""
    P = np.eye(What.shape[0]) - What @ What.T
    return np.concatenate([What, P @ Ytil], axis=1)
