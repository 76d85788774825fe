"""Seeded synthetic inputs for the randomized DOT hot path.

This module draws and lays out inputs only: grid geometry, the Gaussian source and
detector columns B and C, PaLS parameter vectors, the sampling matrices W and V,
and the noise draws used to perturb computed data.  It holds none of the method's
arithmetic (no discretized operator, no PaLS evaluation, no solve), so the same
inputs can be fed both to the CUDA path and to the independent FP64 oracle.

Conventions (the paper leaves them open; Sec. 2 only says "finite difference
discretization" and puts sources on the top and detectors on the bottom):
  * cell-centred grid of nx*ny*nz cells of size h, cell (i, j, k) centred at
    ((i+1/2)h, (j+1/2)h, (k+1/2)h); voxel index v = i + nx*(j + ny*k);
    the face z = 0 is the top (sources), z = nz*h the bottom (detectors);
  * boundary flags per face in the order -x, +x, -y, +y, -z (top), +z (bottom),
    ROBIN = 0, DIRICHLET = 1;
  * PaLS parameters per RBF in the order (alpha, beta, chi_x, chi_y, chi_z), five per
    RBF as in the 3D experiment of Sec. 4;
  * W = l_s^{-1/2} [w_1 ... w_ls] and V = l_d^{-1/2} [v_1 ... v_ld] as in
    Eqs. (defW), (defV), with Rademacher or Gaussian entries;
  * sparse B, C are CSC (int64 colptr, int32 rows, float64 values).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

ROBIN = 0
DIRICHLET = 1

# mu_s' = 10 / cm, background mu_a = 0.05 / cm, anomaly mu_a = 0.2 / cm.
MUS_PRIME = 10.0
MU_OUT = 0.05
MU_IN = 0.2
# omega / nu for a 100 MHz modulation in tissue of refractive index 1.4 (cm^-1).
OMEGA_NU_100MHZ = 2.0 * math.pi * 1.0e8 / (2.99792458e10 / 1.4)

SEED_BASE = 1706055860


@dataclasses.dataclass(frozen=True)
class Workload:
    """Shape of one synthetic DOT problem (all lengths in cm)."""
    name: str
    nx: int
    ny: int
    nz: int
    h: float
    omega_nu: float
    src_grid: tuple  # (gx, gy) lattice of sources on the top face
    det_grid: tuple  # (gx, gy) lattice of detectors on the bottom face
    ls: int
    ld: int
    m0: int
    sampling: str = "gaussian"  # "rademacher" | "gaussian"
    rtol: float = 1e-10
    seed_index: int = 0
    rbf_radius: float = 1.0
    gamma: float = 1e-2
    cutoff: float = 0.0
    noise: float = 0.01
    bc: tuple = (ROBIN,) * 6

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def ns(self) -> int:
        return self.src_grid[0] * self.src_grid[1]

    @property
    def nd(self) -> int:
        return self.det_grid[0] * self.det_grid[1]

    @property
    def k(self) -> int:
        return self.ls + self.ld

    @property
    def np_(self) -> int:
        return 5 * self.m0

    @property
    def eps(self) -> float:
        # smoothed-Heaviside half width, taken numerically equal to h
        return self.h


# The five workloads: 1M voxels (the 128x128x64 frequency-domain case) is the
# headline; the 32x32x16 case is the small one the oracle finishes in seconds.
WORKLOADS = {
    "dot32x32x16": Workload("dot32x32x16", 32, 32, 16, 0.25, 0.0, (4, 4), (4, 4), 2, 2, 27,
                            sampling="rademacher", rtol=1e-10, seed_index=1),
    "dot64x64x32": Workload("dot64x64x32", 64, 64, 32, 0.125, 0.0, (8, 8), (8, 8), 12, 12, 125,
                            sampling="gaussian", rtol=1e-10, seed_index=2),
    "dot128x128x64_w100MHz": Workload("dot128x128x64_w100MHz", 128, 128, 64, 0.0625, OMEGA_NU_100MHZ,
                                      (16, 16), (16, 16), 32, 32, 125,
                                      sampling="gaussian", rtol=1e-10, seed_index=3),
    "dot128x128x128": Workload("dot128x128x128", 128, 128, 128, 0.0625, 0.0, (16, 32), (16, 32),
                               32, 32, 1000, sampling="gaussian", rtol=1e-10, seed_index=4),
    # the 1M-cell frequency-domain workload with half the columns (16 + 16): the same
    # kernels in about 7 GB of device memory, for profiler captures of many passes
    "dot128x128x64_w100MHz_k32": Workload("dot128x128x64_w100MHz_k32", 128, 128, 64, 0.0625, OMEGA_NU_100MHZ,
                                          (16, 16), (16, 16), 16, 16, 125,
                                          sampling="gaussian", rtol=1e-10, seed_index=3),
}


# Eight independent inversions with uneven grids n x n x n/2 (h = 8/n cm, 8 x 8 x 4 cm
# box, 96 <= n <= 256, 23,281,664 cells in all) and alternating omega = 0 / 100 MHz,
# each with 1,024 sources and 1,024 detectors sampled by 40 + 40 columns.
BATCH8 = tuple(
    Workload(f"batch8_{n}", n, n, n // 2, 8.0 / n, (0.0 if i % 2 == 0 else OMEGA_NU_100MHZ), (32, 32), (32, 32),
             40, 40, 125, sampling="gaussian", rtol=1e-10, seed_index=20 + i)
    for i, n in enumerate((96, 112, 128, 144, 160, 192, 224, 256)))


def small_workload(nx, ny, nz, h, *, omega_nu=0.0, src_grid=(2, 2), det_grid=(2, 2), ls=1, ld=1,
                   m0=4, sampling="rademacher", bc=(ROBIN,) * 6, seed_index=11, rbf_radius=None,
                   gamma=1e-2, cutoff=0.0, noise=0.01, name=None) -> Workload:
    """A small odd-shaped workload for brute-force and parity checks."""
    L = min(nx, ny, nz) * h
    if rbf_radius is None:
        rbf_radius = max(0.35 * L, 2.5 * h)
    return Workload(name or f"small{nx}x{ny}x{nz}", nx, ny, nz, h, omega_nu, tuple(src_grid),
                    tuple(det_grid), ls, ld, m0, sampling=sampling, seed_index=seed_index,
                    rbf_radius=rbf_radius, gamma=gamma, cutoff=cutoff, noise=noise, bc=tuple(bc))


def cell_centres(nx, ny, nz, h):
    """Cell-centre coordinates, shape (N, 3), voxel order v = i + nx*(j + ny*k)."""
    i = (np.arange(nx) + 0.5) * h
    j = (np.arange(ny) + 0.5) * h
    k = (np.arange(nz) + 0.5) * h
    Z, Y, X = np.meshgrid(k, j, i, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def _lattice(g, Lx, Ly):
    gx, gy = g
    return [((a + 0.5) * Lx / gx, (b + 0.5) * Ly / gy) for b in range(gy) for a in range(gx)]


def gaussian_columns(wl: Workload, which: str):
    """Sparse CSC columns of truncated Gaussians (sigma = h, cut at 4 sigma).

    which == "src": centred on the top face z = 0, normalised to sum(b) h^3 = 1.
    which == "det": centred on the bottom face z = nz h, normalised to sum(c) = 1.
    """
    nx, ny, nz, h = wl.nx, wl.ny, wl.nz, wl.h
    Lx, Ly, Lz = nx * h, ny * h, nz * h
    sigma = h
    rcut = 4.0 * sigma
    grid = wl.src_grid if which == "src" else wl.det_grid
    zc = 0.0 if which == "src" else Lz
    colptr = [0]
    rows, vals = [], []
    for (sx, sy) in _lattice(grid, Lx, Ly):
        i0, i1 = max(0, int(math.floor((sx - rcut) / h))), min(nx, int(math.ceil((sx + rcut) / h)) + 1)
        j0, j1 = max(0, int(math.floor((sy - rcut) / h))), min(ny, int(math.ceil((sy + rcut) / h)) + 1)
        k0, k1 = max(0, int(math.floor((zc - rcut) / h))), min(nz, int(math.ceil((zc + rcut) / h)) + 1)
        r_list, v_list = [], []
        for kk in range(k0, k1):
            z = (kk + 0.5) * h
            for jj in range(j0, j1):
                y = (jj + 0.5) * h
                for ii in range(i0, i1):
                    x = (ii + 0.5) * h
                    d2 = (x - sx) ** 2 + (y - sy) ** 2 + (z - zc) ** 2
                    if d2 <= rcut * rcut:
                        r_list.append(ii + nx * (jj + ny * kk))
                        v_list.append(math.exp(-d2 / (2.0 * sigma * sigma)))
        order = np.argsort(r_list)
        r_arr = np.asarray(r_list, dtype=np.int32)[order]
        v_arr = np.asarray(v_list, dtype=np.float64)[order]
        if which == "src":
            v_arr = v_arr / (v_arr.sum() * h ** 3)
        else:
            v_arr = v_arr / v_arr.sum()
        rows.append(r_arr)
        vals.append(v_arr)
        colptr.append(colptr[-1] + len(r_arr))
    return (np.asarray(colptr, dtype=np.int64), np.concatenate(rows).astype(np.int32),
            np.concatenate(vals).astype(np.float64))


def csc_to_dense(n, colptr, rows, vals):
    """Dense (n x ncol) copy of a CSC matrix (small cases only)."""
    ncol = len(colptr) - 1
    out = np.zeros((n, ncol))
    for c in range(ncol):
        out[rows[colptr[c]:colptr[c + 1]], c] = vals[colptr[c]:colptr[c + 1]]
    return out


def sampling_matrix(rng, n, l, kind):
    """l^{-1/2} [w_1 ... w_l] with i.i.d. zero-mean, unit-variance entries, Eqs. (defW)/(defV)."""
    if kind == "rademacher":
        w = rng.integers(0, 2, size=(n, l)).astype(np.float64) * 2.0 - 1.0
    elif kind == "gaussian":
        w = rng.standard_normal((n, l))
    else:
        raise ValueError(kind)
    return np.asfortranarray(w / math.sqrt(l))


@dataclasses.dataclass
class Inputs:
    wl: Workload
    p_true: np.ndarray
    p0: np.ndarray
    W: np.ndarray
    V: np.ndarray
    xi: np.ndarray        # (nd, ns) noise draws (real part)
    xi_im: np.ndarray     # (nd, ns) noise draws (imaginary part)
    B: tuple              # CSC (colptr, rows, vals)
    C: tuple


def draw(wl: Workload) -> Inputs:
    """All random inputs of a workload, from PCG64(1706055860 + seed_index).

    Draw order: RBF centres, RBF weights, W, V, noise, then the p0 perturbation.
    """
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + wl.seed_index))
    Lx, Ly, Lz = wl.nx * wl.h, wl.ny * wl.h, wl.nz * wl.h
    shrink = min(0.5, 0.25 * min(Lx, Ly, Lz))
    lo = np.array([shrink, shrink, shrink])
    hi = np.array([Lx - shrink, Ly - shrink, Lz - shrink])
    centres = lo + (hi - lo) * rng.random((wl.m0, 3))
    alpha = rng.standard_normal(wl.m0)
    beta = np.full(wl.m0, 1.0 / wl.rbf_radius)
    p_true = np.empty(5 * wl.m0)
    p_true[0::5] = alpha
    p_true[1::5] = beta
    p_true[2::5] = centres[:, 0]
    p_true[3::5] = centres[:, 1]
    p_true[4::5] = centres[:, 2]
    W = sampling_matrix(rng, wl.ns, wl.ls, wl.sampling)
    V = sampling_matrix(rng, wl.nd, wl.ld, wl.sampling)
    xi = rng.standard_normal((wl.nd, wl.ns))
    xi_im = rng.standard_normal((wl.nd, wl.ns))
    p0 = p_true.copy()
    p0[0::5] += 0.3 * rng.standard_normal(wl.m0)
    dchi = 0.2 * rng.standard_normal((wl.m0, 3)) * (wl.rbf_radius / 1.0)
    p0[2::5] += dchi[:, 0]
    p0[3::5] += dchi[:, 1]
    p0[4::5] += dchi[:, 2]
    B = gaussian_columns(wl, "src")
    C = gaussian_columns(wl, "det")
    return Inputs(wl, p_true, p0, W, V, xi, xi_im, B, C)


def diffusion_from_mua(mua, mus_prime=MUS_PRIME):
    """Diffusion coefficient of the diffusion approximation, D = 1 / (3 (mu_a + mu_s'))."""
    return 1.0 / (3.0 * (np.asarray(mua, dtype=np.float64) + mus_prime))


def add_noise(M_clean, inp: Inputs, level=None):
    """Data with relative Gaussian noise: Re and Im each perturbed by `level` of their own size."""
    lvl = inp.wl.noise if level is None else level
    M_clean = np.asarray(M_clean)
    if np.iscomplexobj(M_clean):
        return (M_clean.real * (1.0 + lvl * inp.xi) + 1j * M_clean.imag * (1.0 + lvl * inp.xi_im))
    return M_clean * (1.0 + lvl * inp.xi)
