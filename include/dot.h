/*
 * dot.h - C ABI of the GB300 hot path for randomized diffuse optical tomography
 * (DOT) with simultaneous random and optimized sources and detectors
 * (Aslan, de Sturler, Kilmer).
 *
 * The library evaluates, for a fixed sampling (W, V), the quantities of Sec. 3:
 *   - forward block solves  A(mu) U = B W    (Eq. (EsTResidual), z_i in the paper)
 *   - adjoint block solves  A^T Z = C V      (Sec. 3.3, y_j in the paper)
 *   - sampled misfit f = ||V^T (C^T A^{-1} B - M) W||_F^2     (Theorem 1)
 *   - sampled mu-Jacobian rows -Z_l (.) U_i  (Eq. (Jacobiancomp) and
 *     Eq. (Jacobian kth column): dA/dmu_v = e_v e_v^T when D is known)
 *   - PaLS chain rule to the shape parameters p   (Sec. 2, Eq. (absorption const))
 *   - misfit gradient 2 Re J^T conj(r_s)          (Eq. (UnbiasedGrad))
 * where A(mu) + i(omega/nu) I is the cell-centred finite-volume form of the
 * diffusion equation of Sec. 2, Eq. (PDE), with Robin or Dirichlet faces.
 *
 * Conventions
 *   - Every call returns an int status: DOT_OK (0) or a negative DOT_E* code.
 *     dot_last_error() returns a message for the calling thread's last error.
 *   - Plain entry points take HOST pointers; the library copies what it needs
 *     into device memory it owns (setters copy, the caller keeps ownership).
 *     Entry points ending in _dev take DEVICE pointers valid on the context's
 *     device; they are read or written in order on the context's stream.
 *   - Dense matrices are column-major.  Complex values (omega != 0) are
 *     interleaved (re, im) pairs of doubles.
 *   - Voxel index v = i + nx (j + ny k) of the cell centred at
 *     ((i+1/2)h, (j+1/2)h, (k+1/2)h); k = 0 is the top face (x3 = 0).
 *   - Face order for boundary flags: -x, +x, -y, +y, -z (top), +z (bottom).
 *   - PaLS parameters: 5 per RBF, (alpha_j, beta_j, chi_xj, chi_yj, chi_zj).
 *   - Sampled Jacobian rows are ordered r = l + l_d * i (vec of V^T R W).
 *   - Results are cached: an evaluation call reuses the block solve while no
 *     setter has changed its inputs.  Every setter invalidates what depends on it.
 *   - A context is not thread-safe; use one context per thread.
 */
#ifndef DOT_H
#define DOT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define DOT_OK          0
#define DOT_EINVAL     -1  /* bad argument (size, pointer, flag)                 */
#define DOT_ESTATE     -2  /* a required setter has not been called              */
#define DOT_ENOMEM     -3  /* device allocation failed                           */
#define DOT_ECUDA      -4  /* CUDA runtime error                                 */
#define DOT_ENOTCONV   -5  /* Krylov solve hit maxit; outputs are still written  */
#define DOT_EBREAKDOWN -6  /* CG/COCG breakdown (zero p^T A p or rho)            */
#define DOT_ETIMEOUT   -7  /* a bounded device-side wait ran out; results invalid */

/* boundary flags */
#define DOT_BC_ROBIN      0  /* 0.25 eta + (D/2) d eta / d xi = 0, Eq. (PDE)      */
#define DOT_BC_DIRICHLET  1  /* eta = 0, Eq. (PDE) lateral faces                  */

/* solver precision */
#define DOT_PREC_FP64   0  /* FP64 / complex128 Jacobi CG (omega = 0) or COCG     */
#define DOT_PREC_MIXED  1  /* FP32 / complex64 CG or COCG recurrence with FP64
                              reliable updates; true residuals, the solution and all
                              outputs FP64 */

typedef struct dot_ctx dot_ctx;

typedef struct dot_stats {
    int32_t k;               /* columns of the last block solve (l_s + l_d)            */
    int32_t iters_max;       /* max over columns of Krylov iterations (summed over
                                refinement steps in mixed precision)                   */
    int64_t iters_sum;       /* sum over columns of Krylov iterations                 */
    int32_t outer_steps;     /* max over columns of FP64 true-residual refreshes
                                (reliable updates) of the last solve                  */
    int32_t status;          /* status of the last block solve                        */
    double  relres_max;      /* max over columns of the FP64 true residual
                                ||b - A x|| / ||b|| at the end of the last solve       */
    int64_t columns_solved;  /* cumulative number of PDE solves (columns)             */
    int64_t block_solves;    /* cumulative number of block solves                     */
    double  ms_setup;        /* last: PaLS + coefficients + right-hand sides          */
    double  ms_solve;        /* last: block Krylov solve                              */
    double  ms_post;         /* last: restriction, misfit, sensitivity, chain rule    */
    int64_t kernel_launches; /* cumulative number of this library's kernel launches   */
    int32_t tuned_tma;       /* stencil path of the last solve, autotuned or default (1 TMA, 0 direct, -1 no solve yet) */
    int32_t tuned_blocks_per_sm; /* blocks per SM of the vector kernels in the last solve (-1 no solve yet) */
    int32_t fused_direction; /* 1: the last solve ran the direction update inside the TMA stencil, 0: as a
                                pass of its own (-1 no solve yet)                                       */
    int32_t reserved;        /* 0                                                                  */
} dot_stats;

/* Per-kernel device time of the Krylov kernels, accumulated while timing is on.
 * Index 0: stencil q = A p with p^T q; 1: r update with r^T M^{-1} r and ||r||^2;
 * 2: direction update p = M^{-1} r + beta p; 3: FP64 refinement round (promotion,
 * residual b - A x, rescaling); 4: x update from the ring of recent directions.
 * bytes: algorithmic DRAM bytes of those launches (each vector element of an
 * active column read or written once, coefficients once per launch). */
typedef struct dot_kernel_timing {
    int64_t launches[5];
    double  ms[5];
    double  bytes[5];
} dot_kernel_timing;

/* Context: binds a CUDA device and owns every device buffer.
 * dot_create: *out receives the handle; device is a CUDA ordinal.  Creates a
 * private non-blocking stream.  Errors: DOT_EINVAL, DOT_ECUDA. */
int dot_create(dot_ctx** out, int device);
/* Frees every device buffer and the private stream.  NULL is accepted. */
int dot_destroy(dot_ctx* ctx);
/* Message for the calling thread's last failed call ("" if none).  The pointer
 * stays valid until the thread's next failed call. */
const char* dot_last_error(void);
/* Make subsequent work run on `stream` (a cudaStream_t of the context's device,
 * e.g. torch.cuda.current_stream().cuda_stream); NULL restores the private stream. */
int dot_set_stream(dot_ctx* ctx, void* stream);

/* Grid (Sec. 2, Eq. (PDE) and Eq. (Eq:compmeas)): nx*ny*nz cells of size h (cm),
 * bc[6] boundary flags.  Invalidates everything sized by the grid. */
int dot_set_grid(dot_ctx* ctx, int nx, int ny, int nz, double h, const int bc[6]);
/* omega / nu (cm^-1) of the frequency term i(omega/nu) E, E = I on the
 * cell-centred grid.  0 selects real arithmetic (CG), != 0 complex (COCG). */
int dot_set_omega(dot_ctx* ctx, double omega_over_nu);
/* Diffusion coefficient D (N doubles, cm), known and held fixed (Sec. 2). */
int dot_set_diffusion(dot_ctx* ctx, const double* D);
/* Absorption mu_a (N doubles, cm^-1) set directly; gradients are then taken
 * with respect to mu (N entries).  Replaces any PaLS parameters. */
int dot_set_mua(dot_ctx* ctx, const double* mu);
/* PaLS absorption (Sec. 2): phi(x) = sum_j alpha_j psi(||beta_j (x - chi_j)||^dagger),
 * psi = Wendland psi_{2,1}, ||y||^dagger = sqrt(||y||^2 + gamma^2),
 * mu = mu_in H_eps(phi - c) + mu_out (1 - H_eps(phi - c)) with the C^1 sine ramp
 * H_eps of half width eps.  p: 5*m0 doubles.  Gradients are then with respect to p. */
int dot_set_pals(dot_ctx* ctx, int m0, const double* p, double mu_in, double mu_out,
                 double c, double eps, double gamma);
/* As dot_set_pals with p a device pointer (5*m0 doubles) read on the context stream. */
int dot_set_pals_dev(dot_ctx* ctx, int m0, const double* p_dev, double mu_in, double mu_out,
                     double c, double eps, double gamma);

/* Physical sources B (N x ns) and detectors C (N x nd) as CSC: colptr[ncol+1]
 * (int64), rows[nnz] (int32 voxel indices, each column's rows distinct),
 * vals[nnz] (double).  Eq. (Eq:compmeas): b_i are the source terms, rows of C^T the
 * detectors. */
int dot_set_sources(dot_ctx* ctx, int ns, const int64_t* colptr, const int32_t* rows,
                    const double* vals);
int dot_set_detectors(dot_ctx* ctx, int nd, const int64_t* colptr, const int32_t* rows,
                      const double* vals);
/* Data M (nd x ns, column-major; the paper's D of Eq. (MartixR)).  is_complex = 1:
 * interleaved complex (required when omega != 0), 0: real. */
int dot_set_data(dot_ctx* ctx, const double* M, int is_complex);
/* Sampling matrices W (ns x ls) and V (nd x ld), column-major, already scaled
 * (Eqs. (defW), (defV): l^{-1/2} times i.i.d. zero-mean unit-variance entries,
 * or optimized / complemented columns, Eqs. (newW), (newV)). */
int dot_set_sampling(dot_ctx* ctx, int ls, const double* W, int ld, const double* V);
/* Krylov settings: precision DOT_PREC_*, relative residual target rtol
 * (||b - A x||_2 <= rtol ||b||_2 per column), maxit Krylov iterations per column
 * (per refinement step in mixed precision; 0 selects 10 (nx + ny + nz)).
 * ls + ld (the block width) may not exceed 1024. */
int dot_set_solver(dot_ctx* ctx, int precision, double rtol, int maxit);
/* Mixed precision only: reliable-update threshold delta (default 1e-3).  A column's
 * FP32 recurrence is refreshed from an FP64 true residual b - A x whenever its
 * recurrence residual falls below delta times its largest value since the last
 * refresh, after 256 iterations without a refresh, and whenever it reaches rtol;
 * convergence is always judged on the FP64 true residual. */
int dot_set_refinement(dot_ctx* ctx, double delta);

/* Sampled misfit f = ||V^T (C^T A^{-1} B - M) W||_F^2 (Theorem 1 / Eq. (EsTResidual);
 * no factor 1/2; complex: sum of squared real and imaginary parts).  Solves the
 * l_s + l_d columns [BW | CV] as one block.  Returns DOT_ENOTCONV or
 * DOT_EBREAKDOWN (with f still written) when a column failed. */
int dot_misfit(dot_ctx* ctx, double* f);
/* Sampled computed measurements S = V^T C^T A^{-1} B W (ld x ls, column-major,
 * complex interleaved when omega != 0); with W = I, V = I this is the full
 * C^T A^{-1} B of Eq. (Eq:compmeas).  Does not need data. */
int dot_measurements(dot_ctx* ctx, double* S);
/* Computed measurements of every physical source, C^T A^{-1} B (nd x ns,
 * column-major; complex interleaved when omega != 0): Eq. (Eq:compmeas) for all
 * b_i.  Solves the ns source columns in blocks of 64 with the current solver
 * settings; needs no sampling and no data, and leaves the sampled state as it was
 * (the next evaluation solves again). */
int dot_forward_model(dot_ctx* ctx, double* M);
/* f and its gradient: g (5*m0 doubles) with respect to p after dot_set_pals,
 * or (N doubles) with respect to mu after dot_set_mua.  g = 2 Re J^T conj(vec R_s)
 * with J the sampled Jacobian of Eq. (Jacobian kth column). */
int dot_gradient(dot_ctx* ctx, double* f, double* g);
/* dot_gradient with device outputs: f_dev (1 double) and g_dev (as for g) are device
 * pointers of the context's device; they are written on the context's stream, which
 * has completed when the call returns.  Lets a framework keep the gradient on the
 * device (no host round trip). */
int dot_gradient_dev(dot_ctx* ctx, double* f_dev, double* g_dev);
/* Sampled mu-Jacobian J_mu[(l + ld i), v] = -Z_l[v] U_i[v]  ((ls*ld) x N,
 * column-major; complex interleaved when omega != 0).  (ls*ld*N) values. */
int dot_jacobian_mua(dot_ctx* ctx, double* J);
/* Sampled p-Jacobian J_p = J_mu dmu/dp  ((ls*ld) x 5*m0, column-major; complex
 * interleaved when omega != 0).  Needs dot_set_pals. */
int dot_jacobian_p(dot_ctx* ctx, double* Jp);

/* Optimized simultaneous sources and detectors (Sec. 3.2, Algorithm 1) completed by
 * random ones in the complementary subspace (Eqs. (newW), (newV), Theorem 2), at the
 * current PaLS parameters.  Solves every physical source and detector once
 * (ns + nd <= 1024 columns), forms the Jacobian tensor J_ijk of Eq. (Jtensor), and
 * runs the Tucker2 alternating iteration: q_d leading left singular vectors of
 * J~ = [J_{:,1,:} ... J_{:,ns,:}], then alternately W~ from K~ and V~ from L~ until the
 * projectors change by less than tol or after maxit sweeps.  The outputs are
 *   W = [W^, (I - W^ W^T) Ytil]  (ns x ls, column-major),  V = [V^, (I - V^ V^T) Ztil]
 * (nd x ld): Ytil (ns x (ls - qs)) and Ztil (nd x (ld - qd)) are the caller's random
 * draws, already scaled by (l - q)^{-1/2}; projecting them onto the complement gives the
 * covariance I - W^ W^T of W_c Y for any basis W_c.  Complex J (omega != 0) enters
 * through its real and imaginary parts.  1 <= qs, qd <= 8.  sweeps and objective
 * (||(W^T (x) V^T) J||_F^2) may be NULL.  Does not change the context's sampling. */
int dot_optimized_sampling(dot_ctx* ctx, int qs, int qd, int maxit, double tol, int ls, const double* Ytil,
                           int ld, const double* Ztil, double* W, double* V, int* sweeps, double* objective);
/* Host helper used by dot_optimized_sampling: eigen-decomposition of a symmetric
 * n x n column-major matrix A (Householder tridiagonalisation, implicit QL);
 * eigenvalues ascending in evals (n), eigenvectors in the columns of evecs (n x n). */
int dot_symeig(int n, const double* A, double* evals, double* evecs);

/* Inspection.  dot_get_mua: the absorption field in use (N doubles).
 * dot_get_fields: forward fields U (N x ls) and adjoint fields Z (N x ld),
 * column-major (complex interleaved when omega != 0); either pointer may be NULL.
 * dot_get_stats: counters of the last evaluation. */
int dot_get_mua(dot_ctx* ctx, double* mu);
int dot_get_fields(dot_ctx* ctx, double* U, double* Z);
int dot_get_stats(dot_ctx* ctx, dot_stats* stats);
/* Launch options of the block solve.  graphs != 0 (default) replays each steady
 * batch of Krylov iterations from a CUDA graph captured on the context stream (the
 * stream must be capturable: not the legacy default stream, no other thread queuing
 * on it meanwhile).  autotune != 0 (default 0) times the first batches of a solve with
 * each stencil path that dot_set_stencil_path allows (direct loads; TMA stencil; TMA
 * stencil with the direction update fused in) and 4, 5, 8 or 16 blocks per SM for the
 * vector kernels, keeps the
 * fastest for the rest of the solve and for later solves of the same shape; since the
 * reduction order follows the launch shape, results then agree to rounding (not
 * bitwise) with an untuned run. */
int dot_set_launch_options(dot_ctx* ctx, int graphs, int autotune);
/* Slots of the direction ring (no counterpart in the paper): the search directions of
 * the last `slots` iterations stay on the device and x~ takes their corrections in one
 * pass per ring.  slots = 0 (default) tries 8, then 4, then 2 as device memory allows;
 * 2, 4 or 8 caps the ring at that size.  Every size gives bitwise the same results
 * (each correction is added in iteration order either way); smaller rings stream
 * more bytes per iteration.  Errors: DOT_EINVAL for other values. */
int dot_set_direction_ring(dot_ctx* ctx, int slots);
/* Misfit and gradient of several contexts (independent inversions, e.g. uneven grids
 * and mixed omega) in one call.  The members run one after another, each on its own
 * stream with its own launch configuration (autotuned per member when enabled) and
 * graph-replayed block solve; each member's kernels fill the GPU by themselves, so
 * members are not overlapped.  Same per-context semantics and outputs as dot_gradient
 * (f[i], g[i]); each context must appear once.  The contexts, their data and the
 * output pointers are checked before the first member runs; a member missing another
 * input fails when its turn comes.  Returns the first hard error (later members do
 * not run), else DOT_ENOTCONV / DOT_EBREAKDOWN if a member ended so (every member's
 * outputs are written). */
int dot_gradient_batch(dot_ctx* const* ctxs, int count, double* f, double* const* g);
/* Stencil implementation of the block solve (no counterpart in the paper, which leaves
 * the solver open).  mode 2 (default): wherever the block allows it (FP32/complex64
 * recurrence, nx and ny multiples of 8, padded block width a multiple of 32 real or 16
 * complex columns) one kernel forms the new search direction p = M^{-1} r~ + beta p and
 * applies the stencil to it, staging r~, the old direction and the coefficients
 * through shared memory with tensor-memory-accelerator copies; mode 1: the
 * TMA-staged stencil after a separate direction pass (block width a multiple of 16);
 * mode 0: the direct-load stencil.  Shapes a mode does not take fall back to the next
 * lower one.  Results agree to rounding.  Errors: DOT_EINVAL for other modes. */
int dot_set_stencil_path(dot_ctx* ctx, int mode);
/* Kernel timing: enable != 0 resets the counters and records CUDA events around
 * every Krylov kernel launch (on the context stream); 0 stops recording. */
int dot_set_kernel_timing(dot_ctx* ctx, int enable);
int dot_get_kernel_timing(dot_ctx* ctx, dot_kernel_timing* out);

/* One operator application y = (A(mu) + i(omega/nu) I) x on k columns
 * (N x k, column-major, complex interleaved when omega != 0) in FP64.
 * The 7-point stencil of the block solve, exposed for testing. */
int dot_apply(dot_ctx* ctx, int k, const double* x, double* y);

/* Self-test of the device-side bounded waits (no counterpart in the paper): one warp
 * waits on an mbarrier that nothing ever arrives at, with a budget of budget_cycles
 * SM clock cycles (0 .. 4e9; the stencil kernels use about 4e9, roughly 2 s), gives
 * up, and reports through the same kind of device error word the stencil kernels use.
 * Nothing is in flight when the wait gives up.  Returns DOT_ETIMEOUT (the expected
 * outcome), DOT_EBREAKDOWN if the wait claimed completion, DOT_EINVAL / DOT_ECUDA
 * otherwise.  The context stays usable afterwards. */
int dot_probe_wait(dot_ctx* ctx, int64_t budget_cycles);

/* Allocation-free restriction and misfit (this library's addition; the paper has
 * no counterpart).  For callers that cannot let the library allocate device memory:
 * a latency-critical loop that must not stall on cudaMalloc / cudaFree (which can
 * synchronize the device), or a process whose device memory is owned entirely by
 * another allocator.  Computes, from fields already on the device,
 *   T = C^T U (n_d x l_s),  S = V^T T (l_d x l_s),  R_s = S - P,  f = ||R_s||_F^2,
 * the restriction and misfit of Eq. (EsTResidual) / Theorem 1, with the same kernels
 * as dot_misfit.  All pointers are DEVICE pointers on the current device; the work
 * is queued on `stream` (a cudaStream_t, NULL for the default stream) and nothing
 * is synchronized.
 *   X: block of fields over n cells, element (v, c) at v * kp + c (double, or
 *      interleaved complex when is_complex), kp >= ls, columns 0..ls-1 the forward
 *      fields U (further columns, e.g. the adjoint fields, are not read);
 *   colptrC (nd + 1, int64), rowsC, valsC: detectors C as CSC, every rowsC entry a cell
 *      index in [0, n) (not checked: the arrays stay on the device, and an index outside
 *      the grid makes the restriction read outside X);  V: nd x ld column-major;
 *   P: l_d x l_s interleaved complex V^T M W, or NULL for no data (R_s = S);
 *   S, Rs: l_d x l_s interleaved complex outputs;  f: one double.
 * The only scratch, T, is a fixed device array of DOT_NOALLOC_MAX_T complex entries
 * (1 MiB) that every GPU loading the library holds until the process exits;
 * nd * ls above that limit is rejected with DOT_EINVAL.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress), so make it before any
 * stream capture; the address is kept for the life of the process, so do not use this
 * entry point on a device after cudaDeviceReset (or any other teardown of its primary
 * context) in the same process.  All calls share the array, which keeps the last call's
 * contents (each call overwrites every entry it reads); calls that overlap on the GPU
 * race. */
#define DOT_NOALLOC_MAX_T 65536
int dot_restrict_misfit_noalloc(const double* X, int64_t n, int kp, int ls, int ld, const int64_t* colptrC,
                                const int32_t* rowsC, const double* valsC, int nd, const double* V,
                                const double* P, int is_complex, double* S, double* Rs, double* f,
                                void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DOT_H */
