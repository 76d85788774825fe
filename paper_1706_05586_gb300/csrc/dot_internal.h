// Host-side declarations shared by the runtime (dot_api.cu) and the kernel
// translation units.  Nothing here is part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace dotk {

// Sets the calling thread's dot_last_error() message; returns code.
int record_error(int code, const std::string& msg);

// Per-column Krylov state of one block solve (device pointers, length kp unless noted).
// The recurrence runs on r~ = r / scale; the FP64 solution and true residual are separate.
// Slots of the direction ring: the search directions of up to this many consecutive
// iterations are kept, and x~ takes their corrections in one pass per ring.
constexpr int kDirRingMax = 8;

struct ColState {
    double2* rho;      // r~^T M^{-1} r~ (bilinear; imaginary part 0 in real arithmetic)
    double2* rho_prev; // rho of the previous iteration (the denominator of beta)
    double2* alpha;
    double2* alpha_hist; // [kDirRingMax][kp] alpha of each iteration of the current direction ring (0: not run)
    double2* beta;
    double* rr;        // ||r~||^2 of the recurrence
    double* maxr;      // max ||r~|| since the last reliable update
    double* scale;     // s: r~ = r / s
    double* ratio;     // s_old / s_new of the last refresh
    double* tol2;      // target for ||r~||^2: rtol^2 ||b||^2 / s^2
    double* bb64;      // ||b||^2
    double* rr64;      // ||b - A x||^2 of the FP64 iterate at the last refresh
    int* active;       // 1 while the column iterates
    int* upd;          // 1 while the column waits for a reliable update
    int* iters;        // Krylov iterations taken
    int* updates;      // reliable updates taken
    int* since;        // iterations since the last refresh
    int* status;       // DOT_OK, DOT_ENOTCONV, DOT_EBREAKDOWN
    int* n_active;     // [1] active columns after the last finaliser
    int* n_update;     // [1] active columns waiting for an update
    unsigned* counter; // [1] arrival counter of the group sums (second reduction level)
    int* error;        // [1] nonzero after a bounded wait in a kernel ran out
    double2* partA;    // [grid * kp] per-block partial sums
    double* partB;     // [grid * kp]
    double2* groupA;   // [ceil(grid / kReduceGroup) * kp] per-group sums
    double* groupB;    // [ceil(grid / kReduceGroup) * kp]
    unsigned* gcount;  // [ceil(grid / kReduceGroup)] arrival counters of the groups
};

// Blocks per first-level group of the per-column reductions.
constexpr int kReduceGroup = 16;

// Raw operator coefficients in one precision.
struct OpRaw {
    const void* cf;    // packed (cx, cy, cz, dre) per voxel
    const void* dinv;  // element type: real or complex of the same precision
    double w;
    int nx, ny, nz;
};

enum ElemKind { EK_F64 = 0, EK_C128 = 1, EK_F32 = 2, EK_C64 = 3 };

struct Launch {
    int grid;      // blocks (persistent, multiple of the SM count where possible)
    int slots;     // voxels per block per sweep
    int threads;   // kp * slots
};

// TMA-staged stencil (stencil_tma.cu): tensor map over the p block and launch shape.
// The search directions of the last H iterations: slot (iteration mod H) receives
// the new direction, slot (iteration - 1) mod H holds the previous one.
struct DirRing {
    void* base = nullptr;    // H consecutive slots of n x kp recurrence-type elements
    int64_t slot_elems = 0;  // elements per slot
    int H = 0;               // slots in use: 8, 4 or 2 (a divisor of the poll batch)
    int flush_grid = 0;      // blocks of the flush: one wave at its register limit (0: as the others)
};

struct TmaStencil {
    alignas(64) unsigned char tmap[kDirRingMax][128];  // CUtensorMap of each ring slot
    alignas(64) unsigned char tmap_cf[128];  // CUtensorMap of the packed coefficients
    int kc = 32;                          // columns per tile (64 for FP32, 32, or 16)
    int zc = 0;                           // z planes per work item
    int grid = 0;
    size_t smem = 0;
    // direction update fused into the stencil (k_dpq_tma): maps over r~ and the ring
    // slots with kcf-column boxes, and over the 32-byte coefficient records
    alignas(64) unsigned char tmap_r[128];
    alignas(64) unsigned char tmap_pf[kDirRingMax][128];
    alignas(64) unsigned char tmap_c8[128];
    bool fused = false;
    int kcf = 0, zcf = 0, gridf = 0;
    size_t smemf = 0;
};
bool tma_stencil_eligible(ElemKind inner, int nx, int ny, int kp);
// Launch the bounded-wait self-test: *err (device) becomes 1 when the wait gave up.
cudaError_t wait_probe(int* err, long long budget, cudaStream_t s);
cudaError_t tma_stencil_prepare(ElemKind inner, const DirRing& ring, const void* cf, int nx, int ny, int nz, int kp,
                                int num_sms, TmaStencil* out);
// q = A p for the direction in ring slot `slot` (its alpha goes to row `slot` of the
// step-length history).
cudaError_t tma_stencil_launch(ElemKind inner, const OpRaw& op, const TmaStencil& t, int slot, void* q, int kp,
                               const ColState& st, cudaStream_t s);
// Direction update fused into the stencil: p_new = M^{-1} r~ + beta p_old into ring slot
// `slot` from slot `prev` (running columns; p_old carried over on the others), then
// q = A p_new with p_new^T q.  Eligible for the FP32 / complex64 recurrence with nx, ny
// multiples of 8 and the padded block width a multiple of 32 (real) or 16 (complex).
bool dpq_eligible(ElemKind inner, int nx, int ny, int kp);
cudaError_t dpq_prepare(ElemKind inner, const DirRing& ring, const void* r, const void* cf8, int nx, int ny, int nz,
                        int kp, int num_sms, TmaStencil* out);
cudaError_t dpq_launch(ElemKind inner, const OpRaw& op, const TmaStencil& t, const DirRing& ring, int slot, int prev,
                       void* q, int kp, const ColState& st, cudaStream_t s);

// Launch shape of the scalar kernels (one column per thread, four blocks per SM).
Launch krylov_launch(int64_t n, int kp, int num_sms);
// Launch shape of the vectorised iteration kernels (W columns per thread).
Launch vector_launch(int64_t n, int kp, int w, int num_sms);
// Columns per thread of the iteration kernels for a recurrence type (kp is padded to 4).
int vector_width(ElemKind inner);

// ---- Krylov (krylov.cu); all enqueue on `s`.  `inner` is the recurrence type
// (EK_F32/EK_C64 mixed, EK_F64/EK_C128 FP64); the FP64 vectors b64, x64, r64 match it
// in complexity.
cudaError_t solve_start(ElemKind inner, const OpRaw& op, const void* b64, void* x64, void* x, void* r, void* p,
                        int64_t n, int kp, const ColState& st, double rtol, const Launch& L, cudaStream_t s);
// Krylov iteration m of a batch (the batch starts at a multiple of the ring size):
// [direction update into slot m mod H (fused into the stencil when tma->fused),]
// stencil q = A p with p^T q, r~ update with
// convergence / refresh decisions, and, when slot m mod H is the ring's last, the
// flush x~ += sum_j alpha_j p_j.  ev, when not null, receives four event records
// around the first three launches; evf, when not null, one record after the flush.
cudaError_t kry_step(ElemKind inner, const OpRaw& op, void* x, void* r, const DirRing& ring, int m, void* q,
                     int64_t n, int kp, const ColState& st, double delta, int maxit, bool with_p, const Launch& Lv,
                     const TmaStencil* tma, cudaStream_t s, cudaEvent_t* ev, cudaEvent_t* evf);
// Reliable update of the active columns (after a flush): promote x~, FP64 true
// residual, rescale r~.
cudaError_t solve_refresh(ElemKind inner, const OpRaw& op, const OpRaw& op64, const void* b64, void* x64, void* r64,
                          void* x, void* r, int64_t n, int kp, const ColState& st, double rtol, int maxit,
                          const Launch& L, int num_sms, cudaStream_t s);
// Promote every column's x~; optionally recompute every column's true residual.
cudaError_t solve_finish(ElemKind inner, const OpRaw& op64, const void* b64, void* x64, void* r64, void* x, int64_t n,
                         int kp, const ColState& st, bool residual, const Launch& L, int num_sms, cudaStream_t s);
cudaError_t op_apply(ElemKind ek, const OpRaw& op, const void* x, void* y, int64_t n, int kp,
                     cudaStream_t s);

// ---- field kernels (fields.cu)
cudaError_t pals_eval(const double* p, int m0, double mu_in, double mu_out, double c, double eps,
                      double gamma, int nx, int ny, int nz, double h, double* phi, double* mu,
                      double* wdmu, cudaStream_t s);
// Packed coefficients (cx, cy, cz, dre) per voxel in FP64 (cf64) and FP32 (cf32),
// and the Jacobi inverse diagonal in both precisions; cf8 (optional, 32 B per voxel):
// the FP32 coefficients followed by the FP32 Jacobi inverse (re, im or value, 0) and
// two zero words, the record the fused direction + stencil kernel stages by TMA.
cudaError_t build_coefficients(const double* D, const double* mu, int nx, int ny, int nz, double h,
                               const int bc[6], double w, void* cf64, void* dinv64, bool cplx, void* cf32,
                               void* dinv32, void* cf8, cudaStream_t s);
cudaError_t build_rhs(bool cplx, const int64_t* rowptrB, const int32_t* colB, const double* valB,
                      const double* W, int ns, int ls, const int64_t* rowptrC, const int32_t* colC,
                      const double* valC, const double* V, int nd, int ld, int64_t n, int kp, void* X,
                      cudaStream_t s);
cudaError_t blk_from_colmajor(bool cplx, const double* cm, int64_t n, int k, int kp, int c0,
                              void* blk, cudaStream_t s);
cudaError_t blk_to_colmajor(bool cplx, const void* blk, int64_t n, int kp, int c0, int k, double* cm,
                            cudaStream_t s);
cudaError_t data_projection(bool cplx, const double* M, int nd, int ns, const double* W, int ls,
                            const double* V, int ld, double* MW, double* P, cudaStream_t s);
cudaError_t restriction_misfit(bool cplx, const void* X, int kp, int ls, const int64_t* colptrC,
                               const int32_t* rowsC, const double* valsC, int nd, const double* V,
                               int ld, const double* P, bool have_data, double* T, double* S,
                               double* Rs, double* f, cudaStream_t s);
cudaError_t sensitivity_gmu(bool cplx, const void* X, int64_t n, int kp, int ls, int ld,
                            const double* Rs, double* gmu, cudaStream_t s);
cudaError_t jacobian_mua(bool cplx, const void* X, int64_t n, int kp, int ls, int ld, double* J,
                         cudaStream_t s);
cudaError_t pals_chain_gp(const double* p, int m0, double gamma, int nx, int ny, int nz, double h,
                          const double* wdmu, const double* gmu, double* gp, cudaStream_t s);
// Band lists of the PaLS derivative: per RBF the cells of its support where dmu/dp is
// nonzero, in box order, with the five derivatives.  count: counts[m0]; fill: from the
// exclusive offsets offs[m0 + 1] into cell[offs[m0]] and dval[5 offs[m0]].
cudaError_t pals_band_count(const double* p, int m0, double gamma, int nx, int ny, int nz, double h,
                            const double* wdmu, int64_t* counts, cudaStream_t s);
cudaError_t pals_band_fill(const double* p, int m0, double gamma, int nx, int ny, int nz, double h,
                           const double* wdmu, const int64_t* offs, int64_t* cell, double* dval, cudaStream_t s);
// J_p = J_mu dmu/dp for the block's l_s forward and l_d adjoint columns over the band lists.
cudaError_t pals_chain_jp(bool cplx, int m0, const int64_t* offs, const int64_t* cell, const double* dval,
                          const void* X, int kp, int ls, int ld, double* Jp, cudaStream_t s);

// ---- optimized sources and detectors (optimize.cu)
int symmetric_eigen(int n, std::vector<double>& A, std::vector<double>& w, std::vector<double>& Q);
void complement(int n, int q, const std::vector<double>& What, int m, const double* Ytil, double* out);
// Chunks of the long dimension of the Gram products and the scratch for their partial
// sums (dGpart: kGramPartDoubles doubles).
constexpr int kGramChunks = 64;
constexpr int64_t kGramPartDoubles = (int64_t)1 << 22;
int optimize_from_tensor(bool cplx, const void* Jd, int nd, int ns, int npar, int qs, int qd, int maxit, double tol,
                         void* scratch_K, void* scratch_L, double* dG, double* dGpart, double* dVW, cudaStream_t s,
                         std::vector<double>& What, std::vector<double>& Vhat, int* sweeps, double* objective);

}  // namespace dotk
