// Host-side declarations shared by the runtime (dot_api.cu) and the kernel
// translation units.  Nothing here is part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dotk {

// Per-column Krylov state of one block solve (device pointers, length kp unless noted).
struct ColState {
    double2* rho;      // r^T z (bilinear; imaginary part 0 in real arithmetic)
    double2* alpha;
    double2* beta;
    double* rr;        // ||r||_2^2
    double* bb;        // ||b||_2^2
    int* active;       // 1 while the column iterates
    int* iters;        // iterations taken
    int* status;       // 0 ok, DOT_ENOTCONV, DOT_EBREAKDOWN
    int* n_active;     // [1] number of active columns after the last finaliser
    unsigned* counter; // [1] arrival counter of the last-block finaliser
    double2* partA;    // [grid * kp] per-block partial sums
    double* partB;     // [grid * kp]
};

// Per-column state of the FP64 iterative-refinement loop (mixed precision).
struct RefState {
    double* bb;        // ||b||^2 of the FP64 right-hand side
    double* rr;        // ||b - A x||^2 of the current FP64 iterate
    double* scale;     // ||r|| used to normalise the FP32 correction problem
    int* active;       // 1 while the column still needs refinement
    int* n_active;     // [1]
    unsigned* counter; // [1]
    double* partB;     // [grid * kp]
};

// Raw operator coefficients in one precision.
struct OpRaw {
    const void* cx;
    const void* cy;
    const void* cz;
    const void* dre;
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

Launch krylov_launch(int64_t n, int kp, int num_sms);

// ---- Krylov (krylov.cu); all enqueue on `s`
cudaError_t kry_init(ElemKind ek, const OpRaw& op, const void* b, void* x, void* r, void* p,
                     int64_t n, int kp, const ColState& st, const Launch& L, cudaStream_t s);
cudaError_t kry_init_from64(ElemKind ek32, const OpRaw& op32, const void* r64, const RefState& rs,
                            void* x, void* r, void* p, int64_t n, int kp, const ColState& st,
                            const Launch& L, cudaStream_t s);
// One Krylov iteration = three launches (stencil + p^T A p, x/r update + convergence,
// direction update).  ev, when not null, receives four event records around them.
cudaError_t kry_iteration(ElemKind ek, const OpRaw& op, void* x, void* r, void* p, void* q,
                          int64_t n, int kp, const ColState& st, double rtol, int maxit,
                          const Launch& L, cudaStream_t s, cudaEvent_t* ev);
cudaError_t ref_init(ElemKind ek64, const void* b, void* x, void* r, int64_t n, int kp,
                     const RefState& rs, const Launch& L, cudaStream_t s);
cudaError_t ref_residual(ElemKind ek64, const OpRaw& op64, const void* b, const void* x, void* r,
                         int64_t n, int kp, const RefState& rs, double rtol, const Launch& L,
                         cudaStream_t s);
cudaError_t ref_promote(ElemKind ek64, ElemKind ek32, void* x64, const void* x32, int64_t n, int kp,
                        const RefState& rs, const Launch& L, cudaStream_t s);
cudaError_t op_apply(ElemKind ek, const OpRaw& op, const void* x, void* y, int64_t n, int kp,
                     cudaStream_t s);

// ---- field kernels (fields.cu)
cudaError_t pals_eval(const double* p, int m0, double mu_in, double mu_out, double c, double eps,
                      double gamma, int nx, int ny, int nz, double h, double* phi, double* mu,
                      double* wdmu, cudaStream_t s);
cudaError_t build_coefficients(const double* D, const double* mu, int nx, int ny, int nz, double h,
                               const int bc[6], double w, double* cx, double* cy, double* cz,
                               double* dre, void* dinv64, bool cplx, float* cx32, float* cy32,
                               float* cz32, float* dre32, void* dinv32, cudaStream_t s);
cudaError_t build_rhs(bool cplx, const int64_t* rowptrB, const int32_t* colB, const double* valB,
                      const double* W, int ns, int ls, const int64_t* rowptrC, const int32_t* colC,
                      const double* valC, const double* V, int nd, int ld, int64_t n, void* X,
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
cudaError_t pals_chain_jp(bool cplx, const double* p, int m0, double gamma, int nx, int ny, int nz,
                          double h, const double* wdmu, const void* X, int kp, int ls, int ld,
                          double* Jp, cudaStream_t s);

}  // namespace dotk
