// Block Jacobi-preconditioned CG / COCG with reliable updates (sm_103a).
//
// k independent Krylov recurrences share one operator A (Sec. 3.3: one block holds
// the l_s forward columns B W and the l_d adjoint columns C V; A is symmetric, or
// complex symmetric when omega != 0, so A^T = A and COCG's bilinear form x^T y
// applies).  The paper leaves the solver open ("iterative solvers or sparse direct
// solvers depending on the size"); this is the iterative choice.
//
// Precision: the recurrence runs in an inner type (FP32/complex64 in mixed mode,
// FP64/complex128 otherwise) on a per-column scaled copy r~ = r / s of the residual.
// The solution lives in FP64.  A column is refreshed ("reliable update",
// Sleijpen and van der Vorst 1996) when its recurrence residual has dropped below
// delta times its largest value since the last refresh, or reaches the target: the
// inner correction is added to the FP64 solution, the true residual b - A x is
// recomputed in FP64, and the recurrence continues from it with the same search
// direction.  Convergence is always decided on the FP64 true residual.
//
// Reductions are deterministic: each block of a persistent grid writes per-column
// partial sums, and the last block to arrive sums them in block order and runs the
// per-column scalar update, so no floating-point atomics are used.
#include "dot_kernels.cuh"
#include "dot_internal.h"
#include "dot_reduce.cuh"
#include "dot.h"

namespace dotk {

Launch krylov_launch(int64_t n, int kp, int num_sms) {
    Launch L;
    L.slots = kp >= 256 ? 1 : 256 / kp;
    L.threads = kp * L.slots;
    int64_t need = (n + L.slots - 1) / L.slots;
    int64_t g = (int64_t)num_sms * 4;
    L.grid = (int)(need < g ? need : g);
    if (L.grid < 1) L.grid = 1;
    return L;
}

static size_t red_smem(const Launch& L, int kp) {
    return (size_t)L.slots * kp * (sizeof(double2) + sizeof(double));
}

constexpr int kRefreshEvery = 256;

#define VOXEL_LOOP(v) \
    for (int64_t v = (int64_t)blockIdx.x * slots + slot; v < n; v += (int64_t)gridDim.x * slots)

// ------------------------------------------------------------- start of a solve
// x64 = 0 and ||b||^2 per column; finaliser: scale s = ||b||, activity.
template <typename T64>
__global__ void __launch_bounds__(1024) k_start_norm(const T64* __restrict__ b, T64* __restrict__ x64, int64_t n, int kp, int slots,
                             ColState st, double rtol) {
    const int c = threadIdx.x % kp, slot = threadIdx.x / kp;
    double bb = 0.0;
    VOXEL_LOOP(v) {
        const int64_t e = v * kp + c;
        bb += (double)eabs2(b[e]);
        x64[e] = ezero<T64>();
    }
    column_partials(make_double2(0.0, 0.0), bb, kp, slots, c, slot, nullptr, st.partB);
    const double2* totA;
    const double* totB;
    if (reduce_columns(st, false, true, kp, smem_raw, &totA, &totB)) {
        for (int cc = threadIdx.x; cc < kp; cc += blockDim.x) {
            const double2 a = totA[cc];
            const double bsum = totB[cc];
            const bool fin = isfinite(bsum);
            st.bb64[cc] = bsum;
            st.rr64[cc] = bsum;
            st.scale[cc] = sqrt(bsum);
            st.tol2[cc] = rtol * rtol;
            st.iters[cc] = 0;
            st.upd[cc] = 0;
            st.updates[cc] = 0;
            st.since[cc] = 0;
            st.alpha[cc] = make_double2(0.0, 0.0);
            st.status[cc] = fin ? DOT_OK : DOT_EBREAKDOWN;
            st.active[cc] = fin && bsum > 0.0;
        }
        __syncthreads();
        publish_counts(st, kp);
    }
}

// r~ = b / s, x~ = 0, p = M^{-1} r~; rho = r~^T M^{-1} r~, ||r~||^2.
template <typename T, typename T64>
__global__ void __launch_bounds__(1024) k_start_inner(Op<T> op, const T64* __restrict__ b, T* __restrict__ x, T* __restrict__ r,
                              T* __restrict__ p, int64_t n, int kp, int slots, ColState st) {
    using R = typename Elem<T>::R;
    const int c = threadIdx.x % kp, slot = threadIdx.x / kp;
    const bool act = st.active[c] != 0;
    const double inv = act ? 1.0 / st.scale[c] : 0.0;
    T rho = ezero<T>();
    R rr = 0;
    VOXEL_LOOP(v) {
        const int64_t e = v * kp + c;
        x[e] = ezero<T>();
        if (!act) continue;
        const T rv = enarrow<T>(ewide(escale(inv, b[e])));
        const T z = emul(op.dinv[v], rv);
        r[e] = rv;
        p[e] = z;
        rho = eadd(rho, emul(rv, z));
        rr += eabs2(rv);
    }
    column_partials(ewide(rho), (double)rr, kp, slots, c, slot, st.partA, st.partB);
    const double2* totA;
    const double* totB;
    if (reduce_columns(st, true, true, kp, smem_raw, &totA, &totB)) {
        for (int cc = threadIdx.x; cc < kp; cc += blockDim.x) {
            if (!st.active[cc]) continue;
            const double2 a = totA[cc];
            const double rsum = totB[cc];
            st.rho[cc] = a;
            st.rr[cc] = rsum;
            st.maxr[cc] = sqrt(rsum);
            st.beta[cc] = make_double2(0.0, 0.0);
            if (!zfinite(a) || !isfinite(rsum)) {
                st.status[cc] = DOT_EBREAKDOWN;
                st.active[cc] = 0;
            }
        }
        __syncthreads();
        publish_counts(st, kp);
    }
}

// -------------------------------------------------------------- one iteration
__device__ __forceinline__ bool running(const ColState& st, int c) { return st.active[c] && !st.upd[c]; }

// The one-column-per-thread kernels (start, promotion, true residual, refresh) run
// blocks of kp x slots threads, up to 1024 at the widest block; they are compiled for
// 1024 threads (at most 64 registers), so every block width stays launchable.

// Launch shape of the vectorised iteration kernels: kp / W threads per voxel, about
// 256 threads per block, at most eight blocks per SM (the solver then sets the grid
// from its blocks-per-SM choice).
Launch vector_launch(int64_t n, int kp, int w, int num_sms) {
    Launch L;
    const int tpv = kp / w;
    L.slots = tpv >= 256 ? 1 : 256 / tpv;
    L.threads = tpv * L.slots;
    const int64_t need = (n + L.slots - 1) / L.slots;
    const int64_t g = (int64_t)num_sms * 8;
    L.grid = (int)(need < g ? need : g);
    if (L.grid < 1) L.grid = 1;
    return L;
}

// Per-column partial sums of a thread owning W columns starting at c0.
template <int W>
__device__ __forceinline__ void column_partials_w(const double2 (&a)[W], const double (&b)[W], int kp, int slots,
                                                  int c0, int slot, double2* partA, double* partB) {
    extern __shared__ unsigned char smem_raw[];
    double2* sA = reinterpret_cast<double2*>(smem_raw);
    double* sB = reinterpret_cast<double*>(sA + slots * kp);
#pragma unroll
    for (int u = 0; u < W; ++u) {
        sA[slot * kp + c0 + u] = a[u];
        sB[slot * kp + c0 + u] = b[u];
    }
    __syncthreads();
    if (slot == 0) {
#pragma unroll
        for (int u = 0; u < W; ++u) {
            double2 ta = make_double2(0.0, 0.0);
            double tb = 0.0;
            for (int s = 0; s < slots; ++s) {
                ta.x += sA[s * kp + c0 + u].x;
                ta.y += sA[s * kp + c0 + u].y;
                tb += sB[s * kp + c0 + u];
            }
            if (partA) partA[(int64_t)blockIdx.x * kp + c0 + u] = ta;
            if (partB) partB[(int64_t)blockIdx.x * kp + c0 + u] = tb;
        }
    }
}

// q = A p and pq = p^T q; finaliser alpha = rho / pq.  One 16-byte load per
// neighbour moves W columns (the direct-load form, for shapes the TMA stencil does not
// take).
template <typename T, int MT>
__global__ void __launch_bounds__(MT) k_pq(Op<T> op, const T* __restrict__ p, T* __restrict__ q, int kp,
                                               int slots, ColState st, int hslot) {
    using R = typename Elem<T>::R;
    constexpr int W = Vec16<T>::W;
    const int tpv = kp / W;
    const int t = threadIdx.x % tpv, slot = threadIdx.x / tpv, c0 = t * W;
    bool any = false;
#pragma unroll
    for (int u = 0; u < W; ++u) any = any || running(st, c0 + u);
    // pq is accumulated for every column of the vector; the finaliser reads only the
    // running ones (a paused or stopped column's q is scratch)
    T pq[W];
#pragma unroll
    for (int u = 0; u < W; ++u) pq[u] = ezero<T>();
    if (any) {
        const int nx = op.nx, nxy = nx * op.ny, n = nxy * op.nz;
        const T* __restrict__ pp = p + c0;
        T* __restrict__ qq = q + c0;
        for (int v = blockIdx.x * slots + slot; v < n; v += gridDim.x * slots) {
            const int kz = v / nxy, rem = v - kz * nxy, j = rem / nx, i = rem - j * nx;
            const int64_t e = (int64_t)v * kp;
            const V16<T> pc = ld16(pp + e);
            const Cf4<R> cv = op.cf[v];
            V16<T> acc;
#pragma unroll
            for (int u = 0; u < W; ++u) {
                acc.e[u] = escale(cv.dre, pc.e[u]);
                if (Elem<T>::cplx) acc.e[u] = eadd(acc.e[u], emul_i(op.w, pc.e[u]));
            }
#define DOT_NB(cond, coef, off)                                                     \
    if (cond) {                                                                     \
        const R cf = (coef);                                                        \
        const V16<T> nb = ld16(pp + e + (off));                                     \
        _Pragma("unroll") for (int u = 0; u < W; ++u) acc.e[u] = esub(acc.e[u], escale(cf, nb.e[u])); \
    }
            DOT_NB(i > 0, op.cf[v - 1].cx, -(int64_t)kp)
            DOT_NB(i < nx - 1, cv.cx, (int64_t)kp)
            DOT_NB(j > 0, op.cf[v - nx].cy, -(int64_t)nx * kp)
            DOT_NB(j < op.ny - 1, cv.cy, (int64_t)nx * kp)
            DOT_NB(kz > 0, op.cf[v - nxy].cz, -(int64_t)nxy * kp)
            DOT_NB(kz < op.nz - 1, cv.cz, (int64_t)nxy * kp)
#undef DOT_NB
            st16(qq + e, acc);
#pragma unroll
            for (int u = 0; u < W; ++u) pq[u] = eadd(pq[u], emul(pc.e[u], acc.e[u]));
        }
    }
    double2 pa[W];
    double pb[W];
#pragma unroll
    for (int u = 0; u < W; ++u) {
        pa[u] = ewide(pq[u]);
        pb[u] = 0.0;
    }
    column_partials_w<W>(pa, pb, kp, slots, c0, slot, st.partA, nullptr);
    const double2* totA;
    const double* totB;
    if (reduce_columns(st, true, false, kp, smem_raw, &totA, &totB)) {
        stencil_finalise(st, totA, kp, hslot);
        __syncthreads();
        publish_counts(st, kp);
    }
}

// r~ -= alpha q, rho' = r~^T M^{-1} r~, ||r~||^2 on the running columns (the others
// are left untouched).  The matching x~ += alpha p waits for the flush that closes
// the direction ring (k_flush), so this pass streams two vectors instead of four.
// Finaliser: pause the column for a
// reliable update when ||r~|| reached the target, fell below delta * max||r~|| or
// went kRefreshEvery iterations without a refresh; otherwise beta = rho' / rho.
template <typename T, int MT>
__global__ void __launch_bounds__(MT) k_r(Op<T> op, const T* __restrict__ q, T* __restrict__ r, int64_t n, int kp,
                                           int slots, ColState st, double delta, int maxit) {
    using R = typename Elem<T>::R;
    constexpr int W = Vec16<T>::W;
    const int tpv = kp / W;
    const int t = threadIdx.x % tpv, slot = threadIdx.x / tpv, c0 = t * W;
    bool run[W];
    bool any = false;
    T alpha[W], rho[W];
    R rr[W];
#pragma unroll
    for (int u = 0; u < W; ++u) {
        run[u] = running(st, c0 + u);
        any = any || run[u];
        alpha[u] = run[u] ? enarrow<T>(st.alpha[c0 + u]) : ezero<T>();
        rho[u] = ezero<T>();
        rr[u] = 0;
    }
    if (any) {
        // four cells in flight per thread: the loop is bound by load latency, not issue
#pragma unroll 4
        VOXEL_LOOP(v) {
            const int64_t e = v * kp + c0;
            const V16<T> qv = ld16(q + e);
            V16<T> rv = ld16(r + e);
            const T dv = op.dinv[v];
#pragma unroll
            for (int u = 0; u < W; ++u) {
                if (!run[u]) continue;
                rv.e[u] = esub(rv.e[u], emul(alpha[u], qv.e[u]));
                rho[u] = eadd(rho[u], emul(rv.e[u], emul(dv, rv.e[u])));
                rr[u] += eabs2(rv.e[u]);
            }
            st16(r + e, rv);
        }
    }
    double2 pa[W];
    double pbv[W];
#pragma unroll
    for (int u = 0; u < W; ++u) {
        pa[u] = ewide(rho[u]);
        pbv[u] = (double)rr[u];
    }
    column_partials_w<W>(pa, pbv, kp, slots, c0, slot, st.partA, st.partB);
    const double2* totA;
    const double* totB;
    if (reduce_columns(st, true, true, kp, smem_raw, &totA, &totB)) {
        for (int cc = threadIdx.x; cc < kp; cc += blockDim.x) {
            if (!running(st, cc)) continue;
            const double2 a = totA[cc];
            const double rsum = totB[cc];
            const int it = st.iters[cc] + 1;
            st.iters[cc] = it;
            st.rr[cc] = rsum;
            if (!isfinite(rsum) || !zfinite(a)) {
                st.status[cc] = DOT_EBREAKDOWN;
                st.active[cc] = 0;
                continue;
            }
            const double mr = st.maxr[cc];
            st.rho_prev[cc] = st.rho[cc];
            const int since = st.since[cc] + 1;
            st.since[cc] = since;
            // refresh at the target, after a drop by delta, at the iteration budget, and (in
            // mixed precision) at least every kRefreshEvery iterations so that a recurrence
            // that drifted from the true residual cannot stall the column
            if (rsum <= st.tol2[cc] || rsum < delta * delta * mr * mr || it >= maxit ||
                (delta > 0.0 && since >= kRefreshEvery)) {
                st.upd[cc] = 1;  // wait for the FP64 refresh; rho keeps its old value
                continue;
            }
            const double2 rho_old = st.rho[cc];
            if (rho_old.x == 0.0 && rho_old.y == 0.0) {
                st.status[cc] = DOT_EBREAKDOWN;
                st.active[cc] = 0;
                continue;
            }
            st.beta[cc] = zdiv(a, rho_old);
            st.rho[cc] = a;
            st.maxr[cc] = fmax(mr, sqrt(rsum));
        }
        __syncthreads();
        publish_counts(st, kp);
    }
}

// p_new = M^{-1} r~ + beta p_old on the running columns, where p_old and p_new are
// consecutive slots of the direction ring.  Paused columns carry p_old over, so that
// they resume from the slot the next iteration reads; stopped columns are skipped.
template <typename T, int MT>
__global__ void __launch_bounds__(MT) k_dir(Op<T> op, const T* __restrict__ r, const T* __restrict__ p_old,
                                             T* __restrict__ p_new, int64_t n, int kp, int slots, ColState st) {
    constexpr int W = Vec16<T>::W;
    const int tpv = kp / W;
    const int t = threadIdx.x % tpv, slot = threadIdx.x / tpv, c0 = t * W;
    bool run[W];
    bool anyrun = false, anyact = false;
    T beta[W];
#pragma unroll
    for (int u = 0; u < W; ++u) {
        run[u] = running(st, c0 + u);
        anyrun = anyrun || run[u];
        anyact = anyact || st.active[c0 + u] != 0;
        beta[u] = run[u] ? enarrow<T>(st.beta[c0 + u]) : ezero<T>();
    }
    if (anyrun) {
#pragma unroll 2
        VOXEL_LOOP(v) {
            const int64_t e = v * kp + c0;
            const V16<T> rv = ld16(r + e);
            V16<T> pv = ld16(p_old + e);
            const T dv = op.dinv[v];
#pragma unroll
            for (int u = 0; u < W; ++u)
                if (run[u]) pv.e[u] = eadd(emul(dv, rv.e[u]), emul(beta[u], pv.e[u]));
            st16(p_new + e, pv);
        }
    } else if (anyact) {
        VOXEL_LOOP(v) {
            const int64_t e = v * kp + c0;
            st16(p_new + e, ld16(p_old + e));
        }
    }
}

// x~ += sum_j alpha_j p_j over the H slots of the direction ring, in iteration order
// (the same sequence of roundings as adding each correction when it is made).  A
// slot whose alpha is 0 (the column did not run in that iteration) adds nothing: its
// value is selected away after the load, never multiplied, so a slot that was never
// written for a column cannot reach x~.  When every slot holds a correction for one
// of the thread's columns (the common case) all H loads are issued back to back.
template <typename T, int H, int MT>
__global__ void __launch_bounds__(MT, MT == 256 ? 2 : 1) k_flush(const T* __restrict__ ring, int64_t slot_elems,
                                               T* __restrict__ x, int64_t n, int kp, int slots, ColState st) {
    constexpr int W = Vec16<T>::W;
    const int tpv = kp / W;
    const int t = threadIdx.x % tpv, slot = threadIdx.x / tpv, c0 = t * W;
    static_assert(H * W <= 32, "one mask bit per (slot, column)");
    T al[H][W];
    unsigned on = 0;   // bit j W + u: column c0 + u has a correction in slot j
    unsigned use = 0;  // bit j: some column of this thread has a correction in slot j
#pragma unroll
    for (int j = 0; j < H; ++j) {
#pragma unroll
        for (int u = 0; u < W; ++u) {
            const double2 a = st.alpha_hist[(int64_t)j * kp + c0 + u];
            al[j][u] = enarrow<T>(a);
            if (a.x != 0.0 || a.y != 0.0) {
                on |= 1u << (j * W + u);
                use |= 1u << j;
            }
        }
    }
    if (!use) return;
    VOXEL_LOOP(v) {
        const int64_t e = v * kp + c0;
        V16<T> xv = ld16(x + e);
        V16<T> pv[H];
        if (use == (1u << H) - 1u) {
#pragma unroll
            for (int j = 0; j < H; ++j) pv[j] = ld16(ring + j * slot_elems + e);
        } else {
#pragma unroll
            for (int j = 0; j < H; ++j)
                if (use & (1u << j)) pv[j] = ld16(ring + j * slot_elems + e);
        }
#pragma unroll
        for (int j = 0; j < H; ++j)
#pragma unroll
            for (int u = 0; u < W; ++u)
                if (on & (1u << (j * W + u))) xv.e[u] = eadd(xv.e[u], emul(al[j][u], pv[j].e[u]));
        st16(x + e, xv);
    }
}

// ------------------------------------------------------------ reliable update
// x64 += s x~, x~ = 0 on the active columns (every column when all != 0).  Runs
// between batches, after the flush of the direction ring, so x~ holds every
// correction made so far.
template <typename T64, typename T>
__global__ void __launch_bounds__(1024) k_promote(T64* __restrict__ x64, T* __restrict__ x, int64_t n, int kp, int slots, ColState st,
                          int all) {
    const int c = threadIdx.x % kp, slot = threadIdx.x / kp;
    if (!(all || st.active[c])) return;
    const double s = st.scale[c];
    VOXEL_LOOP(v) {
        const int64_t e = v * kp + c;
        const double2 d = ewide(x[e]);
        x64[e] = eadd(x64[e], enarrow<T64>(make_double2(s * d.x, s * d.y)));
        x[e] = ezero<T>();
    }
}

// r64 = b - A x64 in FP64 on the active columns (every column when all != 0).  A
// refresh round serves every active column at once, so the columns that asked for it
// and those close to asking share one round of launches (refreshing a column early is
// always valid); the pass is bound by the FP64 pipe, 16 fused multiply-adds per complex
// element.
// Finaliser (update mode): converged when ||r64|| <= rtol ||b||, stopped when the
// iteration budget is spent, otherwise the new scale s' = ||r64||, ratio = s / s',
// and the scaled target tol2 = rtol^2 ||b||^2 / s'^2.
// acc + s a for a real scalar s, one fused multiply-add per component.
__device__ __forceinline__ double eaxpy(double s, double a, double acc) { return __fma_rn(s, a, acc); }
__device__ __forceinline__ double2 eaxpy(double s, double2 a, double2 acc) {
    return make_double2(__fma_rn(s, a.x, acc.x), __fma_rn(s, a.y, acc.y));
}

// acc - i w x (complex); nothing in real arithmetic, where A has no frequency term.
__device__ __forceinline__ double sub_iw(double, double, double acc) { return acc; }
__device__ __forceinline__ double2 sub_iw(double w, double2 x, double2 acc) {
    return make_double2(__fma_rn(w, x.y, acc.x), __fma_rn(-w, x.x, acc.y));
}

// r = b - A x at voxel v, column c, folded into fused multiply-adds that start from b:
// 8 (real) or 16 (complex) FP64 FMAs per element, the least the FP64 pipe can do.
template <typename T>
__device__ __forceinline__ T residual_at(const Op<T>& op, const T* __restrict__ b, const T* __restrict__ x, int64_t v,
                                         int kp, int c) {
    const int vi = (int)v;  // grids hold fewer than 2^31 cells
    const int nxy = op.nx * op.ny;
    const int kz = vi / nxy;
    const int rem = vi - kz * nxy;
    const int j = rem / op.nx;
    const int i = rem - j * op.nx;
    const int64_t e = v * kp + c;
    const Cf4<double> cv = op.cf[vi];
    const T xc = x[e];
    T r = sub_iw(op.w, xc, eaxpy(-cv.dre, xc, b[e]));
    if (i > 0)          r = eaxpy(op.cf[vi - 1].cx, x[e - kp], r);
    if (i < op.nx - 1)  r = eaxpy(cv.cx, x[e + kp], r);
    if (j > 0)          r = eaxpy(op.cf[vi - op.nx].cy, x[e - (int64_t)op.nx * kp], r);
    if (j < op.ny - 1)  r = eaxpy(cv.cy, x[e + (int64_t)op.nx * kp], r);
    if (kz > 0)         r = eaxpy(op.cf[vi - nxy].cz, x[e - (int64_t)nxy * kp], r);
    if (kz < op.nz - 1) r = eaxpy(cv.cz, x[e + (int64_t)nxy * kp], r);
    return r;
}

template <typename T64>
__global__ void __launch_bounds__(1024) k_true_residual(Op<T64> op, const T64* __restrict__ b, const T64* __restrict__ x64,
                                T64* __restrict__ r64, int64_t n, int kp, int slots, ColState st, double rtol,
                                int maxit, int all) {
    const int c = threadIdx.x % kp, slot = threadIdx.x / kp;
    const bool sel = all ? true : (st.active[c] != 0);
    double rr = 0.0;
    if (sel) {
        // two cells in flight per thread: their neighbour loads overlap, which keeps the
        // FP64 pipe fed (the sum of |r|^2 keeps its per-thread order)
#pragma unroll 2
        VOXEL_LOOP(v) {
            const int64_t e = v * kp + c;
            const T64 rv = residual_at(op, b, x64, v, kp, c);
            r64[e] = rv;
            rr += (double)eabs2(rv);
        }
    }
    column_partials(make_double2(0.0, 0.0), rr, kp, slots, c, slot, nullptr, st.partB);
    const double2* totA;
    const double* totB;
    if (reduce_columns(st, false, true, kp, smem_raw, &totA, &totB)) {
        for (int cc = threadIdx.x; cc < kp; cc += blockDim.x) {
            const bool s2 = all ? true : (st.active[cc] != 0);
            if (!s2) continue;
            const double2 a = totA[cc];
            const double rsum = totB[cc];
            st.rr64[cc] = rsum;
            if (all) continue;
            st.updates[cc] += 1;
            if (!isfinite(rsum)) {
                st.status[cc] = DOT_EBREAKDOWN;
                st.active[cc] = 0;
                st.upd[cc] = 0;
            } else if (rsum <= rtol * rtol * st.bb64[cc]) {
                st.status[cc] = DOT_OK;
                st.active[cc] = 0;
                st.upd[cc] = 0;
            } else if (st.iters[cc] >= maxit) {
                st.status[cc] = DOT_ENOTCONV;
                st.active[cc] = 0;
                st.upd[cc] = 0;
            } else {
                const double snew = sqrt(rsum);
                st.ratio[cc] = st.scale[cc] / snew;
                st.scale[cc] = snew;
                st.tol2[cc] = rtol * rtol * st.bb64[cc] / rsum;
            }
        }
        __syncthreads();
        publish_counts(st, kp);
    }
}

// r~ = r64 / s' on the refreshed (active) columns; rho' = r~^T M^{-1} r~.  The search
// direction is kept in the old scale, so beta = (rho' / rho_prev) / ratio carries it
// over, where rho_prev is the rho of the iteration that produced the replaced residual.
template <typename T, typename T64>
__global__ void __launch_bounds__(1024) k_refresh(Op<T> op, const T64* __restrict__ r64, T* __restrict__ r, int64_t n, int kp, int slots,
                          ColState st) {
    using R = typename Elem<T>::R;
    const int c = threadIdx.x % kp, slot = threadIdx.x / kp;
    const bool sel = st.active[c] != 0;
    T rho = ezero<T>();
    R rr = 0;
    if (sel) {
        // scale after narrowing: in FP32 the product then runs on the FP32 pipe (this
        // part's FP64 pipe is about 58 times slower); in FP64 it is the same operation
        const R inv = (R)(1.0 / st.scale[c]);
        VOXEL_LOOP(v) {
            const int64_t e = v * kp + c;
            const T rv = escale(inv, enarrow<T>(ewide(r64[e])));
            r[e] = rv;
            rho = eadd(rho, emul(rv, emul(op.dinv[v], rv)));
            rr += eabs2(rv);
        }
    }
    column_partials(ewide(rho), (double)rr, kp, slots, c, slot, st.partA, st.partB);
    const double2* totA;
    const double* totB;
    if (reduce_columns(st, true, true, kp, smem_raw, &totA, &totB)) {
        for (int cc = threadIdx.x; cc < kp; cc += blockDim.x) {
            if (!st.active[cc]) continue;
            const double2 a = totA[cc];
            const double rsum = totB[cc];
            st.upd[cc] = 0;
            const double2 rho_old = st.rho_prev[cc];
            if (!zfinite(a) || !isfinite(rsum) || (rho_old.x == 0.0 && rho_old.y == 0.0)) {
                st.status[cc] = DOT_EBREAKDOWN;
                st.active[cc] = 0;
                continue;
            }
            const double2 bq = zdiv(a, rho_old);
            const double inv_ratio = 1.0 / st.ratio[cc];
            st.beta[cc] = make_double2(bq.x * inv_ratio, bq.y * inv_ratio);
            st.rho[cc] = a;
            st.rr[cc] = rsum;
            st.maxr[cc] = sqrt(rsum);
            st.since[cc] = 0;
        }
        __syncthreads();
        publish_counts(st, kp);
    }
}

template <typename T>
__global__ void k_apply(Op<T> op, const T* __restrict__ x, T* __restrict__ y, int64_t n, int kp) {
    const int64_t total = n * kp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        y[e] = apply_at(op, x, e / kp, kp, (int)(e % kp));
    }
}

// ------------------------------------------------------------------ dispatch
template <typename T>
static Op<T> make_op(const OpRaw& o) {
    using R = typename Elem<T>::R;
    Op<T> op;
    op.cf = static_cast<const Cf4<R>*>(o.cf);
    op.dinv = static_cast<const T*>(o.dinv);
    op.w = (R)o.w;
    op.nx = o.nx;
    op.ny = o.ny;
    op.nz = o.nz;
    return op;
}

// (inner, outer) element-type pairs
#define DOT_DISPATCH2(ek, ...)                                                          \
    switch (ek) {                                                                       \
        case EK_F64: { using T = double; using T64 = double; __VA_ARGS__; } break;      \
        case EK_C128: { using T = double2; using T64 = double2; __VA_ARGS__; } break;   \
        case EK_F32: { using T = float; using T64 = double; __VA_ARGS__; } break;       \
        case EK_C64: { using T = float2; using T64 = double2; __VA_ARGS__; } break;     \
        default: return cudaErrorInvalidValue;                                          \
    }

static int grid_elems(int64_t total, int cap) {
    int64_t b = (total + 255) / 256;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

cudaError_t solve_start(ElemKind inner, const OpRaw& o, const void* b64, void* x64, void* x, void* r, void* p,
                        int64_t n, int kp, const ColState& st, double rtol, const Launch& L, cudaStream_t s) {
    DOT_DISPATCH2(inner, {
        k_start_norm<T64><<<L.grid, L.threads, red_smem(L, kp), s>>>((const T64*)b64, (T64*)x64, n, kp, L.slots, st,
                                                                     rtol);
        k_start_inner<T, T64><<<L.grid, L.threads, red_smem(L, kp), s>>>(make_op<T>(o), (const T64*)b64, (T*)x,
                                                                         (T*)r, (T*)p, n, kp, L.slots, st);
    });
    return cudaGetLastError();
}

// Timing events around the launches of one iteration.  Inside a stream capture a plain
// record only orders work, so the capture records them as event nodes of the graph
// instead; every replay then records them like a direct launch would.
static void record_timing(cudaEvent_t ev, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    if (cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
    else
        cudaEventRecord(ev, s);
}

cudaError_t kry_step(ElemKind inner, const OpRaw& o, void* x, void* r, const DirRing& ring, int m, void* q,
                     int64_t n, int kp, const ColState& st, double delta, int maxit, bool with_p, const Launch& Lv,
                     const TmaStencil* tma, cudaStream_t s, cudaEvent_t* ev, cudaEvent_t* evf) {
    const int H = ring.H;
    const int slot = m % H, prev = (slot + H - 1) % H;
    DOT_DISPATCH2(inner, {
        Op<T> op = make_op<T>(o);
        const size_t sm = red_smem(Lv, kp);
        T* base = static_cast<T*>(ring.base);
        T* p_new = base + slot * ring.slot_elems;
        const T* p_old = base + prev * ring.slot_elems;
        // blocks wider than 256 threads (one column per thread at block widths above
        // 256 x the vector width) take the instantiations compiled for 1024 threads
        const bool wide = Lv.threads > 256;
        // the direction update fused into the TMA stencil: one launch streams r~ and the
        // old direction in and the new direction and q out
        const bool fused = with_p && tma && tma->fused;
        if (ev) record_timing(ev[0], s);
        if (with_p && !fused) {
            if (wide)
                k_dir<T, 1024><<<Lv.grid, Lv.threads, 0, s>>>(op, (const T*)r, p_old, p_new, n, kp, Lv.slots, st);
            else
                k_dir<T, 256><<<Lv.grid, Lv.threads, 0, s>>>(op, (const T*)r, p_old, p_new, n, kp, Lv.slots, st);
        }
        if (ev) record_timing(ev[1], s);
        if (fused) {
            const cudaError_t e = dpq_launch(inner, o, *tma, ring, slot, prev, q, kp, st, s);
            if (e != cudaSuccess) return e;
        } else if (tma) {
            const cudaError_t e = tma_stencil_launch(inner, o, *tma, slot, q, kp, st, s);
            if (e != cudaSuccess) return e;
        } else if (wide) {
            k_pq<T, 1024><<<Lv.grid, Lv.threads, sm, s>>>(op, p_new, (T*)q, kp, Lv.slots, st, slot);
        } else {
            k_pq<T, 256><<<Lv.grid, Lv.threads, sm, s>>>(op, p_new, (T*)q, kp, Lv.slots, st, slot);
        }
        if (ev) record_timing(ev[2], s);
        if (wide)
            k_r<T, 1024><<<Lv.grid, Lv.threads, sm, s>>>(op, (const T*)q, (T*)r, n, kp, Lv.slots, st, delta, maxit);
        else
            k_r<T, 256><<<Lv.grid, Lv.threads, sm, s>>>(op, (const T*)q, (T*)r, n, kp, Lv.slots, st, delta, maxit);
        if (ev) record_timing(ev[3], s);
        if (slot == H - 1) {
            const T* rb = base;
            const int64_t se = ring.slot_elems;
            const int fg = ring.flush_grid > 0 ? ring.flush_grid : Lv.grid;
            if (wide) {
                if (H == 8)
                    k_flush<T, 8, 1024><<<fg, Lv.threads, 0, s>>>(rb, se, (T*)x, n, kp, Lv.slots, st);
                else if (H == 4)
                    k_flush<T, 4, 1024><<<fg, Lv.threads, 0, s>>>(rb, se, (T*)x, n, kp, Lv.slots, st);
                else
                    k_flush<T, 2, 1024><<<fg, Lv.threads, 0, s>>>(rb, se, (T*)x, n, kp, Lv.slots, st);
            } else {
                if (H == 8)
                    k_flush<T, 8, 256><<<fg, Lv.threads, 0, s>>>(rb, se, (T*)x, n, kp, Lv.slots, st);
                else if (H == 4)
                    k_flush<T, 4, 256><<<fg, Lv.threads, 0, s>>>(rb, se, (T*)x, n, kp, Lv.slots, st);
                else
                    k_flush<T, 2, 256><<<fg, Lv.threads, 0, s>>>(rb, se, (T*)x, n, kp, Lv.slots, st);
            }
            if (evf) record_timing(*evf, s);
        }
        (void)sizeof(T64);
    });
    return cudaGetLastError();
}

int vector_width(ElemKind inner) {
    switch (inner) {
        case EK_F32: return 4;
        case EK_C64: return 2;
        case EK_F64: return 2;
        default: return 1;
    }
}

cudaError_t solve_refresh(ElemKind inner, const OpRaw& o, const OpRaw& o64, const void* b64, void* x64, void* r64,
                          void* x, void* r, int64_t n, int kp, const ColState& st, double rtol, int maxit,
                          const Launch& L, int num_sms, cudaStream_t s) {
    (void)num_sms;
    DOT_DISPATCH2(inner, {
        k_promote<T64, T><<<L.grid, L.threads, 0, s>>>((T64*)x64, (T*)x, n, kp, L.slots, st, 0);
        k_true_residual<T64><<<L.grid, L.threads, red_smem(L, kp), s>>>(make_op<T64>(o64), (const T64*)b64,
                                                                        (const T64*)x64, (T64*)r64, n, kp, L.slots,
                                                                        st, rtol, maxit, 0);
        k_refresh<T, T64><<<L.grid, L.threads, red_smem(L, kp), s>>>(make_op<T>(o), (const T64*)r64, (T*)r, n, kp,
                                                                     L.slots, st);
    });
    return cudaGetLastError();
}

cudaError_t solve_finish(ElemKind inner, const OpRaw& o64, const void* b64, void* x64, void* r64, void* x, int64_t n,
                         int kp, const ColState& st, bool residual, const Launch& L, int num_sms, cudaStream_t s) {
    (void)num_sms;
    DOT_DISPATCH2(inner, {
        k_promote<T64, T><<<L.grid, L.threads, 0, s>>>((T64*)x64, (T*)x, n, kp, L.slots, st, 1);
        if (residual)
            k_true_residual<T64><<<L.grid, L.threads, red_smem(L, kp), s>>>(make_op<T64>(o64), (const T64*)b64,
                                                                            (const T64*)x64, (T64*)r64, n, kp,
                                                                            L.slots, st, 0.0, 0, 1);
    });
    return cudaGetLastError();
}

cudaError_t op_apply(ElemKind ek, const OpRaw& o, const void* x, void* y, int64_t n, int kp, cudaStream_t s) {
    const int grid = grid_elems(n * kp, 152 * 16);
    switch (ek) {
        case EK_F64:
            k_apply<double><<<grid, 256, 0, s>>>(make_op<double>(o), (const double*)x, (double*)y, n, kp);
            break;
        case EK_C128:
            k_apply<double2><<<grid, 256, 0, s>>>(make_op<double2>(o), (const double2*)x, (double2*)y, n, kp);
            break;
        case EK_F32:
            k_apply<float><<<grid, 256, 0, s>>>(make_op<float>(o), (const float*)x, (float*)y, n, kp);
            break;
        case EK_C64:
            k_apply<float2><<<grid, 256, 0, s>>>(make_op<float2>(o), (const float2*)x, (float2*)y, n, kp);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace dotk
