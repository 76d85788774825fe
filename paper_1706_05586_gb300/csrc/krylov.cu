// Block Jacobi-preconditioned CG / COCG and FP64 iterative refinement (sm_103a).
//
// k independent Krylov recurrences share one operator A (Sec. 3.3: one block holds
// the l_s forward columns B W and the l_d adjoint columns C V; A is symmetric, or
// complex symmetric when omega != 0, so A^T = A and COCG's bilinear form x^T y
// applies).  The paper leaves the solver open ("iterative solvers or sparse direct
// solvers depending on the size"); this is the iterative choice.
//
// Reductions are deterministic: each block of a persistent grid writes per-column
// partial sums, and the last block to arrive sums them in block order and runs the
// per-column scalar update (alpha, beta, convergence), so no host round trip and
// no floating-point atomics are needed.
#include "dot_kernels.cuh"
#include "dot_internal.h"
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

// -------------------------------------------------------------- block reduction
// Sum per-column values over the block's voxel slots (fixed order) and store the
// block's partial sums.  Then report whether this block arrived last.
__device__ __forceinline__ void column_partials(double2 a, double b, int kp, int slots, int c, int slot,
                                                double2* partA, double* partB) {
    extern __shared__ unsigned char smem_raw[];
    double2* sA = reinterpret_cast<double2*>(smem_raw);
    double* sB = reinterpret_cast<double*>(sA + slots * kp);
    sA[slot * kp + c] = a;
    sB[slot * kp + c] = b;
    __syncthreads();
    if (slot == 0) {
        double2 ta = make_double2(0.0, 0.0);
        double tb = 0.0;
        for (int s = 0; s < slots; ++s) {
            ta.x += sA[s * kp + c].x;
            ta.y += sA[s * kp + c].y;
            tb += sB[s * kp + c];
        }
        if (partA) partA[(int64_t)blockIdx.x * kp + c] = ta;
        if (partB) partB[(int64_t)blockIdx.x * kp + c] = tb;
    }
}

__device__ __forceinline__ bool arrive_last(unsigned* counter) {
    __shared__ int am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(counter, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    return am_last != 0;
}

__device__ __forceinline__ void sum_partials(const double2* partA, const double* partB, int kp, int cc,
                                             double2* a, double* b) {
    double2 ra = make_double2(0.0, 0.0);
    double rb = 0.0;
    for (int g = 0; g < (int)gridDim.x; ++g) {
        if (partA) {
            double2 t = __ldcg(&partA[(int64_t)g * kp + cc]);
            ra.x += t.x;
            ra.y += t.y;
        }
        if (partB) rb += __ldcg(&partB[(int64_t)g * kp + cc]);
    }
    *a = ra;
    *b = rb;
}

// ------------------------------------------------------------------- kernels
// x = 0, r = b, p = z = M^{-1} b; rho = b^T z, bb = ||b||^2.
template <typename T>
__global__ void k_init(Op<T> op, const T* __restrict__ b, T* __restrict__ x, T* __restrict__ r,
                       T* __restrict__ p, int64_t n, int kp, int slots, ColState st) {
    using R = typename Elem<T>::R;
    const int c = threadIdx.x % kp, slot = threadIdx.x / kp;
    T rho = ezero<T>();
    R bb = 0;
    for (int64_t v = (int64_t)blockIdx.x * slots + slot; v < n; v += (int64_t)gridDim.x * slots) {
        const int64_t e = v * kp + c;
        T bv = b[e];
        T z = emul(op.dinv[v], bv);
        x[e] = ezero<T>();
        r[e] = bv;
        p[e] = z;
        rho = eadd(rho, emul(bv, z));
        bb += eabs2(bv);
    }
    column_partials(ewide(rho), (double)bb, kp, slots, c, slot, st.partA, st.partB);
    if (arrive_last(st.counter)) {
        __shared__ int cnt;
        if (threadIdx.x == 0) cnt = 0;
        __syncthreads();
        for (int cc = threadIdx.x; cc < kp; cc += blockDim.x) {
            double2 a;
            double bsum;
            sum_partials(st.partA, st.partB, kp, cc, &a, &bsum);
            st.rho[cc] = a;
            st.bb[cc] = bsum;
            st.rr[cc] = bsum;
            st.beta[cc] = make_double2(0.0, 0.0);
            st.iters[cc] = 0;
            const bool fin = isfinite(bsum) && zfinite(a);
            st.status[cc] = fin ? DOT_OK : DOT_EBREAKDOWN;
            const int act = fin && bsum > 0.0;
            st.active[cc] = act;
            if (act) atomicAdd(&cnt, 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            *st.n_active = cnt;
            *st.counter = 0u;
        }
    }
}

// Correction problem of one refinement step: b32 = r64 / ||r64|| on the columns
// still refining (0 elsewhere), then the same start as k_init.
template <typename T32, typename T64>
__global__ void k_init_from64(Op<T32> op, const T64* __restrict__ r64, RefState rs, T32* __restrict__ x,
                              T32* __restrict__ r, T32* __restrict__ p, int64_t n, int kp, int slots,
                              ColState st) {
    using R = typename Elem<T32>::R;
    const int c = threadIdx.x % kp, slot = threadIdx.x / kp;
    const bool ract = rs.active[c] != 0;
    const double inv = ract ? 1.0 / rs.scale[c] : 0.0;
    T32 rho = ezero<T32>();
    R bb = 0;
    for (int64_t v = (int64_t)blockIdx.x * slots + slot; v < n; v += (int64_t)gridDim.x * slots) {
        const int64_t e = v * kp + c;
        T32 bv = ract ? enarrow<T32>(ewide(escale(inv, r64[e]))) : ezero<T32>();
        T32 z = emul(op.dinv[v], bv);
        x[e] = ezero<T32>();
        r[e] = bv;
        p[e] = z;
        rho = eadd(rho, emul(bv, z));
        bb += eabs2(bv);
    }
    column_partials(ewide(rho), (double)bb, kp, slots, c, slot, st.partA, st.partB);
    if (arrive_last(st.counter)) {
        __shared__ int cnt;
        if (threadIdx.x == 0) cnt = 0;
        __syncthreads();
        for (int cc = threadIdx.x; cc < kp; cc += blockDim.x) {
            double2 a;
            double bsum;
            sum_partials(st.partA, st.partB, kp, cc, &a, &bsum);
            st.rho[cc] = a;
            st.bb[cc] = bsum;
            st.rr[cc] = bsum;
            st.beta[cc] = make_double2(0.0, 0.0);
            st.iters[cc] = 0;
            const bool fin = isfinite(bsum) && zfinite(a);
            st.status[cc] = fin ? DOT_OK : DOT_EBREAKDOWN;
            const int act = fin && bsum > 0.0;
            st.active[cc] = act;
            if (act) atomicAdd(&cnt, 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            *st.n_active = cnt;
            *st.counter = 0u;
        }
    }
}

// q = A p and pq = p^T q; finaliser alpha = rho / pq.
template <typename T>
__global__ void k_pq(Op<T> op, const T* __restrict__ p, T* __restrict__ q, int64_t n, int kp, int slots,
                     ColState st) {
    const int c = threadIdx.x % kp, slot = threadIdx.x / kp;
    const bool act = st.active[c] != 0;
    T pq = ezero<T>();
    if (act) {
        for (int64_t v = (int64_t)blockIdx.x * slots + slot; v < n; v += (int64_t)gridDim.x * slots) {
            const int64_t e = v * kp + c;
            T qv = apply_at(op, p, v, kp, c);
            q[e] = qv;
            pq = eadd(pq, emul(p[e], qv));
        }
    }
    column_partials(ewide(pq), 0.0, kp, slots, c, slot, st.partA, nullptr);
    if (arrive_last(st.counter)) {
        __shared__ int cnt;
        if (threadIdx.x == 0) cnt = 0;
        __syncthreads();
        for (int cc = threadIdx.x; cc < kp; cc += blockDim.x) {
            if (!st.active[cc]) continue;
            double2 a;
            double unused;
            sum_partials(st.partA, nullptr, kp, cc, &a, &unused);
            if (!zfinite(a) || (a.x == 0.0 && a.y == 0.0)) {
                st.status[cc] = DOT_EBREAKDOWN;
                st.active[cc] = 0;
                continue;
            }
            st.alpha[cc] = zdiv(st.rho[cc], a);
            atomicAdd(&cnt, 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            *st.n_active = cnt;
            *st.counter = 0u;
        }
    }
}

// x += alpha p, r -= alpha q, rho' = r^T M^{-1} r, ||r||^2; finaliser: convergence
// test ||r|| <= rtol ||b||, then beta = rho' / rho.
template <typename T>
__global__ void k_xr(Op<T> op, const T* __restrict__ p, const T* __restrict__ q, T* __restrict__ x,
                     T* __restrict__ r, int64_t n, int kp, int slots, ColState st, double rtol, int maxit) {
    using R = typename Elem<T>::R;
    const int c = threadIdx.x % kp, slot = threadIdx.x / kp;
    const bool act = st.active[c] != 0;
    T rho = ezero<T>();
    R rr = 0;
    if (act) {
        const T alpha = enarrow<T>(st.alpha[c]);
        for (int64_t v = (int64_t)blockIdx.x * slots + slot; v < n; v += (int64_t)gridDim.x * slots) {
            const int64_t e = v * kp + c;
            T xv = eadd(x[e], emul(alpha, p[e]));
            T rv = esub(r[e], emul(alpha, q[e]));
            x[e] = xv;
            r[e] = rv;
            T z = emul(op.dinv[v], rv);
            rho = eadd(rho, emul(rv, z));
            rr += eabs2(rv);
        }
    }
    column_partials(ewide(rho), (double)rr, kp, slots, c, slot, st.partA, st.partB);
    if (arrive_last(st.counter)) {
        __shared__ int cnt;
        if (threadIdx.x == 0) cnt = 0;
        __syncthreads();
        for (int cc = threadIdx.x; cc < kp; cc += blockDim.x) {
            if (!st.active[cc]) continue;
            double2 a;
            double rsum;
            sum_partials(st.partA, st.partB, kp, cc, &a, &rsum);
            const int it = st.iters[cc] + 1;
            st.iters[cc] = it;
            st.rr[cc] = rsum;
            if (!isfinite(rsum) || !zfinite(a)) {
                st.status[cc] = DOT_EBREAKDOWN;
                st.active[cc] = 0;
                continue;
            }
            if (rsum <= rtol * rtol * st.bb[cc]) {
                st.status[cc] = DOT_OK;
                st.active[cc] = 0;
                continue;
            }
            if (it >= maxit) {
                st.status[cc] = DOT_ENOTCONV;
                st.active[cc] = 0;
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
            atomicAdd(&cnt, 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            *st.n_active = cnt;
            *st.counter = 0u;
        }
    }
}

// p = M^{-1} r + beta p
template <typename T>
__global__ void k_p(Op<T> op, const T* __restrict__ r, T* __restrict__ p, int64_t n, int kp, int slots,
                    ColState st) {
    const int c = threadIdx.x % kp, slot = threadIdx.x / kp;
    if (!st.active[c]) return;
    const T beta = enarrow<T>(st.beta[c]);
    for (int64_t v = (int64_t)blockIdx.x * slots + slot; v < n; v += (int64_t)gridDim.x * slots) {
        const int64_t e = v * kp + c;
        p[e] = eadd(emul(op.dinv[v], r[e]), emul(beta, p[e]));
    }
}

// ---------------------------------------------------------- FP64 refinement
template <typename T>
__global__ void k_ref_init(const T* __restrict__ b, T* __restrict__ x, T* __restrict__ r, int64_t n, int kp,
                           int slots, RefState rs) {
    const int c = threadIdx.x % kp, slot = threadIdx.x / kp;
    double bb = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * slots + slot; v < n; v += (int64_t)gridDim.x * slots) {
        const int64_t e = v * kp + c;
        T bv = b[e];
        x[e] = ezero<T>();
        r[e] = bv;
        bb += (double)eabs2(bv);
    }
    column_partials(make_double2(0.0, 0.0), bb, kp, slots, c, slot, nullptr, rs.partB);
    if (arrive_last(rs.counter)) {
        __shared__ int cnt;
        if (threadIdx.x == 0) cnt = 0;
        __syncthreads();
        for (int cc = threadIdx.x; cc < kp; cc += blockDim.x) {
            double2 a;
            double bsum;
            sum_partials(nullptr, rs.partB, kp, cc, &a, &bsum);
            rs.bb[cc] = bsum;
            rs.rr[cc] = bsum;
            rs.scale[cc] = sqrt(bsum);
            const int act = isfinite(bsum) && bsum > 0.0;
            rs.active[cc] = act;
            if (act) atomicAdd(&cnt, 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            *rs.n_active = cnt;
            *rs.counter = 0u;
        }
    }
}

// r = b - A x in FP64 on the columns still refining; finaliser: stop a column when
// ||r|| <= rtol ||b||, else record ||r|| as the next correction's scale.
template <typename T>
__global__ void k_ref_resid(Op<T> op, const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ r,
                            int64_t n, int kp, int slots, RefState rs, double rtol) {
    const int c = threadIdx.x % kp, slot = threadIdx.x / kp;
    const bool act = rs.active[c] != 0;
    double rr = 0.0;
    if (act) {
        for (int64_t v = (int64_t)blockIdx.x * slots + slot; v < n; v += (int64_t)gridDim.x * slots) {
            const int64_t e = v * kp + c;
            T rv = esub(b[e], apply_at(op, x, v, kp, c));
            r[e] = rv;
            rr += (double)eabs2(rv);
        }
    }
    column_partials(make_double2(0.0, 0.0), rr, kp, slots, c, slot, nullptr, rs.partB);
    if (arrive_last(rs.counter)) {
        __shared__ int cnt;
        if (threadIdx.x == 0) cnt = 0;
        __syncthreads();
        for (int cc = threadIdx.x; cc < kp; cc += blockDim.x) {
            if (!rs.active[cc]) continue;
            double2 a;
            double rsum;
            sum_partials(nullptr, rs.partB, kp, cc, &a, &rsum);
            rs.rr[cc] = rsum;
            if (!isfinite(rsum) || rsum <= rtol * rtol * rs.bb[cc]) {
                rs.active[cc] = 0;
                continue;
            }
            rs.scale[cc] = sqrt(rsum);
            atomicAdd(&cnt, 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            *rs.n_active = cnt;
            *rs.counter = 0u;
        }
    }
}

template <typename T64, typename T32>
__global__ void k_ref_promote(T64* __restrict__ x64, const T32* __restrict__ x32, int64_t n, int kp, RefState rs) {
    const int64_t total = n * kp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % kp);
        if (!rs.active[c]) continue;
        const double s = rs.scale[c];
        double2 d = ewide(x32[e]);
        T64 add = enarrow<T64>(make_double2(s * d.x, s * d.y));
        x64[e] = eadd(x64[e], add);
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
    op.cx = static_cast<const R*>(o.cx);
    op.cy = static_cast<const R*>(o.cy);
    op.cz = static_cast<const R*>(o.cz);
    op.dre = static_cast<const R*>(o.dre);
    op.dinv = static_cast<const T*>(o.dinv);
    op.w = (R)o.w;
    op.nx = o.nx;
    op.ny = o.ny;
    op.nz = o.nz;
    return op;
}

#define DOT_DISPATCH(ek, ...)                                         \
    switch (ek) {                                                     \
        case EK_F64: { using T = double; __VA_ARGS__; } break;        \
        case EK_C128: { using T = double2; __VA_ARGS__; } break;      \
        case EK_F32: { using T = float; __VA_ARGS__; } break;         \
        case EK_C64: { using T = float2; __VA_ARGS__; } break;        \
        default: return cudaErrorInvalidValue;                        \
    }

cudaError_t kry_init(ElemKind ek, const OpRaw& o, const void* b, void* x, void* r, void* p, int64_t n, int kp,
                     const ColState& st, const Launch& L, cudaStream_t s) {
    DOT_DISPATCH(ek, (k_init<T><<<L.grid, L.threads, red_smem(L, kp), s>>>(
                          make_op<T>(o), (const T*)b, (T*)x, (T*)r, (T*)p, n, kp, L.slots, st)));
    return cudaGetLastError();
}

cudaError_t kry_init_from64(ElemKind ek32, const OpRaw& o, const void* r64, const RefState& rs, void* x,
                            void* r, void* p, int64_t n, int kp, const ColState& st, const Launch& L,
                            cudaStream_t s) {
    if (ek32 == EK_F32)
        k_init_from64<float, double><<<L.grid, L.threads, red_smem(L, kp), s>>>(
            make_op<float>(o), (const double*)r64, rs, (float*)x, (float*)r, (float*)p, n, kp, L.slots, st);
    else if (ek32 == EK_C64)
        k_init_from64<float2, double2><<<L.grid, L.threads, red_smem(L, kp), s>>>(
            make_op<float2>(o), (const double2*)r64, rs, (float2*)x, (float2*)r, (float2*)p, n, kp, L.slots, st);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t kry_iteration(ElemKind ek, const OpRaw& o, void* x, void* r, void* p, void* q, int64_t n, int kp,
                          const ColState& st, double rtol, int maxit, const Launch& L, cudaStream_t s,
                          cudaEvent_t* ev) {
    DOT_DISPATCH(ek, {
        Op<T> op = make_op<T>(o);
        if (ev) cudaEventRecord(ev[0], s);
        k_pq<T><<<L.grid, L.threads, red_smem(L, kp), s>>>(op, (const T*)p, (T*)q, n, kp, L.slots, st);
        if (ev) cudaEventRecord(ev[1], s);
        k_xr<T><<<L.grid, L.threads, red_smem(L, kp), s>>>(op, (const T*)p, (const T*)q, (T*)x, (T*)r, n, kp,
                                                            L.slots, st, rtol, maxit);
        if (ev) cudaEventRecord(ev[2], s);
        k_p<T><<<L.grid, L.threads, 0, s>>>(op, (const T*)r, (T*)p, n, kp, L.slots, st);
        if (ev) cudaEventRecord(ev[3], s);
    });
    return cudaGetLastError();
}

cudaError_t ref_init(ElemKind ek64, const void* b, void* x, void* r, int64_t n, int kp, const RefState& rs,
                     const Launch& L, cudaStream_t s) {
    if (ek64 == EK_F64)
        k_ref_init<double><<<L.grid, L.threads, red_smem(L, kp), s>>>((const double*)b, (double*)x, (double*)r, n,
                                                                      kp, L.slots, rs);
    else if (ek64 == EK_C128)
        k_ref_init<double2><<<L.grid, L.threads, red_smem(L, kp), s>>>((const double2*)b, (double2*)x,
                                                                       (double2*)r, n, kp, L.slots, rs);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t ref_residual(ElemKind ek64, const OpRaw& o, const void* b, const void* x, void* r, int64_t n, int kp,
                         const RefState& rs, double rtol, const Launch& L, cudaStream_t s) {
    if (ek64 == EK_F64)
        k_ref_resid<double><<<L.grid, L.threads, red_smem(L, kp), s>>>(make_op<double>(o), (const double*)b,
                                                                       (const double*)x, (double*)r, n, kp,
                                                                       L.slots, rs, rtol);
    else if (ek64 == EK_C128)
        k_ref_resid<double2><<<L.grid, L.threads, red_smem(L, kp), s>>>(make_op<double2>(o), (const double2*)b,
                                                                        (const double2*)x, (double2*)r, n, kp,
                                                                        L.slots, rs, rtol);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t ref_promote(ElemKind ek64, ElemKind ek32, void* x64, const void* x32, int64_t n, int kp,
                        const RefState& rs, const Launch& L, cudaStream_t s) {
    const int threads = 256;
    int64_t blocks = (n * kp + threads - 1) / threads;
    int grid = (int)(blocks < (int64_t)L.grid * 4 ? blocks : (int64_t)L.grid * 4);
    if (grid < 1) grid = 1;
    if (ek64 == EK_F64 && ek32 == EK_F32)
        k_ref_promote<double, float><<<grid, threads, 0, s>>>((double*)x64, (const float*)x32, n, kp, rs);
    else if (ek64 == EK_C128 && ek32 == EK_C64)
        k_ref_promote<double2, float2><<<grid, threads, 0, s>>>((double2*)x64, (const float2*)x32, n, kp, rs);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t op_apply(ElemKind ek, const OpRaw& o, const void* x, void* y, int64_t n, int kp, cudaStream_t s) {
    const int threads = 256;
    int64_t blocks = (n * kp + threads - 1) / threads;
    int grid = (int)(blocks < 152 * 16 ? blocks : 152 * 16);
    if (grid < 1) grid = 1;
    DOT_DISPATCH(ek, (k_apply<T><<<grid, threads, 0, s>>>(make_op<T>(o), (const T*)x, (T*)y, n, kp)));
    return cudaGetLastError();
}

}  // namespace dotk
