// Deterministic per-column reductions shared by the Krylov kernels (device code only).
#pragma once

#include "dot.h"
#include "dot_kernels.cuh"
#include "dot_internal.h"

namespace dotk {

// Dynamic shared memory of the kernel being compiled.
extern __shared__ __align__(16) unsigned char smem_raw[];

// -------------------------------------------------------------- block reduction
// Sum per-column values over the block's voxel slots (fixed order) and store the
// block's partial sums.
static __device__ __forceinline__ void column_partials(double2 a, double b, int kp, int slots, int c, int slot,
                                                double2* partA, double* partB) {
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

// Totals of G per-block partial sums (rows of kp), computed by every thread of one
// block (scratch: shared memory of at least (blockDim / kp, >= 1) * kp * 24 bytes):
// tpc = blockDim / kp threads share a column, each summing a fixed strided subset of
// the rows with four independent accumulators, and the subsets are combined in a
// fixed order, so the result does not depend on scheduling.  Returns pointers to the
// kp totals in shared memory (valid until the next call or the block's exit); a
// null input gives zeros.
static __device__ __noinline__ void block_sums(const double2* partA, const double* partB, int kp, int G,
                                               void* scratch, const double2** outA, const double** outB) {
    double2* sA = reinterpret_cast<double2*>(scratch);
    const int tpc = max(1, (int)blockDim.x / kp);
    double* sB = reinterpret_cast<double*>(sA + tpc * kp);
    for (int t = threadIdx.x; t < kp * tpc; t += blockDim.x) {
        const int cc = t % kp, q = t / kp;
        // two passes with four independent accumulators each keep the register
        // footprint of this rarely-run code below that of the kernels' main loops
        double2 ta = make_double2(0.0, 0.0);
        if (partA) {
            double2 a0 = ta, a1 = ta, a2 = ta, a3 = ta;
            int g = q;
            for (; g + 3 * tpc < G; g += 4 * tpc) {
                const double2 x0 = __ldcg(&partA[(int64_t)g * kp + cc]);
                const double2 x1 = __ldcg(&partA[(int64_t)(g + tpc) * kp + cc]);
                const double2 x2 = __ldcg(&partA[(int64_t)(g + 2 * tpc) * kp + cc]);
                const double2 x3 = __ldcg(&partA[(int64_t)(g + 3 * tpc) * kp + cc]);
                a0.x += x0.x; a0.y += x0.y;
                a1.x += x1.x; a1.y += x1.y;
                a2.x += x2.x; a2.y += x2.y;
                a3.x += x3.x; a3.y += x3.y;
            }
            for (; g < G; g += tpc) {
                const double2 x0 = __ldcg(&partA[(int64_t)g * kp + cc]);
                a0.x += x0.x;
                a0.y += x0.y;
            }
            ta = make_double2((a0.x + a1.x) + (a2.x + a3.x), (a0.y + a1.y) + (a2.y + a3.y));
        }
        double tb = 0.0;
        if (partB) {
            double b0 = 0.0, b1 = 0.0, b2 = 0.0, b3 = 0.0;
            int g = q;
            for (; g + 3 * tpc < G; g += 4 * tpc) {
                b0 += __ldcg(&partB[(int64_t)g * kp + cc]);
                b1 += __ldcg(&partB[(int64_t)(g + tpc) * kp + cc]);
                b2 += __ldcg(&partB[(int64_t)(g + 2 * tpc) * kp + cc]);
                b3 += __ldcg(&partB[(int64_t)(g + 3 * tpc) * kp + cc]);
            }
            for (; g < G; g += tpc) b0 += __ldcg(&partB[(int64_t)g * kp + cc]);
            tb = (b0 + b1) + (b2 + b3);
        }
        sA[q * kp + cc] = ta;
        sB[q * kp + cc] = tb;
    }
    __syncthreads();
    for (int cc = threadIdx.x; cc < kp; cc += blockDim.x) {
        for (int q = 1; q < tpc; ++q) {
            sA[cc].x += sA[q * kp + cc].x;
            sA[cc].y += sA[q * kp + cc].y;
            sB[cc] += sB[q * kp + cc];
        }
    }
    __syncthreads();
    *outA = sA;
    *outB = sB;
}

// Deterministic two-level reduction of the per-block partial sums (st.partA /
// st.partB, as selected by useA / useB) after every block has written its own.
// Blocks form groups of kReduceGroup consecutive indices; the last block of a group
// to arrive sums that group's rows into st.groupA / st.groupB, and the last group
// to finish sums the group rows.  Both levels add in a fixed order, so the totals do
// not depend on which block arrives last, and no block reads more than
// max(kReduceGroup, ceil(grid / kReduceGroup)) rows.  Returns true in every thread
// of the one block holding the totals (*outA, *outB in shared memory); that block
// re-arms st.counter through publish_counts, each group block its group counter.
static __device__ __noinline__ bool reduce_columns(const ColState& st, bool useA, bool useB, int kp, void* scratch,
                                                   const double2** outA, const double** outB) {
    __shared__ int is_last;
    const int G = gridDim.x;
    const int g = blockIdx.x / kReduceGroup, ng = (G + kReduceGroup - 1) / kReduceGroup;
    const int g0 = g * kReduceGroup, gs = min(kReduceGroup, G - g0);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(&st.gcount[g], 1u) == (unsigned)(gs - 1);
    __syncthreads();
    if (!is_last) return false;
    const double2* tA;
    const double* tB;
    block_sums(useA ? st.partA + (int64_t)g0 * kp : nullptr, useB ? st.partB + (int64_t)g0 * kp : nullptr, kp, gs,
               scratch, &tA, &tB);
    for (int cc = threadIdx.x; cc < kp; cc += blockDim.x) {
        if (useA) st.groupA[(int64_t)g * kp + cc] = tA[cc];
        if (useB) st.groupB[(int64_t)g * kp + cc] = tB[cc];
    }
    if (threadIdx.x == 0) st.gcount[g] = 0u;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(st.counter, 1u) == (unsigned)(ng - 1);
    __syncthreads();
    if (!is_last) return false;
    block_sums(useA ? st.groupA : nullptr, useB ? st.groupB : nullptr, kp, ng, scratch, outA, outB);
    return true;
}

// Finaliser of the stencil kernels: alpha = rho / p^T q on the running columns
// (breakdown on a zero or non-finite p^T q), and row hslot of the step-length
// history records alpha, 0 for every column that did not take this iteration.
static __device__ __noinline__ void stencil_finalise(const ColState& st, const double2* totA, int kp, int hslot) {
    for (int cc = threadIdx.x; cc < kp; cc += blockDim.x) {
        double2 al = make_double2(0.0, 0.0);
        if (st.active[cc] && !st.upd[cc]) {
            const double2 a = totA[cc];
            if (!zfinite(a) || (a.x == 0.0 && a.y == 0.0)) {
                st.status[cc] = DOT_EBREAKDOWN;
                st.active[cc] = 0;
            } else {
                al = zdiv(st.rho[cc], a);
            }
        }
        st.alpha[cc] = al;
        st.alpha_hist[(int64_t)hslot * kp + cc] = al;
    }
}

// Column counters written by the finalisers: active columns and columns paused for
// a reliable update.  Also re-arms the second-level arrival counter.
static __device__ __forceinline__ void publish_counts(const ColState& st, int kp) {
    __shared__ int na, nu;
    if (threadIdx.x == 0) {
        na = 0;
        nu = 0;
    }
    __syncthreads();
    for (int cc = threadIdx.x; cc < kp; cc += blockDim.x) {
        if (st.active[cc]) {
            atomicAdd(&na, 1);
            if (st.upd[cc]) atomicAdd(&nu, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *st.n_active = na;
        *st.n_update = nu;
        *st.counter = 0u;
    }
}


}  // namespace dotk
