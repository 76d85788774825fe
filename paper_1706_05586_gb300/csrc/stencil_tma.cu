// TMA-staged stencil q = A p with the per-column dot products p^T q (sm_103a).
//
// The 7-point operator of Sec. 2 (Eq. (PDE), Eq. (Eq:compmeas)) is applied to a
// block of right-hand-side columns.  A CTA owns a tile of 8 x 8 cells x KC columns
// (KC = 32, or 16 when the block width is an odd multiple of 16; FP32 blocks whose
// width is a multiple of 64 take KC = 64 with two columns per lane)
// and marches it through a range of z planes.  Each plane of the tile, with a
// one-cell halo in x and y, is brought into shared memory by two
// cp.async.bulk.tensor loads completing on one mbarrier: the p values (4-D tensor
// map over [z][y][x][column]) and the packed face/diagonal coefficients of the
// same cells (4-D map over [z][y][x][4 floats]).  Four planes are in the ring, so
// every element of p crosses L2 once per plane instead of once per neighbour, the
// z neighbours are the adjacent planes of the ring, and the inner loop reads only
// shared memory.  Out-of-range halo cells are zero-filled by the copy engine, p and
// coefficients alike, so boundary faces contribute exact zeros without branches.
// A warp owns one tile row; a lane owns one column (two adjacent FP32 columns in
// 64-column tiles), and with KC = 16 a half-warp owns one cell, so every shared-memory
// read and global store of a warp is one contiguous 256-byte (complex64, FP32 pairs)
// or 128-byte run.
//
// Every wait on an mbarrier is bounded by a clock budget; on expiry the CTA records
// an error code, drains its outstanding copies (again bounded) and stops issuing work.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "dot.h"
#include "dot_kernels.cuh"
#include "dot_internal.h"
#include "dot_reduce.cuh"

namespace dotk {

namespace {

constexpr int TX = 8, TY = 8;        // cells per tile
constexpr int HX = TX + 2, HY = TY + 2;
constexpr int NBUF = 4;              // planes in flight
constexpr int THREADS = 32 * TY;     // warp w <-> tile row y = w
constexpr int CF_BYTES = HX * HY * 16;                    // one plane of packed coefficients
constexpr int CF_SLOT = (CF_BYTES + 127) / 128 * 128;     // its room in a ring slot
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz
// Tile rows of the fused direction + stencil kernel: 8 (two 256-thread blocks per SM).
// 16 rows (one 512-thread block per SM, 1.41 instead of 1.56 halo cells per cell) was
// 9% slower at 1M cells x 64 complex64 columns.
constexpr int kDpqRows = 8;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the given phase parity; false if the budget ran out.  The clock is
// read only once the first try has failed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long budget = kWaitCycles) {
    const uint32_t addr = smem_u32(bar);
    if (mbar_try(addr, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try(addr, parity)) return true;
        if (clock64() - t0 > budget) return false;
    }
}

__device__ __forceinline__ void tma_load4(const CUtensorMap* tm, void* dst, uint64_t* bar, int c0, int x, int y,
                                          int z) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load3(const CUtensorMap* tm, void* dst, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// One plane of the tile into one ring slot: p box {KC, HX, HY, 1} at (c0, i0 - 1,
// j0 - 1, z), then the coefficients right behind it; both complete on the slot's
// mbarrier.  The coefficient map views each grid row as one run of 4 nx floats, so a
// plane's 10 x 10 cells arrive as 10 rows of 160 contiguous bytes (x coordinate
// 4 (i0 - 1): a multiple of 16 bytes), laid out in shared memory exactly as cells.
__device__ __forceinline__ void tma_plane(const CUtensorMap* tm, const CUtensorMap* tc, unsigned char* dst,
                                          uint32_t p_bytes, uint64_t* bar, int c0, int x, int y, int z) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, p_bytes + CF_BYTES);
    tma_load4(tm, dst, bar, c0, x, y, z);
    tma_load3(tc, dst + p_bytes, bar, 4 * x, y, z);
}

// Two adjacent real columns carried by one lane (FP32 tiles of 64 columns, so that a
// warp moves 256-byte rows as in the complex64 tiles).  Componentwise arithmetic.
struct alignas(8) RPair {
    float a, b;
};
__device__ __forceinline__ RPair escale(float s, RPair x) { return RPair{s * x.a, s * x.b}; }
__device__ __forceinline__ RPair eadd(RPair x, RPair y) { return RPair{x.a + y.a, x.b + y.b}; }
__device__ __forceinline__ RPair esub(RPair x, RPair y) { return RPair{x.a - y.a, x.b - y.b}; }
__device__ __forceinline__ RPair emul(RPair x, RPair y) { return RPair{x.a * y.a, x.b * y.b}; }
__device__ __forceinline__ double2 ewide(RPair x) { return make_double2(x.a, x.b); }

// What a lane carries in a tile of KC columns of element type T: L, covering CPL columns.
template <typename T, int KC>
struct TmaLane {
    using L = T;
    static constexpr int CPL = 1;
    static __device__ __forceinline__ L zero() { return ezero<T>(); }
};
template <>
struct TmaLane<float, 64> {
    using L = RPair;
    static constexpr int CPL = 2;
    static __device__ __forceinline__ L zero() { return RPair{0.f, 0.f}; }
};

}  // namespace

// Shared memory: NBUF ring slots (a plane of p, then its coefficients), NBUF
// mbarriers, per-CTA column accumulators (kp).  The per-warp partials of a work item
// reuse slot 0 once its planes are consumed, and the finaliser scratch reuses the
// ring.
template <typename T, int KC>
__global__ void __launch_bounds__(THREADS, KC == 16 ? 3 : 2) k_pq_tma(const __grid_constant__ CUtensorMap tm,
                                                       const __grid_constant__ CUtensorMap tc, Op<T> op,
                                                       T* __restrict__ q, int kp, int zc_len, ColState st,
                                                       int hslot) {
    using R = typename Elem<T>::R;
    using Lane = TmaLane<T, KC>;
    using L = typename Lane::L;
    constexpr int CPL = Lane::CPL;       // columns per lane
    constexpr int LPC = KC / CPL;        // lanes per cell
    constexpr int PLANE = KC * HX * HY;  // elements
    constexpr int P_BYTES = PLANE * sizeof(T);
    constexpr int SLOT = P_BYTES + CF_SLOT;
    static_assert(P_BYTES % 128 == 0 && TY * 32 * sizeof(double2) <= P_BYTES, "ring slot layout");
    // ring slots start on a 128-byte boundary (the copy engine's shared-memory alignment)
    unsigned char* base = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + (size_t)NBUF * SLOT);
    double2* acc = reinterpret_cast<double2*>(bar + NBUF);  // NBUF even: 16-byte aligned
    double2* wsum = reinterpret_cast<double2*>(base);
    static_assert(NBUF % 2 == 0, "accumulator alignment");
    static_assert(LPC == 16 || LPC == 32, "column tile");
    constexpr int XS = 32 / LPC;  // cells per warp instruction

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int col = lane % LPC, xsub = lane / LPC;
    const int nx = op.nx, ny = op.ny, nz = op.nz;
    const int tiles_x = nx / TX, tiles_y = ny / TY, tiles_c = kp / KC;
    const int zchunks = (nz + zc_len - 1) / zc_len;
    const int nitems = tiles_x * tiles_y * tiles_c * zchunks;

    if (threadIdx.x == 0) {
        for (int b = 0; b < NBUF; ++b) mbar_init(&bar[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int c = threadIdx.x; c < kp; c += blockDim.x) acc[c] = make_double2(0.0, 0.0);
    __syncthreads();

    uint32_t parity = 0;    // bit b: parity of the next phase of buffer b
    uint32_t pending = 0;   // bit b: a copy into buffer b has been issued and not waited for
    bool failed = false;

    for (int item = blockIdx.x; item < nitems && !failed; item += gridDim.x) {
        int rem = item;
        const int txi = rem % tiles_x;
        rem /= tiles_x;
        const int tyi = rem % tiles_y;
        rem /= tiles_y;
        const int cci = rem % tiles_c;
        const int zci = rem / tiles_c;
        const int i0 = txi * TX, j0 = tyi * TY, c0 = cci * KC;
        const int z0 = zci * zc_len, z1 = min(z0 + zc_len, nz);
        // the lane's columns c0 + CPL col .. c0 + CPL col + CPL - 1
        bool run = false;
#pragma unroll
        for (int u = 0; u < CPL; ++u) {
            const int cu = c0 + CPL * col + u;
            run = run || (st.active[cu] && !st.upd[cu]);
        }
        if (!__syncthreads_or(run)) continue;

        // planes z0-1 .. z1 go to buffers (z - z0 + 1) mod NBUF
        auto slot = [&](int z) { return (z - z0 + 1) & (NBUF - 1); };
        // (the barrier above also ends the previous item's reads of the partials in slot 0)
        if (threadIdx.x == 0) {
            for (int z = z0 - 1; z <= min(z0 + 1, z1); ++z)
                tma_plane(&tm, &tc, base + (size_t)slot(z) * SLOT, P_BYTES, &bar[slot(z)], c0, i0 - 1, j0 - 1, z);
        }
        for (int z = z0 - 1; z <= min(z0 + 1, z1); ++z) pending |= 1u << slot(z);
        bool ok = true;
        for (int z = z0 - 1; z <= z0 && ok; ++z) {
            const int b = slot(z);
            ok = mbar_wait(&bar[b], (parity >> b) & 1u);
            if (ok) {
                parity ^= 1u << b;
                pending &= ~(1u << b);
            }
        }
        failed = __syncthreads_or(!ok);
        L pq = Lane::zero();
        for (int k = z0; k < z1 && !failed; ++k) {
            if (k + 2 <= z1) {
                const int b = slot(k + 2);
                if (threadIdx.x == 0)
                    tma_plane(&tm, &tc, base + (size_t)b * SLOT, P_BYTES, &bar[b], c0, i0 - 1, j0 - 1, k + 2);
                pending |= 1u << b;
            }
            {
                const int b = slot(k + 1);
                ok = mbar_wait(&bar[b], (parity >> b) & 1u);
                if (ok) {
                    parity ^= 1u << b;
                    pending &= ~(1u << b);
                }
            }
            failed = __syncthreads_or(!ok);
            if (failed) break;
            const unsigned char* sm = base + (size_t)slot(k - 1) * SLOT;
            const unsigned char* sc = base + (size_t)slot(k) * SLOT;
            const L* pm = reinterpret_cast<const L*>(sm);
            const L* pc = reinterpret_cast<const L*>(sc);
            const L* pn = reinterpret_cast<const L*>(base + (size_t)slot(k + 1) * SLOT);
            const Cf4<R>* cm = reinterpret_cast<const Cf4<R>*>(sm + P_BYTES);
            const Cf4<R>* cc = reinterpret_cast<const Cf4<R>*>(sc + P_BYTES);
            const int j = j0 + warp;
            const int row = (warp + 1) * HX * LPC;
            const int crow = (warp + 1) * HX;
#pragma unroll 2
            for (int xi = xsub; xi < TX; xi += XS) {
                const int i = i0 + xi;
                const int v = i + nx * (j + ny * k);
                const int o = row + (xi + 1) * LPC + col;
                const int co = crow + xi + 1;
                const Cf4<R> cv = cc[co];
                const L xc = pc[o];
                L a = escale(cv.dre, xc);
                if constexpr (Elem<T>::cplx) a = eadd(a, emul_i(op.w, xc));
                // faces to the -x, -y, -z neighbours carry that neighbour's coefficient
                // (zero outside the grid, where p is zero as well)
                a = esub(a, escale(cc[co - 1].cx, pc[o - LPC]));
                a = esub(a, escale(cv.cx, pc[o + LPC]));
                a = esub(a, escale(cc[co - HX].cy, pc[o - HX * LPC]));
                a = esub(a, escale(cv.cy, pc[o + HX * LPC]));
                a = esub(a, escale(cm[co].cz, pm[o]));
                a = esub(a, escale(cv.cz, pn[o]));
                reinterpret_cast<L*>(q + (int64_t)v * kp + c0)[col] = a;
                pq = eadd(pq, emul(xc, a));
            }
            __syncthreads();  // plane k-1's buffer is refilled in the next iteration
        }
        if (failed) break;
        // fold this item's per-lane sums into the CTA's column accumulators in a fixed
        // order (warp, then half-warp)
        wsum[warp * 32 + lane] = ewide(pq);
        __syncthreads();
        if (threadIdx.x < KC) {
            // column t is component t % CPL of lane t / CPL (a complex lane carries
            // one column as (re, im); a pair lane two real columns)
            const int t = threadIdx.x, lt = t / CPL, comp = t % CPL;
            double2 s = make_double2(0.0, 0.0);
            for (int w = 0; w < TY; ++w)
                for (int h = 0; h < XS; ++h) {
                    const double2 pw = wsum[w * 32 + h * LPC + lt];
                    if (CPL == 1) {
                        s.x += pw.x;
                        s.y += pw.y;
                    } else {
                        s.x += comp ? pw.y : pw.x;
                    }
                }
            acc[c0 + t].x += s.x;
            acc[c0 + t].y += s.y;
        }
        __syncthreads();
    }

    if (failed) {
        if (threadIdx.x == 0) atomicExch(st.error, 1);
        // drain this CTA's copies still in flight before shared memory is released
        for (int b = 0; b < NBUF; ++b)
            if (pending & (1u << b)) mbar_wait(&bar[b], (parity >> b) & 1u);
        __syncthreads();
    }
    for (int c = threadIdx.x; c < kp; c += blockDim.x) st.partA[(int64_t)blockIdx.x * kp + c] = acc[c];
    const double2* totA;
    const double* totB;
    if (reduce_columns(st, true, false, kp, base, &totA, &totB)) {
        stencil_finalise(st, totA, kp, hslot);
        __syncthreads();
        publish_counts(st, kp);
    }
}

// ------------------------------------------------------------------------------
// Direction update fused into the stencil.  One pass computes, for the direction of
// iteration m,
//     p_new = M^{-1} r~ + beta p_old   (running columns; p_old carried over otherwise)
//     q = A p_new,  p_new^T q
// writing p_new into its ring slot and q, so the iteration streams r~ and p_old in and
// p_new and q out (4 block vectors) instead of the 3 + 2 of a direction pass followed
// by the stencil.  Each plane of the tile arrives with its one-cell halo by three
// cp.async.bulk.tensor loads on one mbarrier: r~ and p_old into one of S staging slots
// and the 32-byte records (coefficients, FP32 Jacobi inverse) into a ring of S + 3
// coefficient planes.  The plane is then converted once, halo included, into a ring
// of three p_new planes (k, k + 1 and the one being converted; the -z neighbours of
// plane k stay in registers) that the stencil reads; out-of-grid cells arrive as zeros
// in r~, p_old and M^{-1}, so their p_new is an exact zero as well.  A staging slot is
// refilled after the barrier that follows its plane's conversion, so S planes are in
// flight while a plane is computed.  A lane carries 16 bytes of columns (two complex
// or four real) of one cell; KC = 16 complex or 32 real columns make 128-byte rows.
template <typename T, int KC, int S, int R>
struct DpqLayout {
    static constexpr int HYR = R + 2;                          // halo rows of an R-row tile
    static constexpr int PLANE = KC * HX * HYR;                // elements of one vector plane
    static constexpr int P_BYTES = PLANE * (int)sizeof(T);
    static constexpr int C8_BYTES = HX * HYR * 32;             // one plane of 32-byte records
    static constexpr int C8_SLOT = (C8_BYTES + 127) / 128 * 128;
    static constexpr int NCF = S + 3;                          // coefficient planes alive
    static constexpr int OFF_PN = 0;                           // 3 converted planes
    static constexpr int OFF_ST = OFF_PN + 3 * P_BYTES;        // S x (r~ plane, p_old plane)
    static constexpr int OFF_CF = OFF_ST + S * 2 * P_BYTES;    // NCF coefficient planes
    static constexpr int OFF_BAR = OFF_CF + NCF * C8_SLOT;     // S mbarriers
    static constexpr int OFF_ACC = OFF_BAR + (S * 8 + 15) / 16 * 16;  // kp column accumulators
    static_assert(P_BYTES % 128 == 0 && C8_SLOT % 128 == 0, "TMA destinations on 128-byte boundaries");
};

__device__ __forceinline__ float dinv_of(float4 w, float*) { return w.x; }
__device__ __forceinline__ float2 dinv_of(float4 w, float2*) { return make_float2(w.x, w.y); }

// 16 bytes of consecutive columns carried by one lane of the fused kernel: two
// complex64 or four FP32 columns, moved by one shared-memory or global access.
template <typename T>
struct alignas(16) Pack16 {
    static constexpr int N = 16 / (int)sizeof(T);
    T e[N];
};

template <typename T, int KC, int S, int R>
__global__ void __launch_bounds__(32 * R, R == 8 ? 2 : 1) k_dpq_tma(const __grid_constant__ CUtensorMap tr,
                                                        const __grid_constant__ CUtensorMap tp,
                                                        const __grid_constant__ CUtensorMap tc8, Op<T> op,
                                                        T* __restrict__ p_new, T* __restrict__ q, int kp,
                                                        int zc_len, ColState st, int hslot) {
    using Ly = DpqLayout<T, KC, S, R>;
    constexpr int HY_ = Ly::HYR;
    using P = Pack16<T>;
    constexpr int CPL = P::N;         // columns per lane
    constexpr int LPC = KC / CPL;     // lanes per cell
    constexpr int XS = 32 / LPC;      // cells per warp instruction
    static_assert(LPC == 8, "column tile of 128 bytes");
    constexpr int P_BYTES = Ly::P_BYTES;
    constexpr int PLANE_P = Ly::PLANE / CPL;  // 16-byte units of one plane
    constexpr int NT = TX / XS;               // own cells of a lane in each plane
    // the cells of a plane that the 7-point stencil reads (the tile and its one-cell
    // halo in x and y; the four corners are no cell's neighbour), R XS at a time
    constexpr int NHALO = HX * HY_ - 4;
    constexpr int NPASS = (NHALO + R * XS - 1) / (R * XS);
    constexpr bool EXACT = NHALO % (R * XS) == 0;
    unsigned char* base = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    P* pn_ring = reinterpret_cast<P*>(base + Ly::OFF_PN);
    unsigned char* stg = base + Ly::OFF_ST;
    unsigned char* cfr = base + Ly::OFF_CF;
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + Ly::OFF_BAR);
    double2* acc = reinterpret_cast<double2*>(base + Ly::OFF_ACC);
    // per-lane partial sums of an item, in the p_new ring once its planes are consumed
    // (the staging slots may already hold the next item's first planes)
    double2* wsum = reinterpret_cast<double2*>(base + Ly::OFF_PN);
    static_assert(R * 32 * CPL * (int)sizeof(double2) <= 3 * P_BYTES, "per-lane partials fit in the p_new ring");

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lc = lane % LPC, xsub = lane / LPC;  // the lane's columns CPL lc .. CPL lc + CPL - 1 of the tile
    const int nx = op.nx, ny = op.ny, nz = op.nz;
    const int nxy = nx * ny;
    const int LP = kp / CPL;          // 16-byte units of one cell's columns in global memory
    const int tiles_x = nx / TX, tiles_y = ny / R, tiles_c = kp / KC;
    const int zchunks = (nz + zc_len - 1) / zc_len;
    const int nitems = tiles_x * tiles_y * tiles_c * zchunks;

    // The lane's halo cells, the same in every plane and item: index in the plane of
    // (HX x HY_) cells, offset from the tile origin in the grid (x + nx y), and a bit
    // in hown for each that is one of the tile's own cells (hlive: within the plane)
    int hcell[NPASS], hrel[NPASS];
    uint32_t hown = 0, hlive = 0;
#pragma unroll
    for (int i = 0; i < NPASS; ++i) {
        const int c = warp * XS + xsub + i * R * XS;
        const int hy = c < HX - 2 ? 0 : (c < HX * HY_ - HX - 2 ? 1 + (c - (HX - 2)) / HX : HY_ - 1);
        const int hx = hy == 0 ? c + 1 : (hy == HY_ - 1 ? c - (HX * HY_ - HX - 2) + 1 : (c - (HX - 2)) % HX);
        const bool live = EXACT || c < NHALO;
        hcell[i] = live ? hy * HX + hx : 0;
        hrel[i] = (hx - 1) + nx * (hy - 1);
        if (live) hlive |= 1u << i;
        if (live && hx >= 1 && hx <= TX && hy >= 1 && hy <= R) hown |= 1u << i;
    }
    // the lane's own cells of its tile row (x = xsub + XS t): offsets from the tile origin
    const int row = (warp + 1) * HX * LPC;
    const int crow = (warp + 1) * HX;

    if (threadIdx.x == 0) {
        for (int b = 0; b < S; ++b) mbar_init(&bar[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int c = threadIdx.x; c < kp; c += blockDim.x) acc[c] = make_double2(0.0, 0.0);
    __syncthreads();

    uint32_t parity = 0;    // bit b: parity of the next phase of staging slot b
    uint32_t pending = 0;   // bit b: a copy into staging slot b has been issued and not waited for
    bool failed = false;
    // Planes are numbered in the order this CTA loads them, across its items: the
    // plane with number s lands in staging slot s % S, its records in coefficient slot
    // s % NCF, and it is converted into p_new slot s % 3.  An item's planes z0 - 1 .. z1
    // are numbers seq0 .. seq0 + z1 - z0 + 1; the first S planes of the next item are
    // loaded while this one ends, into the staging slots its last planes leave.
    unsigned seq0 = 0;
    int npref = 0;          // planes of the current item already loaded by the previous one

    // tile of a work item: column tiles fastest, so the tiles sharing a cell's columns run
    // on neighbouring CTAs at the same time and the 256-byte L2 lines their 128-byte rows
    // split are used by both while resident
    struct Tile {
        int i0, j0, c0, z0, z1;
    };
    auto tile_of = [&](int item) {
        int rem = item;
        const int cci = rem % tiles_c;
        rem /= tiles_c;
        const int txi = rem % tiles_x;
        rem /= tiles_x;
        const int tyi = rem % tiles_y;
        const int zci = rem / tiles_y;
        Tile g;
        g.i0 = txi * TX;
        g.j0 = tyi * R;
        g.c0 = cci * KC;
        g.z0 = zci * zc_len;
        g.z1 = min(g.z0 + zc_len, nz);
        return g;
    };
    // the copies of plane z of tile g as plane number s (thread 0 only)
    auto issue = [&](const Tile& g, int z, unsigned s) {
        const int sl = (int)(s % S);
        unsigned char* d = stg + (size_t)sl * 2 * P_BYTES;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bar[sl], 2 * P_BYTES + Ly::C8_BYTES);
        tma_load4(&tr, d, &bar[sl], g.c0, g.i0 - 1, g.j0 - 1, z);
        tma_load4(&tp, d + P_BYTES, &bar[sl], g.c0, g.i0 - 1, g.j0 - 1, z);
        tma_load3(&tc8, cfr + (size_t)(s % Ly::NCF) * Ly::C8_SLOT, &bar[sl], 8 * (g.i0 - 1), g.j0 - 1, z);
    };

    for (int item = blockIdx.x; item < nitems && !failed; item += gridDim.x) {
        const Tile g = tile_of(item);
        const int i0 = g.i0, j0 = g.j0, c0 = g.c0, z0 = g.z0, z1 = g.z1;
        const int cb = c0 + CPL * lc;   // the lane's first column
        const int bcell = i0 + nx * j0; // the tile origin's cell in a plane
        bool run[CPL];
        T bt[CPL];
        bool act = false, anyrun = false;
#pragma unroll
        for (int u = 0; u < CPL; ++u) {
            const bool a = st.active[cb + u] != 0;
            run[u] = a && !st.upd[cb + u];
            bt[u] = run[u] ? enarrow<T>(st.beta[cb + u]) : ezero<T>();
            act = act || a;
            anyrun = anyrun || run[u];
        }
        // the CTA's next item, whose first planes are loaded while this one ends when it
        // has a running column
        const int nitem = item + (int)gridDim.x;
        const Tile gn = tile_of(nitem < nitems ? nitem : item);
        bool nact = false;
        if (nitem < nitems) {
#pragma unroll
            for (int u = 0; u < CPL; ++u) nact = nact || st.active[gn.c0 + CPL * lc + u] != 0;
        }
        // a tile whose columns have all stopped needs neither p_new nor q (it was not
        // prefetched either: npref is 0)
        if (!__syncthreads_or(act)) continue;
        const bool pf = __syncthreads_or(nact);
        bool lane_all = true;
#pragma unroll
        for (int u = 0; u < CPL; ++u) lane_all = lane_all && run[u];
        const bool allrun = __all_sync(0xffffffffu, lane_all);  // warp-uniform: no per-column selects
        P* const pcol = reinterpret_cast<P*>(p_new + cb);
        P* const qcol = reinterpret_cast<P*>(q + cb);
        const unsigned seq_end = seq0 + (unsigned)(z1 - z0 + 2);   // the next item's first plane
        const unsigned npf = pf ? (unsigned)min(S, gn.z1 - gn.z0 + 2) : 0u;

        // this item's first planes that the previous item did not load
        for (unsigned s = seq0 + (unsigned)npref; s < seq0 + (unsigned)min(S, z1 - z0 + 2); ++s) {
            if (threadIdx.x == 0) issue(g, z0 - 1 + (int)(s - seq0), s);
            pending |= 1u << (s % S);
        }
        // after a barrier that ends every read of plane s's staging slot: load plane s + S
        // into it, of this item or, past its end, of the next
        auto refill = [&](unsigned s) {
            const unsigned t = s + S;
            if (t < seq_end) {
                if (threadIdx.x == 0) issue(g, z0 - 1 + (int)(t - seq0), t);
                pending |= 1u << (t % S);
            } else if (t - seq_end < npf) {
                if (threadIdx.x == 0) issue(gn, gn.z0 - 1 + (int)(t - seq_end), t);
                pending |= 1u << (t % S);
            }
        };
        // wait for plane z (number s) and convert it into its p_new slot ps (and, for the
        // chunk's own planes, write the tile's cells to the ring slot in global memory);
        // no barrier: the caller's next barrier ends the reads of the staging slot
        auto convert = [&](int z, unsigned s, int ps) -> bool {
            const int sl = (int)(s % S);
            if (!mbar_wait(&bar[sl], (parity >> sl) & 1u)) return false;
            parity ^= 1u << sl;
            pending &= ~(1u << sl);
            const P* Rr = reinterpret_cast<const P*>(stg + (size_t)sl * 2 * P_BYTES);
            const P* Po = Rr + PLANE_P;
            const float4* cw = reinterpret_cast<const float4*>(cfr + (size_t)(s % Ly::NCF) * Ly::C8_SLOT);
            P* Pn = pn_ring + ps * PLANE_P;
            const bool own = z >= z0 && z < z1;
            P* const pz = pcol + (int64_t)(own ? z : 0) * nxy * LP;
#pragma unroll
            for (int i = 0; i < NPASS; ++i) {
                if (EXACT || ((hlive >> i) & 1u)) {
                    const P po = Po[hcell[i] * LPC + lc];
                    P pn = po;
                    if (allrun) {
                        const P rr = Rr[hcell[i] * LPC + lc];
                        const T dv = dinv_of(cw[2 * hcell[i] + 1], (T*)nullptr);
#pragma unroll
                        for (int u2 = 0; u2 < CPL; ++u2) pn.e[u2] = eadd(emul(dv, rr.e[u2]), emul(bt[u2], po.e[u2]));
                    } else if (anyrun) {
                        const P rr = Rr[hcell[i] * LPC + lc];
                        const T dv = dinv_of(cw[2 * hcell[i] + 1], (T*)nullptr);
#pragma unroll
                        for (int u2 = 0; u2 < CPL; ++u2)
                            if (run[u2]) pn.e[u2] = eadd(emul(dv, rr.e[u2]), emul(bt[u2], po.e[u2]));
                    }
                    Pn[hcell[i] * LPC + lc] = pn;
                    if (own && ((hown >> i) & 1u)) pz[(int64_t)(bcell + hrel[i]) * LP] = pn;
                }
            }
            return true;
        };
        // the lane's own cells: their -z neighbours (p_new and the face coefficient of
        // the plane below) stay in registers from one plane to the next, so a plane's
        // compute reads only planes k and k + 1
        P xd[NT];
        float czd[NT];
        T pq[CPL];
#pragma unroll
        for (int u = 0; u < CPL; ++u) pq[u] = ezero<T>();
        bool ok = convert(z0 - 1, seq0, (int)(seq0 % 3u));
        failed = __syncthreads_or(!ok);
        if (!failed) {
            refill(seq0);
            const P* pl = pn_ring + (seq0 % 3u) * PLANE_P;
            const float4* cl = reinterpret_cast<const float4*>(cfr + (size_t)(seq0 % Ly::NCF) * Ly::C8_SLOT);
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const int xi = xsub + XS * t;
                xd[t] = pl[row + (xi + 1) * LPC + lc];
                czd[t] = cl[2 * (crow + xi + 1)].z;
            }
            ok = convert(z0, seq0 + 1, (int)((seq0 + 1) % 3u));
            failed = __syncthreads_or(!ok);
        }
        if (!failed) {
            refill(seq0 + 1);
            ok = convert(z0 + 1, seq0 + 2, (int)((seq0 + 2) % 3u));
            failed = __syncthreads_or(!ok);
        }
        if (!failed) refill(seq0 + 2);
        // p_new slots of planes k, k + 1, k + 2 and the coefficient slot of plane k,
        // advanced by rotation instead of a modulo per plane
        int ps0 = (int)((seq0 + 1) % 3u), ps1 = (int)((seq0 + 2) % 3u), ps2 = (int)(seq0 % 3u);
        int cs0 = (int)((seq0 + 1) % Ly::NCF);
        for (int k = z0; k < z1 && !failed; ++k) {
            // plane k from planes k and k + 1 (and the registers xd, czd of plane k - 1);
            // then plane k + 2 goes into the p_new slot plane k - 1 left
            {
                const P* pc = pn_ring + ps0 * PLANE_P;
                const P* pn = pn_ring + ps1 * PLANE_P;
                const float4* cc = reinterpret_cast<const float4*>(cfr + (size_t)cs0 * Ly::C8_SLOT);
                P* const qz = qcol + (int64_t)k * nxy * LP;
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    const int xi = xsub + XS * t;
                    const int o = row + (xi + 1) * LPC + lc;
                    const int co = crow + xi + 1;
                    const float4 cv = cc[2 * co];   // (cx, cy, cz, dre)
                    const float cxm = cc[2 * (co - 1)].x, cym = cc[2 * (co - HX)].y;
                    const P xc = pc[o];
                    const P xw = pc[o - LPC], xe = pc[o + LPC], xs = pc[o - HX * LPC], xn = pc[o + HX * LPC];
                    const P xu = pn[o];
                    P a;
#pragma unroll
                    for (int u = 0; u < CPL; ++u) {
                        T r = escale(cv.w, xc.e[u]);
                        if constexpr (Elem<T>::cplx) r = eadd(r, emul_i(op.w, xc.e[u]));
                        r = esub(r, escale(cxm, xw.e[u]));
                        r = esub(r, escale(cv.x, xe.e[u]));
                        r = esub(r, escale(cym, xs.e[u]));
                        r = esub(r, escale(cv.y, xn.e[u]));
                        r = esub(r, escale(czd[t], xd[t].e[u]));
                        r = esub(r, escale(cv.z, xu.e[u]));
                        a.e[u] = r;
                        pq[u] = eadd(pq[u], emul(xc.e[u], r));
                    }
                    qz[(int64_t)(bcell + xi + nx * warp) * LP] = a;
                    xd[t] = xc;
                    czd[t] = cv.z;
                }
            }
            const unsigned s2 = seq0 + (unsigned)(k + 2 - z0 + 1);
            ok = k + 2 > z1 || convert(k + 2, s2, ps2);
            failed = __syncthreads_or(!ok);  // also: plane k's slot is free for plane k + 3
            if (!failed && k + 2 <= z1) refill(s2);
            const int pt = ps0;
            ps0 = ps1;
            ps1 = ps2;
            ps2 = pt;
            cs0 = cs0 + 1 == Ly::NCF ? 0 : cs0 + 1;
        }
        if (failed) break;
        // this item's per-lane sums into the CTA's column accumulators, in a fixed order
#pragma unroll
        for (int u = 0; u < CPL; ++u) wsum[(warp * 32 + lane) * CPL + u] = ewide(pq[u]);
        __syncthreads();
        if (threadIdx.x < KC) {
            const int t = threadIdx.x, tl = t / CPL, tu = t % CPL;
            double2 sm = make_double2(0.0, 0.0);
            for (int w = 0; w < R; ++w)
                for (int h = 0; h < XS; ++h) {
                    const double2 pw = wsum[(w * 32 + h * LPC + tl) * CPL + tu];
                    sm.x += pw.x;
                    sm.y += pw.y;
                }
            acc[c0 + t].x += sm.x;
            acc[c0 + t].y += sm.y;
        }
        __syncthreads();
        seq0 = seq_end;
        npref = (int)npf;
    }

    if (failed) {
        if (threadIdx.x == 0) atomicExch(st.error, 1);
        for (int b = 0; b < S; ++b)
            if (pending & (1u << b)) mbar_wait(&bar[b], (parity >> b) & 1u);
        __syncthreads();
    }
    for (int c = threadIdx.x; c < kp; c += blockDim.x) st.partA[(int64_t)blockIdx.x * kp + c] = acc[c];
    const double2* totA;
    const double* totB;
    if (reduce_columns(st, true, false, kp, base, &totA, &totB)) {
        stencil_finalise(st, totA, kp, hslot);
        __syncthreads();
        publish_counts(st, kp);
    }
}

// Self-test of the bounded wait: one mbarrier that nothing ever arrives at, waited on
// with a budget of `budget` cycles by one warp; the wait must give up and report.
// Nothing is in flight, so giving up leaves no copy behind.
__global__ void k_wait_probe(int* err, long long budget) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0u, budget);
    if (!__syncthreads_or(ok) && threadIdx.x == 0) *err = 1;
}

cudaError_t wait_probe(int* err, long long budget, cudaStream_t s) {
    k_wait_probe<<<1, 32, 0, s>>>(err, budget);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------- host
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool tma_stencil_eligible(ElemKind inner, int nx, int ny, int kp) {
    return (inner == EK_C64 || inner == EK_F32) && nx % TX == 0 && ny % TY == 0 && kp % 16 == 0 && kp <= 1024 &&
           encode_fn() != nullptr;
}

static size_t tma_smem(size_t es, int kc, int kp) {
    return 128 + (size_t)NBUF * ((size_t)kc * HX * HY * es + CF_SLOT) + NBUF * sizeof(uint64_t) +
           (size_t)kp * sizeof(double2);
}

// Shared-memory opt-in and resident blocks per SM of one instantiation.  The opt-in is
// a property of the kernel, shared by every context of the process, so it is set to
// what the widest block (1024 columns) needs: a context preparing a narrower block must
// not lower it under another context's launches.  Occupancy follows the actual size.
template <typename T, int KC>
static cudaError_t tma_configure(size_t smem, int* per_sm) {
    const size_t widest = tma_smem(sizeof(T), KC == 64 ? 64 : KC, 1024);
    cudaError_t e = cudaFuncSetAttribute(k_pq_tma<T, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(smem > widest ? smem : widest));
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_pq_tma<T, KC>, THREADS, smem);
    return e;
}

// z-chunk length of the TMA stencils' work items (a tile marched through zc planes plus
// the two halo planes it converts).  The CTAs resident on an SM share its issue slots,
// so the time follows the planes each SM processes: item i runs on SM i mod num_sms
// (grids are whole multiples of the SM count), ceil(items / num_sms) items of zc + 2
// planes.  At 1M cells x 64 complex64 columns this takes whole 64-plane columns
// (7 x 66 planes per SM) over 32-plane chunks (14 x 34), measured 0.6% faster.
static int zchunk_length(int tiles, int nz, int num_sms) {
    int best = nz;
    double best_cost = 1e300;
    for (int zc : {4, 8, 12, 16, 24, 32, 48, 64, 96, 128, nz}) {
        if (zc > nz || zc < 1) continue;
        const long items = (long)tiles * ((nz + zc - 1) / zc);
        const double cost = (double)((items + num_sms - 1) / num_sms) * (zc + 2);
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = zc;
        }
    }
    return best;
}

cudaError_t tma_stencil_prepare(ElemKind inner, const DirRing& ring, const void* cf, int nx, int ny, int nz, int kp,
                                int num_sms, TmaStencil* out) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const size_t es = inner == EK_C64 ? 8 : 4;
    // FP32: 64-column tiles (two columns per lane) when the block width allows
    const int kc = (inner == EK_F32 && kp % 64 == 0) ? 64 : (kp % 32 == 0 ? 32 : 16);
    const cuuint64_t dims[4] = {(cuuint64_t)kp, (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[3] = {(cuuint64_t)kp * es, (cuuint64_t)kp * nx * es, (cuuint64_t)kp * nx * ny * es};
    const cuuint32_t box[4] = {(cuuint32_t)kc, HX, HY, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    if (ring.H < 1 || ring.H > kDirRingMax) return cudaErrorInvalidValue;
    for (int sl = 0; sl < ring.H; ++sl) {
        void* p = static_cast<unsigned char*>(ring.base) + (size_t)sl * ring.slot_elems * es;
        const CUresult r = enc(reinterpret_cast<CUtensorMap*>(out->tmap[sl]),
                               inner == EK_C64 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                               p, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    // packed coefficients {cx, cy, cz, dre} per cell, FP32 for both recurrence types
    // viewed as [z][y][4 nx floats]: a box of 4 HX floats x HY rows is the plane's cells
    const cuuint64_t cdims[3] = {(cuuint64_t)nx * 4, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t cstrides[2] = {(cuuint64_t)nx * 16, (cuuint64_t)nx * ny * 16};
    const cuuint32_t cbox[3] = {4 * HX, HY, 1};
    const CUresult rc = enc(reinterpret_cast<CUtensorMap*>(out->tmap_cf), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                            const_cast<void*>(cf), cdims, cstrides, cbox, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (rc != CUDA_SUCCESS) return cudaErrorInvalidValue;
    out->kc = kc;
    out->smem = tma_smem(es, kc, kp);
    int per_sm = 0;
    cudaError_t e;
    if (inner == EK_C64)
        e = kc == 32 ? tma_configure<float2, 32>(out->smem, &per_sm) : tma_configure<float2, 16>(out->smem, &per_sm);
    else if (kc == 64)
        e = tma_configure<float, 64>(out->smem, &per_sm);
    else
        e = kc == 32 ? tma_configure<float, 32>(out->smem, &per_sm) : tma_configure<float, 16>(out->smem, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int tiles = (nx / TX) * (ny / TY) * (kp / kc);
    const int grid_cap = per_sm * num_sms;
    const int best = zchunk_length(tiles, nz, num_sms);
    out->zc = best;
    const long items = (long)tiles * ((nz + best - 1) / best);
    out->grid = (int)(items < grid_cap ? items : grid_cap);
    return cudaSuccess;
}

cudaError_t tma_stencil_launch(ElemKind inner, const OpRaw& o, const TmaStencil& t, int slot, void* q, int kp,
                               const ColState& st, cudaStream_t s) {
    if (slot < 0 || slot >= kDirRingMax) return cudaErrorInvalidValue;
    const CUtensorMap* tm = reinterpret_cast<const CUtensorMap*>(t.tmap[slot]);
    const CUtensorMap* tc = reinterpret_cast<const CUtensorMap*>(t.tmap_cf);
    if (inner == EK_C64) {
        Op<float2> op;
        op.cf = static_cast<const Cf4<float>*>(o.cf);
        op.dinv = static_cast<const float2*>(o.dinv);
        op.w = (float)o.w;
        op.nx = o.nx;
        op.ny = o.ny;
        op.nz = o.nz;
        if (t.kc == 32)
            k_pq_tma<float2, 32><<<t.grid, THREADS, t.smem, s>>>(*tm, *tc, op, (float2*)q, kp, t.zc, st, slot);
        else
            k_pq_tma<float2, 16><<<t.grid, THREADS, t.smem, s>>>(*tm, *tc, op, (float2*)q, kp, t.zc, st, slot);
    } else if (inner == EK_F32) {
        Op<float> op;
        op.cf = static_cast<const Cf4<float>*>(o.cf);
        op.dinv = static_cast<const float*>(o.dinv);
        op.w = 0.f;
        op.nx = o.nx;
        op.ny = o.ny;
        op.nz = o.nz;
        if (t.kc == 64)
            k_pq_tma<float, 64><<<t.grid, THREADS, t.smem, s>>>(*tm, *tc, op, (float*)q, kp, t.zc, st, slot);
        else if (t.kc == 32)
            k_pq_tma<float, 32><<<t.grid, THREADS, t.smem, s>>>(*tm, *tc, op, (float*)q, kp, t.zc, st, slot);
        else
            k_pq_tma<float, 16><<<t.grid, THREADS, t.smem, s>>>(*tm, *tc, op, (float*)q, kp, t.zc, st, slot);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ------------------------------------------------- fused direction + stencil (host)
constexpr int kDpqStages = 2;

bool dpq_eligible(ElemKind inner, int nx, int ny, int kp) {
    const int kc = inner == EK_C64 ? 16 : 32;
    return (inner == EK_C64 || inner == EK_F32) && nx % TX == 0 && ny % kDpqRows == 0 && kp % kc == 0 &&
           kp <= 1024 && encode_fn() != nullptr;
}

template <typename T, int KC>
static size_t dpq_smem(int kp) {
    return 128 + (size_t)DpqLayout<T, KC, kDpqStages, kDpqRows>::OFF_ACC + (size_t)kp * sizeof(double2);
}

// As tma_configure: the opt-in covers the widest block, whichever context sets it.
template <typename T, int KC>
static cudaError_t dpq_configure(size_t smem, int* per_sm) {
    const size_t widest = dpq_smem<T, KC>(1024);
    cudaError_t e = cudaFuncSetAttribute(k_dpq_tma<T, KC, kDpqStages, kDpqRows>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(smem > widest ? smem : widest));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_dpq_tma<T, KC, kDpqStages, kDpqRows>,
                                                          32 * kDpqRows, smem);
    return e;
}

cudaError_t dpq_prepare(ElemKind inner, const DirRing& ring, const void* r, const void* cf8, int nx, int ny, int nz,
                        int kp, int num_sms, TmaStencil* out) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc || !dpq_eligible(inner, nx, ny, kp) || !r || !cf8) return cudaErrorNotSupported;
    if (ring.H < 1 || ring.H > kDirRingMax) return cudaErrorInvalidValue;
    const bool cx = inner == EK_C64;
    const size_t es = cx ? 8 : 4;
    const int kc = cx ? 16 : 32;
    const cuuint64_t dims[4] = {(cuuint64_t)kp, (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[3] = {(cuuint64_t)kp * es, (cuuint64_t)kp * nx * es, (cuuint64_t)kp * nx * ny * es};
    const cuuint32_t box[4] = {(cuuint32_t)kc, HX, kDpqRows + 2, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt = cx ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    auto encode = [&](unsigned char* dst, const void* ptr) {
        return enc(reinterpret_cast<CUtensorMap*>(dst), dt, 4, const_cast<void*>(ptr), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    };
    if (encode(out->tmap_r, r) != CUDA_SUCCESS) return cudaErrorInvalidValue;
    for (int sl = 0; sl < ring.H; ++sl) {
        const void* p = static_cast<const unsigned char*>(ring.base) + (size_t)sl * ring.slot_elems * es;
        if (encode(out->tmap_pf[sl], p) != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    // 32-byte records {cx, cy, cz, dre, dinv (re, im or value, 0), 0, 0} per cell
    // viewed as [z][y][8 nx floats]: each plane of the tile arrives as rows of 320 bytes
    const cuuint64_t cdims[3] = {(cuuint64_t)nx * 8, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t cstrides[2] = {(cuuint64_t)nx * 32, (cuuint64_t)nx * ny * 32};
    const cuuint32_t cbox[3] = {8 * HX, kDpqRows + 2, 1};
    if (enc(reinterpret_cast<CUtensorMap*>(out->tmap_c8), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(cf8),
            cdims, cstrides, cbox, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    out->kcf = kc;
    out->smemf = cx ? dpq_smem<float2, 16>(kp) : dpq_smem<float, 32>(kp);
    int per_sm = 0;
    cudaError_t e = cx ? dpq_configure<float2, 16>(out->smemf, &per_sm) : dpq_configure<float, 32>(out->smemf, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int tiles = (nx / TX) * (ny / kDpqRows) * (kp / kc);
    const int grid_cap = per_sm * num_sms;
    const int best = zchunk_length(tiles, nz, num_sms);
    out->zcf = best;
    const long items = (long)tiles * ((nz + best - 1) / best);
    out->gridf = (int)(items < grid_cap ? items : grid_cap);
    out->fused = true;
    return cudaSuccess;
}

cudaError_t dpq_launch(ElemKind inner, const OpRaw& o, const TmaStencil& t, const DirRing& ring, int slot, int prev,
                       void* q, int kp, const ColState& st, cudaStream_t s) {
    if (!t.fused || slot < 0 || slot >= ring.H || prev < 0 || prev >= ring.H) return cudaErrorInvalidValue;
    const CUtensorMap* tr = reinterpret_cast<const CUtensorMap*>(t.tmap_r);
    const CUtensorMap* tp = reinterpret_cast<const CUtensorMap*>(t.tmap_pf[prev]);
    const CUtensorMap* tc = reinterpret_cast<const CUtensorMap*>(t.tmap_c8);
    if (inner == EK_C64) {
        Op<float2> op;
        op.cf = static_cast<const Cf4<float>*>(o.cf);
        op.dinv = static_cast<const float2*>(o.dinv);
        op.w = (float)o.w;
        op.nx = o.nx;
        op.ny = o.ny;
        op.nz = o.nz;
        float2* pn = static_cast<float2*>(ring.base) + (size_t)slot * ring.slot_elems;
        k_dpq_tma<float2, 16, kDpqStages, kDpqRows><<<t.gridf, 32 * kDpqRows, t.smemf, s>>>(*tr, *tp, *tc, op, pn, (float2*)q, kp,
                                                                           t.zcf, st, slot);
    } else if (inner == EK_F32) {
        Op<float> op;
        op.cf = static_cast<const Cf4<float>*>(o.cf);
        op.dinv = static_cast<const float*>(o.dinv);
        op.w = 0.f;
        op.nx = o.nx;
        op.ny = o.ny;
        op.nz = o.nz;
        float* pn = static_cast<float*>(ring.base) + (size_t)slot * ring.slot_elems;
        k_dpq_tma<float, 32, kDpqStages, kDpqRows><<<t.gridf, 32 * kDpqRows, t.smemf, s>>>(*tr, *tp, *tc, op, pn, (float*)q, kp,
                                                                          t.zcf, st, slot);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace dotk
