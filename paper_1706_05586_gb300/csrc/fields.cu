// One-pass kernels of the DOT hot path (sm_103a): PaLS absorption, operator
// coefficients, right-hand-side block, restriction and misfit, sensitivity and the
// PaLS chain rule.  All reductions are deterministic (fixed-order block sums).
#include "dot_kernels.cuh"
#include "dot_internal.h"
#include "dfloat.cuh"
#include "dot.h"

namespace dotk {

static inline int grid_for(int64_t n, int threads, int cap = 152 * 32) {
    int64_t b = (n + threads - 1) / threads;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// ------------------------------------------------------------ PaLS (Sec. 2)
// Wendland psi_{2,1}(r) = (1-r)^4 (4r+1) and psi'(r) = -20 r (1-r)^3 on r < 1.
__device__ __forceinline__ double wendland(double r) {
    double s = 1.0 - r, s2 = s * s;
    return s2 * s2 * (4.0 * r + 1.0);
}
__device__ __forceinline__ double wendland_prime(double r) {
    double s = 1.0 - r;
    return -20.0 * r * s * s * s;
}

// phi(x_v) = sum_j alpha_j psi(sqrt(beta_j^2 |x_v - chi_j|^2 + gamma^2)),
// mu = mu_out + (mu_in - mu_out) H_eps(phi - c), wdmu = (mu_in - mu_out) H_eps'(phi - c),
// with the C^1 sine ramp H_eps (Eq. (absorption const); the ramp is this library's reading).
//
// A block owns a tile of 8 x 8 x 4 cells.  It first lists, in increasing j, the RBFs
// whose support (r < 1) can reach a cell centre of the tile (a conservative test on
// the distance from chi_j to the tile's box of centres), then sums only those.  The
// skipped terms are exact zeros of the sum, and the kept ones are added in the same
// order as a loop over all j, so phi is the same to the last bit.
constexpr int kPalsTx = 8, kPalsTy = 8, kPalsTz = 4;
constexpr int kPalsCullMax = 4096;  // RBFs that the tile list can hold; more: no culling

__global__ void __launch_bounds__(256) k_pals_eval(const double* __restrict__ p, int m0, double mu_in, double mu_out,
                                                   double c, double eps, double gamma, int nx, int ny, int nz, double h,
                                                   double* __restrict__ phi_out, double* __restrict__ mu_out_arr,
                                                   double* __restrict__ wdmu) {
    constexpr int CH = 128;
    __shared__ double sp[5 * CH];
    __shared__ int slist[kPalsCullMax];
    __shared__ unsigned smask[kPalsCullMax / 32];
    __shared__ int soff[kPalsCullMax / 32];
    __shared__ int scount;
    const int tiles_x = (nx + kPalsTx - 1) / kPalsTx, tiles_y = (ny + kPalsTy - 1) / kPalsTy;
    const int tb = blockIdx.x;
    const int ti = tb % tiles_x, tj = (tb / tiles_x) % tiles_y, tk = tb / (tiles_x * tiles_y);
    const int i = ti * kPalsTx + threadIdx.x % kPalsTx;
    const int j = tj * kPalsTy + (threadIdx.x / kPalsTx) % kPalsTy;
    const int k = tk * kPalsTz + threadIdx.x / (kPalsTx * kPalsTy);
    const bool in = i < nx && j < ny && k < nz;
    const double x = (i + 0.5) * h, y = (j + 0.5) * h, z = (k + 0.5) * h;
    const double g2 = gamma * gamma;
    const bool cull = m0 <= kPalsCullMax;
    int cnt = m0;
    if (cull) {
        // box of the tile's cell centres (clipped to the grid)
        const double xlo = (ti * kPalsTx + 0.5) * h, xhi = (min(ti * kPalsTx + kPalsTx, nx) - 0.5) * h;
        const double ylo = (tj * kPalsTy + 0.5) * h, yhi = (min(tj * kPalsTy + kPalsTy, ny) - 0.5) * h;
        const double zlo = (tk * kPalsTz + 0.5) * h, zhi = (min(tk * kPalsTz + kPalsTz, nz) - 0.5) * h;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
        const int nch = (m0 + 31) / 32;
        for (int ch = warp; ch < nch; ch += nwarps) {
            const int jj = ch * 32 + lane;
            bool keep = false;
            if (jj < m0) {
                const double be = p[5 * jj + 1];
                const double cx = p[5 * jj + 2], cy = p[5 * jj + 3], cz = p[5 * jj + 4];
                const double dx = fmax(0.0, fmax(xlo - cx, cx - xhi));
                const double dy = fmax(0.0, fmax(ylo - cy, cy - yhi));
                const double dz = fmax(0.0, fmax(zlo - cz, cz - zhi));
                // drop only when every centre of the tile is certainly outside r < 1
                // (margin for the rounding of the per-cell distance)
                keep = !(be * be * (dx * dx + dy * dy + dz * dz) * (1.0 - 1e-12) + g2 >= 1.0);
            }
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (lane == 0) smask[ch] = m;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int run = 0;
            for (int ch = 0; ch < nch; ++ch) {
                soff[ch] = run;
                run += __popc(smask[ch]);
            }
            scount = run;
        }
        __syncthreads();
        for (int ch = warp; ch < nch; ch += nwarps) {
            const unsigned m = smask[ch];
            if (m & (1u << lane)) slist[soff[ch] + __popc(m & ((1u << lane) - 1u))] = ch * 32 + lane;
        }
        __syncthreads();
        cnt = scount;
    }
    double phi = 0.0;
    for (int q0 = 0; q0 < cnt; q0 += CH) {
        const int nq = min(CH, cnt - q0);
        __syncthreads();
        for (int t = threadIdx.x; t < 5 * nq; t += blockDim.x) {
            const int jj = cull ? slist[q0 + t / 5] : q0 + t / 5;
            sp[t] = p[5 * jj + t % 5];
        }
        __syncthreads();
        if (in) {
            for (int q = 0; q < nq; ++q) {
                const double a = sp[5 * q], be = sp[5 * q + 1];
                const double dx = x - sp[5 * q + 2], dy = y - sp[5 * q + 3], dz = z - sp[5 * q + 4];
                const double d2 = dx * dx + dy * dy + dz * dz;
                const double r2 = be * be * d2 + g2;
                if (r2 < 1.0) phi += a * wendland(sqrt(r2));
            }
        }
    }
    if (in) {
        const int64_t v = i + (int64_t)nx * (j + (int64_t)ny * k);
        const double t = phi - c;
        double H, dH;
        if (t < -eps) {
            H = 0.0;
            dH = 0.0;
        } else if (t > eps) {
            H = 1.0;
            dH = 0.0;
        } else {
            H = 0.5 * (1.0 + t / eps + sinpi(t / eps) / CUDART_PI);
            dH = (1.0 + cospi(t / eps)) / (2.0 * eps);
        }
        phi_out[v] = phi;
        mu_out_arr[v] = mu_in * H + mu_out * (1.0 - H);
        wdmu[v] = (mu_in - mu_out) * dH;
    }
}

cudaError_t pals_eval(const double* p, int m0, double mu_in, double mu_out, double c, double eps, double gamma,
                      int nx, int ny, int nz, double h, double* phi, double* mu, double* wdmu, cudaStream_t s) {
    const int64_t tiles = (int64_t)((nx + kPalsTx - 1) / kPalsTx) * ((ny + kPalsTy - 1) / kPalsTy) *
                          ((nz + kPalsTz - 1) / kPalsTz);
    k_pals_eval<<<(unsigned)tiles, kPalsTx * kPalsTy * kPalsTz, 0, s>>>(p, m0, mu_in, mu_out, c, eps, gamma, nx, ny,
                                                                       nz, h, phi, mu, wdmu);
    return cudaGetLastError();
}

// --------------------------------------------------------- coefficients (Sec. 2)
__device__ __forceinline__ double face_coef(double a, double b, double h2) { return 2.0 * a * b / (a + b) / h2; }
__device__ __forceinline__ double bnd_coef(int flag, double Dc, double h) {
    // Robin: eliminate the face value from eta_b + 2 D (eta_b - eta_c)/(h/2) = 0,
    // outflow eta_b / 2 per area; Dirichlet: eta_b = 0 at distance h/2.
    return flag == DOT_BC_ROBIN ? 2.0 * Dc / (h * (h + 4.0 * Dc)) : 2.0 * Dc / (h * h);
}

struct Bc6 { int f[6]; };

__global__ void k_coefficients(const double* __restrict__ D, const double* __restrict__ mu, int nx, int ny, int nz,
                               double h, Bc6 bc, double w, Cf4<double>* __restrict__ cf64, double* dinv64, int cplx,
                               Cf4<float>* __restrict__ cf32, float* dinv32, float4* __restrict__ cf8) {
    const int64_t n = (int64_t)nx * ny * nz;
    const int64_t nxy = (int64_t)nx * ny;
    const double h2 = h * h;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(v % nx), j = (int)((v / nx) % ny), k = (int)(v / nxy);
        const double Dv = D[v];
        const double fxp = i < nx - 1 ? face_coef(Dv, D[v + 1], h2) : 0.0;
        const double fyp = j < ny - 1 ? face_coef(Dv, D[v + nx], h2) : 0.0;
        const double fzp = k < nz - 1 ? face_coef(Dv, D[v + nxy], h2) : 0.0;
        double d = mu[v];
        d += i > 0 ? face_coef(D[v - 1], Dv, h2) : bnd_coef(bc.f[0], Dv, h);
        d += i < nx - 1 ? fxp : bnd_coef(bc.f[1], Dv, h);
        d += j > 0 ? face_coef(D[v - nx], Dv, h2) : bnd_coef(bc.f[2], Dv, h);
        d += j < ny - 1 ? fyp : bnd_coef(bc.f[3], Dv, h);
        d += k > 0 ? face_coef(D[v - nxy], Dv, h2) : bnd_coef(bc.f[4], Dv, h);
        d += k < nz - 1 ? fzp : bnd_coef(bc.f[5], Dv, h);
        Cf4<double> c64;
        c64.cx = fxp;
        c64.cy = fyp;
        c64.cz = fzp;
        c64.dre = d;
        cf64[v] = c64;
        Cf4<float> c32;
        c32.cx = (float)fxp;
        c32.cy = (float)fyp;
        c32.cz = (float)fzp;
        c32.dre = (float)d;
        cf32[v] = c32;
        float2 di;
        if (cplx) {
            // 1 / (d + i w) = (d - i w) / (d^2 + w^2)
            const double den = d * d + w * w;
            const double re = d / den, im = -w / den;
            reinterpret_cast<double2*>(dinv64)[v] = make_double2(re, im);
            di = make_float2((float)re, (float)im);
            reinterpret_cast<float2*>(dinv32)[v] = di;
        } else {
            dinv64[v] = 1.0 / d;
            di = make_float2((float)(1.0 / d), 0.f);
            dinv32[v] = di.x;
        }
        // 32-byte record of the fused direction + stencil kernel: the four coefficients
        // and the FP32 Jacobi inverse, bitwise the values of cf32 and dinv32
        if (cf8) {
            cf8[2 * v] = make_float4(c32.cx, c32.cy, c32.cz, c32.dre);
            cf8[2 * v + 1] = make_float4(di.x, di.y, 0.f, 0.f);
        }
    }
}

cudaError_t build_coefficients(const double* D, const double* mu, int nx, int ny, int nz, double h, const int bc[6],
                               double w, void* cf64, void* dinv64, bool cplx, void* cf32, void* dinv32, void* cf8,
                               cudaStream_t s) {
    Bc6 b;
    for (int f = 0; f < 6; ++f) b.f[f] = bc[f];
    const int64_t n = (int64_t)nx * ny * nz;
    k_coefficients<<<grid_for(n, 256), 256, 0, s>>>(D, mu, nx, ny, nz, h, b, w, (Cf4<double>*)cf64, (double*)dinv64,
                                                    cplx ? 1 : 0, (Cf4<float>*)cf32, (float*)dinv32, (float4*)cf8);
    return cudaGetLastError();
}

// ------------------------------------------------------ right-hand sides [BW | CV]
// B and C arrive as CSR by voxel (rowptr[n+1]); column c < ls is (B W)_c,
// column ls + l is (C V)_l (Sec. 3.3: one block for both solves).
template <typename T>
__global__ void k_rhs(const int64_t* __restrict__ rpB, const int32_t* __restrict__ ciB, const double* __restrict__ vB,
                      const double* __restrict__ W, int ns, int ls, const int64_t* __restrict__ rpC,
                      const int32_t* __restrict__ ciC, const double* __restrict__ vC, const double* __restrict__ V,
                      int nd, int ld, int64_t n, int kp, T* __restrict__ X) {
    // columns ls + ld .. kp - 1 pad the block to a multiple of 4 and stay zero
    const int64_t total = n * kp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = e / kp;
        const int c = (int)(e % kp);
        double acc = 0.0;
        if (c < ls) {
            for (int64_t t = rpB[v]; t < rpB[v + 1]; ++t) acc += vB[t] * W[ciB[t] + (int64_t)ns * c];
        } else if (c < ls + ld) {
            const int l = c - ls;
            for (int64_t t = rpC[v]; t < rpC[v + 1]; ++t) acc += vC[t] * V[ciC[t] + (int64_t)nd * l];
        }
        X[e] = enarrow<T>(make_double2(acc, 0.0));
    }
}

cudaError_t build_rhs(bool cplx, const int64_t* rpB, const int32_t* ciB, const double* vB, const double* W, int ns,
                      int ls, const int64_t* rpC, const int32_t* ciC, const double* vC, const double* V, int nd,
                      int ld, int64_t n, int kp, void* X, cudaStream_t s) {
    const int g = grid_for(n * kp, 256);
    if (cplx)
        k_rhs<double2><<<g, 256, 0, s>>>(rpB, ciB, vB, W, ns, ls, rpC, ciC, vC, V, nd, ld, n, kp, (double2*)X);
    else
        k_rhs<double><<<g, 256, 0, s>>>(rpB, ciB, vB, W, ns, ls, rpC, ciC, vC, V, nd, ld, n, kp, (double*)X);
    return cudaGetLastError();
}

// ------------------------------------------------------------- layout changes
template <typename T>
__global__ void k_from_cm(const T* __restrict__ cm, int64_t n, int k, int kp, int c0, T* __restrict__ blk) {
    const int64_t total = n * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = e / k;
        const int c = (int)(e % k);
        blk[v * kp + c0 + c] = cm[(int64_t)c * n + v];
    }
}
template <typename T>
__global__ void k_to_cm(const T* __restrict__ blk, int64_t n, int kp, int c0, int k, T* __restrict__ cm) {
    const int64_t total = n * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = e % n;
        const int c = (int)(e / n);
        cm[(int64_t)c * n + v] = blk[v * kp + c0 + c];
    }
}

cudaError_t blk_from_colmajor(bool cplx, const double* cm, int64_t n, int k, int kp, int c0, void* blk,
                              cudaStream_t s) {
    const int g = grid_for(n * k, 256);
    if (cplx)
        k_from_cm<double2><<<g, 256, 0, s>>>((const double2*)cm, n, k, kp, c0, (double2*)blk);
    else
        k_from_cm<double><<<g, 256, 0, s>>>(cm, n, k, kp, c0, (double*)blk);
    return cudaGetLastError();
}

cudaError_t blk_to_colmajor(bool cplx, const void* blk, int64_t n, int kp, int c0, int k, double* cm, cudaStream_t s) {
    const int g = grid_for(n * k, 256);
    if (cplx)
        k_to_cm<double2><<<g, 256, 0, s>>>((const double2*)blk, n, kp, c0, k, (double2*)cm);
    else
        k_to_cm<double><<<g, 256, 0, s>>>((const double*)blk, n, kp, c0, k, cm);
    return cudaGetLastError();
}

// ------------------------------------------------- data projection P = V^T M W
// M, MW, P are complex (double2) even in real arithmetic (imaginary part 0).
__global__ void k_mw(const double2* __restrict__ M, int nd, int ns, const double* __restrict__ W, int ls,
                     double2* __restrict__ MW) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nd * ls) return;
    const int d = t % nd, i = t / nd;
    double2 acc = make_double2(0.0, 0.0);
    for (int s = 0; s < ns; ++s) {
        const double w = W[s + (int64_t)ns * i];
        const double2 m = M[d + (int64_t)nd * s];
        acc.x += m.x * w;
        acc.y += m.y * w;
    }
    MW[d + (int64_t)nd * i] = acc;
}
__global__ void k_vt(const double2* __restrict__ Y, int nd, int ls, const double* __restrict__ V, int ld,
                     double2* __restrict__ P) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ld * ls) return;
    const int l = t % ld, i = t / ld;
    double2 acc = make_double2(0.0, 0.0);
    for (int d = 0; d < nd; ++d) {
        const double vv = V[d + (int64_t)nd * l];
        const double2 y = Y[d + (int64_t)nd * i];
        acc.x += vv * y.x;
        acc.y += vv * y.y;
    }
    P[l + (int64_t)ld * i] = acc;
}

cudaError_t data_projection(bool, const double* M, int nd, int ns, const double* W, int ls, const double* V, int ld,
                            double* MW, double* P, cudaStream_t s) {
    k_mw<<<(nd * ls + 127) / 128, 128, 0, s>>>((const double2*)M, nd, ns, W, ls, (double2*)MW);
    k_vt<<<(ld * ls + 127) / 128, 128, 0, s>>>((const double2*)MW, nd, ls, V, ld, (double2*)P);
    return cudaGetLastError();
}

// ----------------------------------------- restriction S = (CV)^T U, R_s, f
// T[d, i] = sum_v C[v, d] U_i[v] over the support of detector d (one block per d),
// then S = V^T T, R_s = S - V^T M W and f = sum |R_s|^2 (Eq. (EsTResidual), Theorem 1).
template <typename T>
__global__ void k_restrict_T(const T* __restrict__ X, int kp, int ls, const int64_t* __restrict__ cpC,
                             const int32_t* __restrict__ rwC, const double* __restrict__ vC, double2* __restrict__ Tm,
                             int nd) {
    const int d = blockIdx.x;
    for (int i = threadIdx.x; i < ls; i += blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int64_t t = cpC[d]; t < cpC[d + 1]; ++t) {
            const double2 u = ewide(X[(int64_t)rwC[t] * kp + i]);
            acc.x += vC[t] * u.x;
            acc.y += vC[t] * u.y;
        }
        Tm[d + (int64_t)nd * i] = acc;
    }
}

__global__ void k_misfit(const double2* __restrict__ Tm, int nd, int ls, const double* __restrict__ V, int ld,
                         const double2* __restrict__ P, int have_data, double2* __restrict__ S,
                         double2* __restrict__ Rs, double* __restrict__ f) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int t = threadIdx.x; t < ld * ls; t += blockDim.x) {
        const int l = t % ld, i = t / ld;
        double2 sv = make_double2(0.0, 0.0);
        for (int d = 0; d < nd; ++d) {
            const double vv = V[d + (int64_t)nd * l];
            const double2 y = Tm[d + (int64_t)nd * i];
            sv.x += vv * y.x;
            sv.y += vv * y.y;
        }
        S[t] = sv;
        double2 r = sv;
        if (have_data) {
            r.x -= P[t].x;
            r.y -= P[t].y;
        }
        Rs[t] = r;
        acc += r.x * r.x + r.y * r.y;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *f = red[0];
}

cudaError_t restriction_misfit(bool cplx, const void* X, int kp, int ls, const int64_t* cpC, const int32_t* rwC,
                               const double* vC, int nd, const double* V, int ld, const double* P, bool have_data,
                               double* Tm, double* S, double* Rs, double* f, cudaStream_t s) {
    const int th = ls >= 128 ? 128 : ((ls + 31) / 32) * 32;
    if (cplx)
        k_restrict_T<double2><<<nd, th, 0, s>>>((const double2*)X, kp, ls, cpC, rwC, vC, (double2*)Tm, nd);
    else
        k_restrict_T<double><<<nd, th, 0, s>>>((const double*)X, kp, ls, cpC, rwC, vC, (double2*)Tm, nd);
    k_misfit<<<1, 256, 0, s>>>((const double2*)Tm, nd, ls, V, ld, (const double2*)P, have_data ? 1 : 0,
                               (double2*)S, (double2*)Rs, f);
    return cudaGetLastError();
}

// ------------------------------------------------------------- sensitivity
// g_mu[v] = -2 Re sum_{i,l} conj(R_s[l,i]) Z_l[v] U_i[v]: the gradient of
// ||R_s||^2 through J_mu[(l,i), v] = -Z_l[v] U_i[v] (Eq. (Jacobiancomp) with
// dA/dmu_v = e_v e_v^T, sampled as in Eq. (Jacobian kth column)).
//
// l_s l_d complex products per cell: the sums run in double-float arithmetic on the
// FP32 pipe (inputs rounded from FP64 to about 48 bits, accumulation error of the same
// order relative to sum |R_s||Z||U|) instead of on the FP64 pipe.  One thread per cell;
// y_i = sum_l conj(R_s[l,i]) Z_l for a chunk of IC sources at a time keeps the
// accumulators in registers; R_s is split once per block into shared memory.
constexpr int kGmuChunk = 8;
constexpr int kGmuSmemEntries = 3072;  // 48 KiB of (re.hi, re.lo, im.hi, im.lo)

__device__ __forceinline__ float4 df_split2(double2 r) {
    const dfloat a = df_from(r.x), b = df_from(r.y);
    return make_float4(a.hi, a.lo, b.hi, b.lo);
}

template <typename T>
__global__ void __launch_bounds__(128) k_gmu(const T* __restrict__ X, int64_t n, int kp, int ls, int ld,
                                             const double2* __restrict__ Rs, double* __restrict__ gmu) {
    constexpr bool C = Elem<T>::cplx;
    constexpr int IC = kGmuChunk;
    extern __shared__ float4 sRf[];
    const int nr = ls * ld;
    const bool in_smem = nr <= kGmuSmemEntries;
    if (in_smem)
        for (int t = threadIdx.x; t < nr; t += blockDim.x) sRf[t] = df_split2(Rs[t]);
    __syncthreads();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const T* row = X + v * kp;
        dfloat g = df_zero();
        for (int i0 = 0; i0 < ls; i0 += IC) {
            const int nc = min(IC, ls - i0);
            dfloat yr[IC], yi[IC];
#pragma unroll
            for (int c = 0; c < IC; ++c) yr[c] = yi[c] = df_zero();
            for (int l = 0; l < ld; ++l) {
                const double2 z = ewide(row[ls + l]);
                const dfloat zr = df_from(z.x);
                const dfloat zi = C ? df_from(z.y) : df_zero();
#pragma unroll
                for (int c = 0; c < IC; ++c) {
                    if (c >= nc) break;
                    const int e = l + ld * (i0 + c);
                    const float4 r = in_smem ? sRf[e] : df_split2(Rs[e]);
                    const dfloat rr{r.x, r.y};
                    // conj(r) z = (rr zr + ri zi) + i (rr zi - ri zr)
                    yr[c] = df_fma(rr, zr, yr[c]);
                    if (C) {
                        const dfloat ri{r.z, r.w};
                        yr[c] = df_fma(ri, zi, yr[c]);
                        yi[c] = df_fma(rr, zi, yi[c]);
                        yi[c] = df_fma(df_neg(ri), zr, yi[c]);
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < IC; ++c) {
                if (c >= nc) break;
                const double2 u = ewide(row[i0 + c]);
                g = df_fma(yr[c], df_from(u.x), g);
                if (C) g = df_fma(df_neg(yi[c]), df_from(u.y), g);
            }
        }
        gmu[v] = -2.0 * df_to_double(g);
    }
}

cudaError_t sensitivity_gmu(bool cplx, const void* X, int64_t n, int kp, int ls, int ld, const double* Rs, double* gmu,
                            cudaStream_t s) {
    const int nr = ls * ld;
    const size_t sm = nr <= kGmuSmemEntries ? (size_t)nr * sizeof(float4) : 0;
    const int g = grid_for(n, 128);
    if (cplx)
        k_gmu<double2><<<g, 128, sm, s>>>((const double2*)X, n, kp, ls, ld, (const double2*)Rs, gmu);
    else
        k_gmu<double><<<g, 128, sm, s>>>((const double*)X, n, kp, ls, ld, (const double2*)Rs, gmu);
    return cudaGetLastError();
}

// J_mu[(l + ld i) + ls ld v] = -Z_l[v] U_i[v]
template <typename T>
__global__ void k_jmu(const T* __restrict__ X, int64_t n, int kp, int ls, int ld, T* __restrict__ J) {
    const int nr = ls * ld;
    const int64_t total = n * nr;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = e / nr;
        const int row = (int)(e % nr);
        const int l = row % ld, i = row / ld;
        const T* xr = X + v * kp;
        J[e] = escale(-1.0, emul(xr[ls + l], xr[i]));
    }
}

cudaError_t jacobian_mua(bool cplx, const void* X, int64_t n, int kp, int ls, int ld, double* J, cudaStream_t s) {
    const int g = grid_for(n * ls * ld, 256);
    if (cplx)
        k_jmu<double2><<<g, 256, 0, s>>>((const double2*)X, n, kp, ls, ld, (double2*)J);
    else
        k_jmu<double><<<g, 256, 0, s>>>((const double*)X, n, kp, ls, ld, J);
    return cudaGetLastError();
}

// ---------------------------------------------------------- PaLS chain rule
// Cells whose centres can lie in the support r < 1 of RBF j.
struct Box { int i0, i1, j0, j1, k0, k1; };
__device__ __forceinline__ Box rbf_box(double be, double cxj, double cyj, double czj, double gamma, int nx, int ny,
                                       int nz, double h) {
    Box b{0, nx - 1, 0, ny - 1, 0, nz - 1};
    const double lim = 1.0 - gamma * gamma;
    if (lim <= 0.0) {
        b.i1 = -1;  // empty
        return b;
    }
    const double abe = fabs(be);
    if (abe < 1e-300) return b;
    const double rad = sqrt(lim) / abe;
    b.i0 = max(0, (int)floor((cxj - rad) / h - 0.5));
    b.i1 = min(nx - 1, (int)ceil((cxj + rad) / h - 0.5));
    b.j0 = max(0, (int)floor((cyj - rad) / h - 0.5));
    b.j1 = min(ny - 1, (int)ceil((cyj + rad) / h - 0.5));
    b.k0 = max(0, (int)floor((czj - rad) / h - 0.5));
    b.k1 = min(nz - 1, (int)ceil((czj + rad) / h - 0.5));
    return b;
}

// d mu_v / d p_{j,q} for q = alpha, beta, chi_x, chi_y, chi_z (0 outside the support).
__device__ __forceinline__ bool dmu_dp(const double* pj, double gamma, double x, double y, double z, double wd,
                                       double out[5]) {
    const double a = pj[0], be = pj[1];
    const double dx = x - pj[2], dy = y - pj[3], dz = z - pj[4];
    const double d2 = dx * dx + dy * dy + dz * dz;
    const double r2 = be * be * d2 + gamma * gamma;
    if (!(r2 < 1.0)) return false;
    const double r = sqrt(r2);
    const double dpsi = wendland_prime(r);
    const double t = a * dpsi / r;
    out[0] = wd * wendland(r);
    out[1] = wd * t * be * d2;
    out[2] = -wd * t * be * be * dx;
    out[3] = -wd * t * be * be * dy;
    out[4] = -wd * t * be * be * dz;
    return true;
}

// g_p[5j + q] = sum_v dmu_v/dp_{j,q} g_mu[v] over the support of RBF j (one block per j).
__global__ void k_chain_gp(const double* __restrict__ p, int m0, double gamma, int nx, int ny, int nz, double h,
                           const double* __restrict__ wdmu, const double* __restrict__ gmu, double* __restrict__ gp) {
    const int j = blockIdx.x;
    if (j >= m0) return;
    const double* pj = p + 5 * j;
    const Box b = rbf_box(pj[1], pj[2], pj[3], pj[4], gamma, nx, ny, nz, h);
    double acc[5] = {0, 0, 0, 0, 0};
    if (b.i1 >= b.i0 && b.j1 >= b.j0 && b.k1 >= b.k0) {
        const int bx = b.i1 - b.i0 + 1, by = b.j1 - b.j0 + 1, bz = b.k1 - b.k0 + 1;
        const int64_t cnt = (int64_t)bx * by * bz;
        for (int64_t t = threadIdx.x; t < cnt; t += blockDim.x) {
            const int ii = b.i0 + (int)(t % bx);
            const int jj = b.j0 + (int)((t / bx) % by);
            const int kk = b.k0 + (int)(t / ((int64_t)bx * by));
            const int64_t v = ii + (int64_t)nx * (jj + (int64_t)ny * kk);
            const double wd = wdmu[v];
            if (wd == 0.0) continue;
            double d[5];
            if (!dmu_dp(pj, gamma, (ii + 0.5) * h, (jj + 0.5) * h, (kk + 0.5) * h, wd, d)) continue;
            const double g = gmu[v];
            for (int q = 0; q < 5; ++q) acc[q] += d[q] * g;
        }
    }
    __shared__ double red[5][256];
    for (int q = 0; q < 5; ++q) red[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 5; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 5) gp[5 * j + threadIdx.x] = red[threadIdx.x][0];
}

cudaError_t pals_chain_gp(const double* p, int m0, double gamma, int nx, int ny, int nz, double h, const double* wdmu,
                          const double* gmu, double* gp, cudaStream_t s) {
    if (m0 <= 0) return cudaSuccess;
    k_chain_gp<<<m0, 256, 0, s>>>(p, m0, gamma, nx, ny, nz, h, wdmu, gmu, gp);
    return cudaGetLastError();
}

// Band lists: for RBF j, the cells of its support box where the Heaviside derivative is
// nonzero and the cell lies inside the support, in box order, with their five
// d mu / d p_{j,q}.  Pass 1 (cell == nullptr) counts them per RBF; pass 2 writes them
// from offs[j].  One block per RBF; the block keeps the box order by an ordered
// compaction (warp ballots, then warp offsets in warp order).
__global__ void k_band(const double* __restrict__ p, int m0, double gamma, int nx, int ny, int nz, double h,
                       const double* __restrict__ wdmu, int64_t* __restrict__ counts, const int64_t* __restrict__ offs,
                       int64_t* __restrict__ cell, double* __restrict__ dval) {
    __shared__ int wtot[32];
    __shared__ int64_t base;
    const int j = blockIdx.x;
    if (j >= m0) return;
    const double* pj = p + 5 * j;
    const Box b = rbf_box(pj[1], pj[2], pj[3], pj[4], gamma, nx, ny, nz, h);
    const bool nonempty = b.i1 >= b.i0 && b.j1 >= b.j0 && b.k1 >= b.k0;
    const int bx = b.i1 - b.i0 + 1, by = b.j1 - b.j0 + 1, bz = b.k1 - b.k0 + 1;
    const int64_t cnt = nonempty ? (int64_t)bx * by * bz : 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) base = cell ? offs[j] : 0;
    __syncthreads();
    for (int64_t t0 = 0; t0 < cnt; t0 += blockDim.x) {
        const int64_t t = t0 + threadIdx.x;
        double d[5];
        int64_t v = 0;
        bool on = false;
        if (t < cnt) {
            const int ii = b.i0 + (int)(t % bx);
            const int jj = b.j0 + (int)((t / bx) % by);
            const int kk = b.k0 + (int)(t / ((int64_t)bx * by));
            v = ii + (int64_t)nx * (jj + (int64_t)ny * kk);
            const double wd = wdmu[v];
            on = wd != 0.0 && dmu_dp(pj, gamma, (ii + 0.5) * h, (jj + 0.5) * h, (kk + 0.5) * h, wd, d);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, on);
        if (lane == 0) wtot[warp] = __popc(bal);
        __syncthreads();
        int64_t before = base;
        for (int w = 0; w < warp; ++w) before += wtot[w];
        if (on && cell) {
            const int64_t at = before + __popc(bal & ((1u << lane) - 1u));
            cell[at] = v;
            for (int q = 0; q < 5; ++q) dval[5 * at + q] = d[q];
        }
        __syncthreads();
        if (threadIdx.x == 0)
            for (int w = 0; w < nw; ++w) base += wtot[w];
        __syncthreads();
    }
    if (!cell && threadIdx.x == 0) counts[j] = base;
}

// J_p[(l + ld i), 5j + q] = sum_v J_mu[(l + ld i), v] dmu_v/dp_{j,q} over RBF j's band
// list: block (j, g) takes rows g * 256 * RPT ..., each thread RPT rows spaced 256 apart
// (consecutive rows across a warp: consecutive detectors l of one source i, so the
// adjoint-field loads coalesce); band entries staged through shared memory in chunks.
template <typename T, int RPT>
__global__ void __launch_bounds__(256) k_chain_jp(const T* __restrict__ X, int kp, int ls, int ld,
                                                  const int64_t* __restrict__ offs, const int64_t* __restrict__ cell,
                                                  const double* __restrict__ dval, T* __restrict__ Jp) {
    constexpr int CH = 64;
    __shared__ double sd[CH][5];
    __shared__ int64_t sv[CH];
    const int j = blockIdx.x;
    const int nr = ls * ld;
    const int64_t e0 = offs[j], e1 = offs[j + 1];
    int row[RPT], l[RPT], i[RPT];
    T acc[RPT][5];
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
        row[u] = (blockIdx.y * RPT + u) * 256 + threadIdx.x;
        l[u] = row[u] % ld;
        i[u] = row[u] / ld;
#pragma unroll
        for (int q = 0; q < 5; ++q) acc[u][q] = ezero<T>();
    }
    for (int64_t t0 = e0; t0 < e1; t0 += CH) {
        const int m = (int)(e1 - t0 < CH ? e1 - t0 : CH);
        __syncthreads();
        for (int u = threadIdx.x; u < m; u += blockDim.x) {
            sv[u] = cell[t0 + u];
            for (int q = 0; q < 5; ++q) sd[u][q] = dval[5 * (t0 + u) + q];
        }
        __syncthreads();
        for (int e = 0; e < m; ++e) {
            const T* xr = X + sv[e] * kp;
#pragma unroll
            for (int u = 0; u < RPT; ++u) {
                if (row[u] >= nr) continue;
                const T jm = escale(-1.0, emul(xr[ls + l[u]], xr[i[u]]));
#pragma unroll
                for (int q = 0; q < 5; ++q) acc[u][q] = eadd(acc[u][q], escale(sd[e][q], jm));
            }
        }
    }
#pragma unroll
    for (int u = 0; u < RPT; ++u)
        if (row[u] < nr)
            for (int q = 0; q < 5; ++q) Jp[row[u] + (int64_t)nr * (5 * j + q)] = acc[u][q];
}

cudaError_t pals_band_count(const double* p, int m0, double gamma, int nx, int ny, int nz, double h,
                            const double* wdmu, int64_t* counts, cudaStream_t s) {
    if (m0 <= 0) return cudaSuccess;
    k_band<<<m0, 256, 0, s>>>(p, m0, gamma, nx, ny, nz, h, wdmu, counts, nullptr, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t pals_band_fill(const double* p, int m0, double gamma, int nx, int ny, int nz, double h,
                           const double* wdmu, const int64_t* offs, int64_t* cell, double* dval, cudaStream_t s) {
    if (m0 <= 0) return cudaSuccess;
    k_band<<<m0, 256, 0, s>>>(p, m0, gamma, nx, ny, nz, h, wdmu, nullptr, offs, cell, dval);
    return cudaGetLastError();
}

cudaError_t pals_chain_jp(bool cplx, int m0, const int64_t* offs, const int64_t* cell, const double* dval,
                          const void* X, int kp, int ls, int ld, double* Jp, cudaStream_t s) {
    if (m0 <= 0) return cudaSuccess;
    const int64_t nr = (int64_t)ls * ld;
    // four rows per thread once there are enough rows to fill the blocks
    if (nr > 1024) {
        const dim3 grd((unsigned)m0, (unsigned)((nr + 1023) / 1024));
        if (cplx)
            k_chain_jp<double2, 4><<<grd, 256, 0, s>>>((const double2*)X, kp, ls, ld, offs, cell, dval, (double2*)Jp);
        else
            k_chain_jp<double, 4><<<grd, 256, 0, s>>>((const double*)X, kp, ls, ld, offs, cell, dval, Jp);
    } else {
        const dim3 grd((unsigned)m0, (unsigned)((nr + 255) / 256));
        if (cplx)
            k_chain_jp<double2, 1><<<grd, 256, 0, s>>>((const double2*)X, kp, ls, ld, offs, cell, dval, (double2*)Jp);
        else
            k_chain_jp<double, 1><<<grd, 256, 0, s>>>((const double*)X, kp, ls, ld, offs, cell, dval, Jp);
    }
    return cudaGetLastError();
}

}  // namespace dotk
