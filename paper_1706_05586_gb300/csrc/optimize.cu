// Optimized simultaneous sources and detectors (Sec. 3.2, Algorithm 1) and their
// complementary random columns (Eqs. (newW), (newV)).
//
// The Jacobian tensor J_ijk = -c_i^T A^{-1} dA/dp_k A^{-1} b_j (Eq. (Jtensor)) is
// formed on the device from one block solve of every physical source and detector.
// The Tucker2 alternating iteration then needs, per half-sweep, a contraction of J
// with the current detector (or source) vectors and the Gram matrix of the
// resulting unfolding; both run on the device in FP64.  The leading eigenvectors of
// the small symmetric Gram matrices (n_d x n_d or n_s x n_s) are computed on the
// host (Householder tridiagonalisation and implicit QL), since they are the left
// singular vectors of the unfoldings J~, K~, L~ of Eqs. (Jtilde), (Ktilde), (Ltilde).
// A complex J enters with real W, V through Re(X X^H), i.e. its real and imaginary
// parts act as separate parameter columns.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "dot.h"
#include "dot_kernels.cuh"
#include "dot_internal.h"

namespace dotk {

// ------------------------------------------------------------------ device
// Partial Gram sums over one chunk of m: G_s[a, b] = Re sum_{m in chunk s} X[a + ldx m]
// conj(X[b + ldx m]) for a, b < n (16 x 16 tiles; blockIdx.z = chunk s of length mchunk).
template <typename T>
__global__ void k_gram(const T* __restrict__ X, int n, int64_t M, int64_t ldx, int64_t mchunk,
                       double* __restrict__ G) {
    __shared__ double2 sa[16][17];
    __shared__ double2 sb[16][17];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int a = blockIdx.x * 16 + tx, b = blockIdx.y * 16 + ty;
    const int64_t mb = (int64_t)blockIdx.z * mchunk, me = M < mb + mchunk ? M : mb + mchunk;
    G += (size_t)blockIdx.z * n * n;
    double acc = 0.0;
    for (int64_t m0 = mb; m0 < me; m0 += 16) {
        // load X[blockIdx.x*16 + r, m0 + c] and X[blockIdx.y*16 + r, m0 + c]
        const int r = tx, c = ty;
        const int64_t m = m0 + c;
        const int ra = blockIdx.x * 16 + r, rb = blockIdx.y * 16 + r;
        sa[c][r] = (ra < n && m < me) ? ewide(X[ra + ldx * m]) : make_double2(0.0, 0.0);
        sb[c][r] = (rb < n && m < me) ? ewide(X[rb + ldx * m]) : make_double2(0.0, 0.0);
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const double2 xa = sa[u][tx], xb = sb[u][ty];
            acc += xa.x * xb.x + xa.y * xb.y;
        }
        __syncthreads();
    }
    if (a < n && b < n) G[a + (int64_t)n * b] = acc;
}

// K[j + ns (k + npar l)] = sum_m V[m + nd l] J[m + nd j + nd ns k]: one block per (j, k).
template <typename T>
__global__ void k_contract_det(const T* __restrict__ J, int nd, int ns, int npar, const double* __restrict__ V, int q,
                               T* __restrict__ K) {
    __shared__ double2 red[8][256];
    const int j = blockIdx.x % ns, k = blockIdx.x / ns;
    double2 acc[8];
    for (int l = 0; l < 8; ++l) acc[l] = make_double2(0.0, 0.0);
    for (int m = threadIdx.x; m < nd; m += blockDim.x) {
        const double2 x = ewide(J[m + (int64_t)nd * j + (int64_t)nd * ns * k]);
        for (int l = 0; l < q && l < 8; ++l) {
            const double v = V[m + (int64_t)nd * l];
            acc[l].x += v * x.x;
            acc[l].y += v * x.y;
        }
    }
    for (int l = 0; l < q && l < 8; ++l) red[l][threadIdx.x] = acc[l];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int l = 0; l < q && l < 8; ++l) {
                red[l][threadIdx.x].x += red[l][threadIdx.x + w].x;
                red[l][threadIdx.x].y += red[l][threadIdx.x + w].y;
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int l = 0; l < q && l < 8; ++l) K[j + (int64_t)ns * (k + (int64_t)npar * l)] = enarrow<T>(red[l][0]);
}

// L[i + nd (k + npar l)] = sum_m W[m + ns l] J[i + nd m + nd ns k]: one thread per (i, k, l).
template <typename T>
__global__ void k_contract_src(const T* __restrict__ J, int nd, int ns, int npar, const double* __restrict__ W, int q,
                               T* __restrict__ L) {
    const int64_t total = (int64_t)nd * npar * q;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t % nd);
        const int64_t kl = t / nd;
        const int k = (int)(kl % npar), l = (int)(kl / npar);
        double2 acc = make_double2(0.0, 0.0);
        for (int m = 0; m < ns; ++m) {
            const double2 x = ewide(J[i + (int64_t)nd * m + (int64_t)nd * ns * k]);
            const double w = W[m + (int64_t)ns * l];
            acc.x += w * x.x;
            acc.y += w * x.y;
        }
        L[i + (int64_t)nd * (k + (int64_t)npar * l)] = enarrow<T>(acc);
    }
}

// Large Gram matrices (n >= 128): 64 x 64 output tiles, each of the 256 threads holding
// a 4 x 4 block of sums in registers, the rows staged 16 columns at a time through
// shared memory; blockIdx.z = chunk of the long dimension as in k_gram.  Every element
// of X is then read once per tile row and per tile column (n / 64 times) instead of
// n / 16 times, which makes the J~ Gram of a 512 x 512 x 5,000 tensor bound by the FP64
// pipe rather than by L2.
template <typename T>
__global__ void __launch_bounds__(256) k_gram64(const T* __restrict__ X, int n, int64_t M, int64_t ldx,
                                                int64_t mchunk, double* __restrict__ G) {
    __shared__ double2 sa[16][64];
    __shared__ double2 sb[16][64];
    const int t = threadIdx.x;
    const int tr = t % 16, tc = t / 16;   // this thread's rows a0 + 4 tr + u, columns b0 + 4 tc + w
    const int a0 = blockIdx.x * 64, b0 = blockIdx.y * 64;
    const int64_t mb = (int64_t)blockIdx.z * mchunk, me = M < mb + mchunk ? M : mb + mchunk;
    G += (size_t)blockIdx.z * n * n;
    double acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[u][w] = 0.0;
    for (int64_t m0 = mb; m0 < me; m0 += 16) {
        // 64 rows x 16 columns of each operand: thread t loads rows t % 64, columns t / 64 + 4 k
        for (int k = 0; k < 4; ++k) {
            const int r = t % 64, c = t / 64 + 4 * k;
            const int64_t m = m0 + c;
            const int ra = a0 + r, rb = b0 + r;
            sa[c][r] = (ra < n && m < me) ? ewide(X[ra + ldx * m]) : make_double2(0.0, 0.0);
            sb[c][r] = (rb < n && m < me) ? ewide(X[rb + ldx * m]) : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll 4
        for (int c = 0; c < 16; ++c) {
            double2 xa[4], xb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                xa[u] = sa[c][4 * tr + u];
                xb[u] = sb[c][4 * tc + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[u][w] += xa[u].x * xb[w].x + xa[u].y * xb[w].y;
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int a = a0 + 4 * tr + u, b = b0 + 4 * tc + w;
            if (a < n && b < n) G[a + (size_t)n * b] = acc[u][w];
        }
}

// G = sum of the chunk partials in chunk order (deterministic).
__global__ void k_gram_sum(const double* __restrict__ part, int chunks, int64_t nn, double* __restrict__ G) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < chunks; ++c) acc += part[(size_t)c * nn + t];
        G[t] = acc;
    }
}

// Gram matrix of the n rows of X.  Small n gives few 16 x 16 tiles, so the long
// dimension M is split into chunks (about 608 blocks in all, at most kGramChunks) whose
// partial sums go to `part` and are added in chunk order.
static cudaError_t gram(bool cplx, const void* X, int n, int64_t M, int64_t ldx, double* G, double* part,
                        cudaStream_t s) {
    const bool big = n >= 128;
    const int tn = big ? (n + 63) / 64 : (n + 15) / 16;
    int64_t chunks = std::max<int64_t>(1, std::min<int64_t>(kGramChunks, 608 / ((int64_t)tn * tn)));
    chunks = std::min<int64_t>(chunks, std::max<int64_t>(1, M / 256));
    int64_t mchunk = (M + chunks - 1) / chunks;
    mchunk = (mchunk + 15) / 16 * 16;
    chunks = std::max<int64_t>(1, (M + mchunk - 1) / mchunk);
    if ((int64_t)n * n * chunks > kGramPartDoubles) chunks = 1, mchunk = M;
    double* dst = chunks > 1 ? part : G;
    dim3 grd(tn, tn, (unsigned)chunks);
    if (big) {
        if (cplx)
            k_gram64<double2><<<grd, 256, 0, s>>>((const double2*)X, n, M, ldx, mchunk, dst);
        else
            k_gram64<double><<<grd, 256, 0, s>>>((const double*)X, n, M, ldx, mchunk, dst);
    } else {
        dim3 blk(16, 16);
        if (cplx)
            k_gram<double2><<<grd, blk, 0, s>>>((const double2*)X, n, M, ldx, mchunk, dst);
        else
            k_gram<double><<<grd, blk, 0, s>>>((const double*)X, n, M, ldx, mchunk, dst);
    }
    if (chunks > 1) {
        const int64_t nn = (int64_t)n * n;
        k_gram_sum<<<(unsigned)std::min<int64_t>((nn + 255) / 256, 1024), 256, 0, s>>>(part, (int)chunks, nn, G);
    }
    return cudaGetLastError();
}

static cudaError_t contract_det(bool cplx, const void* J, int nd, int ns, int npar, const double* V, int q, void* K,
                                cudaStream_t s) {
    const int th = 128;
    const unsigned blocks = (unsigned)((int64_t)ns * npar);
    if (cplx)
        k_contract_det<double2><<<blocks, th, 0, s>>>((const double2*)J, nd, ns, npar, V, q, (double2*)K);
    else
        k_contract_det<double><<<blocks, th, 0, s>>>((const double*)J, nd, ns, npar, V, q, (double*)K);
    return cudaGetLastError();
}

static cudaError_t contract_src(bool cplx, const void* J, int nd, int ns, int npar, const double* W, int q, void* L,
                                cudaStream_t s) {
    const int64_t total = (int64_t)nd * npar * q;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 32);
    if (blocks < 1) blocks = 1;
    if (cplx)
        k_contract_src<double2><<<blocks, 256, 0, s>>>((const double2*)J, nd, ns, npar, W, q, (double2*)L);
    else
        k_contract_src<double><<<blocks, 256, 0, s>>>((const double*)J, nd, ns, npar, W, q, (double*)L);
    return cudaGetLastError();
}

// ------------------------------------------------------------------- host
// Symmetric eigen-decomposition (column-major n x n A, destroyed): Householder reduction
// to tridiagonal form with the orthogonal factor accumulated, then implicit QL sweeps
// with Wilkinson shifts (Golub and Van Loan, Sec. 8.3).  Eigenvalues ascending in w,
// eigenvectors in the columns of Q.
int symmetric_eigen(int n, std::vector<double>& A, std::vector<double>& w, std::vector<double>& Q) {
    auto at = [&](std::vector<double>& M, int r, int c) -> double& { return M[(size_t)r + (size_t)n * c]; };
    Q.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) at(Q, i, i) = 1.0;
    std::vector<double> v(n), p(n), qv(n);
    std::vector<double> d(n), e(n, 0.0);
    for (int k = 0; k + 2 < n; ++k) {
        double norm = 0.0;
        for (int i = k + 1; i < n; ++i) norm += at(A, i, k) * at(A, i, k);
        norm = std::sqrt(norm);
        if (norm == 0.0) continue;
        const double x0 = at(A, k + 1, k);
        const double alpha = x0 > 0 ? -norm : norm;
        for (int i = 0; i < n; ++i) v[i] = 0.0;
        for (int i = k + 1; i < n; ++i) v[i] = at(A, i, k);
        v[k + 1] -= alpha;
        double vn = 0.0;
        for (int i = k + 1; i < n; ++i) vn += v[i] * v[i];
        vn = std::sqrt(vn);
        if (vn == 0.0) continue;
        for (int i = k + 1; i < n; ++i) v[i] /= vn;
        // A <- H A H on the whole matrix (H = I - 2 v v^T acts on rows/cols k+1..n-1)
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = k + 1; j < n; ++j) s += at(A, i, j) * v[j];
            p[i] = s;
        }
        double K = 0.0;
        for (int i = k + 1; i < n; ++i) K += v[i] * p[i];
        for (int i = 0; i < n; ++i) qv[i] = p[i] - K * v[i];
        for (int c = 0; c < n; ++c)
            for (int r = 0; r < n; ++r) at(A, r, c) -= 2.0 * (v[r] * qv[c] + qv[r] * v[c]);
        // Q <- Q H
        for (int r = 0; r < n; ++r) {
            double s = 0.0;
            for (int j = k + 1; j < n; ++j) s += at(Q, r, j) * v[j];
            for (int j = k + 1; j < n; ++j) at(Q, r, j) -= 2.0 * s * v[j];
        }
    }
    for (int i = 0; i < n; ++i) d[i] = at(A, i, i);
    for (int i = 0; i + 1 < n; ++i) e[i] = at(A, i + 1, i);
    // implicit QL on (d, e).  An off-diagonal is negligible next to its two diagonal
    // neighbours or next to the whole matrix (the largest |d_i| + |e_i|): Gram matrices of
    // low-rank unfoldings have a cluster of eigenvalues that are zero up to rounding,
    // whose rounding-level off-diagonals a purely local test would keep sweeping.
    double tnorm = 0.0;
    for (int i = 0; i < n; ++i) tnorm = std::max(tnorm, std::fabs(d[i]) + (i + 1 < n ? std::fabs(e[i]) : 0.0));
    for (int l = 0; l < n; ++l) {
        int iter = 0;
        while (true) {
            int m = l;
            for (; m + 1 < n; ++m) {
                const double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
                if (std::fabs(e[m]) <= 1e-15 * dd || std::fabs(e[m]) <= 1e-16 * tnorm) break;
            }
            if (m == l) break;
            if (++iter > 60) return record_error(DOT_EBREAKDOWN, "symmetric eigensolver did not converge");
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = std::hypot(g, 1.0);
            g = d[m] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
            double s = 1.0, c = 1.0, pp = 0.0;
            int i = m - 1;
            for (; i >= l; --i) {
                double f = s * e[i], b = c * e[i];
                r = std::hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {
                    d[i + 1] -= pp;
                    e[m] = 0.0;
                    break;
                }
                s = f / r;
                c = g / r;
                g = d[i + 1] - pp;
                r = (d[i] - g) * s + 2.0 * c * b;
                pp = s * r;
                d[i + 1] = g + pp;
                g = c * r - b;
                for (int k = 0; k < n; ++k) {
                    f = at(Q, k, i + 1);
                    at(Q, k, i + 1) = s * at(Q, k, i) + c * f;
                    at(Q, k, i) = c * at(Q, k, i) - s * f;
                }
            }
            if (r == 0.0 && i >= l) continue;
            d[l] -= pp;
            e[l] = g;
            e[m] = 0.0;
        }
    }
    // sort ascending
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return d[a] < d[b]; });
    std::vector<double> Qs((size_t)n * n);
    w.resize(n);
    for (int c = 0; c < n; ++c) {
        w[c] = d[idx[c]];
        for (int r = 0; r < n; ++r) Qs[(size_t)r + (size_t)n * c] = Q[(size_t)r + (size_t)n * idx[c]];
    }
    Q.swap(Qs);
    return DOT_OK;
}

// The q leading eigenvectors (largest eigenvalues first) of a symmetric n x n matrix.
int leading_vectors(int n, const std::vector<double>& G, int q, std::vector<double>& out) {
    std::vector<double> A(G), w, Q;
    const int rc = symmetric_eigen(n, A, w, Q);
    if (rc != DOT_OK) return rc;
    out.assign((size_t)n * q, 0.0);
    for (int c = 0; c < q; ++c)
        for (int r = 0; r < n; ++r) out[(size_t)r + (size_t)n * c] = Q[(size_t)r + (size_t)n * (n - 1 - c)];
    return DOT_OK;
}

double projector_change(int n, int q, const std::vector<double>& A, const std::vector<double>& B) {
    double s = 0.0;
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            double pa = 0.0, pb = 0.0;
            for (int l = 0; l < q; ++l) {
                pa += A[(size_t)r + (size_t)n * l] * A[(size_t)c + (size_t)n * l];
                pb += B[(size_t)r + (size_t)n * l] * B[(size_t)c + (size_t)n * l];
            }
            s += (pa - pb) * (pa - pb);
        }
    return std::sqrt(s);
}

// [What, (I - What What^T) Ytil], n x (q + m), column-major.
void complement(int n, int q, const std::vector<double>& What, int m, const double* Ytil, double* out) {
    for (int c = 0; c < q; ++c)
        for (int r = 0; r < n; ++r) out[(size_t)r + (size_t)n * c] = What[(size_t)r + (size_t)n * c];
    for (int c = 0; c < m; ++c) {
        const double* y = Ytil + (size_t)n * c;
        double* o = out + (size_t)n * (q + c);
        for (int r = 0; r < n; ++r) o[r] = y[r];
        for (int l = 0; l < q; ++l) {
            double dotp = 0.0;
            for (int r = 0; r < n; ++r) dotp += What[(size_t)r + (size_t)n * l] * y[r];
            for (int r = 0; r < n; ++r) o[r] -= dotp * What[(size_t)r + (size_t)n * l];
        }
    }
}

int optimize_from_tensor(bool cplx, const void* Jd, int nd, int ns, int npar, int qs, int qd, int maxit, double tol,
                         void* scratch_K, void* scratch_L, double* dG, double* dGpart, double* dVW, cudaStream_t s,
                         std::vector<double>& What, std::vector<double>& Vhat, int* sweeps, double* objective) {
    const size_t es = cplx ? 16 : 8;
    (void)es;
    std::vector<double> G;
    auto fetch = [&](int n) -> int {
        G.resize((size_t)n * n);
        cudaError_t e = cudaMemcpyAsync(G.data(), dG, (size_t)n * n * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return record_error(DOT_ECUDA, std::string("gram copy: ") + cudaGetErrorString(e));
        return DOT_OK;
    };
    auto upload = [&](const std::vector<double>& h) -> int {
        cudaError_t e = cudaMemcpyAsync(dVW, h.data(), h.size() * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return record_error(DOT_ECUDA, std::string("vector upload: ") + cudaGetErrorString(e));
        return DOT_OK;
    };
#define OPT_TRY(x)              \
    do {                        \
        int rc_ = (x);          \
        if (rc_ != DOT_OK) return rc_; \
    } while (0)
#define OPT_CK(x)                                                                                    \
    do {                                                                                             \
        cudaError_t e_ = (x);                                                                        \
        if (e_ != cudaSuccess) return record_error(DOT_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)
    // step (1): V~ from J~ = [J_{:,1,:} ... J_{:,ns,:}], rows m, columns j + ns k, stride nd
    OPT_CK(gram(cplx, Jd, nd, (int64_t)ns * npar, nd, dG, dGpart, s));
    OPT_TRY(fetch(nd));
    OPT_TRY(leading_vectors(nd, G, qd, Vhat));
    std::vector<double> Wold, Vold;
    int it = 0;
    for (it = 1; it <= maxit; ++it) {
        // step (2): W~ from K~ = [K_1 ... K_qd]
        OPT_TRY(upload(Vhat));
        OPT_CK(contract_det(cplx, Jd, nd, ns, npar, dVW, qd, scratch_K, s));
        OPT_CK(gram(cplx, scratch_K, ns, (int64_t)npar * qd, ns, dG, dGpart, s));
        OPT_TRY(fetch(ns));
        std::vector<double> Wn;
        OPT_TRY(leading_vectors(ns, G, qs, Wn));
        // step (3): V~ from L~ = [L_1 ... L_qs]
        OPT_TRY(upload(Wn));
        OPT_CK(contract_src(cplx, Jd, nd, ns, npar, dVW, qs, scratch_L, s));
        OPT_CK(gram(cplx, scratch_L, nd, (int64_t)npar * qs, nd, dG, dGpart, s));
        OPT_TRY(fetch(nd));
        std::vector<double> Vn;
        OPT_TRY(leading_vectors(nd, G, qd, Vn));
        double change = projector_change(nd, qd, Vn, Vhat);
        if (!What.empty()) change += projector_change(ns, qs, Wn, What);
        What.swap(Wn);
        Vhat.swap(Vn);
        if (it > 1 && change < tol) break;
    }
    if (it > maxit) it = maxit;
    *sweeps = it;
    // objective ||(W^T (x) V^T) J||_F^2 = ||W^T K~||_F^2 with K~ from the final V^
    OPT_TRY(upload(Vhat));
    OPT_CK(contract_det(cplx, Jd, nd, ns, npar, dVW, qd, scratch_K, s));
    OPT_CK(gram(cplx, scratch_K, ns, (int64_t)npar * qd, ns, dG, dGpart, s));
    OPT_TRY(fetch(ns));
    double obj = 0.0;
    for (int l = 0; l < qs; ++l)
        for (int a = 0; a < ns; ++a)
            for (int b = 0; b < ns; ++b)
                obj += What[(size_t)a + (size_t)ns * l] * G[(size_t)a + (size_t)ns * b] * What[(size_t)b + (size_t)ns * l];
    *objective = obj;
    return DOT_OK;
#undef OPT_TRY
#undef OPT_CK
}

}  // namespace dotk

extern "C" int dot_symeig(int n, const double* A, double* evals, double* evecs) {
    if (n < 1 || !A || !evals || !evecs) return dotk::record_error(DOT_EINVAL, "bad dot_symeig arguments");
    std::vector<double> M(A, A + (size_t)n * n), w, Q;
    const int rc = dotk::symmetric_eigen(n, M, w, Q);
    if (rc != DOT_OK) return rc;
    std::memcpy(evals, w.data(), (size_t)n * 8);
    std::memcpy(evecs, Q.data(), (size_t)n * n * 8);
    return DOT_OK;
}
