// Shared device-side definitions of the DOT hot-path kernels (sm_103a).
//
// Element types: double (FP64, omega = 0), double2 (complex128), float (FP32),
// float2 (complex64).  Block vectors are stored RHS-innermost: element (v, c) of a
// block with kp columns lives at v * kp + c, so the k columns of one voxel are
// contiguous and a warp reads consecutive columns of consecutive voxels.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace dotk {

// ------------------------------------------------------------------ element ops
template <typename T> struct Elem;
template <> struct Elem<float>   { using R = float;  static constexpr bool cplx = false; };
template <> struct Elem<float2>  { using R = float;  static constexpr bool cplx = true;  };
template <> struct Elem<double>  { using R = double; static constexpr bool cplx = false; };
template <> struct Elem<double2> { using R = double; static constexpr bool cplx = true;  };

template <typename T> __device__ __forceinline__ T ezero();
template <> __device__ __forceinline__ float   ezero<float>()   { return 0.f; }
template <> __device__ __forceinline__ double  ezero<double>()  { return 0.0; }
template <> __device__ __forceinline__ float2  ezero<float2>()  { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 ezero<double2>() { return make_double2(0.0, 0.0); }

__device__ __forceinline__ float   eadd(float a, float b)     { return a + b; }
__device__ __forceinline__ double  eadd(double a, double b)   { return a + b; }
__device__ __forceinline__ float2  eadd(float2 a, float2 b)   { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 eadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float   esub(float a, float b)     { return a - b; }
__device__ __forceinline__ double  esub(double a, double b)   { return a - b; }
__device__ __forceinline__ float2  esub(float2 a, float2 b)   { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 esub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float   emul(float a, float b)     { return a * b; }
__device__ __forceinline__ double  emul(double a, double b)   { return a * b; }
__device__ __forceinline__ float2  emul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 emul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// real scalar times element
__device__ __forceinline__ float   escale(float s, float a)     { return s * a; }
__device__ __forceinline__ double  escale(double s, double a)   { return s * a; }
__device__ __forceinline__ float2  escale(float s, float2 a)    { return make_float2(s * a.x, s * a.y); }
__device__ __forceinline__ double2 escale(double s, double2 a)  { return make_double2(s * a.x, s * a.y); }
// i * w * a (complex only; real types never carry a frequency term)
__device__ __forceinline__ float   emul_i(float, float)          { return 0.f; }
__device__ __forceinline__ double  emul_i(double, double)        { return 0.0; }
__device__ __forceinline__ float2  emul_i(float w, float2 a)     { return make_float2(-w * a.y, w * a.x); }
__device__ __forceinline__ double2 emul_i(double w, double2 a)   { return make_double2(-w * a.y, w * a.x); }
// |a|^2
__device__ __forceinline__ float   eabs2(float a)   { return a * a; }
__device__ __forceinline__ double  eabs2(double a)  { return a * a; }
__device__ __forceinline__ float   eabs2(float2 a)  { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double  eabs2(double2 a) { return a.x * a.x + a.y * a.y; }
// widen to a complex double pair (real part only for real types)
__device__ __forceinline__ double2 ewide(float a)   { return make_double2((double)a, 0.0); }
__device__ __forceinline__ double2 ewide(double a)  { return make_double2(a, 0.0); }
__device__ __forceinline__ double2 ewide(float2 a)  { return make_double2((double)a.x, (double)a.y); }
__device__ __forceinline__ double2 ewide(double2 a) { return a; }
// narrow a complex double scalar to the element type
template <typename T> __device__ __forceinline__ T enarrow(double2 s);
template <> __device__ __forceinline__ float   enarrow<float>(double2 s)   { return (float)s.x; }
template <> __device__ __forceinline__ double  enarrow<double>(double2 s)  { return s.x; }
template <> __device__ __forceinline__ float2  enarrow<float2>(double2 s)  { return make_float2((float)s.x, (float)s.y); }
template <> __device__ __forceinline__ double2 enarrow<double2>(double2 s) { return s; }

// complex-double scalar arithmetic used by the per-column finalisers
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
    // Smith's algorithm (R. L. Smith, CACM 5(8), 1962) to avoid overflow
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, den = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / den, (a.y - a.x * r) / den);
    }
    double r = b.x / b.y, den = b.x * r + b.y;
    return make_double2((a.x * r + a.y) / den, (a.y * r - a.x) / den);
}
__device__ __forceinline__ bool zfinite(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// ------------------------------------------------------- 16-byte vector access
// A thread of the Krylov kernels owns W = 16 / sizeof(T) consecutive columns of a
// voxel and moves them with one 16-byte load or store (block widths are padded to a
// multiple of 4 columns, so every such access is 16-byte aligned).
template <typename T> struct Vec16;
template <> struct Vec16<float>   { static constexpr int W = 4; using L = float4; };
template <> struct Vec16<float2>  { static constexpr int W = 2; using L = float4; };
template <> struct Vec16<double>  { static constexpr int W = 2; using L = double2; };
template <> struct Vec16<double2> { static constexpr int W = 1; using L = double2; };

template <typename T>
struct alignas(16) V16 {
    T e[Vec16<T>::W];
};

template <typename T>
__device__ __forceinline__ V16<T> ld16(const T* __restrict__ p) {
    typename Vec16<T>::L t = *reinterpret_cast<const typename Vec16<T>::L*>(p);
    V16<T> r;
    memcpy(&r, &t, 16);
    return r;
}
template <typename T>
__device__ __forceinline__ void st16(T* __restrict__ p, const V16<T>& v) {
    typename Vec16<T>::L t;
    memcpy(&t, &v, 16);
    *reinterpret_cast<typename Vec16<T>::L*>(p) = t;
}

// ---------------------------------------------------------------- operator
// Coefficients of (A(mu) + i w I), per unit volume, packed per voxel:
//   (A u)_v = dre_v u_v + i w u_v - sum_faces c_f u_nb
// cx couples v and v+1 (0 on the +x boundary), cy v and v+nx, cz v and v+nx*ny; one
// aligned load brings a voxel's four coefficients.  dinv = 1 / (dre + i w) is the
// Jacobi preconditioner, stored in the element type.
template <typename R>
struct alignas(4 * sizeof(R)) Cf4 {
    R cx, cy, cz, dre;
};

template <typename T>
struct Op {
    using R = typename Elem<T>::R;
    const Cf4<R>* cf;
    const T* dinv;
    R w;
    int nx, ny, nz;
};

// y = A x at voxel v, column c of a block with kp columns.
template <typename T>
__device__ __forceinline__ T apply_at(const Op<T>& op, const T* __restrict__ x, int64_t v, int kp, int c) {
    using R = typename Elem<T>::R;
    // grids hold fewer than 2^31 cells, so the index split runs in 32-bit arithmetic
    const int vi = (int)v;
    const int nxy = op.nx * op.ny;
    const int kz = vi / nxy;
    const int rem = vi - kz * nxy;
    const int j = rem / op.nx;
    const int i = rem - j * op.nx;
    const int64_t e = v * kp + c;
    const Cf4<R> cv = op.cf[vi];
    T xc = x[e];
    T acc = escale(cv.dre, xc);
    if (Elem<T>::cplx) acc = eadd(acc, emul_i(op.w, xc));
    if (i > 0)          acc = esub(acc, escale(op.cf[vi - 1].cx, x[e - kp]));
    if (i < op.nx - 1)  acc = esub(acc, escale(cv.cx, x[e + kp]));
    if (j > 0)          acc = esub(acc, escale(op.cf[vi - op.nx].cy, x[e - (int64_t)op.nx * kp]));
    if (j < op.ny - 1)  acc = esub(acc, escale(cv.cy, x[e + (int64_t)op.nx * kp]));
    if (kz > 0)         acc = esub(acc, escale(op.cf[vi - nxy].cz, x[e - (int64_t)nxy * kp]));
    if (kz < op.nz - 1) acc = esub(acc, escale(cv.cz, x[e + (int64_t)nxy * kp]));
    return acc;
}

}  // namespace dotk
