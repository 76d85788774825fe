"""Thin ctypes binding of libdot.so (the C ABI declared in include/dot.h).

Every function here has the name of the C entry point it marshals to and does
argument marshalling only; all arithmetic runs in the library's CUDA kernels.
Loading fails loudly (ImportError) when libdot.so is missing: there is no CPU
fallback.  Build it with `python -m paper_1706_05586_gb300.build`.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libdot.so")

DOT_OK = 0
DOT_EINVAL = -1
DOT_ESTATE = -2
DOT_ENOMEM = -3
DOT_ECUDA = -4
DOT_ENOTCONV = -5
DOT_EBREAKDOWN = -6
DOT_ETIMEOUT = -7
BC_ROBIN = 0
BC_DIRICHLET = 1
PREC_FP64 = 0
PREC_MIXED = 1

# name -> argument types (all return int unless listed in _RESTYPE)
SIGNATURES = {
    "dot_create": [C.POINTER(C.c_void_p), C.c_int],
    "dot_destroy": [C.c_void_p],
    "dot_last_error": [],
    "dot_set_stream": [C.c_void_p, C.c_void_p],
    "dot_set_grid": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double, C.POINTER(C.c_int)],
    "dot_set_omega": [C.c_void_p, C.c_double],
    "dot_set_diffusion": [C.c_void_p, C.c_void_p],
    "dot_set_mua": [C.c_void_p, C.c_void_p],
    "dot_set_pals": [C.c_void_p, C.c_int, C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double,
                     C.c_double],
    "dot_set_pals_dev": [C.c_void_p, C.c_int, C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double,
                         C.c_double],
    "dot_set_sources": [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p],
    "dot_set_detectors": [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p],
    "dot_set_data": [C.c_void_p, C.c_void_p, C.c_int],
    "dot_set_sampling": [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p],
    "dot_set_solver": [C.c_void_p, C.c_int, C.c_double, C.c_int],
    "dot_set_refinement": [C.c_void_p, C.c_double],
    "dot_misfit": [C.c_void_p, C.c_void_p],
    "dot_measurements": [C.c_void_p, C.c_void_p],
    "dot_forward_model": [C.c_void_p, C.c_void_p],
    "dot_gradient": [C.c_void_p, C.c_void_p, C.c_void_p],
    "dot_gradient_dev": [C.c_void_p, C.c_void_p, C.c_void_p],
    "dot_jacobian_mua": [C.c_void_p, C.c_void_p],
    "dot_jacobian_p": [C.c_void_p, C.c_void_p],
    "dot_get_mua": [C.c_void_p, C.c_void_p],
    "dot_get_fields": [C.c_void_p, C.c_void_p, C.c_void_p],
    "dot_get_stats": [C.c_void_p, C.c_void_p],
    "dot_apply": [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p],
    "dot_probe_wait": [C.c_void_p, C.c_int64],
    "dot_set_kernel_timing": [C.c_void_p, C.c_int],
    "dot_set_stencil_path": [C.c_void_p, C.c_int],
    "dot_set_launch_options": [C.c_void_p, C.c_int, C.c_int],
    "dot_set_direction_ring": [C.c_void_p, C.c_int],
    "dot_gradient_batch": [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p],
    "dot_optimized_sampling": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.c_void_p, C.c_int,
                               C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "dot_symeig": [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p],
    "dot_restrict_misfit_noalloc": [C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p],
    "dot_get_kernel_timing": [C.c_void_p, C.c_void_p],
}
_RESTYPE = {"dot_last_error": C.c_char_p}


class DotStats(C.Structure):
    _fields_ = [("k", C.c_int32), ("iters_max", C.c_int32), ("iters_sum", C.c_int64),
                ("outer_steps", C.c_int32), ("status", C.c_int32), ("relres_max", C.c_double),
                ("columns_solved", C.c_int64), ("block_solves", C.c_int64), ("ms_setup", C.c_double),
                ("ms_solve", C.c_double), ("ms_post", C.c_double), ("kernel_launches", C.c_int64),
                ("tuned_tma", C.c_int32), ("tuned_blocks_per_sm", C.c_int32), ("fused_direction", C.c_int32),
                ("reserved", C.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class DotKernelTiming(C.Structure):
    _fields_ = [("launches", C.c_int64 * 5), ("ms", C.c_double * 5), ("bytes", C.c_double * 5)]

    def as_dict(self):
        names = ("stencil", "update", "direction", "refine_residual", "flush")
        return {nm: {"launches": int(self.launches[i]), "ms": float(self.ms[i]), "bytes": float(self.bytes[i])}
                for i, nm in enumerate(names)}


class DotError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


_lib = None


def load(path: str | None = None):
    """Load libdot.so once; raises ImportError if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libdot.so not found at {path}; run `python -m paper_1706_05586_gb300.build`")
    lib = C.CDLL(path)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = _RESTYPE.get(name, C.c_int)
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _check(rc, allow=()):
    if rc != DOT_OK and rc not in allow:
        raise DotError(rc, load().dot_last_error().decode())
    return rc


def _f64(a, cplx=False):
    a = np.asarray(a)
    if cplx:
        return np.ascontiguousarray(a, dtype=np.complex128)
    return np.ascontiguousarray(a, dtype=np.float64)


def _fortran(a, cplx=False):
    return np.asfortranarray(np.asarray(a, dtype=np.complex128 if cplx else np.float64))


# ------------------------------------------------------------ C-named wrappers
def dot_create(device: int = 0):
    h = C.c_void_p()
    _check(load().dot_create(C.byref(h), device))
    return h


def dot_destroy(ctx):
    return _check(load().dot_destroy(ctx))


def dot_last_error() -> str:
    return load().dot_last_error().decode()


def dot_set_stream(ctx, stream_handle: int | None):
    return _check(load().dot_set_stream(ctx, C.c_void_p(stream_handle) if stream_handle else None))


def dot_set_grid(ctx, nx, ny, nz, h, bc):
    arr = (C.c_int * 6)(*[int(b) for b in bc])
    return _check(load().dot_set_grid(ctx, nx, ny, nz, float(h), arr))


def dot_set_omega(ctx, omega_over_nu):
    return _check(load().dot_set_omega(ctx, float(omega_over_nu)))


def dot_set_diffusion(ctx, D):
    D = _f64(D)
    return _check(load().dot_set_diffusion(ctx, _ptr(D)))


def dot_set_mua(ctx, mu):
    mu = _f64(mu)
    return _check(load().dot_set_mua(ctx, _ptr(mu)))


def dot_set_pals(ctx, p, mu_in, mu_out, c, eps, gamma):
    p = _f64(p)
    return _check(load().dot_set_pals(ctx, p.size // 5, _ptr(p), mu_in, mu_out, c, eps, gamma))


def dot_set_pals_dev(ctx, m0, p_dev_ptr: int, mu_in, mu_out, c, eps, gamma):
    return _check(load().dot_set_pals_dev(ctx, m0, C.c_void_p(p_dev_ptr), mu_in, mu_out, c, eps, gamma))


def _csc(csc):
    colptr, rows, vals = csc
    return (np.ascontiguousarray(colptr, dtype=np.int64), np.ascontiguousarray(rows, dtype=np.int32),
            np.ascontiguousarray(vals, dtype=np.float64))


def dot_set_sources(ctx, csc):
    cp, rw, vv = _csc(csc)
    return _check(load().dot_set_sources(ctx, cp.size - 1, _ptr(cp), _ptr(rw), _ptr(vv)))


def dot_set_detectors(ctx, csc):
    cp, rw, vv = _csc(csc)
    return _check(load().dot_set_detectors(ctx, cp.size - 1, _ptr(cp), _ptr(rw), _ptr(vv)))


def dot_set_data(ctx, M):
    M = np.asarray(M)
    is_c = np.iscomplexobj(M)
    Mf = _fortran(M, is_c)
    return _check(load().dot_set_data(ctx, _ptr(Mf), int(is_c)))


def dot_set_sampling(ctx, W, V):
    Wf, Vf = _fortran(W), _fortran(V)
    return _check(load().dot_set_sampling(ctx, Wf.shape[1], _ptr(Wf), Vf.shape[1], _ptr(Vf)))


def dot_set_solver(ctx, precision, rtol, maxit=0):
    return _check(load().dot_set_solver(ctx, int(precision), float(rtol), int(maxit)))


def dot_set_refinement(ctx, delta):
    return _check(load().dot_set_refinement(ctx, float(delta)))


def dot_misfit(ctx, allow=()):
    f = np.zeros(1)
    rc = _check(load().dot_misfit(ctx, _ptr(f)), allow)
    return float(f[0]), rc


def dot_measurements(ctx, ls, ld, cplx, allow=()):
    S = np.zeros((ld, ls), dtype=np.complex128 if cplx else np.float64, order="F")
    rc = _check(load().dot_measurements(ctx, _ptr(S)), allow)
    return S, rc


def dot_forward_model(ctx, ns, nd, cplx, allow=()):
    M = np.zeros((nd, ns), dtype=np.complex128 if cplx else np.float64, order="F")
    rc = _check(load().dot_forward_model(ctx, _ptr(M)), allow)
    return M, rc


def dot_gradient(ctx, ng, allow=()):
    f = np.zeros(1)
    g = np.zeros(ng)
    rc = _check(load().dot_gradient(ctx, _ptr(f), _ptr(g)), allow)
    return float(f[0]), g, rc


def dot_gradient_dev(ctx, f_ptr, g_ptr, allow=()):
    """dot_gradient into device memory: f_ptr, g_ptr are device addresses (e.g. the
    data_ptr() of float64 CUDA tensors of 1 and n_p elements)."""
    return _check(load().dot_gradient_dev(ctx, C.c_void_p(f_ptr), C.c_void_p(g_ptr)), allow)


def dot_jacobian_mua(ctx, ls, ld, n, cplx, allow=()):
    J = np.zeros((ls * ld, n), dtype=np.complex128 if cplx else np.float64, order="F")
    rc = _check(load().dot_jacobian_mua(ctx, _ptr(J)), allow)
    return J, rc


def dot_jacobian_p(ctx, ls, ld, npar, cplx, allow=()):
    J = np.zeros((ls * ld, npar), dtype=np.complex128 if cplx else np.float64, order="F")
    rc = _check(load().dot_jacobian_p(ctx, _ptr(J)), allow)
    return J, rc


def dot_get_mua(ctx, n):
    mu = np.zeros(n)
    _check(load().dot_get_mua(ctx, _ptr(mu)))
    return mu


def dot_get_fields(ctx, n, ls, ld, cplx):
    dt = np.complex128 if cplx else np.float64
    U = np.zeros((n, ls), dtype=dt, order="F")
    Z = np.zeros((n, ld), dtype=dt, order="F")
    _check(load().dot_get_fields(ctx, _ptr(U), _ptr(Z)))
    return U, Z


def dot_get_stats(ctx) -> dict:
    s = DotStats()
    _check(load().dot_get_stats(ctx, C.byref(s)))
    return s.as_dict()


def dot_optimized_sampling(ctx, qs, qd, ns, nd, ls, ld, Ytil=None, Ztil=None, maxit=100, tol=1e-10):
    W = np.zeros((ns, ls), order="F")
    V = np.zeros((nd, ld), order="F")
    Yf = None if Ytil is None else _fortran(Ytil)
    Zf = None if Ztil is None else _fortran(Ztil)
    sweeps = C.c_int(0)
    obj = C.c_double(0.0)
    _check(load().dot_optimized_sampling(ctx, qs, qd, maxit, tol, ls, _ptr(Yf), ld, _ptr(Zf), _ptr(W), _ptr(V),
                                         C.byref(sweeps), C.byref(obj)))
    return W, V, sweeps.value, obj.value


def dot_symeig(A):
    A = _fortran(A)
    n = A.shape[0]
    w = np.zeros(n)
    Q = np.zeros((n, n), order="F")
    _check(load().dot_symeig(n, _ptr(A), _ptr(w), _ptr(Q)))
    return w, Q


def dot_set_launch_options(ctx, graphs=True, autotune=False):
    return _check(load().dot_set_launch_options(ctx, int(bool(graphs)), int(bool(autotune))))


def dot_set_direction_ring(ctx, slots=0):
    return _check(load().dot_set_direction_ring(ctx, int(slots)))


def dot_gradient_batch(ctxs, ngs, allow=()):
    """Misfit and gradient of several contexts; ngs[i] is the gradient length of ctxs[i]."""
    n = len(ctxs)
    handles = (C.c_void_p * n)(*[c.value if hasattr(c, "value") else c for c in ctxs])
    f = np.zeros(n)
    gs = [np.zeros(m) for m in ngs]
    gp = (C.c_void_p * n)(*[g.ctypes.data for g in gs])
    rc = _check(load().dot_gradient_batch(C.cast(handles, C.c_void_p), n, _ptr(f), C.cast(gp, C.c_void_p)), allow)
    return f, gs, rc


def dot_set_stencil_path(ctx, mode):
    """2: TMA stencil with the direction update fused in (default), 1: TMA stencil after a
    separate direction pass, 0: direct-load stencil."""
    return _check(load().dot_set_stencil_path(ctx, int(mode)))


def dot_set_kernel_timing(ctx, enable):
    return _check(load().dot_set_kernel_timing(ctx, int(bool(enable))))


def dot_get_kernel_timing(ctx) -> dict:
    t = DotKernelTiming()
    _check(load().dot_get_kernel_timing(ctx, C.byref(t)))
    return t.as_dict()


def dot_apply(ctx, X, cplx):
    X = _fortran(X, cplx)
    if X.ndim == 1:
        X = X.reshape(-1, 1, order="F")
    Y = np.zeros_like(X, order="F")
    _check(load().dot_apply(ctx, X.shape[1], _ptr(X), _ptr(Y)))
    return Y


def dot_probe_wait(ctx, budget_cycles, allow=(DOT_ETIMEOUT,)):
    """Self-test of the bounded device waits; returns the status (DOT_ETIMEOUT expected)."""
    return _check(load().dot_probe_wait(ctx, int(budget_cycles)), allow)


def dot_restrict_misfit_noalloc(X, n, kp, ls, ld, colptrC, rowsC, valsC, nd, V, P, is_complex, S, Rs, f,
                                stream=None):
    """Allocation-free restriction and misfit; every array argument is a device pointer (int)."""
    vp = lambda x: None if x is None else C.c_void_p(x)
    return _check(load().dot_restrict_misfit_noalloc(vp(X), n, kp, ls, ld, vp(colptrC), vp(rowsC), vp(valsC), nd,
                                                     vp(V), vp(P), int(bool(is_complex)), vp(S), vp(Rs), vp(f),
                                                     vp(stream)))


class Context:
    """Owning handle: `with Context(0) as ctx: ...` destroys the context on exit."""

    def __init__(self, device: int = 0):
        self.h = dot_create(device)

    def close(self):
        if self.h is not None:
            dot_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self.h

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
