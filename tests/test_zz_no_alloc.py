"""The allocation-free restriction entry point against the context path.

dot_restrict_misfit_noalloc serves callers that cannot let the library allocate
device memory (a loop that must not stall on cudaMalloc / cudaFree, or a process
whose device memory belongs to another allocator): its scratch is a fixed device
array, so the caller hands it device inputs and outputs only.  Here it is fed the
fields of a solved context and must reproduce that context's own measurements and
misfit (dot_measurements, dot_misfit), on two calls in a row, since every call
reuses the same scratch.  This file sorts last so that a run stopping at the first
failure has run every other test already.
"""
import numpy as np
import pytest

from paper_1706_05586_gb300 import dot as D
from paper_1706_05586_gb300 import synth
from tests import problem
from tests.gpu_setup import configure, rel

pytestmark = pytest.mark.gpu

CASES = {
    "cplx_11x6x7": synth.small_workload(11, 6, 7, 0.35, omega_nu=0.3, src_grid=(3, 1), det_grid=(2, 2), ls=3, ld=2,
                                        m0=5, sampling="gaussian", seed_index=62),
    "real_13x10x6": synth.small_workload(13, 10, 6, 0.3, src_grid=(3, 2), det_grid=(2, 3), ls=2, ld=2, m0=3,
                                         seed_index=63),
}


def _reference(pb):
    wl = pb.wl
    cplx = wl.omega_nu != 0.0
    h = D.dot_create(0)
    try:
        configure(h, pb, p=pb.inp.p0, rtol=1e-14)
        f_ref, _ = D.dot_misfit(h)
        S_ref, _ = D.dot_measurements(h, wl.ls, wl.ld, cplx)
        U, Z = D.dot_get_fields(h, wl.n, wl.ls, wl.ld, cplx)
    finally:
        D.dot_destroy(h)
    return f_ref, S_ref, U, Z


@pytest.mark.parametrize("name", list(CASES))
def test_noalloc_restriction_matches_context(name):
    torch = pytest.importorskip("torch")
    pb = problem.build(CASES[name])
    wl = pb.wl
    cplx = wl.omega_nu != 0.0
    f_ref, S_ref, U, Z = _reference(pb)
    dev = torch.device("cuda", 0)
    kp = wl.ls + wl.ld
    dt = torch.complex128 if cplx else torch.float64
    X = torch.zeros((wl.n, kp), dtype=dt)
    X[:, :wl.ls] = torch.from_numpy(np.ascontiguousarray(U))
    X[:, wl.ls:] = torch.from_numpy(np.ascontiguousarray(Z))
    Xd = X.to(dev).contiguous()
    colptr, rows, vals = pb.inp.C
    cp = torch.from_numpy(np.ascontiguousarray(colptr, dtype=np.int64)).to(dev)
    rw = torch.from_numpy(np.ascontiguousarray(rows, dtype=np.int32)).to(dev)
    vv = torch.from_numpy(np.ascontiguousarray(vals, dtype=np.float64)).to(dev)
    Vd = torch.from_numpy(np.asfortranarray(pb.inp.V).ravel(order="F").copy()).to(dev)
    P = (pb.inp.V.T @ pb.M @ pb.inp.W).astype(np.complex128)
    Pd = torch.from_numpy(np.asfortranarray(P).ravel(order="F").view(np.float64).copy()).to(dev)
    S = torch.empty(2 * wl.ls * wl.ld, dtype=torch.float64, device=dev)
    Rs = torch.empty_like(S)
    f = torch.empty(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for _ in range(2):
        S.fill_(float("nan"))
        Rs.fill_(float("nan"))
        f.fill_(float("nan"))
        D.dot_restrict_misfit_noalloc(Xd.data_ptr(), wl.n, kp, wl.ls, wl.ld, cp.data_ptr(), rw.data_ptr(),
                                      vv.data_ptr(), wl.nd, Vd.data_ptr(), Pd.data_ptr(), cplx, S.data_ptr(),
                                      Rs.data_ptr(), f.data_ptr(), stream)
        torch.cuda.synchronize(dev)
        S_h = S.cpu().numpy().view(np.complex128).reshape(wl.ld, wl.ls, order="F")
        R_h = Rs.cpu().numpy().view(np.complex128).reshape(wl.ld, wl.ls, order="F")
        assert rel(S_h if cplx else S_h.real, S_ref) <= 1e-10
        assert np.allclose(R_h, S_h - P, rtol=0, atol=1e-14 * np.abs(S_h).max())
        assert abs(f.item() - f_ref) <= 1e-10 * f_ref


def test_noalloc_rejects_sizes_above_scratch_limit():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    buf = torch.zeros(16, dtype=torch.float64, device=dev)
    ibuf = torch.zeros(16, dtype=torch.int64, device=dev)
    p = buf.data_ptr()
    with pytest.raises(D.DotError) as e:
        D.dot_restrict_misfit_noalloc(p, 4, 2, 1, 1, ibuf.data_ptr(), ibuf.data_ptr(), p, 65537, p, None, False,
                                      p, p, p, None)
    assert e.value.code == D.DOT_EINVAL
    assert "scratch limit" in D.dot_last_error()
