"""Several independent inversions in one call (dot_gradient_batch), CUDA-graph replay
of the iteration batches, and the launch autotuner: the batch reproduces each
context's own evaluation bitwise (same kernels, same launch shapes), graph replay is
bitwise identical to direct launches, and autotuned launches agree to rounding."""
import numpy as np
import pytest

from oracle import dot_oracle as orc
from paper_1706_05586_gb300 import dot as D
from paper_1706_05586_gb300 import synth
from tests import problem
from tests.gpu_setup import configure, rel

pytestmark = pytest.mark.gpu

MEMBERS = [
    synth.small_workload(16, 16, 9, 0.3, src_grid=(4, 4), det_grid=(4, 4), ls=16, ld=16, m0=4, sampling="gaussian",
                         seed_index=66),                                   # TMA-eligible, real
    synth.small_workload(11, 6, 7, 0.35, omega_nu=0.3, src_grid=(3, 1), det_grid=(2, 2), ls=3, ld=2, m0=5,
                         sampling="gaussian", seed_index=62),              # ragged, complex
    synth.small_workload(24, 16, 10, 0.3, omega_nu=0.4, src_grid=(4, 4), det_grid=(4, 4), ls=16, ld=16, m0=5,
                         sampling="gaussian", seed_index=65),              # TMA-eligible, complex
]


@pytest.fixture(scope="module")
def problems():
    return [problem.build(w) for w in MEMBERS]


def _single(pb, prec, rtol, graphs=True, autotune=False):
    h = D.dot_create(0)
    try:
        configure(h, pb, p=pb.inp.p0, prec=prec, rtol=rtol)
        D.dot_set_launch_options(h, graphs, autotune)
        f, g, _ = D.dot_gradient(h, pb.wl.np_)
        return f, g, D.dot_get_stats(h)
    finally:
        D.dot_destroy(h)


@pytest.mark.parametrize("prec,rtol", [(D.PREC_MIXED, 1e-12), (D.PREC_FP64, 1e-13)])
def test_batch_matches_members_bitwise(problems, prec, rtol):
    hs = [D.dot_create(0) for _ in problems]
    try:
        for h, pb in zip(hs, problems):
            configure(h, pb, p=pb.inp.p0, prec=prec, rtol=rtol)
        f, gs, rc = D.dot_gradient_batch(hs, [pb.wl.np_ for pb in problems])
        assert rc == D.DOT_OK
    finally:
        for h in hs:
            D.dot_destroy(h)
    for i, pb in enumerate(problems):
        f1, g1, _ = _single(pb, prec, rtol)
        assert f[i] == f1 and np.array_equal(gs[i], g1)


def test_graph_replay_is_bitwise_identical(problems):
    for pb in problems:
        a = _single(pb, D.PREC_MIXED, 1e-12, graphs=True)
        b = _single(pb, D.PREC_MIXED, 1e-12, graphs=False)
        assert a[0] == b[0] and np.array_equal(a[1], b[1])
        assert a[2]["iters_max"] == b[2]["iters_max"]


def test_autotuned_launches_agree(problems):
    for pb in problems:
        ref = _single(pb, D.PREC_MIXED, 1e-12)
        tuned = _single(pb, D.PREC_MIXED, 1e-12, autotune=True)
        assert abs(tuned[0] - ref[0]) <= 1e-9 * abs(ref[0])
        assert rel(tuned[1], ref[1]) <= 1e-7
        st = tuned[2]
        assert st["tuned_blocks_per_sm"] in (4, 5, 8, 16) and st["tuned_tma"] in (0, 1)


def _tuning_direction_ms(mode):
    """Mean CUDA-event time per launch of the separate direction passes during one
    autotuning solve in stencil mode `mode` (64 x 64 x 32 cells, 16 + 16 complex64
    columns, eligible for the fused kernel)."""
    wl = synth.small_workload(64, 64, 32, 0.125, omega_nu=0.4, src_grid=(4, 4), det_grid=(4, 4), ls=16, ld=16,
                              m0=8, sampling="gaussian", seed_index=93)
    inp = synth.draw(wl)
    h = D.dot_create(0)
    try:
        D.dot_set_grid(h, wl.nx, wl.ny, wl.nz, wl.h, wl.bc)
        D.dot_set_omega(h, wl.omega_nu)
        D.dot_set_diffusion(h, np.full(wl.n, 1.0 / 30.0))
        D.dot_set_pals(h, inp.p0, synth.MU_IN, synth.MU_OUT, wl.cutoff, wl.eps, wl.gamma)
        D.dot_set_sources(h, inp.B)
        D.dot_set_detectors(h, inp.C)
        D.dot_set_data(h, np.zeros((wl.nd, wl.ns)))
        D.dot_set_sampling(h, inp.W, inp.V)
        D.dot_set_solver(h, D.PREC_MIXED, 1e-10, 0)
        D.dot_set_stencil_path(h, mode)
        D.dot_set_launch_options(h, True, True)
        D.dot_set_kernel_timing(h, 1)
        _, _, rc = D.dot_gradient(h, wl.np_)             # the tuning solve
        assert rc == D.DOT_OK
        d = D.dot_get_kernel_timing(h)["direction"]
    finally:
        D.dot_destroy(h)
    assert d["launches"] > 0
    return d["ms"] / d["launches"]


def test_autotune_candidates_run_their_configuration():
    """Each autotuner candidate runs exactly its stencil configuration.  In stencil
    mode 2 the fused kernel's maps are prepared, yet the candidates with a separate
    direction pass (direct and TMA stencils) must run that pass: their direction
    intervals then take as long per launch as in mode 1, where the same two kinds of
    candidate are timed and no fused kernel exists.  A candidate that fused the
    direction into the stencil while timed as a separate pass would add empty
    intervals to mode 2's mean."""
    m1 = _tuning_direction_ms(1)
    m2 = _tuning_direction_ms(2)
    assert m2 >= 0.8 * m1, (m2, m1)


def test_batch_rejects_duplicates(problems):
    h = D.dot_create(0)
    try:
        configure(h, problems[1], p=problems[1].inp.p0)
        with pytest.raises(D.DotError) as e:
            D.dot_gradient_batch([h, h], [problems[1].wl.np_] * 2)
        assert e.value.code == D.DOT_EINVAL
    finally:
        D.dot_destroy(h)


def _timed(pb, graphs):
    h = D.dot_create(0)
    try:
        configure(h, pb, p=pb.inp.p0, prec=D.PREC_MIXED, rtol=1e-12)
        D.dot_set_launch_options(h, graphs, False)
        D.dot_set_kernel_timing(h, 1)
        f, g, _ = D.dot_gradient(h, pb.wl.np_)
        return f, g, D.dot_get_kernel_timing(h)
    finally:
        D.dot_destroy(h)


def test_kernel_timing_under_graph_replay(problems):
    # per-launch timing events are part of the captured graph: the same launches are
    # counted with and without replay, every timed kernel has a positive duration,
    # and timing changes no result
    for pb in problems:
        fa, ga, ka = _timed(pb, True)
        fb, gb, kb = _timed(pb, False)
        assert fa == fb and np.array_equal(ga, gb)
        for nm in ka:
            assert ka[nm]["launches"] == kb[nm]["launches"]
            if ka[nm]["launches"]:
                assert ka[nm]["ms"] > 0.0


def test_batch_with_kernel_timing(problems):
    hs = [D.dot_create(0) for _ in problems]
    try:
        for h, pb in zip(hs, problems):
            configure(h, pb, p=pb.inp.p0, prec=D.PREC_MIXED, rtol=1e-12)
            D.dot_set_kernel_timing(h, 1)
        f, gs, rc = D.dot_gradient_batch(hs, [pb.wl.np_ for pb in problems])
        assert rc == D.DOT_OK
        for h in hs:
            kt = D.dot_get_kernel_timing(h)
            assert sum(kt[nm]["launches"] for nm in kt) > 0
    finally:
        for h in hs:
            D.dot_destroy(h)
    for i, pb in enumerate(problems):
        f1, g1, _ = _single(pb, D.PREC_MIXED, 1e-12)
        assert f[i] == f1 and np.array_equal(gs[i], g1)


def test_stats_report_the_launch_configuration(problems):
    # without the autotuner every solve runs 5 blocks per SM and, where the shape allows
    # it (8-aligned x, y and a block width that is a multiple of 16), the TMA stencil
    for pb in problems:
        st = _single(pb, D.PREC_MIXED, 1e-12)[2]
        kp = -(-(pb.wl.ls + pb.wl.ld) // 4) * 4
        tma_ok = pb.wl.nx % 8 == 0 and pb.wl.ny % 8 == 0 and kp % 16 == 0
        assert st["tuned_blocks_per_sm"] == 5
        assert st["tuned_tma"] == (1 if tma_ok else 0)
        # the direction update runs inside the TMA stencil where the tile width allows it
        fused_ok = tma_ok and kp % (16 if pb.wl.omega_nu else 32) == 0
        assert st["fused_direction"] == (1 if fused_ok else 0)


@pytest.mark.parametrize("prec", [D.PREC_MIXED, D.PREC_FP64])
def test_direction_ring_sizes_give_the_same_results(problems, prec):
    # each correction alpha_j p_j reaches x~ in iteration order whatever the ring size
    out = []
    for slots in (8, 4, 2):
        for pb in problems:
            h = D.dot_create(0)
            try:
                configure(h, pb, p=pb.inp.p0, prec=prec, rtol=1e-12)
                D.dot_set_direction_ring(h, slots)
                f, g, _ = D.dot_gradient(h, pb.wl.np_)
                out.append((slots, pb.wl.name, f, g, D.dot_get_stats(h)["iters_max"]))
            finally:
                D.dot_destroy(h)
    ref = {name: (f, g, it) for s, name, f, g, it in out if s == 8}
    for s, name, f, g, it in out:
        f8, g8, it8 = ref[name]
        assert f == f8 and np.array_equal(g, g8) and it == it8, (s, name)


def test_direction_ring_rejects_other_sizes():
    h = D.dot_create(0)
    try:
        with pytest.raises(D.DotError) as e:
            D.dot_set_direction_ring(h, 3)
        assert e.value.code == D.DOT_EINVAL
    finally:
        D.dot_destroy(h)


@pytest.mark.parametrize("prec,rtol,tol", [(D.PREC_MIXED, 1e-13, 1e-8), (D.PREC_FP64, 2e-15, 1e-10)])
def test_batch_members_match_oracle(problems, prec, rtol, tol):
    """Every member of a dot_gradient_batch call against the FP64 oracle (true relative f
    and g at p0, the parity bars of the path), with a fourth member sampled as in the
    batching workload: q = 2 optimized simultaneous sources and detectors from Algorithm 1
    (dot_optimized_sampling, Sec. 3.2) completed by 6 random ones in the complementary
    subspace (Eqs. (newW), (newV)), fed to dot_set_sampling."""
    opt_pb = problems[2]                      # 16 x 16 physical sources and detectors, complex
    rng = np.random.default_rng(31)
    q, l = 2, 8
    Yt = rng.standard_normal((opt_pb.wl.ns, l - q)) / np.sqrt(l - q)
    Zt = rng.standard_normal((opt_pb.wl.nd, l - q)) / np.sqrt(l - q)
    h = D.dot_create(0)
    try:
        configure(h, opt_pb, p=opt_pb.inp.p0, prec=D.PREC_FP64, rtol=1e-13)
        W_opt, V_opt, _, _ = D.dot_optimized_sampling(h, q, q, opt_pb.wl.ns, opt_pb.wl.nd, l, l, Yt, Zt)
    finally:
        D.dot_destroy(h)
    members = [(pb, pb.inp.W, pb.inp.V) for pb in problems] + [(opt_pb, W_opt, V_opt)]
    hs = [D.dot_create(0) for _ in members]
    try:
        for h, (pb, W, V) in zip(hs, members):
            configure(h, pb, p=pb.inp.p0, prec=prec, rtol=rtol, W=W, V=V)
        f, gs, rc = D.dot_gradient_batch(hs, [pb.wl.np_ for pb, _, _ in members])
        assert rc == D.DOT_OK
    finally:
        for h in hs:
            D.dot_destroy(h)
    for i, (pb, W, V) in enumerate(members):
        mu = pb.mu_of(pb.inp.p0)
        ref = orc.evaluate(pb.D, mu, pb.grid, pb.wl.bc, pb.wl.omega_nu, pb.Bd, pb.Cd, pb.M, W, V,
                           dmu=pb.dmu_of(pb.inp.p0))
        assert abs(f[i] - ref["f"]) <= tol * ref["f"], i
        assert rel(gs[i], ref["g_p"]) <= tol, i


def test_stencil_path_rejects_other_modes():
    h = D.dot_create(0)
    try:
        for bad in (-1, 3):
            with pytest.raises(D.DotError) as e:
                D.dot_set_stencil_path(h, bad)
            assert e.value.code == D.DOT_EINVAL
    finally:
        D.dot_destroy(h)


def test_full_size_batch_member_against_oracle():
    """Two members of the eight-inversion batch workload at full size in one
    dot_gradient_batch call (96 x 96 x 48 real and 144 x 144 x 72 at 100 MHz, 1,024 x 1,024
    physical, 40 + 40 columns, mixed precision to 1e-10, autotuned launches): for the
    complex member the absorption, the FP64 true residual of every column with the
    oracle's A, and its misfit and PaLS gradient against the oracle's loops applied to
    its fields (agreement to rounding: 1e-10 relative)."""
    members = [synth.BATCH8[0], synth.BATCH8[3]]
    rng = np.random.default_rng(19)
    kw = dict(mu_in=synth.MU_IN, mu_out=synth.MU_OUT)
    prep = []
    for wl in members:
        inp = synth.draw(wl)
        X = orc.cell_centres(wl.nx, wl.ny, wl.nz, wl.h)
        k = dict(kw, c=wl.cutoff, eps=wl.eps, gamma=wl.gamma)
        Dfield = synth.diffusion_from_mua(orc.pals_mu(inp.p_true, X, **k))
        M = 1e-6 * rng.standard_normal((wl.nd, wl.ns))
        if wl.omega_nu:
            M = M + 1e-6j * rng.standard_normal((wl.nd, wl.ns))
        prep.append((inp, X, k, Dfield, M))
    hs = [D.dot_create(0) for _ in members]
    try:
        for h, wl, (inp, X, k, Dfield, M) in zip(hs, members, prep):
            D.dot_set_grid(h, wl.nx, wl.ny, wl.nz, wl.h, wl.bc)
            D.dot_set_omega(h, wl.omega_nu)
            D.dot_set_diffusion(h, Dfield)
            D.dot_set_pals(h, inp.p0, synth.MU_IN, synth.MU_OUT, wl.cutoff, wl.eps, wl.gamma)
            D.dot_set_sources(h, inp.B)
            D.dot_set_detectors(h, inp.C)
            D.dot_set_data(h, M)
            D.dot_set_sampling(h, inp.W, inp.V)
            D.dot_set_solver(h, D.PREC_MIXED, 1e-10, 0)
            D.dot_set_launch_options(h, True, True)
        f, gs, rc = D.dot_gradient_batch(hs, [wl.np_ for wl in members])
        assert rc == D.DOT_OK
        wl = members[1]
        U, Z = D.dot_get_fields(hs[1], wl.n, wl.ls, wl.ld, True)
        mu = D.dot_get_mua(hs[1], wl.n)
    finally:
        for h in hs:
            D.dot_destroy(h)
    inp, X, k, Dfield, M = prep[1]
    assert np.max(np.abs(mu - orc.pals_mu(inp.p0, X, **k))) <= 1e-12
    A = orc.assemble(Dfield, mu, wl.nx, wl.ny, wl.nz, wl.h, wl.bc, wl.omega_nu)
    B = orc.sparse_of_csc(wl.n, inp.B)
    C = orc.sparse_of_csc(wl.n, inp.C)
    for F, Rhs in ((U, B @ inp.W), (Z, C @ inp.V)):
        res = np.linalg.norm(Rhs - A @ F, axis=0) / np.linalg.norm(Rhs, axis=0)
        assert np.all(res <= 1.5e-10), res.max()
    R_s = (C @ inp.V).T @ U - inp.V.T @ M @ inp.W
    assert abs(f[1] - float(np.sum(np.abs(R_s) ** 2))) <= 1e-10 * f[1]
    g_mu = np.empty(wl.n)
    for v0 in range(0, wl.n, 8192):
        v1 = min(wl.n, v0 + 8192)
        g_mu[v0:v1] = orc.misfit_gradient(R_s, orc.sampled_jacobian_mua(U[v0:v1], Z[v0:v1], np.eye(wl.ls),
                                                                        np.eye(wl.ld)))
    g_ref = orc.pals_dmu_dp(inp.p0, X, **k).T @ g_mu
    assert np.linalg.norm(gs[1] - g_ref) <= 1e-10 * np.linalg.norm(g_ref)
