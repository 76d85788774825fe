"""Solve counts per evaluation against the statements of Sec. 3 (tests/golden/
solve_counts.txt): the oracle's plain evaluation solves every physical source and
detector (n_s + n_d columns), the library's sampled evaluation l_s + l_d."""
import os

import numpy as np
import pytest

from oracle import dot_oracle as orc
from paper_1706_05586_gb300 import synth
from tests import problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "solve_counts.txt")

WORKLOADS = {
    "cplx_11x6x7": synth.small_workload(11, 6, 7, 0.35, omega_nu=0.3, src_grid=(3, 1), det_grid=(2, 2), ls=3, ld=2,
                                        m0=5, sampling="gaussian", seed_index=62),
    "real_16x16x9": synth.small_workload(16, 16, 9, 0.3, src_grid=(4, 4), det_grid=(4, 4), ls=16, ld=16, m0=4,
                                         sampling="gaussian", seed_index=66),
    "small_8x8x4_l1": synth.small_workload(8, 8, 4, 0.3, src_grid=(2, 2), det_grid=(2, 2), ls=1, ld=1, m0=3,
                                           seed_index=75),
}


def golden():
    rows = {}
    for ln in open(GOLDEN):
        if ln.startswith("#") or not ln.strip():
            continue
        name, *vals = ln.split()
        rows[name] = dict(zip(("ns", "nd", "ls", "ld", "full", "sampled"), map(int, vals)))
    return rows


def test_golden_rows_follow_the_counting_rule():
    for name, g in golden().items():
        wl = WORKLOADS[name]
        assert (g["ns"], g["nd"], g["ls"], g["ld"]) == (wl.ns, wl.nd, wl.ls, wl.ld)
        assert g["full"] == g["ns"] + g["nd"] and g["sampled"] == g["ls"] + g["ld"]


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_oracle_evaluation_solves_every_source_and_detector(name, monkeypatch):
    g = golden()[name]
    pb = problem.build(WORKLOADS[name])
    solved = []
    real_solve = orc.solve

    def counting_solve(A, RHS, *a, **k):
        solved.append(1 if np.ndim(RHS) == 1 else np.shape(RHS)[1])
        return real_solve(A, RHS, *a, **k)

    monkeypatch.setattr(orc, "solve", counting_solve)
    pb.evaluate(pb.inp.p0)
    assert sum(solved) == g["full"]


@pytest.mark.gpu
@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_library_evaluation_solves_the_sampled_columns(name):
    from paper_1706_05586_gb300 import dot as D
    from tests.gpu_setup import configure
    g = golden()[name]
    pb = problem.build(WORKLOADS[name])
    h = D.dot_create(0)
    try:
        configure(h, pb, p=pb.inp.p0, prec=D.PREC_MIXED, rtol=1e-10)
        before = D.dot_get_stats(h)["columns_solved"]
        D.dot_gradient(h, pb.wl.np_)
        assert D.dot_get_stats(h)["columns_solved"] - before == g["sampled"]
        # the computed measurements of every physical source: n_s more solves
        before = D.dot_get_stats(h)["columns_solved"]
        D.dot_forward_model(h, pb.wl.ns, pb.wl.nd, pb.wl.omega_nu != 0.0)
        assert D.dot_get_stats(h)["columns_solved"] - before == g["ns"]
    finally:
        D.dot_destroy(h)
