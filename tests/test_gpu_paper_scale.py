"""Parity at the full paper-scale size (r = 30, ten layers, N = 60000, 88 445 tets,
Neo-Hookean, gravity, 500 cubature tets) in the launch configuration the
benchmark uses: reduced system against the FP64 oracle, decoder outputs on
sampled rows."""
import numpy as np
import pytest

import oracle
from paper_2102_11026_gb300 import synth
from gpu_harness import Gpu, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def paper():
    wl = synth.paper()
    q0 = synth.newton_start(wl.state)
    ref = oracle.reduced_system(wl, q0)
    return wl, q0, ref


@pytest.mark.parametrize("prec,tol1,tol2", [("fp32", 1e-5, 1e-4), ("bf16x3", 1e-4, 1e-3)])
def test_paper_scale_parity(paper, prec, tol1, tol2):
    wl, q0, ref = paper
    g = Gpu(wl, prec)
    try:
        rs = g.reduced(q0)
        for k in ("Mr", "B", "Kr", "aH", "g_int"):
            assert relerr(rs[k], ref[k]) <= tol2, (k, relerr(rs[k], ref[k]))
        assert relerr(rs["phi"], ref["phi"]) <= tol2
        assert relerr(rs["A"], ref["A"]) <= tol2
        assert abs(rs["energy"] - ref["energy"]) <= tol2 * abs(ref["energy"])
        # decoder outputs on 300 sampled rows (oracle evaluates only those rows)
        rows = np.sort(np.random.default_rng(0).choice(wl.dec.n_out, 300, replace=False))
        out = g.derivs(q0, want=("u", "J", "Hqq", "dJ"))
        dref = oracle.derivs(wl.dec, q0, wl.state.qbar, wl.state.qbar_dot, wl.state.dt, rows=rows)
        assert relerr(out["u"][rows], dref["u"]) <= tol1
        assert relerr(out["J"][rows], dref["J"]) <= tol1
        assert relerr(out["Hqq"][rows], dref["Hqq"]) <= tol2
        assert relerr(out["dJ"][rows], dref["dJ"]) <= tol2
        # the full-size Newton step takes the oracle's direction: A delta = -phi
        d_gpu = np.linalg.solve(rs["A"], -rs["phi"])
        d_ref = np.linalg.solve(ref["A"], -ref["phi"])
        kappa = np.linalg.cond(ref["A"])
        bound = kappa * (relerr(rs["A"], ref["A"]) + relerr(rs["phi"], ref["phi"]))
        assert relerr(d_gpu, d_ref) <= 2 * bound + 1e-12
    finally:
        g.close()
