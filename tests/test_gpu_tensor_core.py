"""GPU parity of the tensor-core (tcgen05) precision forms against the FP64 oracle.

Split-BF16x3 recovers FP32-level accuracy (J within 1e-4); plain TF32 and BF16 are
reported forms whose error is bounded by their input rounding (checked against
a band, not a target)."""
import numpy as np
import pytest

import oracle
from paper_2102_11026_gb300 import synth
from gpu_harness import Gpu, colerr, relerr, TOL_BF16X3_J

pytestmark = pytest.mark.gpu

# (first-order tol, higher-order / reduced-system tol)
TOLS = {"bf16x3": (TOL_BF16X3_J, 1e-3), "tf32": (3e-3, 1e-2), "bf16": (3e-2, 6e-2)}


def odd_workload(r, act="tanh", material="stvk", seed=5, gravity=False, hidden=(40, 72)):
    return synth.custom([r, *hidden, 360], (4, 5, 6), 24, seed, act, material, 1e4, 0.35, gravity)


CASES = {
    "small": lambda: synth.small(),
    "r1": lambda: odd_workload(1),
    "r13_nh_grav_sin": lambda: odd_workload(13, act="sin", material="neohookean", gravity=True),
    "r32_deep": lambda: odd_workload(32, seed=9, hidden=(48, 64, 80, 96)),
}


@pytest.mark.parametrize("prec", list(TOLS))
@pytest.mark.parametrize("name", list(CASES))
def test_tensor_core_parity(name, prec):
    wl = CASES[name]()
    g = Gpu(wl, prec)
    try:
        q = synth.newton_start(wl.state) + 0.05 * np.random.default_rng(3).normal(size=wl.dec.r)
        ref = oracle.derivs(wl.dec, q, wl.state.qbar, wl.state.qbar_dot, wl.state.dt)
        out = g.derivs(q, want=("u", "J", "Hqq", "dJ"))
        t1, t2 = TOLS[prec]
        # normwise and per column (elements against their column's largest value)
        for k, t in (("u", t1), ("J", t1), ("Hqq", t2), ("dJ", t2)):
            assert relerr(out[k], ref[k]) <= t, k
            assert colerr(out[k], ref[k]) <= t, (k, colerr(out[k], ref[k]))
        rs = g.reduced(q)
        rr = oracle.reduced_system(wl, q)
        assert relerr(rs["phi"], rr["phi"]) <= t2
        assert relerr(rs["A"], rr["A"]) <= t2
    finally:
        g.close()


def test_bf16x3_newton_step():
    wl = synth.small()
    g = Gpu(wl, "bf16x3")
    try:
        q0 = synth.newton_start(wl.state)
        q, rep = g.newton(q0)
        qo, _ = oracle.newton_solve(wl, q0=q0, max_iter=5)
        assert rep.status == 0
        assert np.linalg.norm(q - qo) <= 1e-3 * np.linalg.norm(qo - q0)
    finally:
        g.close()


def test_precision_switch_keeps_results():
    """dae_decoder_set_precision switches the GEMM arithmetic in place."""
    from paper_2102_11026_gb300 import dae
    wl = odd_workload(7)
    g = Gpu(wl, "fp32")
    try:
        q = synth.newton_start(wl.state)
        a = g.derivs(q, want=("J",))["J"]
        dae.dae_decoder_set_precision(g.ctx, g.dec, "bf16x3")
        b = g.derivs(q, want=("J",))["J"]
        dae.dae_decoder_set_precision(g.ctx, g.dec, "fp32")
        c = g.derivs(q, want=("J",))["J"]
        assert relerr(b, a) <= 1e-4 and np.array_equal(a, c)
    finally:
        g.close()
