"""GPU tests of the exact multicomplex activation (the ablation of the truncated form,
dae_decoder_set_cs_mode): on the FP32 form, every perturbation is its own tricomplex
number evaluated in exact multicomplex arithmetic.  Its derivatives must match the FP64
oracle (exact hyper-dual numbers) within the FP32 bounds, and the truncated form within
FP32 rounding (the two differ by O(h_cs^2) ~ 1e-12 relative)."""
import numpy as np
import pytest

import oracle
from paper_2102_11026_gb300 import dae, synth
from gpu_harness import Gpu, colerr, relerr, TOL_FP32_FIRST, TOL_FP32_HIGHER

pytestmark = pytest.mark.gpu

KEYS = ("u", "J", "Hqq", "dJ", "Hw", "Sdd")


def odd_workload(r, act="tanh", seed=5, hidden=(40, 72)):
    return synth.custom([r, *hidden, 360], (4, 5, 6), 24, seed, act, "stvk", 1e4, 0.35, False)


CASES = {
    "small": lambda: synth.small(),
    "small_sin": lambda: synth.small(act="sin"),
    "r1": lambda: odd_workload(1),
    "r7_sin": lambda: odd_workload(7, act="sin"),
    "r17_deep": lambda: odd_workload(17, seed=9, hidden=(48, 64, 80, 96)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_exact_activation_matches_oracle_and_truncated_form(name):
    wl = CASES[name]()
    q = synth.newton_start(wl.state) + 0.05 * np.random.default_rng(1).normal(size=wl.dec.r)
    ref = oracle.derivs(wl.dec, q, wl.state.qbar, wl.state.qbar_dot, wl.state.dt)
    g = Gpu(wl, "fp32")
    try:
        trunc = g.derivs(q, want=KEYS)
        dae.dae_decoder_set_cs_mode(g.ctx, g.dec, True)
        exact = g.derivs(q, want=KEYS)
        again = g.derivs(q, want=KEYS)
        dae.dae_decoder_set_cs_mode(g.ctx, g.dec, False)
        back = g.derivs(q, want=KEYS)
    finally:
        g.close()
    for k in KEYS:
        tol = TOL_FP32_FIRST if k in ("u", "J") else TOL_FP32_HIGHER
        assert relerr(exact[k], ref[k]) <= tol, (k, relerr(exact[k], ref[k]))
        assert colerr(exact[k], ref[k]) <= tol, (k, colerr(exact[k], ref[k]))
        # both forms carry the same quantities to FP32 rounding
        assert colerr(exact[k], trunc[k]) <= tol, (k, colerr(exact[k], trunc[k]))
        assert np.array_equal(exact[k], again[k]), k          # deterministic
        assert np.array_equal(back[k], trunc[k]), k           # the default form is untouched
    # u of the exact form is the unperturbed network: the same FP32 kernel on column 0
    assert relerr(exact["u"], trunc["u"]) <= 1e-6


def test_exact_mode_is_refused_outside_its_range():
    wl = odd_workload(18)
    g = Gpu(wl, "fp32")
    try:
        with pytest.raises(dae.DaeError) as e:
            dae.dae_decoder_set_cs_mode(g.ctx, g.dec, True)      # 6r + 4 > 112 columns
        assert e.value.status == -9
        # a precision change turns the exact form off
        dae.dae_decoder_set_precision(g.ctx, g.dec, "bf16x3")
        with pytest.raises(dae.DaeError) as e:
            dae.dae_decoder_set_cs_mode(g.ctx, g.dec, True)
        assert e.value.status == -9
    finally:
        g.close()
