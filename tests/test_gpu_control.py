"""GPU tests of the device-side Newton control and of re-planning after a precision
change, against the FP64 oracle.

* The line search (Armijo on |phi|^2 with step halving, reading R6 of the paper's
  silent line search): a start far from the solution on a Neo-Hookean body whose
  full Newton steps first overshoot and later invert a cubature tet, so the control
  must take its halving branch and reject an inverted trial.  The oracle's trail of
  trials fixes every accept / reject decision; its margins are checked first so that
  FP32 rounding cannot flip one.
* The first-trial cap |alpha delta|_inf <= max_step.
* A precision change rebuilds the layer chains (their partial tiles and per-tile
  counters) and must invalidate the cached frame graph and re-size the Gram output
  stage's counters; results after a round trip must equal those before it.
"""
import numpy as np
import pytest

import oracle
from paper_2102_11026_gb300 import dae, synth
from gpu_harness import Gpu, relerr

pytestmark = pytest.mark.gpu


def far_start_workload():
    """Latent 3, 3-40-72-360 tanh decoder with output scale 1 (large displacements),
    4x5x6 Neo-Hookean grid (E = 1e4, nu = 0.35), 24 cubature tets; the start adds
    N(0, 0.5^2) to q0 = qbar + dt qbar_dot."""
    seed = 11
    dec = synth.make_decoder([3, 40, 72, 360], seed, "tanh", out_scale=1.0)
    mesh = synth.make_grid_mesh(4, 5, 6, seed, "neohookean", 1e4, 0.35)
    cub, w = synth.make_cubature(mesh.n_tet, 24, seed)
    st = synth.make_state(3, seed)
    wl = synth.Workload("far_start", dec, mesh, cub, w, st, np.zeros(360, np.float32))
    q0 = synth.newton_start(st) + 0.5 * np.random.default_rng(seed).normal(size=3)
    return wl, q0


def opts_for(max_step):
    o = dae.dae_default_newton_opts()
    o.max_iter = 5
    o.max_evals = 40
    o.max_step = max_step
    return o


def check_margins(trials, margin=0.05):
    """Every Armijo decision of the oracle's trail is at least ``margin`` away from
    its threshold (inverted trials are decided by det F, checked separately)."""
    for it, alpha, ratio in trials:
        if ratio is not None:
            assert abs(ratio - 1.0) >= margin, (it, alpha, ratio)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_line_search_halves_and_rejects_inverted_trial(prec):
    wl, q0 = far_start_workload()
    qo, ro = oracle.newton_solve(wl, q0=q0, max_iter=5, max_step=0.0)
    # the oracle's trail: at least one halving and one inverted trial, decisions clear
    assert any(ratio is None for _, _, ratio in ro["trials"])
    assert any(a < 1.0 for a in ro["alphas"])
    check_margins(ro["trials"])
    g = Gpu(wl, prec)
    try:
        q, rep = g.newton(q0, opts_for(0.0))
    finally:
        g.close()
    assert rep.status == 0
    assert rep.iters == ro["iters"] and rep.evals == ro["evals"]
    # only iterates whose Newton matrix is solved with form A (the first iterate and the
    # accepted trials that do not end the frame); rejected trials and the final accepted
    # one are phi-only evaluations
    assert rep.full_evals == ro["nfull"] and rep.full_evals < rep.evals
    assert rep.alpha == ro["alphas"][-1]                 # powers of two: exact
    assert bool(rep.converged) == ro["converged"]
    tol = 1e-4 if prec == "fp32" else 1e-3
    assert np.linalg.norm(q - qo) <= tol * np.linalg.norm(qo - q0), (q, qo)
    assert abs(rep.phi_norm - ro["phi_hist"][-1]) <= 10 * tol * ro["phi_hist"][0]


def test_first_trial_cap_matches_oracle():
    """max_step = 0.5: every update's first trial is capped to |alpha delta|_inf = 0.5
    (the Newton steps here are 1-10 latent units), and all capped trials pass."""
    wl, q0 = far_start_workload()
    qo, ro = oracle.newton_solve(wl, q0=q0, max_iter=5, max_step=0.5)
    assert ro["iters"] == 5 and all(a < 0.5 for a in ro["alphas"])
    check_margins(ro["trials"])
    g = Gpu(wl, "fp32")
    try:
        q, rep = g.newton(q0, opts_for(0.5))
    finally:
        g.close()
    assert rep.status == 0 and rep.iters == ro["iters"] and rep.evals == ro["evals"]
    # alpha = max_step / |delta|_inf: delta from the FP32 derivative pass
    assert abs(rep.alpha - ro["alphas"][-1]) <= 1e-3 * ro["alphas"][-1]
    assert np.linalg.norm(q - qo) <= 1e-4 * np.linalg.norm(qo - q0), (q, qo)


def test_precision_round_trip_with_large_cubature_set():
    """Gram-form output stage with 12|C| + K rows above the counters the hidden chains
    need (small decoder, K = 1024, |C| = 256: 8 + 24 output tiles against 25
    counters): assemble, switch to BF16 and back, assemble again.  Both results match
    the oracle and each other bit for bit."""
    wl = synth.small()
    cub, w = synth.make_cubature(wl.mesh.n_tet, 256, 1)
    wl.cub_tets, wl.cub_w = cub, w
    q = synth.newton_start(wl.state) + 0.02 * np.random.default_rng(4).normal(size=wl.dec.r)
    ref = oracle.reduced_system(wl, q)
    g = Gpu(wl, "bf16x3")
    try:
        a = g.reduced(q)
        dae.dae_decoder_set_precision(g.ctx, g.dec, "bf16")
        mid = g.reduced(q)
        dae.dae_decoder_set_precision(g.ctx, g.dec, "bf16x3")
        b = g.reduced(q)
    finally:
        g.close()
    for out in (a, b):
        assert relerr(out["phi"], ref["phi"]) <= 1e-3
        assert relerr(out["A"], ref["A"]) <= 1e-3
    assert relerr(mid["A"], ref["A"]) <= 6e-2
    assert np.array_equal(a["phi"], b["phi"]) and np.array_equal(a["A"], b["A"])


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_tensor_core_assembly_repeats_bitwise(prec):
    """The Gram-form output stage writes each cubature row's u and J to a slot of its
    own (cubature tets share vertices, so one DOF appears in several rows): repeated
    assemblies, and a Newton step repeated, give the same bits."""
    wl = synth.small()
    cub, w = synth.make_cubature(wl.mesh.n_tet, 256, 1)
    wl.cub_tets, wl.cub_w = cub, w
    q = synth.newton_start(wl.state) + 0.02 * np.random.default_rng(5).normal(size=wl.dec.r)
    g = Gpu(wl, prec)
    try:
        outs = [g.reduced(q) for _ in range(3)]
        qs = [g.newton(q)[0] for _ in range(2)]
    finally:
        g.close()
    for o in outs[1:]:
        for k in ("phi", "A", "energy", "Kr", "g_int", "aH"):
            assert np.array_equal(o[k], outs[0][k]), k
    assert np.array_equal(qs[0], qs[1])


@pytest.mark.parametrize("other", ["bf16x3", "tf32"])
def test_newton_step_after_precision_change_replays_a_fresh_graph(other):
    """A Newton step caches its frame graph; a precision change (to the same form or a
    round trip through another) rebuilds the chains' buffers, so the next step must
    capture a new graph: its result equals the first step's and the oracle's."""
    wl = synth.small()
    q0 = synth.newton_start(wl.state)
    qo, _ = oracle.newton_solve(wl, q0=q0, max_iter=5)
    g = Gpu(wl, "bf16x3")
    try:
        q1, r1 = g.newton(q0)
        dae.dae_decoder_set_precision(g.ctx, g.dec, other)
        if other != "bf16x3":
            g.newton(q0)
            dae.dae_decoder_set_precision(g.ctx, g.dec, "bf16x3")
        q2, r2 = g.newton(q0)
    finally:
        g.close()
    assert r1.status == 0 and r2.status == 0
    assert np.array_equal(q1, q2) and r1.evals == r2.evals
    assert np.linalg.norm(q2 - qo) <= 1e-3 * np.linalg.norm(qo - q0)
