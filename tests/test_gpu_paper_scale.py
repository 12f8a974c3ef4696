"""Parity at the full paper-scale size (r = 30, ten layers, N = 60000, 88 445 tets,
Neo-Hookean, gravity, 500 cubature tets) in the launch configuration the
benchmark uses: reduced system against the FP64 oracle, decoder outputs on
sampled rows, and rollout frames on device buffers whose solutions the oracle
confirms."""
import numpy as np
import pytest

import oracle
from paper_2102_11026_gb300 import synth
from gpu_harness import Gpu, colerr, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def paper():
    wl = synth.paper()
    q0 = synth.newton_start(wl.state)
    ref = oracle.reduced_system(wl, q0)
    return wl, q0, ref


# (precision, first-order tol, higher-order tol, check the separate terms of A)
# TF32 and BF16 are reported forms: their bands follow from the operand rounding
# (2^-11 and 2^-8 relative) over ten layers.
CASES = [("fp32", 1e-5, 1e-4, True), ("bf16x3", 1e-4, 1e-3, True),
         ("tf32", 3e-3, 5e-3, False), ("bf16", 2e-2, 3e-2, False)]


@pytest.mark.parametrize("prec,tol1,tol2,terms", CASES)
def test_paper_scale_parity(paper, prec, tol1, tol2, terms):
    wl, q0, ref = paper
    g = Gpu(wl, prec)
    try:
        rs = g.reduced(q0)
        if terms:
            for k in ("Mr", "B", "Kr", "aH", "g_int"):
                assert relerr(rs[k], ref[k]) <= tol2, (k, relerr(rs[k], ref[k]))
        assert relerr(rs["phi"], ref["phi"]) <= tol2
        assert relerr(rs["A"], ref["A"]) <= tol2
        assert abs(rs["energy"] - ref["energy"]) <= tol2 * abs(ref["energy"])
        # decoder outputs on 300 sampled rows (oracle evaluates only those rows)
        rows = np.sort(np.random.default_rng(0).choice(wl.dec.n_out, 300, replace=False))
        out = g.derivs(q0, want=("u", "J", "Hqq", "dJ"))
        dref = oracle.derivs(wl.dec, q0, wl.state.qbar, wl.state.qbar_dot, wl.state.dt, rows=rows)
        for k, t in (("u", tol1), ("J", tol1), ("Hqq", tol2), ("dJ", tol2)):
            assert relerr(out[k][rows], dref[k]) <= t, k
            assert colerr(out[k][rows], dref[k]) <= 2 * t, (k, colerr(out[k][rows], dref[k]))
        # the full-size Newton step takes the oracle's direction: A delta = -phi
        d_gpu = np.linalg.solve(rs["A"], -rs["phi"])
        d_ref = np.linalg.solve(ref["A"], -ref["phi"])
        kappa = np.linalg.cond(ref["A"])
        bound = kappa * (relerr(rs["A"], ref["A"]) + relerr(rs["phi"], ref["phi"]))
        assert relerr(d_gpu, d_ref) <= 2 * bound + 1e-12
    finally:
        g.close()


@pytest.mark.parametrize("prec,ratio", [("bf16x3", 1e-4), ("fp32", 1e-4)])
def test_paper_scale_rollout_frames(paper, prec, ratio):
    """Two frames of dae_rollout on device buffers from a torch stream (the
    benchmark's launch configuration).  For each frame the oracle, restarted from
    the GPU's state at the start of the frame with that frame's cubature weights,
    finds |phi| at the GPU's solution a small fraction of |phi| at the frame's
    first iterate, and the latent stays at the scale of the start state."""
    import torch
    import bench
    from paper_2102_11026_gb300 import dae
    wl, _, _ = paper
    d, m = wl.dec, wl.mesh
    r, n = d.r, wl.cub_tets.size
    n_frames = 2
    stream = torch.cuda.Stream()
    ctx = dae.dae_create(0, stream.cuda_stream)
    g = Gpu(wl, prec, ctx=ctx)
    try:
        cw = bench.frame_weights(wl, n_frames, 2)
        dev = lambda x, dt: torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device="cuda")
        q = dev(wl.state.qbar, torch.float64)
        qd = dev(wl.state.qbar_dot, torch.float64)
        traj = torch.zeros((n_frames, r), dtype=torch.float64, device="cuda")
        opts = dae.dae_default_newton_opts()
        opts.max_iter = 5
        with torch.cuda.stream(stream):
            reps = dae.dae_rollout(ctx, g.dec, g.mesh, dev(wl.cub_tets, torch.int32),
                                   dev(cw, torch.float32), n_frames, q, qd, wl.state.dt,
                                   dev(wl.f_ext, torch.float32), opts, traj)
        torch.cuda.synchronize()
        traj = traj.cpu().numpy()
        qbar, qdot = wl.state.qbar.copy(), wl.state.qbar_dot.copy()
        for f in range(n_frames):
            assert reps[f].status == 0
            w = cw[f * n:(f + 1) * n]
            q0 = qbar + wl.state.dt * qdot
            p0 = np.linalg.norm(oracle.phi_only(wl, q0, qbar=qbar, qbar_dot=qdot, cub_w=w))
            p1 = np.linalg.norm(oracle.phi_only(wl, traj[f], qbar=qbar, qbar_dot=qdot, cub_w=w))
            assert p1 <= ratio * p0, (f, p0, p1)
            assert np.abs(traj[f]).max() <= 10 * max(np.abs(wl.state.qbar).max(), 0.1)
            qdot = (traj[f] - qbar) / wl.state.dt
            qbar = traj[f].copy()
    finally:
        g.close()
        dae.dae_destroy(ctx)


def test_paper_scale_autotuned_plan(paper):
    """The tile autotuner on the paper-scale decoder (BF16x3): the tuned plan keeps the
    reduced system within the oracle tolerances and runs the Newton frames no slower than
    the built-in plan (frames timed with CUDA events, the two plans interleaved)."""
    import torch
    import bench
    from paper_2102_11026_gb300 import dae
    wl, q0, ref = paper
    d = wl.dec
    n = wl.cub_tets.size
    stream = torch.cuda.Stream()
    ctx = dae.dae_create(0, stream.cuda_stream)
    g = Gpu(wl, "bf16x3", ctx=ctx)
    try:
        nh = len(d.W) - 1
        plans = {"built-in": [dae.dae_decoder_get_chain_plan(ctx, g.dec, nh, k) for k in (0, 1)]}
        ms = dae.dae_decoder_autotune(ctx, g.dec, reps=10)
        assert ms[1] <= ms[0] and ms[3] <= ms[2]
        plans["tuned"] = [dae.dae_decoder_get_chain_plan(ctx, g.dec, nh, k) for k in (0, 1)]
        rs = g.reduced(q0)
        assert relerr(rs["phi"], ref["phi"]) <= 1e-3 and relerr(rs["A"], ref["A"]) <= 1e-3
        dev = lambda x, dt: torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device="cuda")
        cw = dev(bench.frame_weights(wl, 12, 2), torch.float32)
        cub_t = dev(wl.cub_tets, torch.int32)
        f_ext = dev(wl.f_ext, torch.float32)
        opts = dae.dae_default_newton_opts()
        times = {"built-in": [], "tuned": []}
        with torch.cuda.stream(stream):
            for _ in range(3):
                for name, pl in plans.items():
                    for k in (0, 1):
                        dae.dae_decoder_set_chain_plan(ctx, g.dec, k, pl[k][0], pl[k][1])
                    q = dev(wl.state.qbar, torch.float64)
                    qd = dev(wl.state.qbar_dot, torch.float64)
                    dae.dae_rollout(ctx, g.dec, g.mesh, cub_t, cw[:2 * n], 2, q, qd, wl.state.dt,
                                    f_ext, opts)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    dae.dae_rollout(ctx, g.dec, g.mesh, cub_t, cw[2 * n:], 10, q, qd, wl.state.dt,
                                    f_ext, opts, want_reports=False)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    times[name].append(e0.elapsed_time(e1))
        t_b, t_t = np.median(times["built-in"]), np.median(times["tuned"])
        assert t_t <= 1.03 * t_b, (t_b, t_t, ms)
    finally:
        g.close()
        dae.dae_destroy(ctx)
