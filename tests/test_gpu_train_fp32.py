"""The FP32 form of the decoder training pass (FFMA GEMMs on the CUDA cores): parity
with the FP64 oracle's reverse sweep at FP32 tolerances, the latent gradient of 64
seeded latents of the small (5-64-256-1024-3000) decoder against FP64 central
differences, and a fit of a re-seeded decoder to 4096 poses from implicit-Euler
rollouts of the small workload (batch 256, 100 Adam steps)."""
import numpy as np
import pytest

import oracle
from paper_2102_11026_gb300 import synth
from gpu_harness import relerr
from test_gpu_train import _run, _setup

pytestmark = pytest.mark.gpu

TOL_FWD = 1e-5      # u, J: FP32 GEMMs, FP32 accumulation
TOL_GRAD = 1e-5     # gradients


@pytest.mark.parametrize("B,act", [(64, "tanh"), (37, "sin")])
def test_fp32_train_pass_matches_oracle(B, act):
    widths = synth.SMALL_WIDTHS
    dae, torch, dec, ctx, tr, W, b, Q, gu, gJ, dev = _setup(widths, B, 3, act)
    try:
        dae.dae_trainer_set_precision(tr, "fp32")
        uJ, gq, gW, gb = _run(dae, torch, tr, W, b, Q, gu, gJ, dev)
        r = widths[0]
        for s in (0, B // 2, B - 1):
            jet = oracle.decoder_jets(dec, Q[s], np.eye(r))
            assert relerr(uJ[0, s], jet[0, :, 0]) <= TOL_FWD
            assert relerr(uJ[1:, s].T, jet[:, :, 1].T) <= TOL_FWD
        rq, rW, rb = oracle.decoder_uJ_vjp(dec, Q, gu, gJ)
        assert relerr(gq, rq) <= TOL_GRAD, relerr(gq, rq)
        for l in range(len(widths) - 1):
            assert relerr(gW[l], rW[l]) <= TOL_GRAD, (l, relerr(gW[l], rW[l]))
            assert relerr(gb[l], rb[l]) <= TOL_GRAD, (l, relerr(gb[l], rb[l]))
        # back to split BF16x3 and to FP32 again: each form gives its own results
        dae.dae_trainer_set_precision(tr, "bf16x3")
        x3 = _run(dae, torch, tr, W, b, Q, gu, gJ, dev)
        assert relerr(x3[1], rq) <= 1e-3
        dae.dae_trainer_set_precision(tr, "fp32")
        again = _run(dae, torch, tr, W, b, Q, gu, gJ, dev)
        assert np.array_equal(again[1], gq) and all(np.array_equal(x, y) for x, y in zip(again[2], gW))
    finally:
        dae.dae_trainer_free(tr)
        dae.dae_destroy(ctx)


def test_fp32_latent_gradient_of_64_latents_against_central_differences():
    """L = sum_s gu_s . u(q_s) + sum_{s,j} gJ_s[:, j] . J(q_s) e_j on the small decoder;
    each sample's term depends on its own latent only, so the FP64 central difference
    (h = 1e-6) of dL/dq_s is that of its term, formed with the oracle's jets."""
    widths = synth.SMALL_WIDTHS
    B = 64
    dae, torch, dec, ctx, tr, W, b, Q, gu, gJ, dev = _setup(widths, B, 11)
    try:
        dae.dae_trainer_set_precision(tr, "fp32")
        _, gq, _, _ = _run(dae, torch, tr, W, b, Q, gu, gJ, dev)
    finally:
        dae.dae_trainer_free(tr)
        dae.dae_destroy(ctx)
    r, h = widths[0], 1e-6

    def term(s, q):
        jet = oracle.decoder_jets(dec, q, np.eye(r))
        return gu[s] @ jet[0, :, 0] + np.sum(gJ[s] * jet[:, :, 1].T)

    fd = np.zeros_like(Q)
    for s in range(B):
        for j in range(r):
            e = np.zeros(r)
            e[j] = h
            fd[s, j] = (term(s, Q[s] + e) - term(s, Q[s] - e)) / (2 * h)
    assert relerr(gq, fd) <= TOL_GRAD, relerr(gq, fd)


def test_fp32_fit_to_rollout_poses():
    import torch
    from paper_2102_11026_gb300 import dae
    from paper_2102_11026_gb300.autograd import decoder_uJ
    import bench
    wl = synth.small()
    d, m = wl.dec, wl.mesh
    r = d.r
    torch.cuda.set_device(0)
    ctx = dae.dae_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        dec = dae.dae_load_decoder(ctx, d.widths, d.W, d.b, d.act, "bf16x3")
        mesh = dae.dae_load_mesh(ctx, m.X.reshape(-1), m.tets.reshape(-1), m.vmass, m.material,
                                 m.E, m.nu)
        poses = []
        for k in range(64):
            st = synth.make_state(r, 1000 + k)
            qh, qdh = st.qbar.copy(), st.qbar_dot.copy()
            traj = np.zeros((64, r))
            dae.dae_rollout(ctx, dec, mesh, wl.cub_tets, bench.frame_weights(wl, 64, 1000 + k), 64,
                            qh, qdh, st.dt, wl.f_ext, None, traj)
            poses.append(traj)
        dae.dae_free_decoder(dec)
        dae.dae_free_mesh(mesh)
        poses = torch.as_tensor(np.concatenate(poses), device="cuda")
        assert poses.shape == (4096, r) and torch.isfinite(poses).all()
        tr = dae.dae_trainer_create(ctx, d.widths, d.act, max_batch=256)
        dae.dae_trainer_set_precision(tr, "fp32")
        dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
        teacher = []
        for w, x in zip(d.W, d.b):
            teacher += [dev(w), dev(x)]
        student = synth.make_decoder(d.widths, 77, d.act)
        params = []
        for w, x in zip(student.W, student.b):
            params += [dev(w).requires_grad_(True), dev(x).requires_grad_(True)]
        opt = torch.optim.Adam(params, lr=1e-3)
        losses = []
        for step in range(100):
            i = (step * 256) % 4096
            with torch.no_grad():
                tu, tJ = decoder_uJ(tr, poses[i:i + 256], teacher)
            u, J = decoder_uJ(tr, poses[i:i + 256], params)
            loss = ((u - tu) ** 2).mean() + ((J - tJ) ** 2).mean()
            opt.zero_grad()
            loss.backward()
            opt.step()
            losses.append(float(loss.detach()))
        assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])
        dae.dae_trainer_free(tr)
    finally:
        dae.dae_destroy(ctx)
