"""GPU parity of the decoder training pass (batched first-order forward and its
reverse sweep) against the FP64 oracle, on the small workload's decoder
5-64-256-1024-3000 with a batch of 64 seeded latents, and a short fit."""
import numpy as np
import pytest

import oracle
from paper_2102_11026_gb300 import synth
from gpu_harness import relerr

pytestmark = pytest.mark.gpu

TOL_FWD = 1e-4      # u, J (split BF16x3 GEMMs, FP32 accumulation)
TOL_GRAD = 1e-3     # gradients: four GEMM layers of split BF16x3 each way


def _setup(widths, B, seed, act="tanh", bias=True):
    import torch
    from paper_2102_11026_gb300 import dae
    dec = synth.make_decoder(widths, seed, act, bias=bias)
    rng = np.random.default_rng(seed + 1)
    Q = rng.normal(0, 0.5, (B, widths[0]))
    gu = rng.normal(size=(B, widths[-1]))
    gJ = rng.normal(size=(B, widths[-1], widths[0]))
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = dae.dae_create(0, stream.cuda_stream)
    tr = dae.dae_trainer_create(ctx, widths, act, max_batch=max(B, 64))
    dev = lambda a, t=torch.float32: torch.as_tensor(np.ascontiguousarray(a), dtype=t, device="cuda")
    W = [dev(w) for w in dec.W]
    b = [dev(x) for x in dec.b]
    return dae, torch, dec, ctx, tr, W, b, Q, gu, gJ, dev


def _run(dae, torch, tr, W, b, Q, gu, gJ, dev):
    B, r = Q.shape
    N = W[-1].shape[0]
    q = dev(Q, torch.float64)
    uJ = torch.zeros((1 + r, B, N), device="cuda")
    dae.dae_train_forward(tr, W, b, q, uJ)
    g = torch.zeros((1 + r, B, N), device="cuda")
    g[0] = dev(gu)
    g[1:] = dev(gJ).permute(2, 0, 1)
    gq = torch.zeros((B, r), dtype=torch.float64, device="cuda")
    gW = [torch.zeros_like(w) for w in W]
    gb = [torch.zeros_like(x) for x in b]
    dae.dae_train_backward(tr, W, b, q, g, gq, gW, gb)
    torch.cuda.synchronize()
    return (uJ.cpu().numpy(), gq.cpu().numpy(), [x.cpu().numpy() for x in gW],
            [x.cpu().numpy() for x in gb])


@pytest.mark.parametrize("B,act", [(64, "tanh"), (37, "sin")])
def test_train_pass_matches_oracle(B, act):
    widths = synth.SMALL_WIDTHS
    dae, torch, dec, ctx, tr, W, b, Q, gu, gJ, dev = _setup(widths, B, 3, act)
    try:
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
    finally:
        dae.dae_trainer_free(tr)
        dae.dae_destroy(ctx)


def test_train_pass_batch_changes_and_repeats():
    """A smaller batch after a larger one (stale batch columns must not leak into the
    weight gradients) and a repeat give the same results."""
    widths = [4, 48, 96, 300]
    dae, torch, dec, ctx, tr, W, b, Q, gu, gJ, dev = _setup(widths, 64, 5)
    try:
        a = _run(dae, torch, tr, W, b, Q, gu, gJ, dev)
        c = _run(dae, torch, tr, W, b, Q[:19], gu[:19], gJ[:19], dev)
        d = _run(dae, torch, tr, W, b, Q[:19], gu[:19], gJ[:19], dev)
        rq, rW, rb = oracle.decoder_uJ_vjp(dec, Q[:19], gu[:19], gJ[:19])
        assert relerr(c[1], rq) <= TOL_GRAD
        for l in range(3):
            assert relerr(c[2][l], rW[l]) <= TOL_GRAD
        assert all(np.array_equal(x, y) for x, y in zip(c[2], d[2]))
        assert np.array_equal(c[1], d[1])
        assert a[1].shape == (64, 4)
    finally:
        dae.dae_trainer_free(tr)
        dae.dae_destroy(ctx)


def test_latent_gradient_against_central_differences():
    """d/dq of the loss by the library against FP64 central differences (h = 1e-6)
    of the same loss evaluated with the oracle's jets."""
    widths = [3, 24, 40, 60]
    dae, torch, dec, ctx, tr, W, b, Q, gu, gJ, dev = _setup(widths, 4, 9)
    try:
        _, gq, _, _ = _run(dae, torch, tr, W, b, Q, gu, gJ, dev)
        h = 1e-6

        def loss(Qm):
            tot = 0.0
            for s in range(Qm.shape[0]):
                jet = oracle.decoder_jets(dec, Qm[s], np.eye(3))
                tot += gu[s] @ jet[0, :, 0] + np.sum(gJ[s] * jet[:, :, 1].T)
            return tot

        fd = np.zeros_like(Q)
        for s in range(4):
            for j in range(3):
                Qp, Qm = Q.copy(), Q.copy()
                Qp[s, j] += h
                Qm[s, j] -= h
                fd[s, j] = (loss(Qp) - loss(Qm)) / (2 * h)
        assert relerr(gq, fd) <= TOL_GRAD
    finally:
        dae.dae_trainer_free(tr)
        dae.dae_destroy(ctx)


def test_autograd_function_and_short_fit():
    """torch.autograd through the library's backward equals its direct gradients, and
    100 Adam steps of a re-seeded decoder towards a teacher's u and J (batch 256)
    reduce the loss."""
    import torch
    from paper_2102_11026_gb300 import dae
    from paper_2102_11026_gb300.autograd import decoder_uJ
    widths = [5, 64, 256, 600]
    teacher = synth.make_decoder(widths, 1, "tanh")
    student = synth.make_decoder(widths, 2, "tanh")
    torch.cuda.set_device(0)
    ctx = dae.dae_create(0, torch.cuda.current_stream().cuda_stream)
    tr = dae.dae_trainer_create(ctx, widths, "tanh", max_batch=256)
    try:
        dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
        Tp = []
        for w, x in zip(teacher.W, teacher.b):
            Tp += [dev(w), dev(x)]
        Sp = []
        for w, x in zip(student.W, student.b):
            Sp += [dev(w).clone().requires_grad_(True), dev(x).clone().requires_grad_(True)]
        rng = np.random.default_rng(0)
        poses = dev(rng.normal(0, 0.5, (1024, 5))).double()
        with torch.no_grad():
            tu, tJ = decoder_uJ(tr, poses[:256], Tp)
        u, J = decoder_uJ(tr, poses[:256], Sp)
        loss = ((u - tu) ** 2).sum() + ((J - tJ) ** 2).sum()
        grads = torch.autograd.grad(loss, Sp)
        # the same gradients from the direct entry point
        g_uJ = torch.zeros((6, 256, 600), device="cuda")
        g_uJ[0] = 2 * (u - tu).detach()
        g_uJ[1:] = (2 * (J - tJ).detach()).permute(2, 0, 1)
        gW = [torch.empty_like(p) for p in Sp[0::2]]
        gb = [torch.empty_like(p) for p in Sp[1::2]]
        dae.dae_train_backward(tr, [p.detach() for p in Sp[0::2]], [p.detach() for p in Sp[1::2]],
                               poses[:256].contiguous(), g_uJ, None, gW, gb)
        torch.cuda.synchronize()
        for a, c in zip(grads[0::2], gW):
            assert torch.allclose(a, c, rtol=1e-5, atol=1e-7)
        opt = torch.optim.Adam(Sp, lr=1e-3)
        first = None
        for step in range(100):
            qb = poses[(step * 256) % 1024:(step * 256) % 1024 + 256]
            with torch.no_grad():
                tu, tJ = decoder_uJ(tr, qb, Tp)
            u, J = decoder_uJ(tr, qb, Sp)
            loss = ((u - tu) ** 2).mean() + ((J - tJ) ** 2).mean()
            opt.zero_grad()
            loss.backward()
            opt.step()
            if first is None:
                first = float(loss.detach())
        assert float(loss.detach()) < 0.5 * first, (first, float(loss.detach()))
    finally:
        dae.dae_trainer_free(tr)
        dae.dae_destroy(ctx)
