"""Combined linear (PCA basis U) + filtered nonlinear subspace (Sec. 3.4, Eqs. 9-11) on
the GPU: the reduced system and a Newton step in r = [p; q] against the FP64 oracle, and
the argument checks."""
import numpy as np
import pytest

import oracle
from gpu_harness import Gpu, relerr
from paper_2102_11026_gb300 import dae, synth

pytestmark = pytest.mark.gpu

NP = 3


def _case(prec="bf16x3"):
    wl = synth.small()
    g = Gpu(wl, prec)
    U = synth.make_linear_basis(wl.dec.n_out, NP, 6)          # (N, np) float32
    dae.dae_decoder_attach_linear(g.ctx, g.dec, np.ascontiguousarray(U.T))
    pb, pd = synth.make_linear_state(NP, 6)
    rbar = np.concatenate([pb, wl.state.qbar])
    rdot = np.concatenate([pd, wl.state.qbar_dot])
    return wl, g, U.astype(np.float64), rbar, rdot


def _assemble(g, wl, r, rbar, rdot):
    n = r.size
    phi, A, en = np.zeros(n), np.zeros(n * n), np.zeros(1)
    terms = np.zeros(4 * n * n + n)
    dae.dae_assemble_reduced(g.ctx, g.dec, g.mesh, wl.cub_tets, wl.cub_w, r, rbar, rdot,
                             wl.state.dt, wl.f_ext, phi, A, en, terms)
    return phi, A.reshape(n, n).T, en[0], terms


def test_linear_subspace_system_matches_oracle():
    wl, g, U, rbar, rdot = _case()
    try:
        rng = np.random.default_rng(3)
        for k in range(2):
            r = rbar + wl.state.dt * rdot + rng.normal(0, 0.02, rbar.size) * k
            phi, A, en, terms = _assemble(g, wl, r, rbar, rdot)
            o = oracle.linear_subspace_system(wl, U, r, rbar, rdot)
            assert relerr(phi, o["phi"]) <= 1e-3, relerr(phi, o["phi"])
            assert relerr(A, o["A"]) <= 1e-3, relerr(A, o["A"])
            assert abs(en - o["energy"]) <= 1e-4 * abs(o["energy"])
            # the p block of A is U^T M U + dt^2 U^T K U
            n = r.size
            Kr = terms[3 * n * n:4 * n * n].reshape(n, n).T
            assert relerr(Kr, o["Kr"]) <= 1e-3
    finally:
        g.close()


def test_linear_subspace_newton_step_matches_oracle():
    wl, g, U, rbar, rdot = _case()
    try:
        r0 = rbar + wl.state.dt * rdot
        r = r0.copy()
        rep = dae.dae_newton_step(g.ctx, g.dec, g.mesh, wl.cub_tets, wl.cub_w, r, rbar, rdot,
                                  wl.state.dt, wl.f_ext)
        ro, _ = oracle.newton_solve(wl, q0=r0, qbar=rbar, qbar_dot=rdot, U=U, max_iter=5)
        assert rep.status == 0 and rep.evals >= 2
        step = np.linalg.norm(ro - r0)
        assert step > 1e-6
        assert np.linalg.norm(r - ro) <= 1e-4 * step, (r, ro)
    finally:
        g.close()


def test_linear_subspace_rollout_frame_two():
    """Two frames; frame 2 restarted in the oracle from the GPU's state after frame 1."""
    wl, g, U, rbar, rdot = _case()
    try:
        n = rbar.size
        dt = wl.state.dt
        q, qd = rbar.copy(), rdot.copy()
        traj = np.zeros(2 * n)
        cw = np.concatenate([wl.cub_w, wl.cub_w])
        reps = dae.dae_rollout(g.ctx, g.dec, g.mesh, wl.cub_tets, cw, 2, q, qd, dt, wl.f_ext,
                               q_traj=traj)
        assert all(rp.status == 0 for rp in reps)
        r1 = traj[:n]
        rb2, rd2 = r1, (r1 - rbar) / dt
        r02 = rb2 + dt * rd2
        ro, _ = oracle.newton_solve(wl, q0=r02, qbar=rb2, qbar_dot=rd2, U=U, max_iter=5)
        step = np.linalg.norm(ro - r02)
        assert np.linalg.norm(traj[n:] - ro) <= 1e-4 * max(step, 1e-12)
        assert np.allclose(q, traj[n:]) and np.allclose(qd, (traj[n:] - r1) / dt)
    finally:
        g.close()


def test_linear_subspace_argument_checks():
    wl = synth.small()
    g = Gpu(wl, "fp32")
    try:
        U = synth.make_linear_basis(wl.dec.n_out, 2, 1).T
        with pytest.raises(dae.DaeError) as e:
            dae.dae_decoder_attach_linear(g.ctx, g.dec, U)
        assert e.value.status == -9
    finally:
        g.close()
    g = Gpu(wl, "bf16x3")
    try:
        big = synth.make_linear_basis(wl.dec.n_out, 32 - wl.dec.r + 1, 1).T
        with pytest.raises(dae.DaeError) as e:
            dae.dae_decoder_attach_linear(g.ctx, g.dec, big)
        assert e.value.status == -9
        U = synth.make_linear_basis(wl.dec.n_out, 2, 1).T
        dae.dae_decoder_attach_linear(g.ctx, g.dec, U)
        with pytest.raises(dae.DaeError) as e:
            dae.dae_decoder_attach_linear(g.ctx, g.dec, U)
        assert e.value.status == -1
    finally:
        g.close()


def test_grouped_step_with_linear_subspaces():
    """Strings with and without a linear subspace in one grouped step equal their
    single-system steps (r = [p; q] for the former)."""
    wls = synth.strings(4, seed=17, v_range=(200, 500))
    ctx = dae.dae_create(0)
    loaded, starts = [], []
    try:
        for k, wl in enumerate(wls):
            d, m = wl.dec, wl.mesh
            dec = dae.dae_load_decoder(ctx, d.widths, d.W, d.b, d.act, "bf16x3")
            mesh = dae.dae_load_mesh(ctx, m.X.reshape(-1), m.tets.reshape(-1), m.vmass,
                                     m.material, m.E, m.nu)
            rbar, rdot = wl.state.qbar, wl.state.qbar_dot
            if k % 2 == 0:
                U = synth.make_linear_basis(d.n_out, 2, 30 + k)
                dae.dae_decoder_attach_linear(ctx, dec, np.ascontiguousarray(U.T))
                pb, pd = synth.make_linear_state(2, 30 + k, p_std=0.1)
                rbar, rdot = np.concatenate([pb, rbar]), np.concatenate([pd, rdot])
            loaded.append((dec, mesh))
            starts.append((rbar, rdot))
        q0 = [rb + wls[0].state.dt * rd for rb, rd in starts]
        qs = [q.copy() for q in q0]
        ys = [dict(dec=dec, mesh=mesh, cub_tets=wl.cub_tets, cub_w=wl.cub_w, q=qs[i],
                   qbar=starts[i][0], qbar_dot=starts[i][1])
              for i, (wl, (dec, mesh)) in enumerate(zip(wls, loaded))]
        reps = dae.dae_newton_step_batched(ctx, ys, wls[0].state.dt)
        for i, wl in enumerate(wls):
            dec, mesh = loaded[i]
            assert reps[i].status == 0
            q1 = q0[i].copy()
            dae.dae_newton_step(ctx, dec, mesh, wl.cub_tets, wl.cub_w, q1, starts[i][0],
                                starts[i][1], wl.state.dt)
            step = np.linalg.norm(q1 - q0[i])
            assert np.linalg.norm(qs[i] - q1) <= 1e-5 * max(step, 1e-12), (i, qs[i], q1)
    finally:
        for dec, mesh in loaded:
            dae.dae_free_decoder(dec)
            dae.dae_free_mesh(mesh)
        dae.dae_destroy(ctx)
