"""Cubature weights predicted by the weight network at run time (Sec. 5, "Weight
Prediction"): the composed first layer against the FP64 oracle's plain definition, a
Newton step and a rollout with predicted weights against the oracle, and the argument
checks."""
import numpy as np
import pytest

import oracle
from gpu_harness import Gpu, relerr
from paper_2102_11026_gb300 import dae, synth

pytestmark = pytest.mark.gpu


def _attach(g, seed=5):
    wl = g.wl
    net = synth.make_wnet(wl.dec.n_out, wl.mesh.n_tet, seed)
    dae.dae_decoder_attach_wnet(g.ctx, g.dec, net.widths, net.W, net.b)
    return net


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16x3", 2e-4)])
def test_predicted_weights_match_oracle(prec, tol):
    wl = synth.small()
    g = Gpu(wl, prec)
    try:
        net = _attach(g)
        for q in (synth.newton_start(wl.state), np.zeros(wl.dec.r), 1.5 * wl.state.qbar):
            w = dae.dae_predict_weights(g.ctx, g.dec, q, wl.cub_tets)
            wo = oracle.wnet_weights(net, wl.dec, q, wl.cub_tets)
            assert relerr(w, wo) <= tol, (prec, relerr(w, wo))
            assert np.all(w >= 0)
        # every element, not only the cubature set
        allt = np.arange(wl.mesh.n_tet, dtype=np.int32)
        w = dae.dae_predict_weights(g.ctx, g.dec, synth.newton_start(wl.state), allt)
        wo = oracle.wnet_weights(net, wl.dec, synth.newton_start(wl.state))
        assert relerr(w, wo) <= tol
    finally:
        g.close()


def test_assemble_with_predicted_weights_equals_explicit_weights():
    wl = synth.small()
    g = Gpu(wl, "bf16x3")
    try:
        _attach(g)
        q = synth.newton_start(wl.state)
        w = dae.dae_predict_weights(g.ctx, g.dec, q, wl.cub_tets)
        a = g.reduced(q, cub_w=w)
        r = wl.dec.r
        phi, A, en = np.zeros(r), np.zeros(r * r), np.zeros(1)
        dae.dae_assemble_reduced(g.ctx, g.dec, g.mesh, wl.cub_tets, None, q, wl.state.qbar,
                                 wl.state.qbar_dot, wl.state.dt, wl.f_ext, phi, A, en)
        assert relerr(phi, a["phi"]) <= 1e-6 and relerr(A.reshape(r, r).T, a["A"]) <= 1e-6
        # and not the seeded weights
        b = g.reduced(q)
        assert relerr(phi, b["phi"]) > 1e-3
    finally:
        g.close()


def test_newton_step_with_predicted_weights_matches_oracle():
    wl = synth.small()
    g = Gpu(wl, "bf16x3")
    try:
        net = _attach(g)
        q0 = synth.newton_start(wl.state)
        q = q0.copy()
        rep = dae.dae_newton_step(g.ctx, g.dec, g.mesh, wl.cub_tets, None, q, wl.state.qbar,
                                  wl.state.qbar_dot, wl.state.dt, wl.f_ext)
        w0 = oracle.wnet_weights(net, wl.dec, q0, wl.cub_tets)
        qo, _ = oracle.newton_solve(wl, q0=q0, max_iter=5, cub_w=w0)
        assert rep.status == 0 and rep.evals >= 2
        step = np.linalg.norm(qo - q0)
        assert np.linalg.norm(q - qo) <= 1e-4 * max(step, 1e-12), (q, qo)
        # the predicted weights differ from the seeded ones, and so does the solution
        qs, _ = oracle.newton_solve(wl, q0=q0, max_iter=5)
        assert np.linalg.norm(qs - qo) > 1e-3 * step
    finally:
        g.close()


def test_rollout_predicts_weights_every_frame():
    """Two frames with predicted weights; frame 2 restarted in the oracle from the GPU's
    state after frame 1, with weights predicted at its first iterate."""
    wl = synth.small()
    g = Gpu(wl, "bf16x3")
    try:
        net = _attach(g)
        r = wl.dec.r
        dt = wl.state.dt
        q = wl.state.qbar.copy()
        qd = wl.state.qbar_dot.copy()
        traj = np.zeros(2 * r)
        reps = dae.dae_rollout(g.ctx, g.dec, g.mesh, wl.cub_tets, None, 2, q, qd, dt, wl.f_ext,
                               q_traj=traj)
        assert all(rp.status == 0 for rp in reps)
        q1 = traj[:r]
        qbar2, qdot2 = q1, (q1 - wl.state.qbar) / dt
        q02 = qbar2 + dt * qdot2
        w2 = oracle.wnet_weights(net, wl.dec, q02, wl.cub_tets)
        qo, _ = oracle.newton_solve(wl, q0=q02, max_iter=5, cub_w=w2, qbar=qbar2, qbar_dot=qdot2)
        step = np.linalg.norm(qo - q02)
        assert np.linalg.norm(traj[r:] - qo) <= 1e-4 * max(step, 1e-12), (traj[r:], qo)
    finally:
        g.close()


def test_weight_network_argument_checks():
    wl = synth.small()
    g = Gpu(wl, "bf16x3")
    try:
        q = synth.newton_start(wl.state)
        with pytest.raises(dae.DaeError) as e:          # no network attached
            dae.dae_newton_step(g.ctx, g.dec, g.mesh, wl.cub_tets, None, q.copy(), wl.state.qbar,
                                wl.state.qbar_dot, wl.state.dt, wl.f_ext)
        assert e.value.status == -1
        with pytest.raises(dae.DaeError) as e:
            dae.dae_predict_weights(g.ctx, g.dec, q, wl.cub_tets)
        assert e.value.status == -1
        net = synth.make_wnet(wl.dec.n_out + 3, wl.mesh.n_tet, 1)   # wrong input width
        with pytest.raises(dae.DaeError) as e:
            dae.dae_decoder_attach_wnet(g.ctx, g.dec, net.widths, net.W, net.b)
        assert e.value.status == -1
    finally:
        g.close()


def test_grouped_step_with_predicted_weights():
    """Strings with their own weight networks in one grouped step equal their
    single-system steps with predicted weights."""
    wls = synth.strings(4, seed=13, v_range=(200, 500))
    ctx = dae.dae_create(0)
    loaded = []
    try:
        for k, wl in enumerate(wls):
            d, m = wl.dec, wl.mesh
            dec = dae.dae_load_decoder(ctx, d.widths, d.W, d.b, d.act, "bf16x3")
            mesh = dae.dae_load_mesh(ctx, m.X.reshape(-1), m.tets.reshape(-1), m.vmass,
                                     m.material, m.E, m.nu)
            net = synth.make_wnet(d.n_out, m.n_tet, 20 + k)
            dae.dae_decoder_attach_wnet(ctx, dec, net.widths, net.W, net.b)
            loaded.append((dec, mesh, net))
        q0 = [synth.newton_start(wl.state) for wl in wls]
        qs = [q.copy() for q in q0]
        ys = [dict(dec=dec, mesh=mesh, cub_tets=wl.cub_tets, cub_w=None, q=qs[i],
                   qbar=wl.state.qbar, qbar_dot=wl.state.qbar_dot)
              for i, (wl, (dec, mesh, _)) in enumerate(zip(wls, loaded))]
        reps = dae.dae_newton_step_batched(ctx, ys, wls[0].state.dt)
        for i, wl in enumerate(wls):
            dec, mesh, net = loaded[i]
            assert reps[i].status == 0
            q1 = q0[i].copy()
            dae.dae_newton_step(ctx, dec, mesh, wl.cub_tets, None, q1, wl.state.qbar,
                                wl.state.qbar_dot, wl.state.dt)
            step = np.linalg.norm(q1 - q0[i])
            assert np.linalg.norm(qs[i] - q1) <= 1e-5 * max(step, 1e-12), (i, qs[i], q1)
            w0 = oracle.wnet_weights(net, wl.dec, q0[i], wl.cub_tets)
            qo, _ = oracle.newton_solve(wl, q0=q0[i], max_iter=5, cub_w=w0)
            assert np.linalg.norm(qs[i] - qo) <= 1e-4 * max(np.linalg.norm(qo - q0[i]), 1e-12)
    finally:
        for dec, mesh, _ in loaded:
            dae.dae_free_decoder(dec)
            dae.dae_free_mesh(mesh)
        dae.dae_destroy(ctx)
