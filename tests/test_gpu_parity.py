"""GPU parity: the C-ABI library against the FP64 oracle, element by element on
the same seeded inputs (small and odd shapes), FP32 path."""
import numpy as np
import pytest

import oracle
from paper_2102_11026_gb300 import synth
from gpu_harness import Gpu, colerr, relerr, TOL_FP32_FIRST, TOL_FP32_HIGHER

pytestmark = pytest.mark.gpu


def odd_workload(r, act="tanh", material="stvk", seed=5, gravity=False, hidden=(40, 72)):
    grid = (4, 5, 6)                      # 120 vertices: N = 360 = 2 x 128 + 104 ragged rows
    wl = synth.custom([r, *hidden, 360], grid, 24, seed, act, material, 1e4, 0.35, gravity)
    return wl


CASES = {
    "small": lambda: synth.small(),
    "r1": lambda: odd_workload(1),
    "r7_sin": lambda: odd_workload(7, act="sin"),
    "r13_nh_grav": lambda: odd_workload(13, material="neohookean", gravity=True),
    "r31": lambda: odd_workload(31, seed=8),
    "r32_deep": lambda: odd_workload(32, seed=9, hidden=(48, 64, 80, 96)),
}


@pytest.fixture(scope="module")
def gpus():
    made = {}
    yield made
    for g in made.values():
        g.close()


def get(gpus, name):
    if name not in gpus:
        gpus[name] = Gpu(CASES[name]())
    return gpus[name]


@pytest.mark.parametrize("name", list(CASES))
def test_eval_derivs_parity(gpus, name):
    g = get(gpus, name)
    wl = g.wl
    q = synth.newton_start(wl.state) + 0.05 * np.random.default_rng(1).normal(size=wl.dec.r)
    ref = oracle.derivs(wl.dec, q, wl.state.qbar, wl.state.qbar_dot, wl.state.dt)
    out = g.derivs(q, want=("u", "J", "Hqq", "dJ", "Hw", "Sdd"))
    # normwise, then every column: each element within the tolerance times its column's
    # largest value (one wrong tile, ragged tail or column of J cannot hide in the rest)
    for k in ("u", "J"):
        assert relerr(out[k], ref[k]) <= TOL_FP32_FIRST, k
        assert colerr(out[k], ref[k]) <= TOL_FP32_FIRST, (k, colerr(out[k], ref[k]))
    for k in ("Hqq", "dJ", "Hw", "Sdd"):
        assert relerr(out[k], ref[k]) <= TOL_FP32_HIGHER, k
        assert colerr(out[k], ref[k]) <= TOL_FP32_HIGHER, (k, colerr(out[k], ref[k]))


@pytest.mark.parametrize("name", list(CASES))
def test_assemble_reduced_parity(gpus, name):
    g = get(gpus, name)
    wl = g.wl
    q = synth.newton_start(wl.state) + 0.02 * np.random.default_rng(2).normal(size=wl.dec.r)
    ref = oracle.reduced_system(wl, q)
    out = g.reduced(q)
    for k in ("Mr", "B", "Kr", "aH", "g_int"):
        assert relerr(out[k], ref[k]) <= TOL_FP32_HIGHER, (k, relerr(out[k], ref[k]))
    assert relerr(out["phi"], ref["phi"]) <= TOL_FP32_HIGHER
    assert relerr(out["A"], ref["A"]) <= TOL_FP32_HIGHER
    assert abs(out["energy"] - ref["energy"]) <= 1e-5 * abs(ref["energy"])


def test_linear_decoder_has_zero_hessian_terms():
    wl = odd_workload(5, act="linear")
    g = Gpu(wl)
    try:
        out = g.derivs(synth.newton_start(wl.state), want=("Hqq", "dJ", "Hw", "Sdd"))
        for k, v in out.items():
            assert np.all(v == 0.0), k
    finally:
        g.close()


def test_no_cubature_and_zero_state():
    """n_cub = 0: phi and A hold only the inertial terms; Delta = 0, qbar_dot = 0
    makes A symmetric (then z = 0 and dJ = 0)."""
    wl = odd_workload(6)
    wl.cub_tets = wl.cub_tets[:0]
    wl.cub_w = wl.cub_w[:0]
    wl.state.qbar_dot = np.zeros(6)
    g = Gpu(wl)
    try:
        q = wl.state.qbar.copy()
        out = g.reduced(q)
        ref = oracle.reduced_system(wl, q)
        assert np.all(out["Kr"] == 0) and np.all(out["g_int"] == 0)
        assert relerr(out["A"], ref["A"]) <= TOL_FP32_HIGHER
        assert np.abs(out["A"] - out["A"].T).max() <= 1e-6 * np.abs(out["A"]).max()
    finally:
        g.close()


def test_newton_step_matches_oracle():
    wl = synth.small()
    g = Gpu(wl)
    try:
        q0 = synth.newton_start(wl.state)
        q, rep = g.newton(q0)
        qo, ro = oracle.newton_solve(wl, q0=q0, max_iter=5)
        assert rep.status == 0 and rep.evals >= 2
        step = np.linalg.norm(qo - q0)
        assert np.linalg.norm(q - qo) <= 1e-4 * max(step, 1e-12), (q, qo)
        # the GPU's final residual is at the FP32 noise floor of phi
        assert rep.phi_norm <= 1e-3 * rep.phi_norm0
    finally:
        g.close()


def test_host_and_device_pointers_agree_and_repeat_bitwise():
    import torch
    wl = odd_workload(9)
    g = Gpu(wl)
    try:
        q = synth.newton_start(wl.state)
        a = g.reduced(q)
        b = g.reduced(q)
        assert np.array_equal(a["A"], b["A"]) and np.array_equal(a["phi"], b["phi"])
        from paper_2102_11026_gb300 import dae
        dev = lambda x, dt: torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device="cuda")
        r = wl.dec.r
        phi = torch.zeros(r, dtype=torch.float64, device="cuda")
        A = torch.zeros(r * r, dtype=torch.float64, device="cuda")
        dae.dae_assemble_reduced(g.ctx, g.dec, g.mesh, dev(wl.cub_tets, torch.int32),
                                 dev(wl.cub_w, torch.float32), dev(q, torch.float64),
                                 dev(wl.state.qbar, torch.float64),
                                 dev(wl.state.qbar_dot, torch.float64), wl.state.dt,
                                 dev(wl.f_ext, torch.float32), phi, A)
        dae.dae_sync(g.ctx)
        assert np.array_equal(phi.cpu().numpy(), a["phi"])
        assert np.array_equal(A.cpu().numpy().reshape(r, r).T, a["A"])
    finally:
        g.close()


def test_invalid_arguments_raise():
    from paper_2102_11026_gb300 import dae
    wl = odd_workload(4)
    g = Gpu(wl)
    try:
        bad = wl.cub_tets.copy()
        bad[0] = wl.mesh.n_tet + 5
        with pytest.raises(dae.DaeError) as e:
            dae.dae_assemble_reduced(g.ctx, g.dec, g.mesh, bad, wl.cub_w,
                                     synth.newton_start(wl.state), wl.state.qbar,
                                     wl.state.qbar_dot, wl.state.dt, None, np.zeros(4))
        assert e.value.status == -1
        with pytest.raises(dae.DaeError):
            dae.dae_eval_derivs(g.ctx, g.dec, synth.newton_start(wl.state), wl.state.qbar,
                                wl.state.qbar_dot, -1.0, u=np.zeros(360, np.float32))
        with pytest.raises(dae.DaeError) as e:
            dae.dae_load_decoder(g.ctx, [33, 8, 9], [np.zeros((8, 33), np.float32),
                                                     np.zeros((9, 8), np.float32)],
                                 [np.zeros(8, np.float32), np.zeros(9, np.float32)])
        assert e.value.status == -9
    finally:
        g.close()


def test_inverted_neohookean_tet_reports_inverted():
    from paper_2102_11026_gb300 import dae
    wl = odd_workload(3, material="neohookean")
    wl.dec.W[-1] *= 400.0                  # huge displacements invert cubature tets
    wl.dec.b[-1] *= 400.0
    g = Gpu(wl)
    try:
        with pytest.raises(dae.DaeError) as e:
            g.reduced(synth.newton_start(wl.state))
        assert e.value.status == -7
    finally:
        g.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_latent_the_decoder_ignores_reports_singular(prec):
    """With column 0 of the first layer zero the decoder does not depend on q_0: row
    and column 0 of A vanish (J e_0 = 0, H[., e_0] = 0, dJ e_0 = 0) while phi stays
    nonzero, so the Newton step must report DAE_ERR_SINGULAR instead of a step."""
    from paper_2102_11026_gb300 import dae
    wl = odd_workload(4)
    wl.dec.W[0][:, 0] = 0.0
    g = Gpu(wl, prec)
    try:
        q0 = synth.newton_start(wl.state)
        try:
            _, rep = g.newton(q0)
            status = rep.status
        except dae.DaeError as e:
            status = e.status
        assert status == -6
    finally:
        g.close()


def test_newton_step_solves_reduced_system():
    """The device Newton step solves A delta = -phi to FP64 accuracy: one update from
    q0 with the line search off equals q0 + A^{-1}(-phi) formed on the host from the
    same library's A and phi."""
    from paper_2102_11026_gb300 import dae
    wl = odd_workload(7, seed=11)
    g = Gpu(wl)
    try:
        q0 = synth.newton_start(wl.state)
        rs = g.reduced(q0)
        delta = np.linalg.solve(rs["A"], -rs["phi"])
        opts = dae.dae_default_newton_opts()
        opts.max_iter = 1
        opts.max_step = 0.0
        opts.xtol = 0.0
        opts.c_armijo = -1e30       # accept the full step
        q, rep = g.newton(q0, opts)
        assert rep.iters == 1
        assert np.linalg.norm(q - (q0 + delta)) <= 1e-12 * np.linalg.norm(delta)
    finally:
        g.close()


def test_rollout_frames_restart_parity():
    """Two implicit-Euler frames on the device; each frame's solution matches the
    oracle restarted from the GPU's state at the start of that frame."""
    from paper_2102_11026_gb300 import dae
    wl = synth.small()
    g = Gpu(wl)
    try:
        r = wl.dec.r
        n_frames = 2
        cw = np.concatenate([synth.make_cubature(wl.mesh.n_tet, 64, 1, frame=f)[1]
                             for f in range(n_frames)])
        q = wl.state.qbar.copy()
        qd = wl.state.qbar_dot.copy()
        traj = np.zeros((n_frames, r))
        reps = dae.dae_rollout(g.ctx, g.dec, g.mesh, wl.cub_tets, cw, n_frames, q, qd,
                               wl.state.dt, wl.f_ext, None, traj)
        qbar, qdot = wl.state.qbar.copy(), wl.state.qbar_dot.copy()
        for f in range(n_frames):
            qo, _ = oracle.newton_solve(wl, max_iter=5, cub_w=cw[f * 64:(f + 1) * 64],
                                        qbar=qbar, qbar_dot=qdot)
            step = np.linalg.norm(qo - (qbar + wl.state.dt * qdot))
            assert np.linalg.norm(traj[f] - qo) <= 1e-4 * max(step, 1e-12)
            assert reps[f].status == 0
            qdot = (traj[f] - qbar) / wl.state.dt
            qbar = traj[f].copy()
        assert np.allclose(q, traj[-1]) and np.allclose(qd, qdot)
    finally:
        g.close()
