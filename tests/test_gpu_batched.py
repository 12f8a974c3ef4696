"""Grouped Newton step of independent strings (dae_newton_step_batched): every string's
step against the FP64 oracle and against its own single-system dae_newton_step, mixed
host / device arrays, bitwise repeatability, strings that finish early, and the
argument checks."""
import numpy as np
import pytest

import oracle
from paper_2102_11026_gb300 import dae, synth

pytestmark = pytest.mark.gpu


def _load(ctx, wl, prec):
    d, m = wl.dec, wl.mesh
    dec = dae.dae_load_decoder(ctx, d.widths, d.W, d.b, d.act, prec)
    mesh = dae.dae_load_mesh(ctx, m.X.reshape(-1), m.tets.reshape(-1), m.vmass, m.material, m.E,
                             m.nu)
    return dec, mesh


class Strings:
    def __init__(self, n, seed, prec="bf16x3", v_range=(200, 800)):
        self.wls = synth.strings(n, seed=seed, v_range=v_range)
        self.ctx = dae.dae_create(0)
        self.loaded = [_load(self.ctx, wl, prec) for wl in self.wls]

    def systems(self, qs, device=None):
        import torch
        out = []
        for i, (wl, (dec, mesh)) in enumerate(zip(self.wls, self.loaded)):
            y = dict(dec=dec, mesh=mesh, cub_tets=wl.cub_tets, cub_w=wl.cub_w, q=qs[i],
                     qbar=wl.state.qbar, qbar_dot=wl.state.qbar_dot)
            if device is not None and device(i):
                for k in ("cub_tets", "cub_w", "qbar", "qbar_dot"):
                    y[k] = torch.from_numpy(np.ascontiguousarray(y[k])).cuda()
            out.append(y)
        return out

    def starts(self):
        return [synth.newton_start(wl.state) for wl in self.wls]

    def close(self):
        for dec, mesh in self.loaded:
            dae.dae_free_decoder(dec)
            dae.dae_free_mesh(mesh)
        dae.dae_destroy(self.ctx)


@pytest.fixture(scope="module")
def strings():
    S = Strings(10, seed=7)
    yield S
    S.close()


def test_batched_step_matches_oracle_and_single_steps(strings):
    S = strings
    q0 = S.starts()
    qs = [q.copy() for q in q0]
    reps = dae.dae_newton_step_batched(S.ctx, S.systems(qs), S.wls[0].state.dt)
    assert len({wl.dec.r for wl in S.wls}) > 2          # several column counts in one launch
    for i, wl in enumerate(S.wls):
        assert reps[i].status == 0 and reps[i].evals >= 2, (i, reps[i].as_dict())
        qo, _ = oracle.newton_solve(wl, q0=q0[i], max_iter=5)
        step = np.linalg.norm(qo - q0[i])
        assert np.linalg.norm(qs[i] - qo) <= 1e-4 * max(step, 1e-12), (i, qs[i], qo)
        # the same string through the single-system entry point
        dec, mesh = S.loaded[i]
        q1 = q0[i].copy()
        r1 = dae.dae_newton_step(S.ctx, dec, mesh, wl.cub_tets, wl.cub_w, q1, wl.state.qbar,
                                 wl.state.qbar_dot, wl.state.dt)
        assert r1.status == 0
        assert np.linalg.norm(qs[i] - q1) <= 1e-5 * max(step, 1e-12), (i, qs[i], q1)


def test_batched_mixed_pointers_repeat_bitwise(strings):
    import torch
    S = strings
    q0 = S.starts()
    runs = []
    for _ in range(2):
        qs = [torch.from_numpy(q.copy()).cuda() if i % 2 else q.copy() for i, q in enumerate(q0)]
        dae.dae_newton_step_batched(S.ctx, S.systems(qs, device=lambda i: i % 3 == 0),
                                    S.wls[0].state.dt, want_reports=False)
        torch.cuda.synchronize()
        runs.append([q.cpu().numpy() if hasattr(q, "cpu") else q for q in qs])
    qh = [q.copy() for q in q0]
    dae.dae_newton_step_batched(S.ctx, S.systems(qh), S.wls[0].state.dt)
    for a, b, c in zip(runs[0], runs[1], qh):
        assert np.array_equal(a, b) and np.array_equal(a, c)


def test_batched_finished_strings_are_skipped(strings):
    """Strings that start at their solution stop after one evaluation while the others
    iterate; every result still equals the all-moving run."""
    S = strings
    q0 = S.starts()
    qa = [q.copy() for q in q0]
    ra = dae.dae_newton_step_batched(S.ctx, S.systems(qa), S.wls[0].state.dt)
    qb = [qa[i].copy() if i % 2 == 0 else q0[i].copy() for i in range(len(q0))]
    rb = dae.dae_newton_step_batched(S.ctx, S.systems(qb), S.wls[0].state.dt)
    for i in range(len(q0)):
        if i % 2 == 0:
            assert rb[i].evals <= 2 and rb[i].converged, rb[i].as_dict()
            step = np.linalg.norm(qa[i] - q0[i])
            assert np.linalg.norm(qb[i] - qa[i]) <= 1e-6 * max(step, 1e-12)
        else:
            assert rb[i].evals == ra[i].evals
            assert np.array_equal(qb[i], qa[i])
    assert max(r.evals for r in rb) > 2


def test_batched_explicit_launches_match_graph(strings):
    """With phase profiling on, the step runs as explicit launches (host loop over the
    evaluations) and gives the graph's result bit for bit."""
    S = strings
    q0 = S.starts()
    qa = [q.copy() for q in q0]
    dae.dae_newton_step_batched(S.ctx, S.systems(qa), S.wls[0].state.dt)
    dae.dae_profile_read(S.ctx)
    dae.dae_profile_enable(S.ctx, True)
    try:
        qb = [q.copy() for q in q0]
        rb = dae.dae_newton_step_batched(S.ctx, S.systems(qb), S.wls[0].state.dt)
    finally:
        dae.dae_profile_enable(S.ctx, False)
    prof = dae.dae_profile_read(S.ctx)
    assert prof["fwd_out"][1] >= max(r.evals for r in rb)
    for a, b in zip(qa, qb):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_batched_other_precisions_match_single(prec):
    S = Strings(4, seed=9, prec=prec, v_range=(200, 500))
    try:
        q0 = S.starts()
        qs = [q.copy() for q in q0]
        reps = dae.dae_newton_step_batched(S.ctx, S.systems(qs), S.wls[0].state.dt)
        for i, wl in enumerate(S.wls):
            assert reps[i].status == 0
            dec, mesh = S.loaded[i]
            q1 = q0[i].copy()
            dae.dae_newton_step(S.ctx, dec, mesh, wl.cub_tets, wl.cub_w, q1, wl.state.qbar,
                                wl.state.qbar_dot, wl.state.dt)
            step = np.linalg.norm(q1 - q0[i])
            # both forms round the same operands; only the GEMMs' K-split order differs
            assert np.linalg.norm(qs[i] - q1) <= 1e-3 * max(step, 1e-12), (i, qs[i], q1)
    finally:
        S.close()


def test_batched_argument_checks(strings):
    S = strings
    q0 = S.starts()
    ys = S.systems([q.copy() for q in q0])
    with pytest.raises(dae.DaeError) as e:
        dae.dae_newton_step_batched(S.ctx, [ys[0], ys[0]], 1.0 / 60)
    assert e.value.status == -1
    wl = S.wls[0]
    dec32, mesh32 = _load(S.ctx, wl, "fp32")
    try:
        y = dict(ys[0], dec=dec32, mesh=mesh32)
        with pytest.raises(dae.DaeError) as e:
            dae.dae_newton_step_batched(S.ctx, [y], 1.0 / 60)
        assert e.value.status == -9
    finally:
        dae.dae_free_decoder(dec32)
        dae.dae_free_mesh(mesh32)
    with pytest.raises(dae.DaeError) as e:
        dae.dae_newton_step_batched(S.ctx, ys[:2], 0.0)
    assert e.value.status == -1
    assert dae.dae_newton_step_batched(S.ctx, [], 1.0 / 60) == []


def test_batched_more_systems_than_one_chain_group():
    """More systems than one grouped chain stage holds (512 jobs): the step runs as
    several chain launches per direction and still equals the single-system steps."""
    wls = []
    for s in range(520):
        wl = synth.custom([3, 32, 48, 3 * 2 * 2 * 10], (2, 2, 10), 8, 1000 + s)
        wl.dec.b = [np.zeros_like(x) for x in wl.dec.b]
        wls.append(wl)
    ctx = dae.dae_create(0)
    loaded = [_load(ctx, wl, "bf16x3") for wl in wls]
    try:
        q0 = [synth.newton_start(wl.state) for wl in wls]
        qs = [q.copy() for q in q0]
        ys = [dict(dec=dec, mesh=mesh, cub_tets=wl.cub_tets, cub_w=wl.cub_w, q=qs[i],
                   qbar=wl.state.qbar, qbar_dot=wl.state.qbar_dot)
              for i, (wl, (dec, mesh)) in enumerate(zip(wls, loaded))]
        try:
            reps = dae.dae_newton_step_batched(ctx, ys, wls[0].state.dt)
        except dae.DaeError:
            reps = None      # a system's own Newton failure: compared below per system
        for i in (0, 255, 511, 512, 519):
            wl = wls[i]
            dec, mesh = loaded[i]
            q1 = q0[i].copy()
            try:
                r1 = dae.dae_newton_step(ctx, dec, mesh, wl.cub_tets, wl.cub_w, q1, wl.state.qbar,
                                         wl.state.qbar_dot, wl.state.dt)
            except dae.DaeError:
                continue
            assert r1.status == 0
            step = np.linalg.norm(q1 - q0[i])
            assert np.linalg.norm(qs[i] - q1) <= 1e-5 * max(step, 1e-12), (i, qs[i], q1)
        assert reps is None or sum(rp.evals for rp in reps) >= 520
    finally:
        for dec, mesh in loaded:
            dae.dae_free_decoder(dec)
            dae.dae_free_mesh(mesh)
        dae.dae_destroy(ctx)
