"""GPU parity of coupled substructures (Sec. 6, deformation substructuring; the ties
read as penalty springs between coinciding interface vertices and anchors at a root's
base): dae_newton_step_coupled against the FP64 oracle's coupled_system and
coupled_newton_solve on synthetic string trees."""
import numpy as np
import pytest

import oracle
from paper_2102_11026_gb300 import dae, synth
from gpu_harness import relerr

pytestmark = pytest.mark.gpu


class Loaded:
    def __init__(self, cm, prec="bf16x3"):
        self.cm = cm
        self.ctx = dae.dae_create(0)
        self.decs, self.meshes = [], []
        for wl in cm.domains:
            d, m = wl.dec, wl.mesh
            self.decs.append(dae.dae_load_decoder(self.ctx, d.widths, d.W, d.b, d.act, prec))
            self.meshes.append(dae.dae_load_mesh(self.ctx, m.X.reshape(-1), m.tets.reshape(-1),
                                                 m.vmass, m.material, m.E, m.nu))

    def systems(self, Q):
        off = np.concatenate([[0], np.cumsum([wl.dec.r for wl in self.cm.domains])])
        qs = [np.array(Q[off[k]:off[k + 1]]) for k in range(len(self.cm.domains))]
        ys = []
        for k, wl in enumerate(self.cm.domains):
            ys.append(dict(dec=self.decs[k], mesh=self.meshes[k], cub_tets=wl.cub_tets,
                           cub_w=wl.cub_w, q=qs[k], qbar=wl.state.qbar,
                           qbar_dot=wl.state.qbar_dot, f_ext=wl.f_ext))
        return ys, qs

    def step(self, Q, opts=None, pairs=None, anchors=None, k_c=None):
        cm = self.cm
        ys, qs = self.systems(Q)
        rep = dae.dae_newton_step_coupled(self.ctx, ys, cm.pairs if pairs is None else pairs,
                                          cm.anchors if anchors is None else anchors,
                                          cm.k_c if k_c is None else k_c,
                                          cm.domains[0].state.dt, opts)
        return np.concatenate(qs), rep

    def close(self):
        for d in self.decs:
            dae.dae_free_decoder(d)
        for m in self.meshes:
            dae.dae_free_mesh(m)
        dae.dae_destroy(self.ctx)


def start(cm):
    Qb = np.concatenate([wl.state.qbar for wl in cm.domains])
    Qd = np.concatenate([wl.state.qbar_dot for wl in cm.domains])
    return Qb, Qd, Qb + cm.domains[0].state.dt * Qd


TREES = {
    # a root with two children, one of which has a child
    "tree4": lambda: synth.coupled_strings([-1, 0, 0, 1], seed=8, bias=True, q_std=0.1, k_c=3e4),
    # two separate trees (two anchored roots): two components solved side by side
    "forest5": lambda: synth.coupled_strings([-1, 0, -1, 2, 3], seed=4, q_std=0.1),
}


@pytest.mark.parametrize("name", list(TREES))
def test_one_full_newton_step_matches_oracle_system(name):
    """One undamped Newton update from Q0 (no line search, no cap): Q1 - Q0 =
    -A(Q0)^{-1} phi(Q0) with the oracle's global phi and A, tie blocks included; the
    report's |phi(Q0)| and the energy at Q1 (domains' cubature plus ties)."""
    cm = TREES[name]()
    Qb, Qd, Q0 = start(cm)
    rs = oracle.coupled_system(cm, Q0, Qb, Qd)
    step = np.linalg.solve(rs["A"], -rs["phi"])
    opts = dae.dae_default_newton_opts()
    opts.max_iter = 1
    opts.max_step = 0.0
    opts.xtol = 0.0
    opts.c_armijo = -1e30
    g = Loaded(cm)
    try:
        Q1, rep = g.step(Q0, opts)
    finally:
        g.close()
    assert rep.status == 0 and rep.iters == 1 and rep.full_evals == 1
    assert relerr(Q1 - Q0, step) <= 2e-3, relerr(Q1 - Q0, step)
    assert abs(rep.phi_norm0 - np.linalg.norm(rs["phi"])) <= 1e-3 * np.linalg.norm(rs["phi"])
    e1 = oracle.coupled_system(cm, Q1, Qb, Qd)["energy"]
    assert abs(rep.energy - e1) <= 1e-3 * abs(e1)


@pytest.mark.parametrize("name", list(TREES))
def test_coupled_newton_matches_oracle(name):
    cm = TREES[name]()
    Qb, Qd, Q0 = start(cm)
    Qo, ro = oracle.coupled_newton_solve(cm, Q0=Q0)
    g = Loaded(cm)
    try:
        Q, rep = g.step(Q0)
    finally:
        g.close()
    assert rep.status == 0
    # the FP32 residual can stop above the FP64 one's tolerance, so the GPU may end on the
    # step test of one more Newton matrix
    assert abs(rep.iters - ro["iters"]) <= 1
    assert ro["nfull"] <= rep.full_evals <= ro["nfull"] + 1 and rep.full_evals >= rep.iters
    assert np.linalg.norm(Q - Qo) <= 1e-3 * np.linalg.norm(Qo - Q0), (Q, Qo)
    # the oracle's |phi| at the GPU's end point is as small as at its own ("tree4" stops
    # at max_iter before convergence: its first steps are capped at max_step)
    p1 = np.linalg.norm(oracle.coupled_system(cm, Q, Qb, Qd)["phi"])
    assert p1 <= 1.01 * ro["phi_hist"][-1] + 1e-6 * ro["phi_hist"][0], (p1, ro["phi_hist"])
    assert bool(rep.converged) == ro["converged"]


def test_anchored_strings_without_pairs_are_independent():
    """Only anchors (every string on a fixed base): the global system is block diagonal,
    one component per string, and equals the oracle's."""
    cm = synth.coupled_strings([-1, -1, -1], seed=5, q_std=0.1)
    assert len(cm.pairs) == 0
    Qb, Qd, Q0 = start(cm)
    Qo, _ = oracle.coupled_newton_solve(cm, Q0=Q0)
    g = Loaded(cm)
    try:
        Q, rep = g.step(Q0)
    finally:
        g.close()
    assert rep.status == 0
    assert np.linalg.norm(Q - Qo) <= 1e-3 * np.linalg.norm(Qo - Q0)


def test_invalid_ties_are_refused():
    cm = TREES["tree4"]()
    _, _, Q0 = start(cm)
    g = Loaded(cm)
    try:
        cyc = np.concatenate([cm.pairs, [[3, 0, 2, 0]]])      # 3-1-0-2-3: a cycle
        with pytest.raises(dae.DaeError) as e:
            g.step(Q0, pairs=cyc)
        assert e.value.status == -9
        with pytest.raises(dae.DaeError) as e:
            g.step(Q0, pairs=[[1, 0, 1, 3]])                   # a domain tied to itself
        assert e.value.status == -1
        with pytest.raises(dae.DaeError) as e:
            g.step(Q0, anchors=[[0, 10 ** 6]])                 # vertex out of range
        assert e.value.status == -1
        # a valid step still runs after the refusals
        _, rep = g.step(Q0)
        assert rep.status == 0
    finally:
        g.close()
