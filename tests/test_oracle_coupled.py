"""Pins of the FP64 oracle for coupled substructures (Sec. 6, deformation
substructuring; the ties read as penalty springs between interface vertices that
coincide at rest, and anchors that hold a root's base at rest): the tie energy's
closed forms, its gradient against central differences of the energy, the global
Newton matrix against central differences of phi (off-diagonal blocks included), the
reduction to independent domains without ties, a one-step textbook solve for linear
decoders, and quadratic convergence."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2102_11026_gb300 import synth


def _state(cm):
    Qb = np.concatenate([wl.state.qbar for wl in cm.domains])
    Qd = np.concatenate([wl.state.qbar_dot for wl in cm.domains])
    return Qb, Qd, cm.domains[0].state.dt


def _relerr(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def tree():
    # a root with two children, one of which has a child: pairs across three interfaces
    return synth.coupled_strings([-1, 0, 0, 1], seed=8, bias=True, q_std=0.1, k_c=3e4)


def test_tie_energy_closed_forms():
    cm = synth.coupled_strings([-1, 0, 1], seed=3)
    rng = np.random.default_rng(0)
    t = rng.normal(size=3)
    # every vertex of every domain displaced by the same t: pairs are slack, each
    # anchor stores k_c/2 |t|^2 and pulls back with k_c t
    us = [np.tile(t, wl.mesh.n_vert) for wl in cm.domains]
    E, g = oracle.coupling_energy(cm, us)
    na = len(cm.anchors)
    assert np.isclose(E, 0.5 * cm.k_c * na * float(t @ t), rtol=1e-14)
    gs = sum(gd.reshape(-1, 3).sum(0) for gd in g)
    assert np.allclose(gs, cm.k_c * na * t, rtol=1e-13)
    for d, i in cm.anchors:
        assert np.allclose(g[d][3 * i:3 * i + 3], cm.k_c * t)
    # random displacements: the pair forces cancel in the sum (action = reaction),
    # so the net tie force is the anchors' pull alone
    us = [rng.normal(size=3 * wl.mesh.n_vert) for wl in cm.domains]
    E, g = oracle.coupling_energy(cm, us)
    net = sum(gd.reshape(-1, 3).sum(0) for gd in g)
    pull = sum(cm.k_c * us[d][3 * i:3 * i + 3] for d, i in cm.anchors)
    assert np.allclose(net, pull, rtol=1e-12, atol=1e-9)
    # one pair stretched by s alone: energy k_c/2 |s|^2
    us = [np.zeros(3 * wl.mesh.n_vert) for wl in cm.domains]
    d, i, e, j = cm.pairs[0]
    s = np.array([0.3, -0.2, 0.1])
    us[d][3 * i:3 * i + 3] = s
    E, g = oracle.coupling_energy(cm, us)
    assert np.isclose(E, 0.5 * cm.k_c * float(s @ s), rtol=1e-14)
    assert np.allclose(g[e][3 * j:3 * j + 3], -cm.k_c * s)


def test_tie_terms_of_phi_are_the_energy_gradient(tree):
    """phi's tie part, dt^2 J_d^T g_d, against central differences of E_c(D(q))."""
    cm = tree
    Qb, Qd, dt = _state(cm)
    Q = Qb + dt * Qd + 0.02
    free = dataclasses.replace(cm, k_c=0.0)
    tied_phi = oracle.coupled_system(cm, Q, Qb, Qd)["phi"]
    free_phi = oracle.coupled_system(free, Q, Qb, Qd)["phi"]
    off = np.concatenate([[0], np.cumsum([wl.dec.r for wl in cm.domains])])

    def Ec(x):
        us = [oracle.decode(wl.dec, x[off[d]:off[d + 1]]) for d, wl in enumerate(cm.domains)]
        return oracle.coupling_energy(cm, us)[0]
    h = 1e-6
    grad = np.array([(Ec(Q + h * e) - Ec(Q - h * e)) / (2 * h) for e in np.eye(Q.size)])
    assert np.linalg.norm(grad) > 1.0
    assert _relerr((tied_phi - free_phi) / dt ** 2, grad) <= 1e-7


def test_coupled_A_is_the_jacobian_of_phi(tree):
    cm = tree
    Qb, Qd, dt = _state(cm)
    rng = np.random.default_rng(5)
    Q = Qb + dt * Qd + rng.normal(0, 0.03, Qb.size)
    rs = oracle.coupled_system(cm, Q, Qb, Qd)
    h = 1e-6
    cols = []
    for e in np.eye(Q.size):
        p = oracle.coupled_system(cm, Q + h * e, Qb, Qd)["phi"]
        m = oracle.coupled_system(cm, Q - h * e, Qb, Qd)["phi"]
        cols.append((p - m) / (2 * h))
    Afd = np.array(cols).T
    assert _relerr(rs["A"], Afd) <= 1e-6, _relerr(rs["A"], Afd)
    r = cm.domains[0].dec.r
    # tied domains couple: the blocks of domain 1 with its parent 0 and child 3
    assert np.linalg.norm(rs["A"][r:2 * r, 0:r]) > 1e-3 * np.linalg.norm(rs["A"])
    assert np.linalg.norm(rs["A"][r:2 * r, 3 * r:4 * r]) > 1e-3 * np.linalg.norm(rs["A"])
    # untied domains do not: 2 and 3 share no interface
    assert np.all(rs["A"][2 * r:3 * r, 3 * r:4 * r] == 0)
    # planted mistakes fail the pin: the tie force left out of a (so out of a^T H) ...
    off = np.concatenate([[0], np.cumsum([wl.dec.r for wl in cm.domains])])
    no_aH = rs["A"].copy()
    for d, wl in enumerate(cm.domains):
        s = slice(off[d], off[d + 1])
        no_aH[s, s] -= oracle.aTH(wl.dec, Q[s], dt ** 2 * rs["g"][d])
    assert _relerr(no_aH, Afd) > 1e2 * _relerr(rs["A"], Afd)
    # ... and the off-diagonal tie blocks with the wrong sign
    flip = rs["A"].copy()
    for d in range(len(cm.domains)):
        for e in range(len(cm.domains)):
            if d != e:
                flip[off[d]:off[d + 1], off[e]:off[e + 1]] *= -1
    assert _relerr(flip, Afd) > 1e2 * _relerr(rs["A"], Afd)


def test_without_ties_domains_are_independent(tree):
    cm = dataclasses.replace(tree, k_c=0.0)
    Qb, Qd, dt = _state(cm)
    Q = Qb + dt * Qd + 0.01
    rs = oracle.coupled_system(cm, Q, Qb, Qd)
    off = np.concatenate([[0], np.cumsum([wl.dec.r for wl in cm.domains])])
    for d, wl in enumerate(cm.domains):
        s = slice(off[d], off[d + 1])
        own = oracle.reduced_system(wl, Q[s], qbar=Qb[s], qbar_dot=Qd[s], dt=dt)
        assert np.array_equal(rs["phi"][s], own["phi"])
        assert np.array_equal(rs["A"][s, s], own["A"])
        rest = np.ones(Q.size, bool)
        rest[s] = False
        assert np.all(rs["A"][s][:, rest] == 0)


def test_linear_decoders_take_one_textbook_step():
    """Linear decoders u_d = B_d q_d and no elastic stiffness (E = 0): the coupled step
    is the linear implicit-Euler system of the spring-tied subspaces,
      (B^T M B + dt^2 B^T K_c B) Q = B^T M B (Qbar + dt Qdot) + dt^2 B^T f_ext,
    with K_c assembled here in full space from the pair and anchor lists; Newton
    reaches it in one step."""
    cm = synth.coupled_strings([-1, 0, 1, 1], seed=11, act="linear", E=0.0, k_c=2e3)
    Qb, Qd, dt = _state(cm)
    Bs = []
    for wl in cm.domains:
        B = np.eye(wl.dec.r)
        for W in wl.dec.W:
            B = np.asarray(W, np.float64) @ B
        Bs.append(B)
    Nn = np.concatenate([[0], np.cumsum([B.shape[0] for B in Bs])])
    Rn = np.concatenate([[0], np.cumsum([B.shape[1] for B in Bs])])
    Bg = np.zeros((Nn[-1], Rn[-1]))
    for d, B in enumerate(Bs):
        Bg[Nn[d]:Nn[d + 1], Rn[d]:Rn[d + 1]] = B
    M = np.concatenate([np.repeat(wl.mesh.vmass, 3) for wl in cm.domains])
    f = np.concatenate([np.asarray(wl.f_ext, np.float64) for wl in cm.domains])
    K = np.zeros((Nn[-1], Nn[-1]))
    for d, i, e, j in cm.pairs:
        for c in range(3):
            a, b = Nn[d] + 3 * i + c, Nn[e] + 3 * j + c
            K[a, a] += cm.k_c
            K[b, b] += cm.k_c
            K[a, b] -= cm.k_c
            K[b, a] -= cm.k_c
    for d, i in cm.anchors:
        for c in range(3):
            K[Nn[d] + 3 * i + c, Nn[d] + 3 * i + c] += cm.k_c
    BMB = Bg.T @ (M[:, None] * Bg)
    lhs = BMB + dt ** 2 * Bg.T @ K @ Bg
    rhs = BMB @ (Qb + dt * Qd) + dt ** 2 * Bg.T @ f
    Qx = np.linalg.solve(lhs, rhs)
    Q, rep = oracle.coupled_newton_solve(cm, max_iter=3, max_step=0.0, xtol=0.0, tol=1e-12)
    assert rep["iters"] >= 1
    assert _relerr(Q, Qx) <= 1e-10, _relerr(Q, Qx)
    assert rep["phi_hist"][1] <= 1e-10 * rep["phi_hist"][0]


def test_coupled_newton_converges_quadratically():
    cm = synth.coupled_strings([-1, 0, 0, 1, 2], seed=4)
    Q, rep = oracle.coupled_newton_solve(cm, max_iter=8, xtol=0.0, tol=1e-12)
    h = rep["phi_hist"]
    assert rep["converged"] and len(h) <= 6, h
    for k in range(1, len(h) - 1):
        if h[k] < 1e-2 and h[k + 1] > 1e-13:
            assert h[k + 1] <= 10.0 * h[k] ** 2, h
    # the solution satisfies every domain's equations with the ties, not without them
    Qb, Qd, dt = _state(cm)
    free = oracle.coupled_system(dataclasses.replace(cm, k_c=0.0), Q, Qb, Qd)
    assert np.linalg.norm(free["phi"]) > 1e3 * max(h[-1], 1e-12)
