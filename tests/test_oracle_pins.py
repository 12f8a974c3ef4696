"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
closed forms, central differences, symmetries, the paper's printed formulas and
textbook material energies.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_2102_11026_gb300 import synth


def tiny_net(widths, seed, act="tanh", scale=1.0):
    dec = synth.make_decoder(widths, seed, act, out_scale=scale)
    return dec


def relerr(x, ref):
    return np.linalg.norm(np.asarray(x) - np.asarray(ref)) / max(np.linalg.norm(ref), 1e-300)


# ---------------------------------------------------------------- decoder --

ACTS = {
    "tanh": (np.tanh,
             lambda x: 1 - np.tanh(x) ** 2,
             lambda x: -2 * np.tanh(x) * (1 - np.tanh(x) ** 2),
             lambda x: -2 * (1 - np.tanh(x) ** 2) * (1 - 3 * np.tanh(x) ** 2)),
    "sin": (np.sin, np.cos, lambda x: -np.sin(x), lambda x: -np.cos(x)),
}


@pytest.mark.parametrize("act", ["tanh", "sin"])
def test_one_hidden_layer_closed_forms(act):
    """u = W2 s(W1 q + b1) + b2; J = W2 diag(s') W1; H[n,i,j] = sum_k W2 s'' W1 W1;
    S likewise with s'''.  Written with the chain rule, not with jets."""
    r, K, N = 4, 7, 9
    dec = tiny_net([r, K, N], 11, act)
    W1, W2 = dec.W[0].astype(np.float64), dec.W[1].astype(np.float64)
    b1, b2 = dec.b[0].astype(np.float64), dec.b[1].astype(np.float64)
    rng = np.random.default_rng(3)
    q, qbar, qd = rng.normal(0, .5, r), rng.normal(0, .5, r), rng.normal(0, .3, r)
    dt = 0.1
    s0, s1, s2, s3 = ACTS[act]
    zz = W1 @ q + b1
    D = q - qbar
    w = 3 * D - dt * qd
    u = W2 @ s0(zz) + b2
    J = W2 @ (s1(zz)[:, None] * W1)
    H = np.einsum("nk,k,ki,kj->nij", W2, s2(zz), W1, W1)
    S = np.einsum("nk,k,ki,kj,kl->nijl", W2, s3(zz), W1, W1, W1)
    d = oracle.derivs(dec, q, qbar, qd, dt)
    assert relerr(d["u"], u) < 1e-14
    assert relerr(d["J"], J) < 1e-13
    assert relerr(d["HDe"], np.einsum("nij,i->nj", H, D)) < 1e-12
    assert relerr(d["Hw"], np.einsum("nij,i->nj", H, w)) < 1e-12
    assert relerr(d["HDD"], np.einsum("nij,i,j->n", H, D, D)) < 1e-12
    assert relerr(d["Sdd"], np.einsum("nijl,j,l->ni", S, D, D)) < 1e-12
    assert relerr(d["Hqq"], np.einsum("nij,i,j->n", H, D / dt, D / dt)) < 1e-12
    a = rng.normal(0, 1, N)
    assert relerr(oracle.aTH(dec, q, a), np.einsum("n,nij->ij", a, H)) < 1e-12


def test_linear_net_has_zero_hessian():
    """Linear activation: D(q) = W3 W2 W1 q + c, so J = W3 W2 W1 and H = S = 0
    exactly (the remark after Eq. 6: the nonlinear reduction collapses to Eq. 3)."""
    dec = tiny_net([3, 6, 5, 12], 5, "linear")
    rng = np.random.default_rng(0)
    q, qbar, qd = rng.normal(0, 1, 3), rng.normal(0, 1, 3), rng.normal(0, 1, 3)
    d = oracle.derivs(dec, q, qbar, qd, 0.05)
    Wp = dec.W[2].astype(np.float64) @ dec.W[1].astype(np.float64) @ dec.W[0].astype(np.float64)
    assert relerr(d["J"], Wp) < 1e-14
    for k in ("HDe", "Hw", "Sdd", "dJ", "HDD"):
        assert np.all(d[k] == 0.0), k
    assert np.all(oracle.aTH(dec, q, rng.normal(size=12)) == 0.0)


def _fd_J(dec, q, eps=1e-5):
    cols = []
    for j in range(q.size):
        e = np.zeros(q.size); e[j] = eps
        cols.append((oracle.decode(dec, q + e) - oracle.decode(dec, q - e)) / (2 * eps))
    return np.stack(cols, 1)


@pytest.mark.parametrize("act", ["tanh", "sin"])
def test_deep_net_against_central_differences(act):
    """Depth-3 net of width <= 8: J from central differences of u; H[., e_j] from
    central differences of J; S[e_j, D, D] from central differences of H[D, D]."""
    r = 3
    dec = tiny_net([r, 8, 8, 6, 9], 21, act)
    rng = np.random.default_rng(7)
    q, qbar, qd = rng.normal(0, .5, r), rng.normal(0, .5, r), rng.normal(0, .3, r)
    dt = 0.2
    d = oracle.derivs(dec, q, qbar, qd, dt)
    assert relerr(d["J"], _fd_J(dec, q)) < 1e-8
    D = q - qbar
    w = 3 * D - dt * qd
    eps = 1e-4
    # H[e_j, v] = d/de (J v)(q + e e_j)
    HDe, Hw = np.zeros_like(d["J"]), np.zeros_like(d["J"])
    for j in range(r):
        e = np.zeros(r); e[j] = eps
        Jp, Jm = _fd_J(dec, q + e, 1e-4), _fd_J(dec, q - e, 1e-4)
        HDe[:, j] = (Jp - Jm) @ D / (2 * eps)
        Hw[:, j] = (Jp - Jm) @ w / (2 * eps)
    assert relerr(d["HDe"], HDe) < 1e-5
    assert relerr(d["Hw"], Hw) < 1e-5
    # H[D,D] from second differences of the plain forward pass
    h = 1e-3
    HDD = (oracle.decode(dec, q + h * D) - 2 * oracle.decode(dec, q)
           + oracle.decode(dec, q - h * D)) / h ** 2
    assert relerr(d["HDD"], HDD) < 1e-5
    # S[e_j, D, D] = d/de H[D,D](q + e e_j), with H[D,D] from the oracle (pinned above)
    Sdd = np.zeros_like(d["J"])
    for j in range(r):
        e = np.zeros(r); e[j] = eps
        Hp = oracle.derivs(dec, q + e, qbar + e, qd, dt)["HDD"]   # same D
        Hm = oracle.derivs(dec, q - e, qbar - e, qd, dt)["HDD"]
        Sdd[:, j] = (Hp - Hm) / (2 * eps)
    assert relerr(d["Sdd"], Sdd) < 1e-6


def test_jet_symmetries():
    """S[e_j, D, D] = S[D, e_j, D] (seed in another slot) and
    sum_j H[D, e_j] D_j = H[D, D]."""
    r = 4
    dec = tiny_net([r, 8, 8, 10], 31, "tanh")
    rng = np.random.default_rng(1)
    q, D = rng.normal(0, .5, r), rng.normal(0, .2, r)
    E = np.eye(r)
    a = oracle.decoder_jets(dec, q, E, D, D)[:, :, 7]
    b = oracle.decoder_jets(dec, q, D, E, D)[:, :, 7]
    assert relerr(a, b) < 1e-13
    d = oracle.derivs(dec, q, q - D, np.zeros(r), 0.1)
    assert relerr(d["HDe"] @ D, d["HDD"]) < 1e-13


def test_sin_jet_matches_bicomplex_formulas():
    """App. A gives sin(a + b i1 + c i2 + d i1 i2) for a bicomplex argument.  With
    b, c ~ h and d ~ h^2, dividing the i1, i2, i1i2 parts by h, h, h^2 gives the
    hyper-dual jet up to O(h^2).  (The first-order formula printed in App. A swaps
    sin/sinh; the second-order a'..d' are used here.)"""
    a0, b0, c0, d0 = 0.7, -1.3, 0.4, 2.1
    h = 1e-5
    a, b, c, d = a0, b0 * h, c0 * h, d0 * h * h
    A = np.sin(a) * np.cosh(b) * np.cosh(c) * np.cos(d) - np.cos(a) * np.sinh(b) * np.sinh(c) * np.sin(d)
    B = np.sin(a) * np.cosh(b) * np.sinh(c) * np.sin(d) + np.cos(a) * np.sinh(b) * np.cosh(c) * np.cos(d)
    C = np.cos(a) * np.cosh(b) * np.sinh(c) * np.cos(d) + np.sin(a) * np.sinh(b) * np.cosh(c) * np.sin(d)
    Dp = np.cos(a) * np.cosh(b) * np.cosh(c) * np.sin(d) - np.sin(a) * np.sinh(b) * np.sinh(c) * np.cos(d)
    jet = oracle.act_jet("sin", [a0, b0, c0, d0, 0, 0, 0, 0])
    assert abs(jet[0] - A) < 1e-9
    assert abs(jet[1] - B / h) < 1e-8
    assert abs(jet[2] - C / h) < 1e-8
    assert abs(jet[3] - Dp / h ** 2) < 1e-5 * max(1, abs(jet[3]))


def test_tanh_jet_matches_complex_step():
    """First-order complex step on tanh (Eq. 15): Im tanh(a + i h)/h -> tanh'(a)."""
    a0 = 0.37
    h = 1e-20
    jet = oracle.act_jet("tanh", [a0, 1, 0, 0, 0, 0, 0, 0])
    assert abs(jet[1] - np.tanh(a0 + 1j * h).imag / h) < 1e-15


def test_aTH_regrouped_equals_plain():
    dec = tiny_net([3, 8, 8, 15], 41, "tanh")
    rng = np.random.default_rng(2)
    q, a = rng.normal(0, .5, 3), rng.normal(0, 1, 15)
    assert relerr(oracle.aTH_regrouped(dec, q, a), oracle.aTH(dec, q, a)) < 1e-13


# -------------------------------------------------------------------- FEM --

def unit_tet_mesh(material="stvk", E=1e5, nu=0.4):
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) * 1.3 + 0.2
    return synth.Mesh(X, np.array([[0, 1, 2, 3]], np.int32), np.ones(4), material, E, nu)


@pytest.mark.parametrize("mat", ["stvk", "neohookean"])
def test_rest_state_is_force_free(mat):
    m = unit_tet_mesh(mat)
    en, f, K, st = oracle.tets_fk(m, np.zeros(12), [0])
    assert st[0] == 0 and abs(en[0]) < 1e-9 and np.abs(f).max() < 1e-9


@pytest.mark.parametrize("mat", ["stvk", "neohookean"])
def test_uniform_stretch_energy(mat):
    """x = s X: F = s I.  StVK: E = (s^2-1)/2 I, Psi = 3 mu e^2 + lam/2 (3e)^2.
    NH: Psi = mu/2 (3 s^2 - 3) - mu ln s^3 + lam/2 (ln s^3)^2.  Times V = |det Dm|/6."""
    m = unit_tet_mesh(mat, 2e4, 0.3)
    s = 1.07
    u = ((s - 1) * m.X).reshape(-1)
    en, f, K, st = oracle.tets_fk(m, u, [0])
    mu, lam = oracle.lame(m.E, m.nu)
    V = 1.3 ** 3 / 6
    if mat == "stvk":
        e = (s * s - 1) / 2
        psi = 3 * mu * e * e + lam / 2 * (3 * e) ** 2
    else:
        lj = np.log(s ** 3)
        psi = mu / 2 * (3 * s * s - 3) - mu * lj + lam / 2 * lj * lj
    assert abs(en[0] - V * psi) < 1e-10 * abs(V * psi)


@pytest.mark.parametrize("mat", ["stvk", "neohookean"])
def test_force_and_stiffness_by_differences(mat):
    """f = grad(V Psi) and K = grad f by central differences; K symmetric;
    energy invariant under a rigid rotation and forces rotate with it."""
    m = unit_tet_mesh(mat)
    rng = np.random.default_rng(4)
    u = rng.normal(0, 0.05, 12)
    en, f, K, st = oracle.tets_fk(m, u, [0])
    eps = 1e-6
    fd_f, fd_K = np.zeros(12), np.zeros((12, 12))
    for a in range(12):
        e = np.zeros(12); e[a] = eps
        ep, fp, _, _ = oracle.tets_fk(m, u + e, [0])
        em, fm, _, _ = oracle.tets_fk(m, u - e, [0])
        fd_f[a] = (ep[0] - em[0]) / (2 * eps)
        fd_K[:, a] = (fp[0] - fm[0]) / (2 * eps)
    assert relerr(f[0], fd_f) < 1e-7
    assert relerr(K[0], fd_K) < 1e-7
    assert np.abs(K[0] - K[0].T).max() < 1e-9 * np.abs(K[0]).max()
    th = 0.9
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    x = m.X + u.reshape(4, 3)
    ur = (x @ R.T - m.X).reshape(-1)
    en2, f2, _, _ = oracle.tets_fk(m, ur, [0])
    assert abs(en2[0] - en[0]) < 1e-10 * abs(en[0])
    assert relerr(f2[0].reshape(4, 3), f[0].reshape(4, 3) @ R.T) < 1e-10


def test_inverted_neohookean_tet_is_flagged():
    m = unit_tet_mesh("neohookean")
    u = np.zeros((4, 3)); u[3, 2] = -2.0 * 1.3   # push apex through the base
    _, _, _, st = oracle.tets_fk(m, u.reshape(-1), [0])
    assert st[0] == -7


# --------------------------------------------------------- reduced system --

def tiny_workload(act="tanh", material="stvk", seed=3, gravity=True, qd_scale=1.0):
    wl = synth.custom([3, 8, 8, 3 * 27], (3, 3, 3), 12, seed, act, material, 1e3, 0.3, gravity)
    wl.dec.W[-1] *= 3.0
    wl.state.qbar_dot = wl.state.qbar_dot * qd_scale * 20
    wl.state.dt = 0.05
    return wl


@pytest.mark.parametrize("material", ["stvk", "neohookean"])
def test_newton_matrix_is_jacobian_of_phi(material):
    """A (Eq. 11 with n_p = 0, '+' sign on the H^T (f_int - f_ext) term) equals the
    central-difference Jacobian of phi (Eq. 7).  The printed '-' sign fails this."""
    wl = tiny_workload(material=material)
    rng = np.random.default_rng(9)
    q = wl.state.qbar + wl.state.dt * wl.state.qbar_dot + rng.normal(0, 0.05, 3)
    rs = oracle.reduced_system(wl, q)
    eps = 1e-6
    A_fd = np.zeros((3, 3))
    for k in range(3):
        e = np.zeros(3); e[k] = eps
        A_fd[:, k] = (oracle.phi_only(wl, q + e) - oracle.phi_only(wl, q - e)) / (2 * eps)
    assert relerr(rs["A"], A_fd) < 1e-6
    assert relerr(rs["phi"], oracle.phi_only(wl, q)) < 1e-14
    wrong = rs["A"] - 2 * wl.state.dt ** 2 * oracle.aTH(wl.dec, q, rs["fC"] - wl.f_ext)
    assert relerr(wrong, A_fd) > 1e-3


def test_phi_terms_against_plain_differences():
    """phi recomputed from Eq. 7 with J and H[D,D] taken from central / second
    differences of the plain forward pass (no jets)."""
    wl = tiny_workload()
    st = wl.state
    rng = np.random.default_rng(5)
    q = st.qbar + st.dt * st.qbar_dot + rng.normal(0, 0.05, 3)
    D = q - st.qbar
    z = D - st.dt * st.qbar_dot
    J = _fd_J(wl.dec, q)
    h = 1e-3
    HDD = (oracle.decode(wl.dec, q + h * D) - 2 * oracle.decode(wl.dec, q)
           + oracle.decode(wl.dec, q - h * D)) / h ** 2
    u = oracle.decode(wl.dec, q)
    en, fe, _, _ = oracle.tets_fk(wl.mesh, u, wl.cub_tets, want_K=False)
    dofs = oracle.tet_dofs(wl.mesh, wl.cub_tets)
    fC = np.zeros(u.size)
    np.add.at(fC, dofs.reshape(-1), (wl.cub_w.astype(float)[:, None] * fe).reshape(-1))
    M = np.repeat(wl.mesh.vmass, 3)
    phi = J.T @ (M * (J @ z + HDD)) + st.dt ** 2 * J.T @ (fC - wl.f_ext)
    assert relerr(oracle.reduced_system(wl, q)["phi"], phi) < 1e-6


def test_cubature_force_is_energy_gradient():
    """g_int = J^T f_C = d/dq sum_e w_e V_e Psi_e(D(q))."""
    wl = tiny_workload()
    rng = np.random.default_rng(6)
    q = rng.normal(0, 0.3, 3)
    rs = oracle.reduced_system(wl, q)
    cw = wl.cub_w.astype(float)

    def Ec(qq):
        en, _, _, _ = oracle.tets_fk(wl.mesh, oracle.decode(wl.dec, qq), wl.cub_tets, want_K=False)
        return float(np.sum(cw * en))

    g = np.array([(Ec(q + e) - Ec(q - e)) / 2e-6 for e in np.eye(3) * 1e-6])
    assert relerr(rs["g_int"], g) < 1e-6
    assert abs(rs["energy"] - Ec(q)) < 1e-12 * abs(Ec(q))


def test_newton_matrix_symmetric_cases():
    """A is symmetric when Delta = 0 and qbar_dot = 0 (then z = 0 and dJ = 0), and
    for linear decoders (H = S = 0); not in general."""
    wl = tiny_workload()
    q = wl.state.qbar.copy()
    rs = oracle.reduced_system(wl, q, qbar_dot=np.zeros(3))
    A = rs["A"]
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    wl2 = tiny_workload(act="linear")
    q2 = wl2.state.qbar + 0.1
    A2 = oracle.reduced_system(wl2, q2)["A"]
    assert np.abs(A2 - A2.T).max() <= 1e-12 * np.abs(A2).max()
    A3 = oracle.reduced_system(wl, q + 0.1)["A"]
    assert np.abs(A3 - A3.T).max() > 1e-6 * np.abs(A3).max()


@pytest.mark.parametrize("material", ["stvk", "neohookean"])
def test_newton_converges_quadratically(material):
    wl = synth.custom([3, 8, 8, 3 * 27], (3, 3, 3), 12, 3, "tanh", material, 1e3, 0.3, True)
    wl.state.dt = 1.0 / 60.0
    wl.state.qbar_dot = wl.state.qbar_dot * 20
    q, rep = oracle.newton_solve(wl, max_iter=12, tol=1e-12, xtol=0.0)
    assert rep["converged"], rep["phi_hist"]
    h = rep["phi_hist"]
    assert np.linalg.norm(oracle.phi_only(wl, q)) <= 1e-12 * max(1, h[0])
    # quadratic tail: once small, the residual at least squares (up to a constant)
    assert len(h) <= 7
    # quadratic tail: e_{k+1} <= C e_k^2 with a modest C
    for a, b in zip(h[2:], h[3:]):
        assert b <= 1e3 * a * a + 1e-15


def test_small_workload_shapes():
    wl = synth.small()
    assert wl.dec.n_params == 5 * 64 + 64 * 256 + 256 * 1024 + 1024 * 3000
    assert wl.mesh.n_tet == 3645 and wl.dec.n_out == 3 * wl.mesh.n_vert
    assert len(set(wl.cub_tets.tolist())) == 64
    assert wl.cub_w.min() >= 0.5 and wl.cub_w.max() <= 2.0


def test_newton_step_cap_and_step_tolerance():
    """max_step caps the first trial of an update in the max-norm (the accepted
    iterate lies on the Newton direction at distance max_step); the xtol stop ends
    at an iterate whose remaining Newton correction is below xtol, which is that
    close to the tightly converged solution."""
    wl = synth.custom([3, 8, 8, 3 * 27], (3, 3, 3), 12, 3, "tanh", "stvk", 1e3, 0.3, True)
    wl.state.qbar_dot = wl.state.qbar_dot * 20
    q0 = synth.newton_start(wl.state)
    rs = oracle.reduced_system(wl, q0)
    delta = np.linalg.solve(rs["A"], -rs["phi"])
    cap = 0.25 * np.abs(delta).max()
    q1, rep1 = oracle.newton_solve(wl, q0=q0, max_iter=1, max_step=cap, xtol=0.0)
    step = q1 - q0
    assert abs(np.abs(step).max() - cap) <= 1e-12 * cap
    assert np.allclose(step, cap * delta / np.abs(delta).max(), rtol=1e-10, atol=0)
    # no cap: the full Newton step is taken
    qf, _ = oracle.newton_solve(wl, q0=q0, max_iter=1, max_step=0.0, xtol=0.0)
    assert np.allclose(qf - q0, delta, rtol=1e-10, atol=1e-14)
    # step tolerance against the tightly converged solution
    qt, rt = oracle.newton_solve(wl, q0=q0, max_iter=20, tol=1e-13, xtol=0.0)
    qx, rx = oracle.newton_solve(wl, q0=q0, max_iter=20, tol=0.0, xtol=1e-6)
    assert rt["converged"] and rx["converged"]
    assert np.abs(qx - qt).max() <= 2e-6 * max(1.0, np.abs(qt).max())
    assert rx["iters"] <= rt["iters"]


def test_simplified_newton_stop_agrees_with_the_full_step():
    """After an accepted trial, the stop on the simplified-Newton estimate -A_prev^{-1}
    phi(q) takes the same decision as the full step -A(q)^{-1} phi(q) on a
    quadratically converging frame: the same iterate and count of iterations, one Newton
    matrix fewer, and the true remaining step at the end is below xtol.  (An estimate
    formed with the previous residual, or with the sign of a step already taken, would
    not stop, and the count of matrices would not drop.)"""
    wl = synth.custom([3, 8, 8, 3 * 27], (3, 3, 3), 12, 3, "tanh", "stvk", 1e3, 0.3, True)
    q0 = synth.newton_start(wl.state)
    xtol = 1e-6
    qe, re = oracle.newton_solve(wl, q0=q0, max_iter=20, tol=0.0, xtol=xtol)
    system = lambda x: oracle.reduced_system(wl, x)
    qn, rn = oracle.newton_iterate(system, q0, 20, tol=0.0, xtol=xtol, estimate=False)
    assert re["converged"] and rn["converged"]
    assert re["iters"] == rn["iters"] >= 2 and np.array_equal(qe, qn)
    assert re["nfull"] == re["iters"] and rn["nfull"] == rn["iters"] + 1
    rs = oracle.reduced_system(wl, qe)
    step = np.linalg.solve(rs["A"], -rs["phi"])
    assert np.abs(step).max() <= xtol * max(1.0, np.abs(qe).max())


# --------------------------------------------- decoder backward (u, J) ---

def _uJ_loss(dec, Q, gu, gJ):
    """L = sum_s gu_s . u(q_s) + sum_{s,j} gJ_s[:, j] . J(q_s) e_j, with u and J from
    the hyper-dual jets (independent of the reverse sweep)."""
    r = dec.r
    tot = 0.0
    for s in range(Q.shape[0]):
        jet = oracle.decoder_jets(dec, Q[s], np.eye(r))
        u = jet[0, :, 0]
        J = jet[:, :, 1].T
        tot += gu[s] @ u + np.sum(gJ[s] * J)
    return tot


@pytest.mark.parametrize("act", ["tanh", "sin", "linear"])
def test_uJ_vjp_against_central_differences(act):
    """Every latent gradient and a sample of weight / bias gradients against FP64
    central differences of the jet-evaluated loss: h = 1e-6 on the FP64 latents,
    h = 2^-12 on the weights and biases (stored in FP32 by the decoder, so the step
    must be exactly representable next to them)."""
    import copy
    dec = tiny_net([3, 5, 6, 9], 21, act)
    rng = np.random.default_rng(4)
    B, r, N = 2, 3, 9
    Q = rng.normal(0, 0.6, (B, r))
    gu = rng.normal(size=(B, N))
    gJ = rng.normal(size=(B, N, r))
    gq, gW, gb = oracle.decoder_uJ_vjp(dec, Q, gu, gJ)
    h = 1e-6
    fd = np.zeros_like(Q)
    for s in range(B):
        for j in range(r):
            Qp, Qm = Q.copy(), Q.copy()
            Qp[s, j] += h
            Qm[s, j] -= h
            fd[s, j] = (_uJ_loss(dec, Qp, gu, gJ) - _uJ_loss(dec, Qm, gu, gJ)) / (2 * h)
    assert relerr(gq, fd) < 1e-6
    hw = np.float32(2.0 ** -12)
    for l in range(3):
        for (i, k) in [(0, 0), (1, 2), (dec.W[l].shape[0] - 1, dec.W[l].shape[1] - 1)]:
            dp, dm = copy.deepcopy(dec), copy.deepcopy(dec)
            dp.W[l][i, k] += hw
            dm.W[l][i, k] -= hw
            step = float(dp.W[l][i, k]) - float(dm.W[l][i, k])
            g = (_uJ_loss(dp, Q, gu, gJ) - _uJ_loss(dm, Q, gu, gJ)) / step
            assert abs(gW[l][i, k] - g) <= 1e-6 * max(1.0, abs(g)), (l, i, k, gW[l][i, k], g)
        dp, dm = copy.deepcopy(dec), copy.deepcopy(dec)
        dp.b[l][1] += hw
        dm.b[l][1] -= hw
        step = float(dp.b[l][1]) - float(dm.b[l][1])
        g = (_uJ_loss(dp, Q, gu, gJ) - _uJ_loss(dm, Q, gu, gJ)) / step
        assert abs(gb[l][1] - g) <= 1e-6 * max(1.0, abs(g))


def test_uJ_vjp_one_hidden_layer_closed_form():
    """u = W2 t + b2, J = W2 diag(t') W1 with t = tanh(W1 q + b1); the gradients written
    out by hand: dL/dW2 = gu t^T + sum_j gJ_j (t' * W1 e_j)^T, dL/db2 = gu,
    dL/dz = t' (W2^T gu) + t'' sum_j (W1 e_j) (W2^T gJ_j),
    dL/dW1 = dL/dz q^T + sum_j (t' W2^T gJ_j) e_j^T, dL/db1 = dL/dz, dL/dq = W1^T dL/dz."""
    r, K, N = 4, 7, 9
    dec = tiny_net([r, K, N], 12, "tanh")
    W1, W2 = dec.W[0].astype(np.float64), dec.W[1].astype(np.float64)
    b1 = dec.b[0].astype(np.float64)
    rng = np.random.default_rng(8)
    q = rng.normal(0, .5, r)
    gu = rng.normal(size=N)
    gJ = rng.normal(size=(N, r))
    z = W1 @ q + b1
    t = np.tanh(z)
    t1 = 1 - t ** 2
    t2 = -2 * t * t1
    gW2 = np.outer(gu, t) + sum(np.outer(gJ[:, j], t1 * W1[:, j]) for j in range(r))
    gz = t1 * (W2.T @ gu) + t2 * sum(W1[:, j] * (W2.T @ gJ[:, j]) for j in range(r))
    gW1 = np.outer(gz, q) + sum(np.outer(t1 * (W2.T @ gJ[:, j]), np.eye(r)[j]) for j in range(r))
    gq, gW, gb = oracle.decoder_uJ_vjp(dec, q[None], gu[None], gJ[None])
    assert relerr(gW[1], gW2) < 1e-13
    assert relerr(gb[1], gu) < 1e-13
    assert relerr(gW[0], gW1) < 1e-13
    assert relerr(gb[0], gz) < 1e-13
    assert relerr(gq[0], W1.T @ gz) < 1e-13


# ------------------------------------------------------------ weight network --
def _wnet(widths, W, b):
    return synth.WNet(list(widths), [np.asarray(w, np.float32) for w in W],
                      [np.asarray(x, np.float32) for x in b])


def test_wnet_layer_order_on_selected_dofs():
    """Sec. 5, Weight Prediction: u = D(q), four FC layers, sin after the first three,
    a square after the last.  With one-hot first-layer rows picking DOFs d_i and
    identity layers after it, w_i = sin(sin(sin(u_{d_i})))^2 exactly: a dropped sin, a
    sin on the last layer or a square in the wrong place fails."""
    wl = synth.small()
    dec = wl.dec
    N = dec.n_out
    q = synth.newton_start(wl.state)
    d = np.array([0, 17, 512, N - 1])
    W1 = np.zeros((4, N), np.float32)
    W1[np.arange(4), d] = 1.0
    I4 = np.eye(4, dtype=np.float32)
    net = _wnet([N, 4, 4, 4, 4], [W1, I4, I4, I4], [np.zeros(4)] * 4)
    u = oracle.decode(dec, q)
    want = np.sin(np.sin(np.sin(u[d]))) ** 2
    got = oracle.wnet_weights(net, dec, q)
    assert np.allclose(got, want, rtol=1e-12, atol=0)
    # biases enter before each activation: a zero last-layer row gives b^2
    net2 = _wnet([N, 4, 4, 4, 2], [W1, I4, I4, np.zeros((2, 4))],
                 [np.zeros(4), np.zeros(4), np.zeros(4), np.array([0.5, -1.5])])
    assert np.allclose(oracle.wnet_weights(net2, dec, q), [0.25, 2.25], rtol=1e-7)


def test_wnet_at_rest_shape_closed_form():
    """A bias-free odd decoder maps q = 0 to the rest shape (u = 0 exactly), so the
    network reduces to its biases: w = (W4 sin(W3 sin(W2 sin(b1) + b2) + b3) + b4)^2."""
    wl = synth.small()
    dec = wl.dec
    net = synth.make_wnet(dec.n_out, wl.mesh.n_tet, 3, hidden=(16, 12, 8))
    W = [w.astype(np.float64) for w in net.W]
    b = [x.astype(np.float64) for x in net.b]
    h = np.sin(b[0])
    h = np.sin(W[1] @ h + b[1])
    h = np.sin(W[2] @ h + b[2])
    want = (W[3] @ h + b[3]) ** 2
    got = oracle.wnet_weights(net, dec, np.zeros(dec.r))
    assert np.allclose(got, want, rtol=1e-12, atol=1e-15)
    sel = np.array([3, 40, 7])
    assert np.array_equal(oracle.wnet_weights(net, dec, np.zeros(dec.r), sel), got[sel])


def test_wnet_weights_are_nonnegative_and_depend_on_q():
    wl = synth.small()
    net = synth.make_wnet(wl.dec.n_out, wl.mesh.n_tet, 5)
    q = synth.newton_start(wl.state)
    w0 = oracle.wnet_weights(net, wl.dec, q, wl.cub_tets)
    w1 = oracle.wnet_weights(net, wl.dec, 2.0 * q, wl.cub_tets)
    assert w0.shape == wl.cub_tets.shape and np.all(w0 >= 0) and np.all(w1 >= 0)
    assert np.max(np.abs(w1 - w0)) > 1e-6
    assert 0.2 < np.median(w0) < 5.0


# ---------------------------------------------------- linear + nonlinear subspace --
def _linear_case(n_p=2, material="stvk"):
    wl = tiny_workload(material=material)
    U = synth.make_linear_basis(wl.dec.n_out, n_p, 4).astype(np.float64)
    pb, pd = synth.make_linear_state(n_p, 4, p_std=0.3)
    rbar = np.concatenate([pb, wl.state.qbar])
    rdot = np.concatenate([pd, wl.state.qbar_dot])
    rng = np.random.default_rng(11)
    r = rbar + wl.state.dt * rdot + rng.normal(0, 0.05, rbar.size)
    return wl, U, r, rbar, rdot


@pytest.mark.parametrize("material", ["stvk", "neohookean"])
def test_linear_subspace_A_is_jacobian_of_phi(material):
    """Eq. 11 for r = [p; q]: every block of A (U^T M U, U^T M (J + dJ), J^T M U, the
    q block with a^T H, dt^2 Jt^T K Jt) equals the central-difference Jacobian of phi."""
    wl, U, r, rbar, rdot = _linear_case(material=material)
    rs = oracle.linear_subspace_system(wl, U, r, rbar, rdot)
    n = r.size
    eps = 1e-6
    A_fd = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n); e[k] = eps
        A_fd[:, k] = (oracle.linear_subspace_system(wl, U, r + e, rbar, rdot, want_A=False)["phi"]
                      - oracle.linear_subspace_system(wl, U, r - e, rbar, rdot, want_A=False)["phi"]) / (2 * eps)
    assert relerr(rs["A"], A_fd) < 1e-6
    # the p block is the linear subspace's own inertia + stiffness
    n_p = U.shape[1]
    assert relerr(rs["A"][:n_p, :n_p], U.T @ (oracle.mass_diag(wl.mesh)[:, None] * U)
                  + wl.state.dt ** 2 * rs["Kr"][:n_p, :n_p]) < 1e-12


def test_linear_subspace_without_basis_is_the_decoder_system():
    wl = tiny_workload()
    q = synth.newton_start(wl.state)
    U0 = np.zeros((wl.dec.n_out, 0))
    a = oracle.linear_subspace_system(wl, U0, q, wl.state.qbar, wl.state.qbar_dot)
    b = oracle.reduced_system(wl, q)
    assert relerr(a["phi"], b["phi"]) < 1e-13 and relerr(a["A"], b["A"]) < 1e-13


def test_filtered_decoder_is_orthogonal_to_the_linear_subspace():
    """The filtering layer makes U^T Dt(q) = 0 and U^T Jt_q = 0 (Eq. 9's constraint), and
    u = U p + Dt(q)."""
    wl, U, r, rbar, rdot = _linear_case(n_p=3)
    rs = oracle.linear_subspace_system(wl, U, r, rbar, rdot)
    n_p = U.shape[1]
    Dt = rs["u"] - U @ r[:n_p]
    # U holds FP32 values (orthonormal to ~1e-7): the projector is exact up to that
    e = np.max(np.abs(U.T @ U - np.eye(n_p)))
    assert e < 1e-6
    assert np.max(np.abs(U.T @ Dt)) < 10 * e * np.max(np.abs(Dt))
    assert np.max(np.abs(U.T @ rs["Jt"][:, n_p:])) < 10 * e * np.max(np.abs(rs["Jt"][:, n_p:]))
    assert np.allclose(U.T @ rs["u"], (U.T @ U) @ r[:n_p], atol=10 * e * np.max(np.abs(Dt)))


def test_linear_subspace_newton_converges_quadratically():
    wl, U, r, rbar, rdot = _linear_case()
    r0 = rbar + wl.state.dt * rdot
    rq, rep = oracle.newton_solve(wl, q0=r0, qbar=rbar, qbar_dot=rdot, U=U, max_iter=6, xtol=0)
    h = rep["phi_hist"]
    assert rep["converged"] and len(h) >= 3
    assert h[-1] < 1e-10 * h[0]
    ks = [k for k in range(1, len(h) - 1) if h[k] < 1e-2 * h[0] and h[k + 1] > 1e-14]
    assert all(h[k + 1] <= 10.0 * h[k] ** 2 / h[0] for k in ks)
