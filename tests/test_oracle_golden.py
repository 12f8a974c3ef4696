"""Oracle pins against printed values and textbook forms (CPU):

* the paper's worked example of complex-step backpropagation (Sec. 4.4, Fig. 5:
  w = (x y)^2 at x = 2, y = 3 gives 36 and 18; ``golden/fig5_complex_step_bp.json``)
  reproduced by a complex-step backward pass written here, which then pins the
  oracle's hyper-dual a^T H on deep tanh / sin decoders from outside its own code;
* the cubature force with every tet at weight 1 is the full mesh's internal force
  (central differences of the total elastic energy);
* at rest, a linear decoder's Newton matrix and first Newton step equal the textbook
  reduced linear-elastic implicit-Euler step, with the element stiffness assembled here
  in Voigt notation (StVK linearises to isotropic linear elasticity at F = I)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2102_11026_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


# ----------------------------------------------------- complex-step BP (Fig. 5) --

def test_fig5_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "fig5_complex_step_bp.json")))
    h = 1e-20
    x = complex(g["point"]["x"], h)
    y = g["point"]["y"]
    z = x * y
    # backward pass in complex arithmetic: dw/dz = 2 z, dw/dx = dw/dz * y
    dw_dz = 2.0 * z
    dw_dx = dw_dz * y
    assert dw_dz.real == g["dw_dz_at_perturbed_point"]["real"]
    assert dw_dz.imag / h == pytest.approx(g["dw_dz_at_perturbed_point"]["imag_over_h"], rel=1e-15)
    assert dw_dx.real == g["dw_dx"]
    assert dw_dx.imag / h == pytest.approx(g["d2w_dx2"], rel=1e-15)


def _act(act, z):
    return {"tanh": np.tanh, "sin": np.sin, "linear": lambda t: t}[act](z)


def _dact(act, z):
    return {"tanh": lambda t: 1.0 - np.tanh(t) ** 2, "sin": np.cos,
            "linear": lambda t: np.ones_like(t)}[act](z)


def complex_step_bp_aTH(dec, q, a, h=1e-20):
    """Column j of a^T H: forward pass with q_j + h i in complex arithmetic, backward
    pass of g(q) = a . D(q) in complex arithmetic, imaginary part of the input signal
    divided by h (Sec. 4.4)."""
    W = [np.asarray(w, np.float64) for w in dec.W]
    b = [np.asarray(x, np.float64) for x in dec.b]
    r = q.size
    out = np.zeros((r, r))
    for j in range(r):
        x = q.astype(complex)
        x[j] += 1j * h
        zs = []
        act = x
        for l in range(len(W)):
            z = W[l] @ act + b[l]
            if l < len(W) - 1:
                zs.append(z)
                act = _act(dec.act, z)
            else:
                act = z
        delta = np.asarray(a, complex)              # dg/du, the output layer is linear
        for l in range(len(W) - 1, 0, -1):
            delta = (W[l].T @ delta) * _dact(dec.act, zs[l - 1])
        grad = W[0].T @ delta
        out[:, j] = grad.imag / h
    return out


@pytest.mark.parametrize("act", ["tanh", "sin"])
def test_oracle_aTH_matches_complex_step_backprop(act):
    wl = synth.custom([4, 24, 32, 24, 3 * 2 * 2 * 4], (2, 2, 4), 6, 31, act=act)
    rng = np.random.default_rng(2)
    q = rng.normal(0, 0.4, 4)
    a = rng.normal(0, 1.0, wl.dec.n_out)
    ref = complex_step_bp_aTH(wl.dec, q, a)
    got = oracle.aTH(wl.dec, q, a)
    assert np.linalg.norm(ref) > 1e-3
    assert relerr(got, ref) <= 1e-12, relerr(got, ref)
    assert np.allclose(ref, ref.T, rtol=0, atol=1e-12 * np.abs(ref).max())


# ------------------------------------------------------------- full-mesh force --

def test_unit_weights_on_every_tet_give_the_full_mesh_force():
    wl = synth.custom([3, 16, 3 * 2 * 2 * 3], (2, 2, 3), 100, 12, material="neohookean")
    n_tet = wl.mesh.n_tet
    wl.cub_tets = np.arange(n_tet, dtype=np.int32)
    wl.cub_w = np.ones(n_tet, np.float32)
    q = np.random.default_rng(3).normal(0, 0.2, 3)
    rs = oracle.reduced_system(wl, q)
    u = rs["u"]

    def E(uu):
        return float(np.sum(oracle.tets_fk(wl.mesh, uu, np.arange(n_tet), want_K=False)[0]))
    eps = 1e-6
    f_int = np.array([(E(u + eps * e) - E(u - eps * e)) / (2 * eps) for e in np.eye(u.size)])
    assert np.linalg.norm(f_int) > 1.0
    assert relerr(rs["fC"], f_int) <= 1e-7
    assert relerr(rs["g_int"], rs["J"].T @ f_int) <= 1e-7


# ------------------------------------------------- textbook linear-elastic step --

def linear_tet_stiffness(X, E, nu):
    """12 x 12 linear-elastic stiffness of a 4-node tet: V B^T C B with the Voigt
    strain-displacement matrix B of the linear shape functions and the isotropic
    elasticity matrix C (engineering shear strains)."""
    Dm = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
    V = abs(np.linalg.det(Dm)) / 6.0
    G = np.linalg.inv(Dm)                  # row a-1: gradient of shape function a >= 1
    grads = np.vstack([-G.sum(0), G])
    B = np.zeros((6, 12))
    for a, (bx, by, bz) in enumerate(grads):
        c = 3 * a
        B[0, c] = bx
        B[1, c + 1] = by
        B[2, c + 2] = bz
        B[3, c + 1], B[3, c + 2] = bz, by
        B[4, c], B[4, c + 2] = bz, bx
        B[5, c], B[5, c + 1] = by, bx
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[[0, 1, 2], [0, 1, 2]] += 2 * mu
    C[[3, 4, 5], [3, 4, 5]] = mu
    return V * B.T @ C @ B


def test_linear_decoder_step_at_rest_is_the_textbook_linear_elastic_step():
    V = 2 * 2 * 4
    wl = synth.custom([5, 12, 3 * V], (2, 2, 4), 1000, 21, act="linear", gravity=True)
    wl.dec.b = [np.zeros_like(x) for x in wl.dec.b]
    n_tet = wl.mesh.n_tet
    rng = np.random.default_rng(8)
    wl.cub_tets = np.arange(n_tet, dtype=np.int32)
    wl.cub_w = rng.uniform(0.5, 2.0, n_tet).astype(np.float32)
    dt = wl.state.dt
    qdot = rng.normal(0, 0.1, 5)
    qbar = -dt * qdot                           # first iterate q0 = qbar + dt qdot = 0
    B = np.eye(5)
    for W in wl.dec.W:
        B = np.asarray(W, np.float64) @ B
    K0 = np.zeros((3 * V, 3 * V))
    for e in range(n_tet):
        T = wl.mesh.tets[e]
        Ke = linear_tet_stiffness(wl.mesh.X[T], wl.mesh.E, wl.mesh.nu)
        dofs = (3 * T[:, None] + np.arange(3)).reshape(-1)
        K0[np.ix_(dofs, dofs)] += float(wl.cub_w[e]) * Ke
    M = np.repeat(wl.mesh.vmass, 3)
    f = np.asarray(wl.f_ext, np.float64)
    BMB = B.T @ (M[:, None] * B)
    A_txt = BMB + dt ** 2 * B.T @ K0 @ B
    q1_txt = np.linalg.solve(A_txt, BMB @ (qbar + dt * qdot) + dt ** 2 * B.T @ f)
    rs = oracle.reduced_system(wl, np.zeros(5), qbar=qbar, qbar_dot=qdot)
    assert relerr(rs["A"], A_txt) <= 1e-10, relerr(rs["A"], A_txt)
    q1 = np.linalg.solve(rs["A"], -rs["phi"])
    assert np.linalg.norm(q1_txt) > 1e-6
    assert relerr(q1, q1_txt) <= 1e-10, relerr(q1, q1_txt)
