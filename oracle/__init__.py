"""FP64 CPU oracle for the reduced implicit-Euler Newton step -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline
leg and ``--impl reference``) may import this package.  The product path never
calls it; it shares no code with the CUDA library.

It evaluates the plain definitions of every quantity in the paper's reduced
system (Sec. 3, Eqs. 6-12; Sec. 5 cubature), in FP64, with exact hyper-dual
derivatives of the decoder (``hyperdual.c``), and the Newton iteration with a
dense LU solve (``numpy.linalg.solve``).

Notation (r = latent size, N = 3V output DOFs, vertex-major x0,y0,z0,x1,...):
  Delta = q - qbar,   z = Delta - dt*qbar_dot,   w = 3*Delta - dt*qbar_dot
  J = dD/dq (N x r),  H = d2D/dq2,  S = d3D/dq3 (never formed in full)
  HDD    = H[Delta, Delta]                    (f_fict = M HDD, Eq. 8)
  Hqq    = H[qdot, qdot], qdot = Delta/dt     (the inertial term of Eq. 5)
  dJ     = S[.,Delta,Delta] + H[., w]         (Eq. 12)
  f_C    = sum_{e in C} w_e scatter(f_e)      (cubature force, Sec. 5)
  phi    = J^T M (J z + HDD) + dt^2 (J^T f_C - J^T f_ext)        (Eq. 7, x dt^2 form)
  a      = M (J z + HDD) + dt^2 (f_C - f_ext)
  A      = a^T H + J^T M (J + dJ) + dt^2 K_r,  K_r = sum w_e J_e^T K_e J_e   (Eq. 11, n_p = 0)

Coupled substructures (Sec. 6, deformation substructuring): domains tied by penalty
springs between interface vertices that coincide at rest (and anchors holding a root's
base at rest); ``coupled_system`` stacks every domain's Eq. 10 residual with the tie
force among its forces and adds the ties' Hessian blocks to the global Newton matrix;
``coupled_newton_solve`` runs the same Newton iteration on the stacked latents.

Readings of the paper taken here (each also listed in the design notes):
  * Eq. 11 prints "- h^2 H^T (f_int - f_ext)"; differentiating Eq. 10 gives "+".
    ``tests/test_oracle_pins.py`` pins A against central differences of phi.
  * Eq. 11 is not symmetric in general (J^T M dJ is not), so the Newton step uses
    LU with partial pivoting rather than the Cholesky the paper mentions.
  * The paper does not specify a line search; backtracking (Armijo on |phi|^2,
    c = 1e-4, step halving, at most 8 halvings) is used.
  * The paper defers the coupling of its domains to Barbic & Zhao (2011) and states no
    formulation; the ties are read as penalty springs (stiffness k_c) between
    coinciding interface vertices, in one global Newton system over all domains.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hyperdual.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

ACT = {"tanh": 0, "sin": 1, "linear": 2}
MAT = {"stvk": 0, "neohookean": 1}


def build(force=False):
    """Compile hyperdual.c into oracle/_build/liboracle.so with gcc (+OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c99", "-fsigned-char",
           _SRC, "-o", _LIB + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        fpp = ctypes.POINTER(ctypes.POINTER(ctypes.c_float))
        L.orc_act_jet.argtypes = [ctypes.c_int, dp, dp]
        L.orc_decoder_jets.argtypes = [ctypes.c_int, ip, fpp, fpp, ctypes.c_int, ctypes.c_int,
                                       dp, ctypes.c_int, dp, dp, dp, ctypes.c_int, ip, dp]
        L.orc_decoder_jets.restype = ctypes.c_int
        L.orc_tets_fk.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_double, dp, dp, dp, ip]
        L.orc_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def num_threads():
    return lib().orc_num_threads()


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


class _DecoderView:
    """Keeps the float32 weight arrays alive and exposes them as C pointer arrays."""

    def __init__(self, dec):
        self.dec = dec
        self.W = [np.ascontiguousarray(w, dtype=np.float32) for w in dec.W]
        self.b = [np.ascontiguousarray(x, dtype=np.float32) for x in dec.b]
        fp = ctypes.POINTER(ctypes.c_float)
        self.Wp = (fp * len(self.W))(*[w.ctypes.data_as(fp) for w in self.W])
        self.bp = (fp * len(self.b))(*[x.ctypes.data_as(fp) for x in self.b])
        self.widths = np.asarray(dec.widths, dtype=np.int32)


_views = {}


def _view(dec):
    v = _views.get(id(dec))
    if v is None or v.dec is not dec:
        v = _DecoderView(dec)
        _views[id(dec)] = v
    return v


# ----------------------------------------------------------------- decoder --

def act_jet(act, x8):
    """Activation applied to one 8-component hyper-dual jet."""
    x8 = np.ascontiguousarray(x8, dtype=np.float64)
    out = np.zeros(8)
    lib().orc_act_jet(ACT[act], _dp(x8), _dp(out))
    return out


def decoder_jets(dec, q, s1=None, s2=None, s3=None, rows=None, n_run=None):
    """Jets of D(q + e1 s1 + e2 s2 + e3 s3).

    s1, s2, s3: None, (r,) or (n_seed, r) seed directions.  Returns an array of
    shape (n_seed, n_rows, 8) with components [u, D[s1], D[s2], D2[s1,s2], D[s3],
    D2[s1,s3], D2[s2,s3], D3[s1,s2,s3]] (or the hidden activations after
    ``n_run`` layers when n_run < number of layers).
    """
    v = _view(dec)
    L = len(dec.W)
    r = dec.r
    n_run = L if n_run is None else n_run
    seeds = [s for s in (s1, s2, s3) if s is not None]
    n_seed = max([np.atleast_2d(s).shape[0] for s in seeds], default=1)

    def prep(s):
        if s is None:
            return None
        s = np.atleast_2d(np.asarray(s, dtype=np.float64))
        if s.shape[0] == 1 and n_seed > 1:
            s = np.repeat(s, n_seed, 0)
        assert s.shape == (n_seed, r)
        return np.ascontiguousarray(s)

    S1, S2, S3 = prep(s1), prep(s2), prep(s3)
    q = np.ascontiguousarray(q, dtype=np.float64)
    if n_run == L and rows is not None:
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        n_rows = rows.size
        rp = _ip(rows)
    else:
        rows = None
        n_rows = dec.widths[n_run]
        rp = None
    out = np.zeros((n_seed, n_rows, 8))
    nul = ctypes.POINTER(ctypes.c_double)()
    st = lib().orc_decoder_jets(L, _ip(v.widths), v.Wp, v.bp, ACT[dec.act], n_run, _dp(q),
                                n_seed, _dp(S1) if S1 is not None else nul,
                                _dp(S2) if S2 is not None else nul,
                                _dp(S3) if S3 is not None else nul, n_rows, rp, _dp(out))
    if st != 0:
        raise RuntimeError("orc_decoder_jets failed: %d" % st)
    return out


def decode(dec, q, rows=None):
    """u = D(q) (FP64)."""
    return decoder_jets(dec, q, rows=rows)[0, :, 0]


def derivs(dec, q, qbar, qbar_dot, dt, rows=None):
    """All first-, second- and third-order quantities of the decoder at q.

    Returns dict with u (N), J (N,r), HDe (N,r) = H[Delta, e_j], Hw (N,r) = H[w, e_j],
    Sdd (N,r) = S[e_j, Delta, Delta], dJ = Sdd + Hw (Eq. 12), HDD (N) = H[Delta,Delta],
    Hqq (N) = H[qdot,qdot] with qdot = Delta/dt.
    """
    r = dec.r
    q = np.asarray(q, np.float64)
    D = q - qbar
    w = 3.0 * D - dt * qbar_dot
    E = np.eye(r)
    # job j: seeds (e_j, Delta, Delta) -> [1]=J e_j, [3]=H[e_j,D], [6]=H[D,D], [7]=S[e_j,D,D]
    j1 = decoder_jets(dec, q, E, D, D, rows=rows)
    # job j: seeds (e_j, w) -> [3]=H[e_j,w]
    j2 = decoder_jets(dec, q, E, w, None, rows=rows)
    u = j1[0, :, 0]
    J = j1[:, :, 1].T.copy()
    HDe = j1[:, :, 3].T.copy()
    Sdd = j1[:, :, 7].T.copy()
    Hw = j2[:, :, 3].T.copy()
    HDD = j1[0, :, 6].copy()
    return dict(u=u, J=J, HDe=HDe, Hw=Hw, Sdd=Sdd, dJ=Sdd + Hw, HDD=HDD, Hqq=HDD / dt ** 2)


def _act_d2(act, z):
    """act(z), act'(z), act''(z) by their plain definitions (FP64)."""
    if act == "tanh":
        t = np.tanh(z)
        s1 = 1.0 - t * t
        return t, s1, -2.0 * t * s1
    if act == "sin":
        return np.sin(z), np.cos(z), -np.sin(z)
    return z, np.ones_like(z), np.zeros_like(z)


def decoder_uJ_vjp(dec, Q, gu, gJ):
    """Gradient of the scalar

        L = sum_s [ gu_s . u(q_s) + sum_j gJ_s[:, j] . J(q_s) e_j ]

    with respect to every latent q_s and every decoder weight W_l and bias b_l, in
    FP64.  u = D(q) and J = dD/dq are formed by first-order forward differentiation
    (a value and r tangents per layer, Sec. 3.5's MLP); the gradient is the reverse
    sweep of the chain rule through that computation (the backpropagation Sec. 4.4
    builds on).  Per layer z = W x + b, zt_j = W xt_j, and for hidden layers
    a = act(z), at_j = act'(z) zt_j; the reverse of the activation is
        gz = act'(z) ga + act''(z) sum_j zt_j gat_j,   gzt_j = act'(z) gat_j.

    Q (B, r), gu (B, N), gJ (B, N, r).  Returns gq (B, r), gW (list of (n_out, n_in)),
    gb (list of (n_out,)).
    """
    W = [np.asarray(w, np.float64) for w in dec.W]
    bb = [np.asarray(x, np.float64) for x in dec.b]
    L = len(W)
    Q = np.atleast_2d(np.asarray(Q, np.float64))
    B, r = Q.shape
    gu = np.asarray(gu, np.float64).reshape(B, -1)
    gJ = np.asarray(gJ, np.float64).reshape(B, -1, r)
    xs, xts, zs, zts = [], [], [], []
    x = Q.copy()
    xt = np.repeat(np.eye(r)[None], B, 0)          # (B, r, n): tangent j of sample s
    for l in range(L):
        xs.append(x)
        xts.append(xt)
        z = x @ W[l].T + bb[l]
        zt = xt @ W[l].T
        zs.append(z)
        zts.append(zt)
        if l < L - 1:
            a, s1, _ = _act_d2(dec.act, z)
            x = a
            xt = s1[:, None, :] * zt
    gz = gu.copy()
    gzt = np.transpose(gJ, (0, 2, 1)).copy()       # (B, r, N)
    gW, gb = [None] * L, [None] * L
    gq = None
    for l in range(L - 1, -1, -1):
        gW[l] = gz.T @ xs[l] + np.einsum("bjo,bji->oi", gzt, xts[l])
        gb[l] = gz.sum(0)
        gx = gz @ W[l]
        gxt = gzt @ W[l]
        if l > 0:
            _, s1, s2 = _act_d2(dec.act, zs[l - 1])
            gz = s1 * gx + s2 * np.einsum("bjn,bjn->bn", zts[l - 1], gxt)
            gzt = s1[:, None, :] * gxt
        else:
            gq = gx
    return gq, gW, gb


def aTH(dec, q, a):
    """(a^T H)[i,j] = sum_n a_n H[n,i,j]: the plain definition, one second-order
    jet per pair (i <= j) over all N outputs."""
    r = dec.r
    E = np.eye(r)
    I, Jx = np.triu_indices(r)
    jets = decoder_jets(dec, q, E[I], E[Jx])          # (npairs, N, 8)
    vals = jets[:, :, 3] @ np.asarray(a, np.float64)
    out = np.zeros((r, r))
    out[I, Jx] = vals
    out[Jx, I] = vals
    return out


def aTH_regrouped(dec, q, a):
    """Same contraction for large decoders: with a linear output layer,
    sum_n a_n H[n,i,j] = (W_L^T a) . d2h_{L-1}[e_i,e_j] where h_{L-1} is the last
    hidden activation (associativity of the output layer's sum).  Pinned against
    ``aTH`` in the tests."""
    r = dec.r
    L = len(dec.W)
    E = np.eye(r)
    I, Jx = np.triu_indices(r)
    v = dec.W[L - 1].astype(np.float64).T @ np.asarray(a, np.float64)
    jets = decoder_jets(dec, q, E[I], E[Jx], n_run=L - 1)   # (npairs, K, 8)
    vals = jets[:, :, 3] @ v
    out = np.zeros((r, r))
    out[I, Jx] = vals
    out[Jx, I] = vals
    return out


# -------------------------------------------------------------------- FEM --

def wnet_weights(wnet, dec, q, tet_ids=None):
    """Cubature weights predicted by the weight network W (Sec. 5, "Weight Prediction"):
    the latent is decoded to the full displacement u = D(q), then the four FC layers of
    W follow, sin after each of the first three and a square after the last (the
    non-negativity constraint).  Returns w_e for the elements tet_ids (all when None).
    The plain definition: every layer applies to the previous layer's full output."""
    h = decode(dec, q)
    L = len(wnet.W)
    for l in range(L):
        z = np.asarray(wnet.W[l], np.float64) @ h + np.asarray(wnet.b[l], np.float64)
        h = np.sin(z) if l < L - 1 else z * z
    return h if tet_ids is None else h[np.asarray(tet_ids)]


def lame(E, nu):
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def tets_fk(mesh, u, tet_ids, want_K=True):
    """Energy, force and stiffness of the listed tets at displacement u (FP64)."""
    tet_ids = np.asarray(tet_ids, dtype=np.int64)
    n = tet_ids.size
    T = mesh.tets[tet_ids]                                # (n,4)
    X = mesh.X[T].reshape(n, 12)
    x = X + np.asarray(u, np.float64).reshape(-1, 3)[T].reshape(n, 12)
    X = np.ascontiguousarray(X)
    x = np.ascontiguousarray(x)
    mu, lam = lame(mesh.E, mesh.nu)
    en = np.zeros(n)
    f = np.zeros((n, 12))
    K = np.zeros((n, 144)) if want_K else None
    st = np.zeros(n, dtype=np.int32)
    lib().orc_tets_fk(n, _dp(X), _dp(x), MAT[mesh.material], mu, lam, _dp(en), _dp(f),
                      _dp(K) if want_K else ctypes.POINTER(ctypes.c_double)(), _ip(st))
    return en, f, (K.reshape(n, 12, 12) if want_K else None), st


def tet_dofs(mesh, tet_ids):
    T = mesh.tets[np.asarray(tet_ids, dtype=np.int64)]
    return (3 * T[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 12)


def mass_diag(mesh):
    return np.repeat(mesh.vmass, 3)


# --------------------------------------------------------- reduced system --

class Inverted(RuntimeError):
    pass


def reduced_system(wl, q, qbar=None, qbar_dot=None, dt=None, cub_w=None, aH="auto"):
    """phi (r), A (r x r), elastic cubature energy and intermediates at q.

    Follows Eq. 7/8 (phi, multiplied through by dt^2 as in Eq. 10) and Eq. 11
    with n_p = 0 (A), Eq. 12 (dJ), and the cubature sums of Sec. 5.
    """
    dec, mesh = wl.dec, wl.mesh
    st = wl.state
    qbar = st.qbar if qbar is None else qbar
    qbar_dot = st.qbar_dot if qbar_dot is None else qbar_dot
    dt = st.dt if dt is None else dt
    cw = np.asarray(wl.cub_w if cub_w is None else cub_w, np.float64)
    q = np.asarray(q, np.float64)
    D = q - qbar
    z = D - dt * qbar_dot
    d = derivs(dec, q, qbar, qbar_dot, dt)
    J, HDD, dJ, u = d["J"], d["HDD"], d["dJ"], d["u"]
    Mdiag = mass_diag(mesh)
    fext = np.asarray(wl.f_ext, np.float64)
    # cubature: f_e, K_e at the deformed cubature tets
    en, fe, Ke, stat = tets_fk(mesh, u, wl.cub_tets)
    if np.any(stat == -7):
        raise Inverted("inverted cubature tet")
    dofs = tet_dofs(mesh, wl.cub_tets)                    # (C,12)
    fC = np.zeros(dec.n_out)
    np.add.at(fC, dofs.reshape(-1), (cw[:, None] * fe).reshape(-1))
    Je = J[dofs]                                          # (C,12,r)
    Kr = np.einsum("e,eai,eab,ebj->ij", cw, Je, Ke, Je)
    energy = float(np.sum(cw * en))
    y = J @ z + HDD
    phi = J.T @ (Mdiag * y) + dt ** 2 * (J.T @ fC - J.T @ fext)
    a = Mdiag * y + dt ** 2 * (fC - fext)
    if aH == "auto":
        aH = "plain" if dec.n_params < 20_000_000 else "regrouped"
    aHm = aTH(dec, q, a) if aH == "plain" else aTH_regrouped(dec, q, a)
    Mr = J.T @ (Mdiag[:, None] * J)
    B = J.T @ (Mdiag[:, None] * dJ)
    A = aHm + Mr + B + dt ** 2 * Kr
    return dict(phi=phi, A=A, energy=energy, a=a, aH=aHm, Mr=Mr, B=B, Kr=Kr, fC=fC,
                g_int=J.T @ fC, **d)


def phi_only(wl, q, qbar=None, qbar_dot=None, dt=None, cub_w=None):
    """phi alone (no second-order terms beyond H[Delta,Delta]); used by the
    line search and by the finite-difference pin of A."""
    dec, mesh = wl.dec, wl.mesh
    st = wl.state
    qbar = st.qbar if qbar is None else qbar
    qbar_dot = st.qbar_dot if qbar_dot is None else qbar_dot
    dt = st.dt if dt is None else dt
    cw = np.asarray(wl.cub_w if cub_w is None else cub_w, np.float64)
    q = np.asarray(q, np.float64)
    D = q - qbar
    z = D - dt * qbar_dot
    r = dec.r
    j1 = decoder_jets(dec, q, np.eye(r), D, D)
    u = j1[0, :, 0]
    J = j1[:, :, 1].T
    HDD = j1[0, :, 6]
    en, fe, _, stat = tets_fk(mesh, u, wl.cub_tets, want_K=False)
    if np.any(stat == -7):
        raise Inverted("inverted cubature tet")
    dofs = tet_dofs(mesh, wl.cub_tets)
    fC = np.zeros(dec.n_out)
    np.add.at(fC, dofs.reshape(-1), (cw[:, None] * fe).reshape(-1))
    Mdiag = mass_diag(mesh)
    y = J @ z + HDD
    fext = np.asarray(wl.f_ext, np.float64)
    return J.T @ (Mdiag * y) + dt ** 2 * (J.T @ fC - J.T @ fext)


def _split(U, r):
    U = np.asarray(U, np.float64)
    n_p = U.shape[1]
    r = np.asarray(r, np.float64)
    return U, n_p, r[:n_p], r[n_p:]


def linear_subspace_system(wl, U, r, rbar, rbar_dot, dt=None, cub_w=None, want_A=True):
    """phi and A of the combined linear + nonlinear subspace (Sec. 3.4, Eqs. 9-11):
    u = U p + Dt(q) with the filtered decoder Dt = (I - U U^T) D (the filtering layer),
    generalized coordinate r = [p; q], Jt = [U, (I - U U^T) J] (N x (n_p + n_q)),
    Ht = diag(0, (I - U U^T) H).  With Delta = r - rbar, z = Delta - dt rbar_dot,
      y   = U z_p + Jt_q z_q + Ht[Delta_q, Delta_q]
      phi = Jt^T M y + dt^2 Jt^T (f_C - f_ext)
      A   = Jt^T M [U, Jt_q + dJt] + diag(0, a^T Ht_q) + dt^2 Jt^T K Jt,
      a   = M y + dt^2 (f_C - f_ext),
    dJt the filtered Eq. 12 term of the decoder.  Plain N-row definitions, FP64."""
    dec, mesh = wl.dec, wl.mesh
    dt = wl.state.dt if dt is None else dt
    cw = np.asarray(wl.cub_w if cub_w is None else cub_w, np.float64)
    U, n_p, p, q = _split(U, r)
    _, _, pbar, qbar = _split(U, rbar)
    _, _, pdot, qdot = _split(U, rbar_dot)
    filt = lambda X: X - U @ (U.T @ X)
    d = derivs(dec, q, qbar, qbar_dot=qdot, dt=dt)
    Jq = filt(d["J"])
    HDD = filt(d["HDD"])
    dJ = filt(d["dJ"])
    u = U @ p + filt(d["u"])
    Jt = np.concatenate([U, Jq], axis=1)
    zp = (p - pbar) - dt * pdot
    zq = (q - qbar) - dt * qdot
    Mdiag = mass_diag(mesh)
    fext = np.asarray(wl.f_ext, np.float64)
    en, fe, Ke, stat = tets_fk(mesh, u, wl.cub_tets, want_K=want_A)
    if np.any(stat == -7):
        raise Inverted("inverted cubature tet")
    dofs = tet_dofs(mesh, wl.cub_tets)
    fC = np.zeros(dec.n_out)
    np.add.at(fC, dofs.reshape(-1), (cw[:, None] * fe).reshape(-1))
    y = U @ zp + Jq @ zq + HDD
    a = Mdiag * y + dt ** 2 * (fC - fext)
    phi = Jt.T @ (Mdiag * y) + dt ** 2 * (Jt.T @ fC - Jt.T @ fext)
    out = dict(phi=phi, u=u, Jt=Jt, energy=float(np.sum(cw * en)), a=a)
    if want_A:
        n = Jt.shape[1]
        Je = Jt[dofs]
        Kr = np.einsum("e,eai,eab,ebj->ij", cw, Je, Ke, Je)
        right = np.concatenate([U, Jq + dJ], axis=1)
        aH = np.zeros((n, n))
        aH[n_p:, n_p:] = aTH(dec, q, filt(a))       # a^T Ht_q = ((I - U U^T) a)^T H
        out.update(A=Jt.T @ (Mdiag[:, None] * right) + aH + dt ** 2 * Kr, Kr=Kr, aH=aH)
    return out


def newton_solve(wl, q0=None, max_iter=None, tol=1e-8, c_armijo=1e-4, max_halvings=8,
                 cub_w=None, qbar=None, qbar_dot=None, dt=None, max_step=0.5, xtol=1e-6, U=None):
    """Implicit-Euler Newton iteration on phi(q) = 0 (Eq. 7) with A from Eq. 11.

    Each iteration solves A delta = -phi (LU, partial pivoting) and backtracks
    on |phi|^2 (Armijo), starting from the step length alpha = min(1,
    max_step / |delta|_inf) (no cap when max_step is 0).  Stops when
    |phi| <= tol * max(1, |phi_0|), or when the next step is negligible,
    |delta|_inf <= xtol * max(1, |q|_inf) (q is then the solution; xtol = 0 turns
    this test off), delta either the Newton step at q or, right after a step is
    accepted, its simplified-Newton estimate -A_prev^{-1} phi(q) with the previous
    iterate's Newton matrix.  Returns (q, report dict).  With a linear basis U (N x n_p) the
    unknown is r = [p; q] and the system is linear_subspace_system (qbar, qbar_dot and
    q0 are then (n_p + n_q)-vectors).
    """
    st = wl.state
    qbar = st.qbar if qbar is None else qbar
    qbar_dot = st.qbar_dot if qbar_dot is None else qbar_dot
    dt = st.dt if dt is None else dt
    q = (qbar + dt * qbar_dot) if q0 is None else np.asarray(q0, np.float64).copy()
    max_iter = wl.max_iter if max_iter is None else max_iter

    def system(x):
        if U is None:
            return reduced_system(wl, x, qbar=qbar, qbar_dot=qbar_dot, dt=dt, cub_w=cub_w)
        return linear_subspace_system(wl, U, x, qbar, qbar_dot, dt, cub_w)
    q, rep = newton_iterate(system, q, max_iter, tol, c_armijo, max_halvings, max_step, xtol)
    rep["qdot"] = (q - qbar) / dt
    return q, rep


def newton_iterate(system, q, max_iter, tol=1e-8, c_armijo=1e-4, max_halvings=8,
                   max_step=0.5, xtol=1e-6, estimate=True):
    """The Newton iteration of ``newton_solve`` on any system: ``system(x)`` returns a
    dict with ``phi`` and its Jacobian ``A`` at x, or raises ``Inverted`` (a trial
    point the line search then halves away from).  ``estimate``: after an accepted
    trial, stop when the simplified-Newton step with the previous Newton matrix is below
    ``xtol`` (else only the full step at the new iterate is tested).  Returns
    (q, report dict)."""
    q = np.asarray(q, np.float64).copy()
    rs = system(q)
    phi0 = np.linalg.norm(rs["phi"])
    hist = [phi0]
    # the line search's trail, for comparing control decisions: every trial as
    # (iteration, alpha, |phi(trial)|^2 / Armijo threshold, or None for an inverted
    # trial), the accepted step lengths, and the number of system evaluations
    trials, alphas, evals = [], [], 1
    nfull = 0      # iterates whose Newton matrix was used (solved with)
    it = 0
    converged = phi0 <= tol * max(1.0, phi0)
    while not converged and it < max_iter:
        delta = np.linalg.solve(rs["A"], -rs["phi"])
        nfull += 1
        m0 = float(rs["phi"] @ rs["phi"])
        dn = float(np.max(np.abs(delta)))
        if xtol > 0 and dn <= xtol * max(1.0, float(np.max(np.abs(q)))):
            converged = True
            break
        alpha = max_step / dn if (max_step > 0 and dn > max_step) else 1.0
        for _ in range(max_halvings + 1):
            qt = q + alpha * delta
            evals += 1
            try:
                rt = system(qt)
                mt = float(rt["phi"] @ rt["phi"])
                thr = (1.0 - 2.0 * c_armijo * alpha) * m0
                ok = mt <= thr
                trials.append((it, alpha, mt / thr if thr > 0 else np.inf))
            except Inverted:
                ok = False
                trials.append((it, alpha, None))
            if ok:
                break
            alpha *= 0.5
        else:
            break
        A_prev = rs["A"]
        q, rs = qt, rt
        it += 1
        alphas.append(alpha)
        hist.append(float(np.linalg.norm(rs["phi"])))
        converged = hist[-1] <= tol * max(1.0, phi0)
        if estimate and not converged and it < max_iter and xtol > 0:
            # simplified-Newton estimate of the next step with the previous Newton matrix:
            # when it is negligible the iterate is the solution (no new A is needed)
            est = np.linalg.solve(A_prev, -rs["phi"])
            if float(np.max(np.abs(est))) <= xtol * max(1.0, float(np.max(np.abs(q)))):
                converged = True
    return q, dict(iters=it, converged=bool(converged), phi_hist=hist, final=rs,
                   trials=trials, alphas=alphas, evals=evals, nfull=nfull)


# --------------------------------------------------- coupled substructures --

def _v3(i):
    return slice(3 * int(i), 3 * int(i) + 3)


def coupling_energy(cm, us):
    """Ties between substructures (deformation substructuring, Sec. 6), read as
    penalty springs of stiffness k_c: every interface pair (d, i, e, j) coincides at
    rest and every anchor (d, i) holds its vertex at rest, so with displacements u_d
      E_c = k_c/2 (sum_pairs |u_d[i] - u_e[j]|^2 + sum_anchors |u_d[i]|^2).
    Returns E_c and the per-domain gradients g_d = dE_c/du_d (N_d each)."""
    k = float(cm.k_c)
    g = [np.zeros(np.asarray(u).size) for u in us]
    E = 0.0
    for d, i, e, j in cm.pairs:
        s = us[d][_v3(i)] - us[e][_v3(j)]
        E += 0.5 * k * float(s @ s)
        g[d][_v3(i)] += k * s
        g[e][_v3(j)] -= k * s
    for d, i in cm.anchors:
        s = us[d][_v3(i)]
        E += 0.5 * k * float(s @ s)
        g[d][_v3(i)] += k * s
    return E, g


def _offsets(cm):
    return np.concatenate([[0], np.cumsum([wl.dec.r for wl in cm.domains])]).astype(int)


def coupled_system(cm, Q, Qbar, Qdot, dt=None, cub_w=None):
    """phi and A of one implicit-Euler step of the coupled domains, unknown the stacked
    latents Q = [q_1; ...; q_D].  Domain d's rows are its own Eq. 10 residual with the
    tie force -g_d among its forces (g_d joins f_C in phi and in a, hence in a^T H), and
    with the Hessian of E_c (k_c [[I, -I], [-I, I]] per pair, k_c I per anchor):
      A_dd = A_d(with g_d) + dt^2 k_c (sum_{pairs at d} J_d[i]^T J_d[i]
                                       + sum_{anchors at d} J_d[i]^T J_d[i]),
      A_de = -dt^2 k_c sum_{pairs (d,i,e,j)} J_d[i]^T J_e[j],
    J_d[i] the 3 rows of J_d at vertex i.  ``cub_w`` is one weight array per domain."""
    off = _offsets(cm)
    dt = cm.domains[0].state.dt if dt is None else dt
    Q, Qbar, Qdot = (np.asarray(x, np.float64) for x in (Q, Qbar, Qdot))
    sl = [slice(off[d], off[d + 1]) for d in range(len(cm.domains))]
    us = [decode(wl.dec, Q[sl[d]]) for d, wl in enumerate(cm.domains)]
    Ec, g = coupling_energy(cm, us)
    n = off[-1]
    phi = np.zeros(n)
    A = np.zeros((n, n))
    Js = []
    energy = Ec
    for d, wl in enumerate(cm.domains):
        tied = dataclasses.replace(wl, f_ext=np.asarray(wl.f_ext, np.float64) - g[d])
        rs = reduced_system(tied, Q[sl[d]], qbar=Qbar[sl[d]], qbar_dot=Qdot[sl[d]], dt=dt,
                            cub_w=None if cub_w is None else cub_w[d])
        phi[sl[d]] = rs["phi"]
        A[sl[d], sl[d]] = rs["A"]
        Js.append(rs["J"])
        energy += rs["energy"]
    c = dt * dt * float(cm.k_c)
    for d, i, e, j in cm.pairs:
        Ji, Jj = Js[d][_v3(i)], Js[e][_v3(j)]
        A[sl[d], sl[d]] += c * Ji.T @ Ji
        A[sl[e], sl[e]] += c * Jj.T @ Jj
        A[sl[d], sl[e]] -= c * Ji.T @ Jj
        A[sl[e], sl[d]] -= c * Jj.T @ Ji
    for d, i in cm.anchors:
        Ji = Js[d][_v3(i)]
        A[sl[d], sl[d]] += c * Ji.T @ Ji
    return dict(phi=phi, A=A, energy=energy, coupling_energy=Ec, u=us, g=g, J=Js)


def coupled_newton_solve(cm, Q0=None, Qbar=None, Qdot=None, dt=None, max_iter=None,
                         cub_w=None, **kw):
    """The Newton iteration of ``newton_solve`` on the coupled system (one global LU
    solve per iteration over all domains' latents; every accepted unconverged iterate
    forms the global Newton matrix, with no simplified-Newton stop).  Defaults: Qbar,
    Qdot stacked from the domains' states, Q0 = Qbar + dt Qdot."""
    dt = cm.domains[0].state.dt if dt is None else dt
    Qbar = np.concatenate([wl.state.qbar for wl in cm.domains]) if Qbar is None else Qbar
    Qdot = np.concatenate([wl.state.qbar_dot for wl in cm.domains]) if Qdot is None else Qdot
    Q0 = Qbar + dt * Qdot if Q0 is None else Q0
    max_iter = cm.domains[0].max_iter if max_iter is None else max_iter
    kw.setdefault("estimate", False)
    Q, rep = newton_iterate(lambda x: coupled_system(cm, x, Qbar, Qdot, dt, cub_w), Q0,
                            max_iter, **kw)
    rep["qdot"] = (Q - Qbar) / dt
    return Q, rep
