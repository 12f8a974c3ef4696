"""Helpers for the GPU parity tests: upload a synthetic workload through the C ABI
and compare against the FP64 oracle."""
import numpy as np

import oracle
from paper_2102_11026_gb300 import dae

# Tolerances (normwise relative error against the FP64 oracle)
TOL_FP32_FIRST = 1e-5      # u, J on the FP32 path
TOL_FP32_HIGHER = 1e-4     # second/third-order terms, phi, A
TOL_BF16X3_J = 1e-4        # J on the split-BF16 path


def relerr(x, ref):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.linalg.norm(ref)
    return np.linalg.norm(x - ref) / (den if den > 0 else 1.0)


def colerr(x, ref):
    """Largest per-column element error relative to that column's scale:
    max_j max_i |x[i, j] - ref[i, j]| / max_i |ref[i, j]| (a vector is one column).
    Unlike ``relerr`` it cannot dilute one wrong tile, row block or column of J in
    the rest of the output; columns of exact zeros must come out exactly zero."""
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    if ref.ndim == 1:
        x, ref = x[:, None], ref[:, None]
    err = np.abs(x - ref).max(axis=0)
    scale = np.abs(ref).max(axis=0)
    out = np.where(scale > 0, err / np.where(scale > 0, scale, 1.0), np.where(err > 0, np.inf, 0.0))
    return float(out.max())


class Gpu:
    def __init__(self, wl, prec="fp32", ctx=None):
        self.wl = wl
        self.ctx = ctx or dae.dae_create(0)
        self.own_ctx = ctx is None
        d = wl.dec
        self.dec = dae.dae_load_decoder(self.ctx, d.widths, d.W, d.b, d.act, prec)
        m = wl.mesh
        self.mesh = dae.dae_load_mesh(self.ctx, m.X.reshape(-1), m.tets.reshape(-1), m.vmass,
                                      m.material, m.E, m.nu)

    def close(self):
        dae.dae_free_decoder(self.dec)
        dae.dae_free_mesh(self.mesh)
        if self.own_ctx:
            dae.dae_destroy(self.ctx)

    def derivs(self, q, want=("u", "J", "Hqq", "dJ")):
        wl = self.wl
        N, r = wl.dec.n_out, wl.dec.r
        out = {}
        shapes = {"u": (N,), "J": (r, N), "Hqq": (N,), "dJ": (r, N), "Hw": (r, N), "Sdd": (r, N)}
        for k in want:
            out[k] = np.zeros(shapes[k], np.float32)
        dae.dae_eval_derivs(self.ctx, self.dec, np.asarray(q, np.float64), wl.state.qbar,
                            wl.state.qbar_dot, wl.state.dt, **{k: out[k] for k in want})
        for k in ("J", "dJ", "Hw", "Sdd"):
            if k in out:
                out[k] = out[k].T          # column-major N x r -> (N, r)
        return out

    def reduced(self, q, cub_w=None, f_ext="wl"):
        wl = self.wl
        r = wl.dec.r
        phi = np.zeros(r)
        A = np.zeros(r * r)
        en = np.zeros(1)
        terms = np.zeros(4 * r * r + r)
        fe = wl.f_ext if isinstance(f_ext, str) else f_ext
        cw = wl.cub_w if cub_w is None else cub_w
        dae.dae_assemble_reduced(self.ctx, self.dec, self.mesh, wl.cub_tets, cw,
                                 np.asarray(q, np.float64), wl.state.qbar, wl.state.qbar_dot,
                                 wl.state.dt, fe, phi, A, en, terms)
        rr = r * r
        T = dict(aH=terms[:rr].reshape(r, r).T, Mr=terms[rr:2 * rr].reshape(r, r).T,
                 B=terms[2 * rr:3 * rr].reshape(r, r).T, Kr=terms[3 * rr:4 * rr].reshape(r, r).T,
                 g_int=terms[4 * rr:])
        return dict(phi=phi, A=A.reshape(r, r).T, energy=en[0], **T)

    def newton(self, q0, opts=None):
        wl = self.wl
        q = np.array(q0, np.float64)
        rep = dae.dae_newton_step(self.ctx, self.dec, self.mesh, wl.cub_tets, wl.cub_w, q,
                                  wl.state.qbar, wl.state.qbar_dot, wl.state.dt, wl.f_ext, opts)
        return q, rep
