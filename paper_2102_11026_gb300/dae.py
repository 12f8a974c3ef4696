"""ctypes binding of the C ABI in include/dae.h (argument marshalling only).

Every function has the name of its C entry point.  Arrays may be numpy arrays
(host memory) or torch tensors (host or CUDA); the library itself detects where
each pointer lives.  A missing or unbuildable ``libdae.so`` raises -- there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdae.so")
_lib = None

STATUS = {0: "DAE_OK", -1: "DAE_ERR_INVALID_ARG", -2: "DAE_ERR_CUDA", -3: "DAE_ERR_OOM",
          -4: "DAE_ERR_NOT_CONVERGED", -5: "DAE_ERR_NONFINITE", -6: "DAE_ERR_SINGULAR",
          -7: "DAE_ERR_INVERTED", -8: "DAE_ERR_TIMEOUT", -9: "DAE_ERR_UNSUPPORTED"}
ACT = {"tanh": 0, "sin": 1, "linear": 2}
PREC = {"fp32": 0, "tf32": 1, "bf16": 2, "bf16x3": 3}
MATERIAL = {"stvk": 0, "neohookean": 1}


class DaeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class dae_newton_opts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int), ("max_evals", ctypes.c_int),
                ("max_halvings", ctypes.c_int), ("tol", ctypes.c_double),
                ("c_armijo", ctypes.c_double), ("h_cs", ctypes.c_double),
                ("max_step", ctypes.c_double), ("xtol", ctypes.c_double)]


class dae_newton_report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("evals", ctypes.c_int), ("converged", ctypes.c_int),
                ("status", ctypes.c_int), ("phi_norm0", ctypes.c_double),
                ("phi_norm", ctypes.c_double), ("energy", ctypes.c_double),
                ("alpha", ctypes.c_double), ("full_evals", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double

class dae_system(ctypes.Structure):
    _fields_ = [("dec", ctypes.c_void_p), ("mesh", ctypes.c_void_p), ("n_cub", ctypes.c_int),
                ("cub_tets", ctypes.c_void_p), ("cub_w", ctypes.c_void_p),
                ("q", ctypes.c_void_p), ("qbar", ctypes.c_void_p), ("qbar_dot", ctypes.c_void_p),
                ("f_ext", ctypes.c_void_p)]


SIGNATURES = {
    "dae_version": ([], _i),
    "dae_status_string": ([_i], ctypes.c_char_p),
    "dae_create": ([ctypes.POINTER(_vp), _i, _vp], _i),
    "dae_destroy": ([_vp], _i),
    "dae_last_error": ([_vp], ctypes.c_char_p),
    "dae_sync": ([_vp], _i),
    "dae_default_newton_opts": ([ctypes.POINTER(dae_newton_opts)], None),
    "dae_load_decoder": ([_vp, _i, _vp, _vp, _vp, _i, _i, ctypes.POINTER(_vp)], _i),
    "dae_free_decoder": ([_vp], _i),
    "dae_decoder_set_precision": ([_vp, _i], _i),
    "dae_decoder_set_cs_mode": ([_vp, _i], _i),
    "dae_decoder_get_chain_plan": ([_vp, _i, _vp, _vp], _i),
    "dae_decoder_set_chain_plan": ([_vp, _i, _vp, _vp], _i),
    "dae_decoder_autotune": ([_vp, _i, _vp], _i),
    "dae_load_mesh": ([_vp, _i, _vp, _i, _vp, _vp, _i, _d, _d, ctypes.POINTER(_vp)], _i),
    "dae_free_mesh": ([_vp], _i),
    "dae_eval_derivs": ([_vp, _vp, _vp, _vp, _vp, _d, _vp, _vp, _vp, _vp, _vp, _vp], _i),
    "dae_assemble_reduced": ([_vp, _vp, _vp, _i, _vp, _vp, _vp, _vp, _vp, _d, _vp, _vp, _vp,
                              _vp, _vp], _i),
    "dae_newton_step": ([_vp, _vp, _vp, _i, _vp, _vp, _vp, _vp, _vp, _d, _vp,
                         ctypes.POINTER(dae_newton_opts), ctypes.POINTER(dae_newton_report)], _i),
    "dae_last_report": ([_vp, ctypes.POINTER(dae_newton_report)], _i),
    "dae_decoder_attach_wnet": ([_vp, _vp, _vp, _vp], _i),
    "dae_decoder_attach_linear": ([_vp, _i, _vp], _i),
    "dae_predict_weights": ([_vp, _vp, _vp, _i, _vp, _vp], _i),
    "dae_newton_step_batched": ([_vp, _i, ctypes.POINTER(dae_system), _d,
                                 ctypes.POINTER(dae_newton_opts), ctypes.POINTER(dae_newton_report)], _i),
    "dae_newton_step_coupled": ([_vp, _i, ctypes.POINTER(dae_system), _i, _vp, _i, _vp, _d, _d,
                                 ctypes.POINTER(dae_newton_opts), ctypes.POINTER(dae_newton_report)], _i),
    "dae_reduce_rows_noalloc": ([_i, _i, _vp, _vp, _vp, _vp, _vp, _vp, _d, _vp, _vp, _vp, _vp], _i),
    "dae_profile_enable": ([_vp, ctypes.c_uint], _i),
    "dae_profile_read": ([_vp, _vp, _vp], _i),
    "dae_launch_count": ([_vp], ctypes.c_longlong),
    "dae_selftest_bounded_waits": ([_vp], _i),
    "dae_trainer_create": ([_vp, _i, _vp, _i, _i, ctypes.POINTER(_vp)], _i),
    "dae_trainer_free": ([_vp], _i),
    "dae_trainer_set_precision": ([_vp, _i], _i),
    "dae_train_forward": ([_vp, _vp, _vp, _i, _vp, _vp], _i),
    "dae_train_backward": ([_vp, _vp, _vp, _i, _vp, _vp, _vp, _vp, _vp], _i),
    "dae_rollout": ([_vp, _vp, _vp, _i, _vp, _vp, _i, _vp, _vp, _d, _vp,
                     ctypes.POINTER(dae_newton_opts), _vp, ctypes.POINTER(dae_newton_report)], _i),
}


def lib():
    """Load libdae.so (building it first if the sources are newer)."""
    global _lib
    if _lib is None:
        from . import build as _build
        if not _build.up_to_date():
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library %s is missing; run paper_2102_11026_gb300.build" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


# ------------------------------------------------------------- marshalling --
_DT = {np.float64: "float64", np.float32: "float32", np.int32: "int32"}


def _ptr(x, dtype=None, n=None):
    """Raw pointer of a contiguous numpy array / torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):          # torch tensor
        if dtype is not None and str(x.dtype).split(".")[-1] != _DT[dtype]:
            raise TypeError("expected %s tensor, got %s" % (_DT[dtype], x.dtype))
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if n is not None and x.numel() < n:
            raise ValueError("tensor has %d elements, need %d" % (x.numel(), n))
        return x.data_ptr()
    a = x
    if dtype is not None and a.dtype != dtype:
        raise TypeError("expected %s array, got %s" % (np.dtype(dtype), a.dtype))
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    if n is not None and a.size < n:
        raise ValueError("array has %d elements, need %d" % (a.size, n))
    return a.ctypes.data


def _check(ctx, st):
    if st != 0:
        msg = lib().dae_last_error(ctx).decode() if ctx else ""
        raise DaeError(st, msg)


def dae_version():
    return lib().dae_version()


def dae_status_string(st):
    return lib().dae_status_string(st).decode()


def dae_create(device=0, stream=None):
    h = _vp()
    st = lib().dae_create(ctypes.byref(h), device, stream)
    if st != 0:
        raise DaeError(st, "dae_create failed")
    return h.value


def dae_destroy(ctx):
    _check(None, lib().dae_destroy(ctx))


def dae_last_error(ctx):
    return lib().dae_last_error(ctx).decode()


def dae_sync(ctx):
    _check(ctx, lib().dae_sync(ctx))


def dae_default_newton_opts():
    o = dae_newton_opts()
    lib().dae_default_newton_opts(ctypes.byref(o))
    return o


def dae_load_decoder(ctx, widths, W, b, act="tanh", prec="fp32"):
    """W[l]: (widths[l+1], widths[l]) float32, b[l]: (widths[l+1],) float32."""
    L = len(widths) - 1
    assert len(W) == L and len(b) == L
    w = (ctypes.c_int * (L + 1))(*widths)
    for l in range(L):
        if tuple(W[l].shape) != (widths[l + 1], widths[l]):
            raise ValueError("W[%d] has shape %s" % (l, tuple(W[l].shape)))
    Wp = (_vp * L)(*[_ptr(W[l], np.float32) for l in range(L)])
    bp = (_vp * L)(*[_ptr(b[l], np.float32, widths[l + 1]) for l in range(L)])
    h = _vp()
    _check(ctx, lib().dae_load_decoder(ctx, L, ctypes.cast(w, _vp), ctypes.cast(Wp, _vp),
                                       ctypes.cast(bp, _vp), ACT[act], PREC[prec], ctypes.byref(h)))
    return h.value


def dae_free_decoder(dec):
    _check(None, lib().dae_free_decoder(dec))


def dae_decoder_set_precision(ctx, dec, prec):
    _check(ctx, lib().dae_decoder_set_precision(dec, PREC[prec]))


def dae_decoder_set_cs_mode(ctx, dec, exact):
    """True: dae_eval_derivs evaluates the activation in exact multicomplex arithmetic
    (FP32 form only); False: the truncated shared-column form."""
    _check(ctx, lib().dae_decoder_set_cs_mode(dec, 1 if exact else 0))


def dae_decoder_get_chain_plan(ctx, dec, n_hidden, direction):
    """(split, rep) int arrays of the hidden layers for direction 0 (forward) or 1 (reverse)."""
    split = np.zeros(n_hidden, np.int32)
    rep = np.zeros(n_hidden, np.int32)
    _check(ctx, lib().dae_decoder_get_chain_plan(dec, int(direction), split.ctypes.data,
                                                 rep.ctypes.data))
    return split, rep


def dae_decoder_set_chain_plan(ctx, dec, direction, split=None, rep=None):
    """Set a direction's plan (None: the built-in plan)."""
    if split is None or rep is None:
        _check(ctx, lib().dae_decoder_set_chain_plan(dec, int(direction), None, None))
        return
    split = np.ascontiguousarray(split, np.int32)
    rep = np.ascontiguousarray(rep, np.int32)
    _check(ctx, lib().dae_decoder_set_chain_plan(dec, int(direction), split.ctypes.data,
                                                 rep.ctypes.data))


def dae_decoder_autotune(ctx, dec, reps=20):
    """Tune both chains' plans; returns (fwd ms before, after, rev ms before, after)."""
    ms = np.zeros(4)
    _check(ctx, lib().dae_decoder_autotune(dec, int(reps), ms.ctypes.data))
    return tuple(float(x) for x in ms)


def dae_load_mesh(ctx, X, tets, vmass, material="stvk", E=1e5, nu=0.4):
    X = np.ascontiguousarray(X, dtype=np.float64) if isinstance(X, np.ndarray) else X
    tets = np.ascontiguousarray(tets, dtype=np.int32) if isinstance(tets, np.ndarray) else tets
    vmass = np.ascontiguousarray(vmass, dtype=np.float64) if isinstance(vmass, np.ndarray) else vmass
    nv = vmass.shape[0]
    nt = (tets.numel() if hasattr(tets, "numel") else tets.size) // 4
    h = _vp()
    _check(ctx, lib().dae_load_mesh(ctx, nv, _ptr(X, np.float64, 3 * nv), nt,
                                    _ptr(tets, np.int32, 4 * nt), _ptr(vmass, np.float64, nv),
                                    MATERIAL[material], float(E), float(nu), ctypes.byref(h)))
    return h.value


def dae_free_mesh(mesh):
    _check(None, lib().dae_free_mesh(mesh))


def dae_eval_derivs(ctx, dec, q, qbar, qbar_dot, dt, u=None, J=None, Hqq=None, dJ=None,
                    Hw=None, Sdd=None):
    _check(ctx, lib().dae_eval_derivs(
        ctx, dec, _ptr(q, np.float64), _ptr(qbar, np.float64), _ptr(qbar_dot, np.float64),
        float(dt), _ptr(u, np.float32), _ptr(J, np.float32), _ptr(Hqq, np.float32),
        _ptr(dJ, np.float32), _ptr(Hw, np.float32), _ptr(Sdd, np.float32)))


def dae_assemble_reduced(ctx, dec, mesh, cub_tets, cub_w, q, qbar, qbar_dot, dt, f_ext=None,
                         phi=None, A=None, energy=None, terms=None):
    n = int(cub_tets.shape[0]) if cub_tets is not None else 0
    _check(ctx, lib().dae_assemble_reduced(
        ctx, dec, mesh, n, _ptr(cub_tets, np.int32), _ptr(cub_w, np.float32),
        _ptr(q, np.float64), _ptr(qbar, np.float64), _ptr(qbar_dot, np.float64), float(dt),
        _ptr(f_ext, np.float32), _ptr(phi, np.float64), _ptr(A, np.float64),
        _ptr(energy, np.float64), _ptr(terms, np.float64)))


def dae_newton_step(ctx, dec, mesh, cub_tets, cub_w, q, qbar, qbar_dot, dt, f_ext=None,
                    opts=None, want_report=True):
    n = int(cub_tets.shape[0]) if cub_tets is not None else 0
    rep = dae_newton_report() if want_report else None
    _check(ctx, lib().dae_newton_step(
        ctx, dec, mesh, n, _ptr(cub_tets, np.int32), _ptr(cub_w, np.float32),
        _ptr(q, np.float64), _ptr(qbar, np.float64), _ptr(qbar_dot, np.float64), float(dt),
        _ptr(f_ext, np.float32), ctypes.byref(opts) if opts is not None else None,
        ctypes.byref(rep) if rep is not None else None))
    return rep


def dae_newton_step_batched(ctx, systems, dt, opts=None, want_reports=True):
    """systems: list of dicts with keys dec, mesh, cub_tets, cub_w, q, qbar, qbar_dot and
    optionally f_ext (arrays as for dae_newton_step; q is updated in place)."""
    n = len(systems)
    arr = (dae_system * max(n, 1))()
    for i, y in enumerate(systems):
        ct = y.get("cub_tets")
        nc = int(ct.shape[0]) if ct is not None else 0
        arr[i] = dae_system(y["dec"], y["mesh"], nc, _ptr(ct, np.int32),
                            _ptr(y.get("cub_w"), np.float32, nc), _ptr(y["q"], np.float64),
                            _ptr(y["qbar"], np.float64), _ptr(y["qbar_dot"], np.float64),
                            _ptr(y.get("f_ext"), np.float32))
    reps = (dae_newton_report * max(n, 1))() if want_reports else None
    _check(ctx, lib().dae_newton_step_batched(
        ctx, n, arr, float(dt), ctypes.byref(opts) if opts is not None else None,
        ctypes.cast(reps, ctypes.POINTER(dae_newton_report)) if reps is not None else None))
    return list(reps)[:n] if reps is not None else None


def _system_array(systems):
    n = len(systems)
    arr = (dae_system * max(n, 1))()
    for i, y in enumerate(systems):
        ct = y.get("cub_tets")
        nc = int(ct.shape[0]) if ct is not None else 0
        arr[i] = dae_system(y["dec"], y["mesh"], nc, _ptr(ct, np.int32),
                            _ptr(y.get("cub_w"), np.float32, nc), _ptr(y["q"], np.float64),
                            _ptr(y["qbar"], np.float64), _ptr(y["qbar_dot"], np.float64),
                            _ptr(y.get("f_ext"), np.float32))
    return arr


def dae_newton_step_coupled(ctx, systems, pairs, anchors, k_c, dt, opts=None):
    """Coupled step of the systems (dicts as for dae_newton_step_batched) tied by pairs
    ((P, 4) ints d, i, e, j) and anchors ((Q, 2) ints d, i) of stiffness k_c; q is updated
    in place; returns the step's report."""
    arr = _system_array(systems)
    pr = np.ascontiguousarray(np.asarray(pairs, np.int32).reshape(-1, 4))
    an = np.ascontiguousarray(np.asarray(anchors, np.int32).reshape(-1, 2))
    rep = dae_newton_report()
    _check(ctx, lib().dae_newton_step_coupled(
        ctx, len(systems), arr, int(pr.shape[0]), pr.ctypes.data if pr.size else None,
        int(an.shape[0]), an.ctypes.data if an.size else None, float(k_c), float(dt),
        ctypes.byref(opts) if opts is not None else None, ctypes.byref(rep)))
    return rep


def dae_decoder_attach_linear(ctx, dec, U):
    """U: (np, N) float32 rows = basis vectors (host numpy or device tensor)."""
    Uc = U if hasattr(U, "data_ptr") else np.ascontiguousarray(U, np.float32)
    n_p = int(Uc.shape[0])
    _check(ctx, lib().dae_decoder_attach_linear(dec, n_p, _ptr(Uc, np.float32)))


def dae_decoder_attach_wnet(ctx, dec, widths, W, b):
    """W, b: lists of 4 row-major float32 arrays (host numpy or device tensors)."""
    wa = (ctypes.c_int * 5)(*[int(x) for x in widths])
    Ws = [np.ascontiguousarray(w, np.float32) if not hasattr(w, "data_ptr") else w for w in W]
    bs = [np.ascontiguousarray(x, np.float32) if not hasattr(x, "data_ptr") else x for x in b]
    Wp = (ctypes.c_void_p * 4)(*[_ptr(w, np.float32) for w in Ws])
    bp = (ctypes.c_void_p * 4)(*[_ptr(x, np.float32) for x in bs])
    _check(ctx, lib().dae_decoder_attach_wnet(dec, wa, Wp, bp))


def dae_predict_weights(ctx, dec, q, tet_ids, w=None):
    n = int(tet_ids.shape[0])
    out = np.zeros(n, np.float32) if w is None else w
    _check(ctx, lib().dae_predict_weights(ctx, dec, _ptr(q, np.float64), n, _ptr(tet_ids, np.int32),
                                          _ptr(out, np.float32, n)))
    return out


def dae_last_report(ctx):
    rep = dae_newton_report()
    _check(ctx, lib().dae_last_report(ctx, ctypes.byref(rep)))
    return rep


def dae_rollout(ctx, dec, mesh, cub_tets, cub_w, n_frames, q, qdot, dt, f_ext=None, opts=None,
                q_traj=None, want_reports=True):
    n = int(cub_tets.shape[0]) if cub_tets is not None else 0
    reps = (dae_newton_report * max(n_frames, 1))() if want_reports else None
    _check(ctx, lib().dae_rollout(
        ctx, dec, mesh, n, _ptr(cub_tets, np.int32), _ptr(cub_w, np.float32, n * n_frames),
        n_frames, _ptr(q, np.float64), _ptr(qdot, np.float64), float(dt), _ptr(f_ext, np.float32),
        ctypes.byref(opts) if opts is not None else None, _ptr(q_traj, np.float64),
        ctypes.cast(reps, ctypes.POINTER(dae_newton_report)) if reps is not None else None))
    return list(reps)[:n_frames] if reps is not None else None


PHASES = ["fwd_hidden", "fwd_out", "rows", "cubature", "wta", "bwd", "assemble", "seed"]


def dae_profile_enable(ctx, phases=None):
    """phases: None/True = all, False/() = off, or an iterable of phase names."""
    if phases is None or phases is True:
        mask = (1 << len(PHASES)) - 1
    elif phases is False:
        mask = 0
    else:
        mask = 0
        for p in phases:
            mask |= 1 << PHASES.index(p)
    _check(ctx, lib().dae_profile_enable(ctx, mask))


def dae_profile_read(ctx):
    """{phase: (total_ms, count)} since the previous read (synchronizes)."""
    ms = np.zeros(len(PHASES))
    cnt = np.zeros(len(PHASES), np.int64)
    _check(ctx, lib().dae_profile_read(ctx, ms.ctypes.data, cnt.ctypes.data))
    return {p: (float(ms[i]), int(cnt[i])) for i, p in enumerate(PHASES)}


def dae_selftest_bounded_waits(ctx):
    _check(ctx, lib().dae_selftest_bounded_waits(ctx))


def dae_launch_count(ctx):
    return int(lib().dae_launch_count(ctx))


def dae_reduce_rows_noalloc(N, r, J, dJ, HDD, mdof, f_ext, z, dt, phi_dense=None, Mr=None, B=None,
                            stream=None):
    """Row reductions with no device allocation (all arrays device tensors)."""
    st = lib().dae_reduce_rows_noalloc(int(N), int(r), _ptr(J, np.float32), _ptr(dJ, np.float32),
                                       _ptr(HDD, np.float32), _ptr(mdof, np.float32),
                                       _ptr(f_ext, np.float32), _ptr(z, np.float32), float(dt),
                                       _ptr(phi_dense, np.float64), _ptr(Mr, np.float64),
                                       _ptr(B, np.float64), stream)
    if st != 0:
        raise DaeError(st, "dae_reduce_rows_noalloc failed")


# ------------------------------------------------------------- training --
class Trainer:
    """Handle of a dae_trainer (decoder training pass)."""

    def __init__(self, ctx, handle, widths, act):
        self.ctx = ctx
        self.handle = handle
        self.widths = list(widths)
        self.act = act


def _devptr_array(tensors):
    arr = (_vp * len(tensors))()
    for i, t in enumerate(tensors):
        if not (hasattr(t, "is_cuda") and t.is_cuda and t.dtype.itemsize == 4 and t.is_contiguous()):
            raise ValueError("trainer arrays must be contiguous float32 CUDA tensors")
        arr[i] = t.data_ptr()
    return arr


def dae_trainer_create(ctx, widths, act="tanh", max_batch=256):
    w = (ctypes.c_int * len(widths))(*[int(x) for x in widths])
    h = _vp()
    _check(ctx, lib().dae_trainer_create(ctx, len(widths) - 1, w, ACT[act], int(max_batch),
                                         ctypes.byref(h)))
    return Trainer(ctx, h, widths, act)


def dae_trainer_free(tr):
    lib().dae_trainer_free(tr.handle)


def dae_trainer_set_precision(tr, prec):
    """'bf16x3' (tensor cores, default) or 'fp32' (CUDA cores)."""
    _check(tr.ctx, lib().dae_trainer_set_precision(tr.handle, PREC[prec]))


def _tensor_ptr(t, dtype):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError("expected a contiguous %s CUDA tensor" % dtype)
    return _vp(t.data_ptr())


def dae_train_forward(tr, W, b, q, uJ):
    """W, b: lists of float32 CUDA tensors; q (B, r) float64; uJ (1 + r, B, N) float32."""
    import torch
    B = int(q.shape[0])
    _check(tr.ctx, lib().dae_train_forward(tr.handle, _devptr_array(W), _devptr_array(b), B,
                                           _tensor_ptr(q, torch.float64), _tensor_ptr(uJ, torch.float32)))


def dae_train_backward(tr, W, b, q, g_uJ, g_q, g_W, g_b):
    import torch
    B = int(q.shape[0])
    _check(tr.ctx, lib().dae_train_backward(
        tr.handle, _devptr_array(W), _devptr_array(b), B, _tensor_ptr(q, torch.float64),
        _tensor_ptr(g_uJ, torch.float32),
        _tensor_ptr(g_q, torch.float64) if g_q is not None else None,
        _devptr_array(g_W), _devptr_array(g_b)))
