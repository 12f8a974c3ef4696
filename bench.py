#!/usr/bin/env python
"""Benchmark: reduced implicit-Euler Newton iterations per second on one GB300.

Workload (default "paper"): latent r = 30, ten-layer tanh decoder
30-128-256-512-1024-2048-2048-2048-4096-4096-60000 (282 M weights), 20x20x50
vertex grid (88 445 tets), Neo-Hookean E = 5e5, nu = 0.45, 500 cubature tets
with per-frame weights in [0.5, 2], gravity, dt = 1/60, at most 5 Newton
updates per frame.  All inputs are seeded and synthetic (the paper ships no
meshes or trained decoders).

A step is one implicit-Euler frame: the device Newton control evaluates the
stacked complex-step forward pass, the output-layer reductions, the cubature and
phi at every iterate; an accepted iterate that starts a new Newton step also runs
the complex-step reverse pass, forms A (Eq. 11) and solves A delta = -phi (LU);
rejected, converged or stopped trials are phi-only evaluations.
``value`` = reduced Newton iterations per second: accepted Newton updates (an
A-assembly, a solve and the line-search trials until one is accepted) over the
timed frames, device-resident inputs; evaluations/s and frames/s are reported
beside it.  ``e2e`` = the same metric through the public C ABI with host buffers,
one ``dae_rollout`` call per frame.  ``forms`` = every precision form on the
paper-scale and the small workload: iterations/s and the normwise relative error
of u, J, H[qdot,qdot], dJ, phi and A against the FP64 oracle at the first iterate.

--impl reference times the FP64 CPU oracle (the baseline this library is
checked against): one whole Newton iteration of the same workload per step.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="paper", choices=["paper", "small", "medium"],
                    help="medium: the paper-scale hidden layers onto a 20x20x17 grid, for "
                         "profiler captures")
    ap.add_argument("--prec", default="bf16x3", choices=["fp32", "tf32", "bf16", "bf16x3"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--np", type=int, default=0,
                    help="add a linear (PCA-style) subspace of this size to the decoder")
    ap.add_argument("--wnet", action="store_true",
                    help="predict the cubature weights with a weight network (N-64-64-64-n_tet)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="run the tile autotuner on the decoder before timing (set-up, untimed)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the grouped-strings and training-pass records of the default line")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the per-precision-form rates and oracle errors")
    ap.add_argument("--form-frames", type=int, default=20,
                    help="timed frames per precision form (the small workload runs 5x more)")
    ap.add_argument("--n-strings", type=int, default=320)
    ap.add_argument("--cub-sizes", default="64,500,6600,11400,88445",
                    help="cubsweep: cubature set sizes |C| (88445 = every tet of the mesh)")
    ap.add_argument("--mode", default="newton", choices=["newton", "train", "strings", "cubsweep"],
                    help="train: fit a re-seeded small-workload decoder to 4096 rollout poses "
                         "(batch 256, 100 Adam steps) and time the library's backward pass")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(name):
    from paper_2102_11026_gb300 import synth
    return {"paper": synth.paper, "small": synth.small, "medium": synth.medium}[name]()


def frame_weights(wl, n_frames, seed, start=0):
    from paper_2102_11026_gb300 import synth
    return np.concatenate([synth.make_cubature(wl.mesh.n_tet, wl.cub_tets.size, seed, frame=f)[1]
                           for f in range(start, start + n_frames)]).astype(np.float32)


# --------------------------------------------------------------- roofline --
def hidden_chain_bytes(wl, prec):
    """Algorithmic DRAM bytes of one hidden forward chain launch (the dominant kernel):
    every hidden layer's weights once, its stacked input columns read and output columns
    written once (operand form), act'(z) and act''(z) b_j written, and the FP32 copy of
    the output layer's input."""
    d = wl.dec
    r = d.r
    C = 4 + 3 * r
    wbytes = {"fp32": 4, "tf32": 4, "bf16": 2, "bf16x3": 4}[prec]
    tot = 0
    for l in range(len(d.W) - 1):
        n_out, n_in = d.W[l].shape
        tot += n_out * n_in * wbytes + C * n_in * wbytes + C * n_out * wbytes + n_out * (1 + r) * 4
    tot += C * d.widths[-2] * 4
    return tot


def output_stage_bytes(wl, prec):
    """Algorithmic DRAM bytes of the Newton path's output stage (Gram form), which runs as
    the last job of the forward chain's launch: the stacked operand [G ; W_L rows at the
    12|C| cubature DOFs] once (K + 12|C| rows of K, operand form), its input columns once,
    and u and J at the cubature DOFs written."""
    d = wl.dec
    r, K = d.r, d.widths[-2]
    C = 4 + 3 * r
    wbytes = {"fp32": 4, "tf32": 4, "bf16": 2, "bf16x3": 4}[prec]
    rows = K + 12 * wl.cub_tets.size
    return rows * K * wbytes + C * K * wbytes + 12 * wl.cub_tets.size * (1 + r) * 4


def algorithmic_flops(wl, gram=True):
    """2 [sum_hidden P_l C_f + P_out C_f + sum_hidden P_l (1 + r) + K]: the stacked forward
    over all C_f = 3r + 4 columns (the output stage in Gram form: K x K of G plus the 12|C|
    cubature rows of W_L; else all N x K of W_L), the complex reverse pass through the
    hidden layers, W_L^T a."""
    d = wl.dec
    r = d.r
    P = [w.size for w in d.W]
    K = d.widths[-2]
    P_out = (K * K + 12 * wl.cub_tets.size * K) if gram else P[-1]
    return 2.0 * ((sum(P[:-1]) + P_out) * (3 * r + 4) + sum(P[:-1]) * (1 + r) + K)


L2_BYTES = 129e6   # GB300 L2


def l2_note(d):
    """How the timed frames relate to L2: the FP32 decoder weights (the GEMM operands are
    at least as large in BF16x3) against the 129 MB L2; no flush is done either way."""
    wb = sum(w.nbytes for w in d.W)
    if wb > L2_BYTES:
        return "inputs larger than L2 (decoder weights %.0f MB)" % (wb / 1e6)
    return ("decoder weights %.0f MB fit in L2 (129 MB): frames run back to back on "
            "L2-resident weights, as in a simulation loop, no flush" % (wb / 1e6))


def workload_config(args, wl, K, evals_all=None, flops=None, ms=None, world=1):
    """The config block shared by both arms of the benchmark."""
    d = wl.dec
    cfg = {"workload": ("paper-scale decoder r=30, 30-128-256-512-1024-2048-2048-2048-"
                        "4096-4096-60000 tanh, 20x20x50 grid (88445 tets), Neo-Hookean, "
                        "500 cubature tets, gravity, dt=1/60, <=5 Newton updates/frame")
           if args.workload == "paper" else
           ("paper-scale hidden layers r=30, 30-...-4096-20400 tanh, 20x20x17 grid, Neo-Hookean"
            if args.workload == "medium" else "small decoder r=5 5-64-256-1024-3000"),
           "step": "one implicit-Euler frame", "frames": K,
           "cubature_weights": ("predicted per frame by a weight network N-64-64-64-n_tet (sin, squared)"
                                if getattr(args, "wnet", False) else "seeded per frame, U[0.5, 2]"),
           "linear_subspace": getattr(args, "np", 0),
           "l2": l2_note(d),
           "parallelism": "replicas" if world > 1 else "single GPU"}
    if evals_all is not None:
        cfg["full_evaluations"] = int(evals_all)
        cfg["algorithmic_gflop_per_full_evaluation"] = flops / 1e9
        cfg["derivative_pass_tflops_over_step"] = flops * evals_all / (ms / 1e3) / 1e12
    return cfg


def pinned_copy(a):
    """A copy of a host array in page-locked memory (a numpy view of a pinned tensor,
    which the view keeps alive)."""
    import torch
    a = np.ascontiguousarray(a)
    t = torch.empty(a.shape, dtype=torch.from_numpy(a).dtype, pin_memory=True)
    v = t.numpy()
    v[...] = a
    return v


def reduce_over_ranks(ms, evals, device):
    """Max of the timed region and sum of the evaluations over all ranks."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e = torch.tensor([float(evals)], dtype=torch.float64, device=device)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), float(e.item())


# ---------------------------------------------------------------- oracle --
ORACLE_SAMPLE = ("one whole Newton iteration of the FP64 oracle from the frame's first "
                 "iterate q0 = qbar + dt qbar_dot: reduced_system (phi and A: hyper-dual "
                 "derivative passes of the full decoder, a^T H, cubature FEM, assembly), "
                 "the LU solve of A delta = -phi and phi_only at the first trial point")


def oracle_iteration(wl, max_step=0.5):
    """Time one Newton iteration of the FP64 oracle at q0, the unit of the metric:
    the reduced system (phi and A), the solve and phi at the line search's first
    trial.  Returns (seconds, OpenMP threads, the reduced system at q0)."""
    import oracle
    from paper_2102_11026_gb300 import synth
    q0 = synth.newton_start(wl.state)
    t0 = time.perf_counter()
    rs = oracle.reduced_system(wl, q0)
    delta = np.linalg.solve(rs["A"], -rs["phi"])
    dn = float(np.max(np.abs(delta)))
    alpha = max_step / dn if (max_step > 0 and dn > max_step) else 1.0
    oracle.phi_only(wl, q0 + alpha * delta)
    t = time.perf_counter() - t0
    return t, oracle.num_threads(), rs


def run_reference(args):
    """The oracle arm: each timed step is one whole oracle Newton iteration of the
    workload (``oracle_iteration``); each warm-up step one phi-only evaluation of it
    (touches the whole decoder and the cubature, warming caches and the thread pool)."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    wl = make_workload(args.workload)
    import oracle
    from paper_2102_11026_gb300 import synth
    oracle.build()
    q0 = synth.newton_start(wl.state)
    t_all = time.perf_counter()
    for _ in range(args.warmup):
        oracle.phi_only(wl, q0)
    times = []
    T = oracle.num_threads()
    for _ in range(args.steps):
        t, T, _ = oracle_iteration(wl)
        times.append(t)
    total = time.perf_counter() - t_all
    ms = 1e3 * float(np.sum(times)) / len(times)
    value = 1e3 / ms
    line = {
        "impl": "reference", "metric": "reduced Newton iterations/s", "value": value,
        "unit": "iterations/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, wl, args.steps),
        "cpu_baseline": {"value": value, "unit": "iterations/s", "cores": T, "kind": "oracle",
                         "sample": ORACLE_SAMPLE + "; one per timed step (warm-up steps: "
                                   "phi_only at q0)"},
        "e2e": {"value": value, "unit": "iterations/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "step_seconds": {"min": float(np.min(times)), "median": float(np.median(times)),
                         "max": float(np.max(times))},
        "wall_seconds": total,
    }
    print(json.dumps(line))


# ------------------------------------------------------------------- ours --
def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2102_11026_gb300 import dae

    wl = make_workload(args.workload)
    d, m = wl.dec, wl.mesh
    stream = torch.cuda.Stream()
    ctx = dae.dae_create(torch.cuda.current_device(), stream.cuda_stream)
    dec = dae.dae_load_decoder(ctx, d.widths, d.W, d.b, d.act, args.prec)
    mesh = dae.dae_load_mesh(ctx, m.X.reshape(-1), m.tets.reshape(-1), m.vmass, m.material,
                             m.E, m.nu)
    tuned = None
    if getattr(args, "autotune", False) and args.prec != "fp32":
        tuned = [round(x, 4) for x in dae.dae_decoder_autotune(ctx, dec, reps=20)]
    if args.wnet:
        from paper_2102_11026_gb300 import synth
        net = synth.make_wnet(d.n_out, m.n_tet, 7)
        dae.dae_decoder_attach_wnet(ctx, dec, net.widths, net.W, net.b)
    QBAR0, QDOT0 = wl.state.qbar, wl.state.qbar_dot
    if args.np > 0:
        # linear subspace: u = U p + (I - U U^T) D(q), unknown [p; q]
        from paper_2102_11026_gb300 import synth
        U = synth.make_linear_basis(d.n_out, args.np, 8)
        dae.dae_decoder_attach_linear(ctx, dec, np.ascontiguousarray(U.T))
        pb, pd = synth.make_linear_state(args.np, 8, p_std=0.05, pdot_std=0.02)
        QBAR0 = np.concatenate([pb, QBAR0])
        QDOT0 = np.concatenate([pd, QDOT0])
    dev = lambda x, dt: torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device="cuda")
    W, K = args.warmup, args.steps
    n = wl.cub_tets.size
    seed = 2 + rank
    cw_all = frame_weights(wl, W + K + 2, seed)
    cub_t = dev(wl.cub_tets, torch.int32)
    cub_w = dev(cw_all, torch.float32)
    if args.wnet:
        class _NoWeights:            # every slice: predicted weights (NULL)
            def __getitem__(self, k):
                return None
        cub_w = _NoWeights()
    f_ext = dev(wl.f_ext, torch.float32)
    q = dev(QBAR0, torch.float64)
    qd = dev(QDOT0, torch.float64)
    opts = dae.dae_default_newton_opts()
    opts.max_iter = 5

    with torch.cuda.stream(stream):
        # warm-up frames (untimed)
        dae.dae_rollout(ctx, dec, mesh, cub_t, cub_w[:W * n], W, q, qd, wl.state.dt, f_ext, opts)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        sampler = ClockSampler(torch.cuda.current_device())
        sampler.start()
        time.sleep(0.3)
        dae.dae_profile_read(ctx)
        dae.dae_profile_enable(ctx, False)           # timed region: the captured frame graph
        launches0 = dae.dae_launch_count(ctx)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        reps = dae.dae_rollout(ctx, dec, mesh, cub_t, cub_w[W * n:(W + K) * n], K, q, qd,
                               wl.state.dt, f_ext, opts)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        launches = dae.dae_launch_count(ctx) - launches0
        clocks = sampler.stop()
        # dominant-kernel time: CUDA events around every output-layer launch of the same
        # frames replayed with explicit launches (events cannot sit inside graph loops)
        q2, qd2 = q.clone(), qd.clone()
        q2.copy_(dev(QBAR0, torch.float64))
        qd2.copy_(dev(QDOT0, torch.float64))
        dae.dae_rollout(ctx, dec, mesh, cub_t, cub_w[:W * n], W, q2, qd2, wl.state.dt, f_ext, opts)
        dae.dae_profile_read(ctx)
        dae.dae_profile_enable(ctx, ["fwd_hidden"])
        reps1 = dae.dae_rollout(ctx, dec, mesh, cub_t, cub_w[W * n:(W + K) * n], K, q2, qd2,
                                wl.state.dt, f_ext, opts)
        dae.dae_profile_enable(ctx, False)
        prof = dae.dae_profile_read(ctx)
        # phase shares from a fully instrumented pass over 2 more frames
        dae.dae_profile_enable(ctx, True)
        reps2 = dae.dae_rollout(ctx, dec, mesh, cub_t, cub_w[(W + K) * n:(W + K + 2) * n], 2, q2, qd2,
                                wl.state.dt, f_ext, opts)
        dae.dae_profile_enable(ctx, False)
        prof_all = dae.dae_profile_read(ctx)
        evals2 = max(1, sum(rp.evals for rp in reps2))
        full2 = max(1, sum(rp.full_evals for rp in reps2))
    evals = sum(rp.evals for rp in reps)
    iters = sum(rp.iters for rp in reps)
    full = sum(rp.full_evals for rp in reps)
    if world > 1:
        ms, iters_all = reduce_over_ranks(ms, iters, "cuda")
        _, evals_all = reduce_over_ranks(ms, evals, "cuda")
        _, full_all = reduce_over_ranks(ms, full, "cuda")
    else:
        iters_all, evals_all, full_all = iters, evals, full
    value = iters_all / (ms / 1e3)

    # ---- roofline of the dominant kernel (the persistent hidden forward chain), timed
    # live with CUDA events around every launch
    peaks, peak_src = load_peaks()
    t_hid, c_hid = prof["fwd_hidden"]
    avg_ms = t_hid / max(c_hid, 1)
    # the tensor-core forms run the Gram-form output stage as the chain launch's last job
    fused = args.prec != "fp32"
    bytes_hid = hidden_chain_bytes(wl, args.prec) + (output_stage_bytes(wl, args.prec) if fused else 0)
    achieved = bytes_hid / (avg_ms / 1e3) / 1e9
    hbm = peaks["hbm_gbs"]
    traffic = load_traffic(args.workload, args.prec + ("/fused" if fused else ""))
    tc = args.prec != "fp32"
    flops_hid = hidden_chain_flops(wl) + (output_stage_flops(wl) if fused else 0.0)
    tf_hid = flops_hid / (avg_ms / 1e3) / 1e12
    tpeak = tensor_peak(peaks, args.prec)
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": traffic,
            "kernel": ("forward chain: %d hidden layers + Gram-form output stage (k_chain, one "
                       "launch, %s)" % (len(d.W) - 1, args.prec)) if fused else
                      "hidden forward chain (k_chain, %d layers, %s)" % (len(d.W) - 1, args.prec),
            "peak_source": "%s hbm_gbs" % peak_src,
            "avg_launch_ms": avg_ms, "algorithmic_bytes_per_launch": bytes_hid}
    tot_ph = sum(v[0] for v in prof_all.values())
    phase_share = {k: round(v[0] / max(tot_ph, 1e-9), 4) for k, v in prof_all.items()}
    phase_ms_per_eval = {k: round(v[0] / evals2, 4) for k, v in prof_all.items()}
    flops = algorithmic_flops(wl, gram=tc)
    # the derivative pass (hidden chain, output stage, reverse pass) of a full evaluation
    t_der = (prof_all["fwd_hidden"][0] + prof_all["fwd_out"][0] + prof_all["bwd"][0] +
             prof_all["wta"][0])
    tf_der = flops * full2 / max(t_der / 1e3, 1e-12) / 1e12
    if tpeak is not None:
        roof["tensor"] = {
            "unit": "TFLOP/s", "peak": tpeak["peak"], "peak_source": "%s %s" % (peak_src, tpeak["src"]),
            "hidden_chain": {"achieved": tf_hid, "frac": tf_hid / tpeak["peak"],
                             "algorithmic_flops_per_launch": flops_hid,
                             "executed_frac": tf_hid * tpeak["mma_per_product"] / tpeak["peak"]},
            "derivative_pass": {"achieved": tf_der, "frac": tf_der / tpeak["peak"],
                                "algorithmic_flops_per_full_evaluation": flops,
                                "executed_frac": tf_der * tpeak["mma_per_product"] / tpeak["peak"]},
            "note": "algorithmic flops (one product per weight and stacked column); split-BF16x3 "
                    "executes %d MMAs per product (executed_frac)" % tpeak["mma_per_product"]}

    # ---- end to end through the C ABI with host buffers (one dae_rollout per frame): every
    # input and output of a frame in page-locked host memory, copied by the call
    e2e = None
    if not args.no_e2e:
        qh = pinned_copy(QBAR0)
        qdh = pinned_copy(QDOT0)
        cwh = pinned_copy(frame_weights(wl, K, seed, start=W))
        tets_h = pinned_copy(wl.cub_tets)
        fext_h = pinned_copy(wl.f_ext) if wl.f_ext is not None else None
        it_tot = 0
        dae.dae_rollout(ctx, dec, mesh, tets_h, None if args.wnet else cwh[:n], 1, qh, qdh,
                        wl.state.dt, fext_h, opts)
        qh[...] = QBAR0
        qdh[...] = QDOT0
        t0 = time.perf_counter()
        for f in range(K):
            rp = dae.dae_rollout(ctx, dec, mesh, tets_h,
                                 None if args.wnet else cwh[f * n:(f + 1) * n], 1, qh, qdh,
                                 wl.state.dt, fext_h, opts)
            it_tot += rp[0].iters
        te = time.perf_counter() - t0
        r = d.r + args.np
        h2d = 2 * r * 8 + n * 4 + (0 if args.wnet else n * 4) + wl.f_ext.nbytes
        d2h = 2 * r * 8 + ctypes_report_bytes()
        e2e = {"value": it_tot / te, "unit": "iterations/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "host_memory": "pinned"}

    # ---- the FP64 oracle: one whole Newton iteration at q0 on the host cores (also the
    # reference values of the precision forms below)
    cpu, ref_paper = None, None
    if rank == 0 and world == 1 and not (args.no_cpu and args.no_forms):
        t_or, T, ref_paper = oracle_iteration(wl)
        if not args.no_cpu:
            cpu = {"value": 1.0 / t_or, "unit": "iterations/s", "cores": T, "kind": "oracle",
                   "sample": ORACLE_SAMPLE + " (%.2f s)" % t_or}
    forms = None
    if rank == 0 and world == 1 and not args.no_forms and args.np == 0 and not args.wnet:
        with torch.cuda.stream(stream):
            forms = {args.workload: measure_forms(ctx, stream, wl, dec, mesh, ref_paper, args,
                                                  args.form_frames)}
            if args.workload != "small":
                from paper_2102_11026_gb300 import synth
                ws = synth.small()
                import oracle
                ref_small = oracle.reduced_system(ws, synth.newton_start(ws.state))
                ds, msh = ws.dec, ws.mesh
                dec_s = dae.dae_load_decoder(ctx, ds.widths, ds.W, ds.b, ds.act, "fp32")
                mesh_s = dae.dae_load_mesh(ctx, msh.X.reshape(-1), msh.tets.reshape(-1),
                                           msh.vmass, msh.material, msh.E, msh.nu)
                forms["small"] = measure_forms(ctx, stream, ws, dec_s, mesh_s, ref_small, args,
                                               5 * args.form_frames)
                dae.dae_free_decoder(dec_s)
                dae.dae_free_mesh(mesh_s)
        for wk, fm in forms.items():
            base = fm["fp32"]["iterations_per_s"]
            for pr, rec in fm.items():
                rec["vs_fp32"] = rec["iterations_per_s"] / base if base > 0 else None

    dae.dae_free_decoder(dec)
    dae.dae_free_mesh(mesh)
    dae.dae_destroy(ctx)
    if rank != 0:
        return
    extra = None
    if world == 1 and not args.no_extra and args.np == 0 and not args.wnet:
        extra = measure_extra(args)
    line = {
        "metric": "reduced Newton iterations/s", "value": value, "unit": "iterations/s",
        "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": ms / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "tf32": "tf32", "bf16": "bf16", "bf16x3": "bf16x3"}[args.prec],
        "data": "synthetic",
        "config": dict(workload_config(args, wl, K, full_all, flops, ms, world),
                       tile_plan="autotuned (forward ms before/after, reverse before/after: %s)" % tuned
                       if tuned else "built-in"),
        "rates": {"newton_iterations_per_s": value, "evaluations_per_s": evals_all / (ms / 1e3),
                  "full_evaluations_per_s": full_all / (ms / 1e3),
                  "frames_per_s": K * world / (ms / 1e3)},
        "newton": {"evals_per_frame": evals / K, "full_evals_per_frame": full / K,
                   "iters_per_frame": iters / K,
                   "converged_frames": sum(rp.converged for rp in reps),
                   "phi_norm0_first": reps[0].phi_norm0, "phi_norm_first": reps[0].phi_norm,
                   "status": sorted(set(rp.status for rp in reps))},
        "roofline": roof, "phase_share": phase_share, "phase_ms_per_evaluation": phase_ms_per_eval,
        "clocks": clocks,
        "gpu_launches": int(launches), "cpu_baseline": cpu, "e2e": e2e, "forms": forms,
        "other_workloads": extra,
    }
    print(json.dumps(line))


def measure_extra(args):
    """The grouped-strings step (320 independent depth-8 string decoders in one graph,
    against per-string launches) and the training pass of the small decoder in both
    forms, in the same run (short: 3 timed steps / 10 timed backward calls)."""
    import copy
    out = {}
    a = copy.copy(args)
    a.steps, a.warmup, a.prec = 3, 2, "bf16x3"
    st = run_strings(a, emit=False)
    keep = ("metric", "value", "unit", "ms_per_step", "per_string_launches", "roofline", "clocks")
    out["strings"] = {k: st[k] for k in keep if k in st}
    out["strings"]["config"] = st["config"]["workload"]
    for prec in ("bf16x3", "fp32"):
        a = copy.copy(args)
        a.steps, a.warmup, a.prec = 10, 3, prec
        tr = run_train(a, emit=False)
        out["train_" + prec] = {k: tr[k] for k in ("metric", "value", "unit", "ms_per_step",
                                                   "roofline", "fit", "dtype") if k in tr}
    return out


def ctypes_report_bytes():
    from paper_2102_11026_gb300 import dae
    import ctypes
    return ctypes.sizeof(dae.dae_newton_report)


def tensor_peak(peaks, prec):
    """Dense tensor-core peak for the precision form: the measured BF16 burst peak (the
    kernels are timed alone inside a ~1 ms frame, well below the power cap); TF32 at the
    nominal TF32/BF16 ratio (1.1 / 2.25 PFLOP/s); split-BF16x3 executes three BF16 MMAs
    per product."""
    bf = peaks.get("bf16_tflops")
    if bf is None or prec == "fp32":
        return None
    if prec == "tf32":
        return {"peak": bf * 1.1 / 2.25, "src": "bf16_tflops x 1.1/2.25 (nominal TF32/BF16)",
                "mma_per_product": 1}
    return {"peak": bf, "src": "bf16_tflops (burst)", "mma_per_product": 3 if prec == "bf16x3" else 1}


def hidden_chain_flops(wl):
    """Algorithmic flops of one hidden forward chain launch: 2 P_l (3r + 4) per hidden
    layer (every stacked complex-step column of the shared-column form)."""
    d = wl.dec
    return 2.0 * sum(w.size for w in d.W[:-1]) * (3 * d.r + 4)


def output_stage_flops(wl):
    """2 (K^2 + 12|C| K)(3r + 4): the Gram-form output stage over the stacked columns."""
    d = wl.dec
    K = d.widths[-2]
    return 2.0 * (K * K + 12 * wl.cub_tets.size * K) * (3 * d.r + 4)


def measure_forms(ctx, stream, wl, dec, mesh, ref, args, n_frames):
    """Every precision form of the decoder GEMMs on one workload: Newton iterations/s
    over ``n_frames`` frames (device buffers, CUDA events on the context's stream, after
    two warm-up frames) and the normwise relative error of u, J, H[qdot,qdot], dJ, phi
    and A at the first iterate q0 against the FP64 oracle's values there (``ref``)."""
    import torch
    from paper_2102_11026_gb300 import dae, synth
    d = wl.dec
    r, N, n = d.r, d.n_out, wl.cub_tets.size
    q0 = synth.newton_start(wl.state)
    dev = lambda x, dt: torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device="cuda")
    cw = dev(frame_weights(wl, n_frames + 2, 11), torch.float32)
    cub_t = dev(wl.cub_tets, torch.int32)
    f_ext = dev(wl.f_ext, torch.float32)
    opts = dae.dae_default_newton_opts()
    opts.max_iter = 5
    rel = lambda x, y: float(np.linalg.norm(np.asarray(x, np.float64) - y) /
                             max(np.linalg.norm(y), 1e-300))
    out = {}
    for prec in ("fp32", "tf32", "bf16", "bf16x3"):
        dae.dae_decoder_set_precision(ctx, dec, prec)
        u = np.zeros(N, np.float32)
        J = np.zeros((r, N), np.float32)
        Hqq = np.zeros(N, np.float32)
        dJ = np.zeros((r, N), np.float32)
        dae.dae_eval_derivs(ctx, dec, q0, wl.state.qbar, wl.state.qbar_dot, wl.state.dt,
                            u=u, J=J, Hqq=Hqq, dJ=dJ)
        phi, A = np.zeros(r), np.zeros(r * r)
        dae.dae_assemble_reduced(ctx, dec, mesh, wl.cub_tets, wl.cub_w, q0, wl.state.qbar,
                                 wl.state.qbar_dot, wl.state.dt, wl.f_ext, phi, A)
        err = {"u": rel(u, ref["u"]), "J": rel(J.T, ref["J"]), "Hqq": rel(Hqq, ref["Hqq"]),
               "dJ": rel(dJ.T, ref["dJ"]), "phi": rel(phi, ref["phi"]),
               "A": rel(A.reshape(r, r).T, ref["A"])}
        q = dev(wl.state.qbar, torch.float64)
        qd = dev(wl.state.qbar_dot, torch.float64)
        dae.dae_rollout(ctx, dec, mesh, cub_t, cw[:2 * n], 2, q, qd, wl.state.dt, f_ext, opts)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        reps = dae.dae_rollout(ctx, dec, mesh, cub_t, cw[2 * n:], n_frames, q, qd, wl.state.dt,
                               f_ext, opts)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        it = sum(rp.iters for rp in reps)
        ev = sum(rp.evals for rp in reps)
        out[prec] = {"iterations_per_s": it / (ms / 1e3), "evaluations_per_s": ev / (ms / 1e3),
                     "frames_per_s": n_frames / (ms / 1e3), "evals_per_frame": ev / n_frames,
                     "iters_per_frame": it / n_frames,
                     "status": sorted(set(rp.status for rp in reps)), "rel_err": err,
                     "l2": l2_note(d)}
    dae.dae_decoder_set_precision(ctx, dec, args.prec)
    return out


def load_traffic(workload, prec):
    """DRAM bytes per launch of the timed forward kernel from the committed ncu summary, if
    any ("<workload>/<precision>[/fused]": the fused key for the chain launch that also
    runs the output stage)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("%s/%s" % (workload, prec))
    return None


# ------------------------------------------------------------------ train --
def train_flops(widths, B):
    """Algorithmic flops of one backward call at batch B: weight gradients of every
    layer, W^T Z̄ for layers 2..L, and the forward of the hidden layers it needs, each
    2 n_out n_in C with C = B (1 + r) columns."""
    P = [widths[l] * widths[l + 1] for l in range(len(widths) - 1)]
    C = B * (1 + widths[0])
    return 2.0 * C * (sum(P) + sum(P[1:]) + sum(P[:-1]))


def run_train(args, emit=True):
    import torch
    from paper_2102_11026_gb300 import dae, synth
    from paper_2102_11026_gb300.autograd import decoder_uJ
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    wl = synth.small()
    d, m = wl.dec, wl.mesh
    r, n = d.r, wl.cub_tets.size
    stream = torch.cuda.current_stream()
    ctx = dae.dae_create(torch.cuda.current_device(), stream.cuda_stream)
    # 4096 poses: 64 implicit-Euler rollouts of 64 frames of the small workload from
    # seeded start states
    dec = dae.dae_load_decoder(ctx, d.widths, d.W, d.b, d.act, "bf16x3")
    mesh = dae.dae_load_mesh(ctx, m.X.reshape(-1), m.tets.reshape(-1), m.vmass, m.material, m.E, m.nu)
    opts = dae.dae_default_newton_opts()
    poses = []
    for k in range(64):
        st = synth.make_state(r, 1000 + k)
        qh, qdh = st.qbar.copy(), st.qbar_dot.copy()
        traj = np.zeros((64, r))
        dae.dae_rollout(ctx, dec, mesh, wl.cub_tets, frame_weights(wl, 64, 1000 + k), 64, qh, qdh,
                        st.dt, wl.f_ext, opts, traj)
        poses.append(traj)
    dae.dae_free_decoder(dec)
    dae.dae_free_mesh(mesh)
    poses = torch.as_tensor(np.concatenate(poses), device="cuda")
    Bt = 256
    tr = dae.dae_trainer_create(ctx, d.widths, d.act, max_batch=Bt)
    # the training GEMMs in split BF16x3 (tensor cores) or FP32 (CUDA cores)
    tprec = "fp32" if args.prec == "fp32" else "bf16x3"
    dae.dae_trainer_set_precision(tr, tprec)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    teacher = []
    for w, x in zip(d.W, d.b):
        teacher += [dev(w), dev(x)]
    st_dec = synth.make_decoder(d.widths, 77, d.act)
    params = []
    for w, x in zip(st_dec.W, st_dec.b):
        params += [dev(w).requires_grad_(True), dev(x).requires_grad_(True)]
    with torch.no_grad():
        tU, tJ = [], []
        for i in range(0, poses.shape[0], Bt):
            u, J = decoder_uJ(tr, poses[i:i + Bt], teacher)
            tU.append(u)
            tJ.append(J)
        tU, tJ = torch.cat(tU), torch.cat(tJ)
    opt = torch.optim.Adam(params, lr=1e-3)
    n_steps = 100
    losses = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for step in range(n_steps):
        i = (step * Bt) % poses.shape[0]
        u, J = decoder_uJ(tr, poses[i:i + Bt], params)
        loss = ((u - tU[i:i + Bt]) ** 2).mean() + ((J - tJ[i:i + Bt]) ** 2).mean()
        opt.zero_grad()
        loss.backward()
        opt.step()
        losses.append(loss.detach())
    e1.record()
    torch.cuda.synchronize()
    fit_ms = e0.elapsed_time(e1)
    losses = [float(x) for x in losses]
    # the backward pass alone, timed over K calls after W warm-up calls
    W_, b_ = [p.detach() for p in params[0::2]], [p.detach() for p in params[1::2]]
    qb = poses[:Bt].contiguous()
    g_uJ = torch.randn((1 + r, Bt, d.n_out), device="cuda")
    gq = torch.empty((Bt, r), dtype=torch.float64, device="cuda")
    gW = [torch.empty_like(w) for w in W_]
    gb = [torch.empty_like(x) for x in b_]
    for _ in range(args.warmup):
        dae.dae_train_backward(tr, W_, b_, qb, g_uJ, gq, gW, gb)
    torch.cuda.synchronize()
    l0 = dae.dae_launch_count(ctx)
    e0.record()
    for _ in range(args.steps):
        dae.dae_train_backward(tr, W_, b_, qb, g_uJ, gq, gW, gb)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    launches = dae.dae_launch_count(ctx) - l0
    flops = train_flops(d.widths, Bt)
    peaks, src = load_peaks()
    tf = flops / (ms / 1e3) / 1e12
    if tprec == "fp32":
        # FP32 FFMA on the CUDA cores: 152 SMs x 128 FP32 lanes x 2 flops x the SM clock
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        alu = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": tf, "peak": alu, "unit": "TFLOP/s", "frac": tf / alu,
                "traffic": None,
                "note": "peak derived: 152 SMs x 128 FP32 FMA lanes x 2 flops x %.0f MHz" % sm_mhz}
    else:
        roof = {"bound": "tensor", "achieved": tf * 3, "peak": peaks["bf16_tflops"],
                "unit": "TFLOP/s", "frac": tf * 3 / peaks["bf16_tflops"], "traffic": None,
                "note": "achieved counts the three BF16 MMAs of each split-BF16x3 product; "
                        "peak: %s bf16 burst" % src}
    dae.dae_trainer_free(tr)
    dae.dae_destroy(ctx)
    if rank != 0:
        return
    out = {
        "metric": "decoder backward-pass TFLOP/s", "value": tf, "unit": "TFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if tprec == "fp32" else "bf16x3",
        "data": "synthetic",
        "config": {"workload": "small decoder 5-64-256-1024-3000 tanh: backward of u and J w.r.t. "
                               "latents, weights and biases, batch 256 (1536 columns)",
                   "poses": "4096 from 64 rollouts x 64 frames of the small workload",
                   "gflop_per_backward": flops / 1e9},
        "roofline": roof,
        "fit": {"steps": n_steps, "batch": Bt, "loss_first": losses[0], "loss_last": losses[-1],
                "ms_per_adam_step": fit_ms / n_steps},
        "gpu_launches": int(launches),
    }
    if not emit:
        return out
    print(json.dumps(out))


# -------------------------------------------------------- grouped strings --
def run_strings(args, emit=True):
    """One implicit-Euler Newton step of every string of the substructured model
    (320 independent strings, depth-8 decoders) per bench step: the grouped entry point
    (all strings in one graph) against per-string dae_newton_step calls.  Under torchrun
    each rank steps its own share of the strings (partitioned by cost, no collective on
    the data path); the timed region is the max over ranks and the evaluations the sum."""
    import torch
    from paper_2102_11026_gb300 import dae, shard, synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > args.n_strings:
        raise SystemExit("more ranks (%d) than strings (%d)" % (world, args.n_strings))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    t0 = time.perf_counter()
    rs, vs = synth.string_shapes(args.n_strings)
    costs = [shard.string_cost(synth.string_widths(r, V)) for r, V in zip(rs, vs)]
    mine = shard.shard_by_cost(costs, world)[rank]
    wls = synth.strings(args.n_strings, only=mine)
    t_gen = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    ctx = dae.dae_create(torch.cuda.current_device(), stream.cuda_stream)
    loaded = []
    for wl in wls:
        d, m = wl.dec, wl.mesh
        loaded.append((dae.dae_load_decoder(ctx, d.widths, d.W, d.b, d.act, args.prec),
                       dae.dae_load_mesh(ctx, m.X.reshape(-1), m.tets.reshape(-1), m.vmass,
                                         m.material, m.E, m.nu)))
    dev = lambda x, dt: torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device="cuda")
    n = len(wls)
    R = 32
    q0_all = torch.zeros(n, R, dtype=torch.float64, device="cuda")
    for i, wl in enumerate(wls):
        q0_all[i, :wl.dec.r] = dev(synth.newton_start(wl.state), torch.float64)
    q_all = q0_all.clone()
    systems = []
    for i, (wl, (dec, mesh)) in enumerate(zip(wls, loaded)):
        systems.append(dict(dec=dec, mesh=mesh, cub_tets=dev(wl.cub_tets, torch.int32),
                            cub_w=dev(wl.cub_w, torch.float32), q=q_all[i],
                            qbar=dev(wl.state.qbar, torch.float64),
                            qbar_dot=dev(wl.state.qbar_dot, torch.float64)))
    dt = wls[0].state.dt
    opts = dae.dae_default_newton_opts()
    opts.max_iter = 5
    W, K = args.warmup, args.steps
    with torch.cuda.stream(stream):
        q_all.copy_(q0_all)
        reps = dae.dae_newton_step_batched(ctx, systems, dt, opts)
        evals = [rp.evals for rp in reps]
        for _ in range(W):
            q_all.copy_(q0_all)
            dae.dae_newton_step_batched(ctx, systems, dt, opts, want_reports=False)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        sampler = ClockSampler(torch.cuda.current_device())
        sampler.start()
        time.sleep(0.3)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(K):
            q_all.copy_(q0_all)
            dae.dae_newton_step_batched(ctx, systems, dt, opts, want_reports=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms = ev0.elapsed_time(ev1)
        clocks = sampler.stop()
        q_grouped = q_all.cpu().numpy().copy()
        # the same step with explicit launches and CUDA events around every phase (the
        # grouped forward chain is the dominant kernel)
        dae.dae_profile_read(ctx)
        dae.dae_profile_enable(ctx, True)
        q_all.copy_(q0_all)
        dae.dae_newton_step_batched(ctx, systems, dt, opts, want_reports=False)
        dae.dae_profile_enable(ctx, False)
        prof = dae.dae_profile_read(ctx)
        q_explicit = q_all.cpu().numpy().copy()
        # per-string launches: the same steps through dae_newton_step, one string at a time
        Kp = max(1, min(K, 3))
        for y in systems[:4]:
            dae.dae_newton_step(ctx, y["dec"], y["mesh"], y["cub_tets"], y["cub_w"], y["q"],
                                y["qbar"], y["qbar_dot"], dt, None, opts, want_report=False)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(Kp):
            q_all.copy_(q0_all)
            for y in systems:
                dae.dae_newton_step(ctx, y["dec"], y["mesh"], y["cub_tets"], y["cub_w"], y["q"],
                                    y["qbar"], y["qbar_dot"], dt, None, opts, want_report=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_single = ev0.elapsed_time(ev1) / Kp
        q_single = q_all.cpu().numpy()
    diff = 0.0
    for i, wl in enumerate(wls):
        r = wl.dec.r
        step = np.linalg.norm(q_grouped[i, :r] - q0_all[i, :r].cpu().numpy())
        diff = max(diff, float(np.linalg.norm(q_grouped[i, :r] - q_single[i, :r]) / max(step, 1e-30)))
    # grouped launches per step: copy in, the graph (begin, per evaluation 12 kernels, end),
    # copy out
    max_ev = max(evals)
    launches_step = 2 + 2 + 12 * max_ev
    for dec, mesh in loaded:
        dae.dae_free_decoder(dec)
        dae.dae_free_mesh(mesh)
    dae.dae_destroy(ctx)
    ev_step = float(sum(evals))
    ms_rank = ms
    if world > 1:
        ms, ev_all = reduce_over_ranks(ms, ev_step, "cuda")
    else:
        ev_all = ev_step
    value = ev_all * K / (ms / 1e3)
    params = [sum(w.size for w in wl.dec.W) for wl in wls]
    bpe = {"bf16x3": 4, "bf16": 2, "tf32": 4}[args.prec]
    peaks, peak_src = load_peaks()
    # every evaluation of a string streams its hidden weights twice (forward chain and the
    # transposed reverse chain) and its stacked Gram operand once ([G ; the W_L rows of its
    # 12 x 32 cubature DOFs], K = 256)
    fwd_bytes = bytes_step = 0.0
    for e, wl in zip(evals, wls):
        r, Kw = wl.dec.r, wl.dec.widths[-2]
        hidden = sum(w.size for w in wl.dec.W[:-1])
        gram = (Kw + 12 * wl.cub_tets.size) * Kw
        cp = (4 + 3 * r + 15) // 16 * 16
        act = sum(cp * n * 2 * bpe // 2 for n in wl.dec.widths[:-1])
        outs = 12 * wl.cub_tets.size * (2 + 2 * r) * 4
        # dominant kernel: the grouped forward chain (hidden layers + Gram operand)
        fwd_bytes += e * ((hidden + gram) * bpe + act + outs)
        bytes_step += e * ((2 * hidden + gram) * bpe)
    step_gbs = bytes_step / (ms_rank / K / 1e3) / 1e9
    t_fwd, c_fwd = prof["fwd_out"]
    achieved = fwd_bytes / (t_fwd / 1e3) / 1e9
    tot_ph = sum(v[0] for v in prof.values())
    phase_share = {k: round(v[0] / max(tot_ph, 1e-9), 4) for k, v in prof.items()}
    explicit_diff = float(np.max(np.abs(q_explicit - q_grouped)))
    if rank != 0:
        return
    line = {
        "metric": "string Newton iterations/s (320 strings, grouped)", "value": value,
        "unit": "iterations/s", "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": ms / K,
        "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None,
        "dtype": {"tf32": "tf32", "bf16": "bf16", "bf16x3": "bf16x3"}[args.prec],
        "data": "synthetic",
        "config": {"workload": "%d strings, depth-8 decoders r-32-64-128-256-256-256-256-3V, "
                               "r ~ U{3..15}, V ~ U[200,2000], 2x2xV/4 grids, StVK, 32 cubature "
                               "tets each; one implicit-Euler Newton step of every string per "
                               "step" % args.n_strings, "params_total": int(sum(params)),
                   "evals_per_step": ev_all, "max_evals": max_ev,
                   "parallelism": ("strings sharded over %d ranks by P*(4r+4), longest "
                                   "first; rank 0 holds %d" % (world, len(mine)))
                   if world > 1 else "single GPU",
                   "l2": "weights %.2f GB > L2%s" % (sum(params) * bpe / 1e9,
                                                      " (rank 0)" if world > 1 else ""),
                   "synth_seconds": round(t_gen, 1)},
        "per_string_launches": {"ms_per_step": ms_single, "value": ev_step / (ms_single / 1e3),
                                "grouped_speedup": ms_single / (ms_rank / K),
                                "max_rel_diff_vs_grouped": diff},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                     "kernel": "grouped forward chain (k_chain, all strings' 8 layers as stages)",
                     "peak_source": "%s hbm_gbs" % peak_src,
                     "avg_launch_ms": t_fwd / max(c_fwd, 1), "launches": c_fwd,
                     "algorithmic_bytes_per_step": fwd_bytes},
        "whole_step_weight_gbs": step_gbs,
        "phase_share": phase_share, "explicit_vs_graph_max_abs_diff": explicit_diff,
        "clocks": clocks, "gpu_launches": int(launches_step * K),
    }
    if not emit:
        return line
    print(json.dumps(line))


# ------------------------------------------------------ cubature |C| sweep --
def cubature_bytes(n_cub, r):
    """Algorithmic bytes of one cubature launch (k_cubature): per tet the decoded u and
    the r columns of J at its 12 DOFs, its 4 vertex ids, Dm^-1 (9 floats), rest volume,
    id and weight read, and its weighted force and DOF ids (12 + 12, read again by
    W_L^T a) written.  The block-summed J_e^T f_e / J_e^T K_e J_e partials (one row of
    r + r(r+1)/2 words and one energy per block of tets) are not counted."""
    read = 12 * 4 * (1 + r) + 4 * 4 + 9 * 4 + 4 + 4 + 4
    write = 12 * 4 + 12 * 4
    return n_cub * (read + write)


def run_cubsweep(args):
    """Achieved HBM bandwidth of the cubature kernel against the cubature set size on the
    paper-scale mesh (20 x 20 x 50 grid, 88445 tets, Neo-Hookean, latent 30): the
    decoder is the paper's latent and output widths with one hidden layer of 256 (the
    cubature kernel sees only u and J at the cubature DOFs), bias-free, at a latent
    near rest.  Each size: one warm-up dae_assemble_reduced, then CUDA events around
    every cubature launch of ``--steps`` more."""
    import torch
    from paper_2102_11026_gb300 import dae, synth
    torch.cuda.set_device(0)
    sizes = [int(x) for x in args.cub_sizes.split(",") if x]
    seed = 2
    dec_w = synth.make_decoder([30, 256, 60000], seed, "tanh", bias=False)
    mesh_w = synth.make_grid_mesh(20, 20, 50, seed, "neohookean", 5e5, 0.45)
    if max(sizes) > mesh_w.n_tet:
        raise SystemExit("|C| > %d tets" % mesh_w.n_tet)
    stream = torch.cuda.Stream()
    ctx = dae.dae_create(0, stream.cuda_stream)
    dec = dae.dae_load_decoder(ctx, dec_w.widths, dec_w.W, dec_w.b, dec_w.act, args.prec)
    mesh = dae.dae_load_mesh(ctx, mesh_w.X.reshape(-1), mesh_w.tets.reshape(-1), mesh_w.vmass,
                             mesh_w.material, mesh_w.E, mesh_w.nu)
    rng = np.random.default_rng(seed)
    r = dec_w.r
    q = rng.normal(0.0, 0.05, r)
    qbar = np.zeros(r)
    qdot = np.zeros(r)
    dt = 1.0 / 60.0
    f_ext = synth.gravity_force(mesh_w.vmass)
    phi, A, en = np.zeros(r), np.zeros(r * r), np.zeros(1)
    peaks, peak_src = load_peaks()
    rows = []
    with torch.cuda.stream(stream):
        for C in sizes:
            cub, w = synth.make_cubature(mesh_w.n_tet, C, seed)
            ct = torch.as_tensor(cub, device="cuda")
            cw = torch.as_tensor(w, device="cuda")
            dae.dae_assemble_reduced(ctx, dec, mesh, ct, cw, q, qbar, qdot, dt, f_ext, phi, A, en)
            dae.dae_profile_read(ctx)
            dae.dae_profile_enable(ctx, ["cubature"])
            for _ in range(args.steps):
                dae.dae_assemble_reduced(ctx, dec, mesh, ct, cw, q, qbar, qdot, dt, f_ext, phi, A,
                                         en)
            dae.dae_profile_enable(ctx, False)
            t, c = dae.dae_profile_read(ctx)["cubature"]
            us = 1e3 * t / max(c, 1)
            b = cubature_bytes(C, r)
            gbs = b / (us / 1e6) / 1e9
            rows.append({"n_cub": C, "us_per_launch": round(us, 2), "launches": c,
                         "algorithmic_bytes": b, "gbs": round(gbs, 1),
                         "frac": round(gbs / peaks["hbm_gbs"], 4),
                         "energy": float(en[0])})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    dae.dae_free_decoder(dec)
    dae.dae_free_mesh(mesh)
    dae.dae_destroy(ctx)
    print(json.dumps({
        "metric": "cubature kernel achieved GB/s vs |C|", "unit": "GB/s",
        "dtype": {"tf32": "tf32", "bf16": "bf16", "bf16x3": "bf16x3", "fp32": "f32"}[args.prec],
        "data": "synthetic",
        "config": {"workload": "20x20x50 grid (88445 tets, Neo-Hookean E=5e5 nu=0.45), "
                               "decoder 30-256-60000 bias-free, q ~ N(0, 0.05^2)",
                   "launches_per_size": args.steps},
        "peak": peaks["hbm_gbs"], "peak_source": "%s hbm_gbs" % peak_src, "sweep": rows}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "train":
        run_train(args)
    elif args.mode == "strings":
        run_strings(args)
    elif args.mode == "cubsweep":
        run_cubsweep(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
