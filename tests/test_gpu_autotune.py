"""GPU tests of the layer chains' work decomposition: every candidate plan of a layer
(P = 1, 2, 4, 8 CTAs per 128-row tile, as a K split or as replicated K loops) must give
the same derivatives and reduced system as the FP64 oracle, on odd shapes with ragged
tiles; invalid plans are refused; the autotuner's plan keeps parity."""
import numpy as np
import pytest

import oracle
from paper_2102_11026_gb300 import dae, synth
from gpu_harness import Gpu, colerr, relerr

pytestmark = pytest.mark.gpu

TOLS = {"bf16x3": (1e-4, 1e-3), "tf32": (3e-3, 1e-2)}


def odd_workload(r, seed, hidden):
    return synth.custom([r, *hidden, 360], (4, 5, 6), 24, seed, "tanh", "stvk", 1e4, 0.35, False)


CASES = {
    "r32_deep": lambda: odd_workload(32, 9, (48, 64, 80, 96)),
    "r13_wide": lambda: odd_workload(13, 7, (200, 520, 300)),
    "small": lambda: synth.small(),
}


def sm_count():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


def candidates(widths, prec, direction, grid):
    """The candidates of every hidden layer l (network order): P CTAs per tile with
    tiles x P <= grid, replicated (1, P) or split (P, 1) with >= 2 k-blocks per CTA."""
    kb = 32 if prec == "tf32" else 64
    out = []
    for l in range(len(widths) - 2):
        n_in, n_out = widths[l], widths[l + 1]
        if direction == 0:
            tiles, nk = -(-n_out // 128), -(-n_in // 64) * 64 // kb
        else:
            tiles, nk = -(-n_in // 128), -(-n_out // 64) * 64 // kb
        c = []
        P = 1
        while P <= 8 and tiles * P <= grid:
            c.append((1, P))
            if P >= 2 and nk >= 2 * P:
                c.append((P, 1))
            P *= 2
        if tiles <= 8 and tiles * nk <= 64:
            c.append((1, 0))      # the whole layer on one CTA
        out.append(c)
    return out


def plans(cands, rng):
    """All P = 1; every small layer on one CTA (consecutive ones without grid barriers);
    the largest replication; the largest split where there is one; two seeded random
    mixes."""
    yield "p1", [(1, 1)] * len(cands)
    yield "solo", [(1, 0) if (1, 0) in cs else (1, 1) for cs in cands]
    yield "rep_max", [max((c for c in cs if c[0] == 1), key=lambda c: c[1]) for cs in cands]
    yield "split_max", [max(cs, key=lambda c: (c[0], c[1])) for cs in cands]
    for k in range(2):
        yield "mix%d" % k, [cs[rng.integers(len(cs))] for cs in cands]


@pytest.mark.parametrize("prec", list(TOLS))
@pytest.mark.parametrize("name", list(CASES))
def test_every_chain_plan_keeps_parity(name, prec):
    wl = CASES[name]()
    d = wl.dec
    grid = sm_count()
    q = synth.newton_start(wl.state) + 0.05 * np.random.default_rng(3).normal(size=d.r)
    ref = oracle.derivs(d, q, wl.state.qbar, wl.state.qbar_dot, wl.state.dt)
    rr = oracle.reduced_system(wl, q)
    q0n = synth.newton_start(wl.state)
    # a full Newton frame through both chains (the small workload converges in a few
    # steps; the odd shapes start far from rest and stop at max_iter, where FP32 rounding
    # differences grow along the iteration)
    newton = prec == "bf16x3" and name == "small"
    qo, _ = oracle.newton_solve(wl, q0=q0n, max_iter=5) if newton else (None, None)
    t1, t2 = TOLS[prec]
    g = Gpu(wl, prec)
    rng = np.random.default_rng(17)
    tried = 0
    try:
        cf = candidates(d.widths, prec, 0, grid)
        cr = candidates(d.widths, prec, 1, grid)
        for (nf, pf), (nr, pr) in zip(plans(cf, rng), plans(cr, rng)):
            dae.dae_decoder_set_chain_plan(g.ctx, g.dec, 0, [p[0] for p in pf], [p[1] for p in pf])
            dae.dae_decoder_set_chain_plan(g.ctx, g.dec, 1, [p[0] for p in pr], [p[1] for p in pr])
            s0, r0 = dae.dae_decoder_get_chain_plan(g.ctx, g.dec, len(d.W) - 1, 0)
            assert list(s0) == [p[0] for p in pf] and list(r0) == [p[1] for p in pf]
            if newton:
                qn, rep = g.newton(synth.newton_start(wl.state))
                assert rep.status == 0 and np.linalg.norm(qn - qo) <= 1e-3 * np.linalg.norm(qo - q0n), nf
            out = g.derivs(q, want=("u", "J", "Hqq", "dJ"))
            for k, t in (("u", t1), ("J", t1), ("Hqq", t2), ("dJ", t2)):
                assert colerr(out[k], ref[k]) <= t, (nf, k, colerr(out[k], ref[k]))
            rs = g.reduced(q)
            assert relerr(rs["phi"], rr["phi"]) <= t2, (nr, relerr(rs["phi"], rr["phi"]))
            assert relerr(rs["A"], rr["A"]) <= t2, (nr, relerr(rs["A"], rr["A"]))
            tried += 1
    finally:
        g.close()
    assert tried == 6


def test_invalid_plans_are_refused():
    wl = CASES["r32_deep"]()
    g = Gpu(wl, "bf16x3")
    try:
        n = len(wl.dec.W) - 1
        for split, rep in (([3] * n, [1] * n), ([2] * n, [2] * n), ([1] * n, [16] * n)):
            with pytest.raises(dae.DaeError) as e:
                dae.dae_decoder_set_chain_plan(g.ctx, g.dec, 0, split, rep)
            assert e.value.status == -1
        g32 = Gpu(wl, "fp32", ctx=g.ctx)
        try:
            with pytest.raises(dae.DaeError) as e:
                dae.dae_decoder_autotune(g.ctx, g32.dec)
            assert e.value.status == -9
        finally:
            dae.dae_free_decoder(g32.dec)
            dae.dae_free_mesh(g32.mesh)
    finally:
        g.close()


def test_autotuned_plan_keeps_parity_and_resets_with_precision():
    wl = CASES["r13_wide"]()
    d = wl.dec
    q0 = synth.newton_start(wl.state)
    qo, _ = oracle.newton_solve(wl, q0=q0, max_iter=5)
    g = Gpu(wl, "bf16x3")
    try:
        default = dae.dae_decoder_get_chain_plan(g.ctx, g.dec, len(d.W) - 1, 0)
        ms = dae.dae_decoder_autotune(g.ctx, g.dec, reps=10)
        assert ms[1] <= ms[0] and ms[3] <= ms[2] and min(ms) > 0
        q, rep = g.newton(q0)
        assert rep.status == 0
        assert np.linalg.norm(q - qo) <= 1e-3 * np.linalg.norm(qo - q0)
        # a precision change returns to the built-in plan
        dae.dae_decoder_set_precision(g.ctx, g.dec, "tf32")
        dae.dae_decoder_set_precision(g.ctx, g.dec, "bf16x3")
        again = dae.dae_decoder_get_chain_plan(g.ctx, g.dec, len(d.W) - 1, 0)
        assert np.array_equal(again[0], default[0]) and np.array_equal(again[1], default[1])
    finally:
        g.close()
