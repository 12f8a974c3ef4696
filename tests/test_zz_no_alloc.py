"""The allocation-free row reductions (dae_reduce_rows_noalloc) give the same sums
as dae_assemble_reduced, on two calls in a row.  Kept in a file that pytest
collects last."""
import numpy as np
import pytest

from paper_2102_11026_gb300 import dae, synth
from gpu_harness import Gpu, relerr, TOL_FP32_FIRST, TOL_FP32_HIGHER

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["small", "gravity"])
def test_no_alloc_rows_match_assemble(name):
    import torch
    if name == "small":
        wl = synth.small()
    else:
        wl = synth.custom([9, 40, 72, 360], (4, 5, 6), 24, 5, "tanh", "neohookean", 1e4, 0.35, True)
    wl.cub_tets = wl.cub_tets[:0]          # no cubature: phi = J^T a_dense
    wl.cub_w = wl.cub_w[:0]
    g = Gpu(wl)
    try:
        st = wl.state
        r, N = wl.dec.r, wl.dec.n_out
        q = synth.newton_start(st) + 0.03 * np.random.default_rng(4).normal(size=r)
        ref = g.reduced(q)
        dev = lambda x, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(x), dtype=dt,
                                                          device="cuda")
        J = torch.zeros(r * N, dtype=torch.float32, device="cuda")
        dJ = torch.zeros(r * N, dtype=torch.float32, device="cuda")
        Hqq = torch.zeros(N, dtype=torch.float32, device="cuda")
        dae.dae_eval_derivs(g.ctx, g.dec, q, st.qbar, st.qbar_dot, st.dt, J=J, dJ=dJ, Hqq=Hqq)
        dae.dae_sync(g.ctx)
        HDD = Hqq * (st.dt ** 2)
        z = dev((q - st.qbar) - st.dt * st.qbar_dot)
        mdof = dev(np.repeat(wl.mesh.vmass, 3))
        f_ext = dev(wl.f_ext)
        outs = []
        for _ in range(2):
            phi = torch.full((r,), np.nan, dtype=torch.float64, device="cuda")
            Mr = torch.full((r * r,), np.nan, dtype=torch.float64, device="cuda")
            B = torch.full((r * r,), np.nan, dtype=torch.float64, device="cuda")
            dae.dae_reduce_rows_noalloc(N, r, J, dJ, HDD, mdof, f_ext, z, st.dt, phi, Mr, B)
            torch.cuda.synchronize()
            outs.append((phi.cpu().numpy(), Mr.cpu().numpy().reshape(r, r).T,
                         B.cpu().numpy().reshape(r, r).T))
        for phi, Mr, B in outs:
            assert relerr(Mr, ref["Mr"]) <= TOL_FP32_FIRST
            assert relerr(B, ref["B"]) <= TOL_FP32_HIGHER
            assert relerr(phi, ref["phi"]) <= TOL_FP32_HIGHER
        assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    finally:
        g.close()


def test_no_alloc_rejects_oversized_problems():
    with pytest.raises(dae.DaeError) as e:
        # 200 000 rows at r = 32 need more partials than the fixed array holds
        dae.dae_reduce_rows_noalloc(200000, 32, 1, 1, 1, 1, None, 1, 0.01, 1, 1, 1)
    assert e.value.status == -1
