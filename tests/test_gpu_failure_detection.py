"""Failure detection without a GPU fault: device-side waits give up after their
limit and report DAE_ERR_TIMEOUT; the context stays usable afterwards.  Host-side
failures (bad indices, inverted tets) are covered in test_gpu_parity.py."""
import time

import numpy as np
import pytest

from paper_2102_11026_gb300 import dae, synth
from gpu_harness import Gpu, relerr

pytestmark = pytest.mark.gpu


def test_bounded_waits_give_up_and_context_survives():
    wl = synth.custom([5, 32, 48, 3 * 60], (3, 4, 5), 8, 2)
    g = Gpu(wl, "bf16x3")
    try:
        q = synth.newton_start(wl.state)
        before = g.reduced(q)
        t0 = time.time()
        dae.dae_selftest_bounded_waits(g.ctx)       # raises unless both waits timed out
        took = time.time() - t0
        assert 3.5 < took < 30.0                    # two 2 s limits, not a hang
        after = g.reduced(q)                        # same context, same results
        assert np.array_equal(before["A"], after["A"])
    finally:
        g.close()
