"""Failure detection on the GPU without a GPU fault.

* Instability: a non-finite population injected from the host is reported
  as FLBM_E_UNSTABLE (tests/test_gpu_parity.py).
* Bounded waits: the TMA row pipeline's mbarrier waits give up after half a
  second to a second.  FLBM_INJECT_STARVE=1 makes a context's row pipeline
  expect 16 bytes more than it copies, so the "full" barrier never
  completes; the wait must run out, the step must return FLBM_E_TIMEOUT, and
  the device must stay usable for the next context.  Both row kernels: one
  node per thread (64-wide rows) and two (256-wide rows, FP32 and FP16).
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nx,precision", [(64, 1), (256, 1), (256, 2)])
def test_row_pipeline_wait_runs_out_and_reports_timeout(monkeypatch, nx, precision):
    from paper_2601_03806_gb300 import flbm
    monkeypatch.setenv("FLBM_INJECT_STARVE", "1")
    g = flbm.Lattice(nx, 4, 3, 0.8, 1e-5, precision=precision)
    monkeypatch.delenv("FLBM_INJECT_STARVE")
    t0 = time.time()
    with pytest.raises(flbm.FlbmError) as ei:
        g.step(1)
    assert ei.value.code == flbm.FLBM_E_TIMEOUT
    assert time.time() - t0 < 30
    g.close()
    # the device and the library stay usable
    h = flbm.Lattice(nx, 4, 3, 0.8, 1e-5, precision=precision)
    h.step(3)
    assert abs(h.stats()["mass"] / (nx * 4 * 3) - 1) < 1e-6


def test_learned_step_tensor_core_wait_runs_out_and_reports_timeout(monkeypatch):
    """FLBM_INJECT_STARVE=1 on a learned-scheme context: the issuer issues
    none of the network's first-layer MMAs and commits nothing, every
    group's bounded wait runs out (half a second to a second) with no
    tensor-core work in flight, the step returns FLBM_E_TIMEOUT and the
    device stays usable."""
    from paper_2601_03806_gb300 import flbm
    import numpy as np
    theta = np.zeros(flbm.MLP_NPARAM, np.float32)
    monkeypatch.setenv("FLBM_INJECT_STARVE", "1")
    g = flbm.Lattice(128, 4, 4, 0.8, 1e-4, scheme=flbm.FLBM_LEARNED)
    monkeypatch.delenv("FLBM_INJECT_STARVE")
    g.set_mlp(theta)
    t0 = time.time()
    with pytest.raises(flbm.FlbmError) as ei:
        g.step(1)
    assert ei.value.code == flbm.FLBM_E_TIMEOUT
    assert time.time() - t0 < 30
    g.close()
    h = flbm.Lattice(128, 4, 4, 0.8, 1e-4, scheme=flbm.FLBM_LEARNED)
    h.set_mlp(theta)
    h.init_thermal(2)
    h.step(3)
    assert abs(h.stats()["mass"] / (128 * 16) - 1) < 1e-2
