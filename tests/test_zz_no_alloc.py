"""flbm_step_noalloc against flbm_step.

Callers whose own allocator owns all device memory cannot let a library call
cudaMalloc; flbm_step_noalloc gives them the same fused step with its scratch
in a static device array.  On the same input, two calls in a row (one from
each AA storage form) must reproduce flbm_step + flbm_stats: the populations
bit for bit (same kernels, same launch shape) and the reduction results
within the tolerance of the other GPU tests.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(64, 6, 5), (30, 4, 3)])   # row pipeline / direct kernel
def test_noalloc_step_matches_flbm_step(shape):
    import torch

    import oracle
    from paper_2601_03806_gb300 import flbm
    from synth import inputs

    nx, ny, nz = shape
    n = nx * ny * nz
    w = oracle.tables()["w"]
    f0 = w[:, None, None, None] * (1 + 0.02 * inputs.population_perturbation(nx, ny, nz, 11))
    ref = flbm.Lattice(nx, ny, nz, 0.7, 1e-4, seed=5, precision=flbm.FLBM_FP32, stats_every=1,
                       torch_memory=True)
    ref.set_populations(f0)
    torch.cuda.synchronize()
    state = ref._buf.clone()          # the caller's own copy of the raw state
    sums = torch.zeros(13, dtype=torch.float64, device="cuda")
    stream = ref.stream.cuda_stream
    for t in range(2):
        rc = flbm.flbm_step_noalloc(C.byref(ref.params), C.c_void_p(state.data_ptr()), t, t % 2,
                                    C.c_void_p(sums.data_ptr()), C.c_void_p(stream))
        assert rc == flbm.FLBM_OK, flbm.flbm_last_error(None)
        ref.step(1)
        torch.cuda.synchronize()
        assert torch.equal(state, ref._buf), t
        st = ref.stats()
        s = sums.cpu().numpy()
        assert st["step"] == t
        assert abs((n * 1.0 + s[0]) - st["mass"]) <= 1e-12 * n
        assert np.allclose(s[1:4], st["mom"], rtol=1e-12, atol=1e-15)
        assert np.allclose(s[4:7] / n, st["u2"], rtol=1e-12, atol=0)
    ref.close()
