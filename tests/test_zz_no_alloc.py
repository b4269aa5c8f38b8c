"""flbm_step_noalloc against flbm_step and against the oracle.

Callers whose own allocator owns all device memory cannot let a library call
cudaMalloc; flbm_step_noalloc gives them the same fused step with its scratch
in a static device array.  On the same input, two calls in a row (one from
each AA storage form) must reproduce flbm_step + flbm_stats: the populations
bit for bit (same kernels, same launch shape) and all 13 reduction sums
within 1e-12 relative (the same FP64 partials, summed in the same order).
Against the FP64 oracle the step is held to the FP32 tolerances of the other
GPU tests: populations within 2e-6 per step, and the sums within the FP32
reduction bound of reduction_sums.py.  The scratch array keeps the last
call's contents, so a call after an unstable one must start from clear flags.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

import reduction_sums as R

pytestmark = pytest.mark.gpu

NAMES = R.NAMES


def _sums_from_stats(st, n, rho0):
    """The 13 sums of one reduced step (after flbm_stats_reset) recovered from
    the flbm_stats fields."""
    mean = np.array(st["m_mean"])
    sq = (np.array(st["m_var"]) + mean ** 2) * n
    return np.array([st["mass"] - n * rho0, *st["mom"], *(np.array(st["u2"]) * n),
                     mean[2] * n, mean[3] * n, *sq])


def _slabs(flbm, lat, n):
    """The context's 27 population slabs (FP32) as a [27, n] view of its
    torch buffer, whose slab stride flbm_state_bytes gives."""
    import torch
    ns = int(flbm.flbm_state_bytes(C.byref(lat.params))) // (27 * 4)
    return lat._buf.view(torch.float32).view(27, ns)[:, :n]


def _call(flbm, params, state, t, sums, stream):
    return flbm.flbm_step_noalloc(C.byref(params), C.c_void_p(state.data_ptr()), t, t % 2,
                                  C.c_void_p(sums.data_ptr()), C.c_void_p(stream))


@pytest.mark.parametrize("scheme", [0, 1, 2])
@pytest.mark.parametrize("shape", [(64, 6, 5), (30, 4, 3)])   # row pipeline / direct kernel
def test_noalloc_step_matches_flbm_step_and_oracle(oracle_mod, scheme, shape):
    import torch

    from paper_2601_03806_gb300 import flbm
    from synth import inputs

    nx, ny, nz = shape
    n = nx * ny * nz
    tau, kT, seed, rho0 = 0.7, 1e-4, 5, 1.0
    w = oracle_mod.tables()["w"]
    f0 = w[:, None, None, None] * (rho0 + 0.02 * inputs.population_perturbation(nx, ny, nz, 11))
    ref = flbm.Lattice(nx, ny, nz, tau, kT, rho0=rho0, seed=seed, scheme=scheme,
                       precision=flbm.FLBM_FP32, stats_every=1, torch_memory=True)
    ref.set_populations(f0)
    torch.cuda.synchronize()
    state = _slabs(flbm, ref, n).clone(memory_format=torch.contiguous_format)   # the caller's own 27 unpadded slabs
    sums = torch.zeros(13, dtype=torch.float64, device="cuda")
    stream = ref.stream.cuda_stream
    box = oracle_mod.Box(nx, ny, nz, tau, kT, rho0=rho0, seed=seed, scheme=scheme)
    box.set_f(f0)
    m = R.nodes_per_thread_bound(nx, ny, nz)
    for t in range(2):
        pre = ref.get_populations()   # pre-collision state at t (equal to the caller's copy)
        S_or, B_or = R.sums_and_bounds(oracle_mod, pre, rho0, m)
        rc = _call(flbm, ref.params, state, t, sums, stream)
        assert rc == flbm.FLBM_OK, flbm.flbm_last_error(None)
        ref.stats_reset()
        ref.step(1)
        box.step(1)
        torch.cuda.synchronize()
        assert torch.equal(state, _slabs(flbm, ref, n)), t
        st = ref.stats()
        assert st["step"] == t
        s = sums.cpu().numpy()
        s_ref = _sums_from_stats(st, n, rho0)
        scale = np.abs(s_ref) + 1e-30
        assert np.all(np.abs(s - s_ref) <= 1e-12 * scale + 1e-12 * (np.abs(s_ref[9:]).max())), \
            dict(zip(NAMES, np.abs(s - s_ref)))
        # against the oracle: the sums of the same pre-collision state ...
        assert np.all(np.abs(s - S_or) <= B_or), dict(zip(NAMES, np.abs(s - S_or) / B_or))
        # ... and the post-collision populations of the oracle's own step
        assert np.abs(ref.get_populations() - box.get_f()).max() < 2e-6 * (t + 1)
    ref.close()


def test_noalloc_flags_cleared_between_calls(oracle_mod):
    """A NaN in the caller's state makes the call return FLBM_E_UNSTABLE; the
    next call, on a clean state, returns FLBM_OK: every call clears the
    flags the shared scratch array kept from the previous one."""
    import torch

    from paper_2601_03806_gb300 import flbm

    nx, ny, nz = 64, 6, 5
    w = oracle_mod.tables()["w"]
    f0 = np.broadcast_to(w[:, None, None, None], (27, nz, ny, nx)).copy()
    ref = flbm.Lattice(nx, ny, nz, 0.8, 1e-4, seed=2, precision=flbm.FLBM_FP32, stats_every=1,
                       torch_memory=True)
    ref.set_populations(f0)
    torch.cuda.synchronize()
    clean = _slabs(flbm, ref, nx * ny * nz).clone(memory_format=torch.contiguous_format)
    sums = torch.zeros(13, dtype=torch.float64, device="cuda")
    stream = ref.stream.cuda_stream
    bad = clean.clone()
    bad[5, 77] = float("nan")
    assert _call(flbm, ref.params, bad, 0, sums, stream) == flbm.FLBM_E_UNSTABLE
    assert _call(flbm, ref.params, clean.clone(), 0, sums, stream) == flbm.FLBM_OK
    torch.cuda.synchronize()
    assert abs(sums[0].item()) < 1e-9                 # rest state: no mass deviation
    ref.close()
