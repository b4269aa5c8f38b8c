"""The padded population layout: 27 slabs of ns >= N elements (N rounded up
to 64, plus a pad that keeps the slabs from starting at addresses with equal
low bits).  The pad is a storage choice, so every result must be the same
bit for bit whatever it is: populations after several steps (both AA forms),
the raw state the host sees (27 N unpadded elements), the reductions, and a
context on a caller's buffer of exactly 27 N elements (unpadded slabs, as an
ensemble replica or a caller without the pad uses) -- and all of them must
match the FP64 oracle to the FP32 tolerance of the other parity tests
(2e-6 per step)."""
import ctypes as C

import numpy as np
import pytest

from synth import inputs

pytestmark = pytest.mark.gpu

PADS = ["0", "2048", "1048576"]


@pytest.fixture(scope="module")
def F():
    from paper_2601_03806_gb300 import flbm
    return flbm


def _f0(O, nx, ny, nz, seed):
    w = O.tables()["w"]
    return w[:, None, None, None] * (1.0 + 0.02 * inputs.population_perturbation(nx, ny, nz, seed))


def _run(F, shape, precision, f0, steps, monkeypatch, pad, torch_memory):
    monkeypatch.setenv("FLBM_SLAB_PAD", pad)
    nx, ny, nz = shape
    with F.Lattice(nx, ny, nz, 0.7, 1e-4, seed=9, precision=precision, torch_memory=torch_memory) as g:
        g.set_populations(f0)
        g.step(steps)
        out = (g.get_populations(), g.get_state(), g.stats())
        # raw state round trip: what get_state gives, set_state takes back
        raw = out[1].copy()
        g.set_state(raw)
        assert np.array_equal(g.get_state(), raw)
    return out


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("shape,steps", [((64, 5, 3), 3), ((130, 3, 2), 4), ((512, 3, 2), 5)])
def test_pad_is_invisible(F, oracle_mod, monkeypatch, precision, shape, steps):
    nx, ny, nz = shape
    f0 = _f0(oracle_mod, nx, ny, nz, seed=nx + ny)
    ref = None
    for pad in PADS:
        for tm in (False, True):
            res = _run(F, shape, precision, f0, steps, monkeypatch, pad, tm)
            if ref is None:
                ref = res
                continue
            assert np.array_equal(res[0], ref[0]), (pad, tm)
            assert np.array_equal(res[1], ref[1]), (pad, tm)
            for k in ("mass", "u2", "m_var"):
                assert np.array_equal(np.asarray(res[2][k]), np.asarray(ref[2][k])), (pad, tm, k)
    o = oracle_mod.Box(nx, ny, nz, 0.7, 1e-4, seed=9)
    o.set_f(f0)
    o.step(steps)
    tol = {0: 1e-12, 1: 2e-6, 2: 2e-5}[precision] * steps
    assert np.abs(ref[0] - o.get_f()).max() < tol


def test_exact_size_caller_buffer_is_unpadded(F, oracle_mod, monkeypatch):
    """flbm_create_ex on a buffer of exactly 27 N FP32 elements keeps the
    slabs unpadded (slot i of node n at element i N + n) and steps like a
    padded context."""
    import torch

    monkeypatch.setenv("FLBM_SLAB_PAD", "1048576")
    nx, ny, nz = 64, 4, 3
    n = nx * ny * nz
    f0 = _f0(oracle_mod, nx, ny, nz, seed=3)
    p = F.make_params(nx, ny, nz, 0.7, 1e-4, seed=9)
    assert F.flbm_state_bytes(C.byref(p)) > 27 * n * 4     # the padded size
    buf = torch.empty(27 * n, dtype=torch.float32, device="cuda")
    h = C.c_void_p()
    stream = torch.cuda.current_stream()
    rc = F.flbm_create_ex(C.byref(p), C.c_void_p(buf.data_ptr()), 27 * n * 4,
                          C.c_void_p(stream.cuda_stream), C.byref(h))
    assert rc == F.FLBM_OK, F.flbm_last_error(None)
    try:
        ff = np.ascontiguousarray(f0, np.float64)
        assert F.lib.flbm_set_populations(h, ff.ctypes.data_as(C.c_void_p)) == F.FLBM_OK
        torch.cuda.synchronize()
        # natural form, unpadded: deviations g_i = f_i - w_i at element i N + n
        w = oracle_mod.tables()["w"]
        dev = (f0 - w[:, None, None, None]).reshape(27, n)
        assert np.abs(buf.view(27, n).cpu().numpy() - dev).max() < 1e-7
        assert F.lib.flbm_step(h, 4) == F.FLBM_OK
        got = np.empty((27, nz, ny, nx))
        assert F.lib.flbm_get_populations(h, got.ctypes.data_as(C.c_void_p)) == F.FLBM_OK
    finally:
        F.lib.flbm_destroy(h)
    with F.Lattice(nx, ny, nz, 0.7, 1e-4, seed=9) as g:
        g.set_populations(f0)
        g.step(4)
        assert np.array_equal(got, g.get_populations())


def test_too_small_caller_buffer_is_refused(F, monkeypatch):
    import torch

    monkeypatch.delenv("FLBM_SLAB_PAD", raising=False)
    nx, ny, nz = 64, 4, 3
    n = nx * ny * nz
    p = F.make_params(nx, ny, nz, 0.7, 1e-4)
    buf = torch.empty(27 * n - 64, dtype=torch.float32, device="cuda")
    h = C.c_void_p()
    rc = F.flbm_create_ex(C.byref(p), C.c_void_p(buf.data_ptr()), (27 * n - 64) * 4, None, C.byref(h))
    assert rc == F.FLBM_E_NOMEM
    assert not h.value
