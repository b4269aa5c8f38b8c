"""C-ABI checks that need no GPU: the library loads, exports every function
include/flbm.h declares, the ctypes structures match the C layout, and
argument validation rejects bad input before touching the device."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "flbm.h")


@pytest.fixture(scope="module")
def F():
    from paper_2601_03806_gb300 import build
    build.build()
    from paper_2601_03806_gb300 import flbm
    return flbm


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(flbm_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(F):
    names = declared_functions()
    assert len(names) >= 19
    out = subprocess.run(["nm", "-D", "--defined-only", F.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(flbm_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(F, n), n          # same-name binding


def test_struct_layout_matches_header(F, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "flbm.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(flbm_params), offsetof(flbm_params, tau),
         offsetof(flbm_params, seed), sizeof(flbm_stats_t), offsetof(flbm_stats_t, er),
         offsetof(flbm_params, state_form));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    assert vals == [C.sizeof(F.flbm_params), F.flbm_params.tau.offset, F.flbm_params.seed.offset,
                    C.sizeof(F.flbm_stats_t), F.flbm_stats_t.er.offset, F.flbm_params.state_form.offset]


@pytest.mark.parametrize("kw,code", [
    (dict(tau=0.5), -1), (dict(tau=0.3), -1), (dict(kT=-1e-5), -1), (dict(rho0=0.0), -1),
    (dict(nx=0), -1), (dict(scheme=7), -1), (dict(precision=3), -1), (dict(stats_every=-1), -1),
    (dict(tau=float("nan")), -1),
])
def test_validation_before_device(F, kw, code):
    args = dict(nx=8, ny=8, nz=8, tau=0.8, kT=1e-5, rho0=1.0, seed=1, scheme=1, precision=1,
                stats_every=1)
    args.update(kw)
    p = F.make_params(args["nx"], args["ny"], args["nz"], args["tau"], args["kT"], args["rho0"],
                      args["seed"], args["scheme"], args["precision"], False, args["stats_every"])
    h = C.c_void_p()
    rc = F.flbm_create_ex(C.byref(p), None, 0, None, C.byref(h))
    assert rc == code
    assert not h.value
    assert F.flbm_last_error(None)


@pytest.mark.parametrize("kw,step,parity,code", [
    (dict(noise_stream=1 << 24), 0, 0, -1), (dict(noise_stream=-1), 0, 0, -1),
    (dict(tau=float("inf")), 0, 0, -1), (dict(kT=float("nan")), 0, 0, -1),
    (dict(rho0=float("inf")), 0, 0, -1), (dict(nx=1 << 14, ny=1 << 14, nz=1 << 12), 0, 0, -1),
    (dict(), -1, 0, -1), (dict(), 0, 2, -1),
    (dict(precision=2), 0, 0, -6), (dict(precision=0), 0, 0, -6), (dict(scheme=3), 0, 0, -6),
    (dict(state_form=1), 0, 0, -6),
])
def test_noalloc_validation_before_device(F, kw, step, parity, code):
    """flbm_step_noalloc checks its parameters as flbm_create does (noise
    stream range, finite tau / kT / rho0, box size) and rejects the storage
    forms and schemes it does not serve, all before any CUDA call: the
    pointers passed here are never dereferenced."""
    args = dict(nx=8, ny=8, nz=8, tau=0.8, kT=1e-5, rho0=1.0, seed=1, scheme=1, precision=1,
                noise_stream=0, state_form=0)
    args.update(kw)
    p = F.make_params(args["nx"], args["ny"], args["nz"], args["tau"], args["kT"], args["rho0"],
                      args["seed"], args["scheme"], args["precision"], False, 1,
                      noise_stream=args["noise_stream"], state_form=args["state_form"])
    rc = F.flbm_step_noalloc(C.byref(p), C.c_void_p(256), step, parity, C.c_void_p(256), None)
    assert rc == code
    assert F.flbm_last_error(None)


def _slab_stride(F, p, es):
    nbytes = F.flbm_state_bytes(C.byref(p))
    assert nbytes % (27 * es) == 0
    return nbytes // (27 * es)


@pytest.mark.parametrize("pad", [None, "0", "2048", "1048576"])
def test_state_bytes_and_params(F, pad, monkeypatch):
    """27 slabs of ns elements: N rounded up to 64 elements, plus 1 MiB for
    slabs of 32 MiB and more, or the FLBM_SLAB_PAD bytes when that is set; a
    pad that is no multiple of 128 bytes is ignored."""
    if pad is None:
        monkeypatch.delenv("FLBM_SLAB_PAD", raising=False)
    else:
        monkeypatch.setenv("FLBM_SLAB_PAD", pad)
    for (nx, ny, nz), prec, es in (((512, 512, 512), 1, 4), ((16, 16, 16), 0, 8), ((130, 3, 2), 2, 2)):
        p = F.make_params(nx, ny, nz, 0.8, 1e-4, precision=prec)
        n = nx * ny * nz
        ns = _slab_stride(F, p, es)
        if pad is None:
            # 1 MiB pad for slabs of 32 MiB and more, none below
            big = n * es >= 32 << 20
            assert ns == (n + 63) // 64 * 64 + ((1 << 20) // es if big else 0)
        else:
            assert ns == (n + 63) // 64 * 64 + int(pad) // es
    monkeypatch.setenv("FLBM_SLAB_PAD", "100")
    p = F.make_params(64, 4, 4, 0.8, 1e-4)
    monkeypatch.delenv("FLBM_SLAB_PAD")
    ns_default = _slab_stride(F, p, 4)
    monkeypatch.setenv("FLBM_SLAB_PAD", "100")
    assert _slab_stride(F, p, 4) == ns_default
    p.tau = 0.4
    assert F.flbm_state_bytes(C.byref(p)) == 0


def test_tuning_struct_layout(F, tmp_path):
    src = tmp_path / "tl.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "flbm.h"
int main(void) {
  printf("%zu %zu\\n", sizeof(flbm_ensemble_tuning), offsetof(flbm_ensemble_tuning, ms_per_step));
  return 0;
}
""")
    exe = tmp_path / "tl"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    assert vals == [C.sizeof(F.flbm_ensemble_tuning), F.flbm_ensemble_tuning.ms_per_step.offset]


def _ens_params(F, n, changes):
    ps = []
    for r in range(n):
        p = F.make_params(32, 4, 2, 0.8, 1e-5, seed=3, noise_stream=r)
        for k, v in changes.get(r, {}).items():
            setattr(p, k, v)
        ps.append(p)
    return ps


@pytest.mark.parametrize("kw,count,code", [
    ({1: dict(seed=4)}, 2, -1),             # one Philox key per ensemble
    ({1: dict(noise_stream=0)}, 2, -1),     # streams must be distinct
    ({0: dict(nx=48)}, 2, -1),              # nx multiple of 32
    ({1: dict(scheme=0)}, 2, -1),
    ({1: dict(stats_every=2)}, 2, -1),
    ({0: dict(tau=0.5)}, 1, -1),
    ({0: dict(noise_stream=1 << 24)}, 1, -1),
    ({0: dict(nx=4096)}, 1, -1),            # two stages of 27 rows exceed shared memory
    ({0: dict(precision=0), 1: dict(precision=0)}, 2, -6),
    ({}, 0, -1),
])
def test_ensemble_validation_before_device(F, kw, count, code):
    ps = _ens_params(F, max(count, 1), kw)
    arr = (F.flbm_params * len(ps))(*ps)
    e = C.c_void_p()
    rc = F.flbm_ensemble_create(arr, count, None, C.byref(e))
    assert rc == code
    assert not e.value
    assert F.flbm_ensemble_last_error(None)


@pytest.mark.parametrize("scheme,precision,form", [
    (0, 1, 1),     # BGK's ghosts keep a memory: no moment state
    (3, 1, 1),     # nor the learned collision
    (1, 0, 1),     # FP32 only
    (2, 2, 1),
    (1, 1, 2),     # unknown form
    (1, 1, -1),
])
def test_state_form_is_validated(F, scheme, precision, form):
    p = F.make_params(8, 8, 8, 0.8, 1e-5, scheme=scheme, precision=precision, state_form=form)
    h = C.c_void_p()
    assert F.flbm_create_ex(C.byref(p), None, 0, None, C.byref(h)) == F.FLBM_E_INVALID
    assert not h.value
    assert b"state_form" in F.flbm_last_error(None) or b"moment-state" in F.flbm_last_error(None)
    ps = _ens_params(F, 2, {1: dict(state_form=1)})
    arr = (F.flbm_params * 2)(*ps)
    e = C.c_void_p()
    assert F.flbm_ensemble_create(arr, 2, None, C.byref(e)) == F.FLBM_E_INVALID
    assert not e.value


def test_noise_stream_is_validated(F):
    p = F.make_params(8, 8, 8, 0.8, 1e-5, noise_stream=-1)
    h = C.c_void_p()
    assert F.flbm_create_ex(C.byref(p), None, 0, None, C.byref(h)) == -1
    assert b"noise_stream" in F.flbm_last_error(None)


def test_null_ensemble_calls_are_rejected(F):
    assert F.flbm_ensemble_step(None, 1) == F.FLBM_E_INVALID
    assert F.flbm_ensemble_count(None) == -1
    assert F.flbm_ensemble_get_step(None) == -1
    assert F.flbm_ensemble_graph(None, 1) == F.FLBM_E_INVALID
    assert F.flbm_ensemble_autotune(None, 1, None) == F.FLBM_E_INVALID
    F.flbm_ensemble_destroy(None)


def test_null_context_calls_are_rejected(F):
    assert F.flbm_step(None, 1) == F.FLBM_E_INVALID
    assert F.flbm_get_step(None) == -1
    assert F.flbm_stats_reset(None) == F.FLBM_E_INVALID
    F.flbm_destroy(None)


def test_mlp_calls_reject_host_pointers(F):
    """Device-array arguments must be device memory: a host array is
    rejected before any kernel could fault on it (the query needs no GPU:
    without a device it fails, which is rejected the same way)."""
    import numpy as np
    p = np.zeros(F.MLP_NPARAM, np.float32)
    x = np.zeros((4, 28), np.float32)
    t = np.zeros((4, 27), np.float32)
    g = np.zeros(F.MLP_NPARAM, np.float32)
    ptr = lambda a: a.ctypes.data_as(C.c_void_p)
    assert F.flbm_mlp_grad(ptr(p), ptr(x), ptr(t), 4, ptr(g), None) == F.FLBM_E_INVALID
    assert F.flbm_mlp_train(ptr(p), ptr(x), ptr(t), 4, 1, 4, 1e-3, 0, None) == F.FLBM_E_INVALID
    assert b"device" in F.flbm_last_error(None)
