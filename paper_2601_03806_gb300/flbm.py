"""Thin ctypes binding of libflbm.so (include/flbm.h), same names as the C ABI.

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch is optional plumbing: ``Lattice(..., torch_memory=True)``
lets torch own the population buffer and the CUDA stream.

If the shared library is missing this module raises at import time; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libflbm.so")

FLBM_BGK, FLBM_GMF, FLBM_REG, FLBM_LEARNED = 0, 1, 2, 3
FLBM_FP64, FLBM_FP32, FLBM_FP16 = 0, 1, 2
FLBM_OK, FLBM_E_INVALID, FLBM_E_NOMEM, FLBM_E_CUDA = 0, -1, -2, -3
FLBM_E_UNSTABLE, FLBM_E_TIMEOUT, FLBM_E_UNSUPPORTED = -4, -5, -6
(FLBM_OBS_RHO, FLBM_OBS_JSUM, FLBM_OBS_PI_DIAG, FLBM_OBS_PI_OFFDIAG,
 FLBM_OBS_JX, FLBM_OBS_JY, FLBM_OBS_JZ) = range(7)
SCHEMES = {"bgk": FLBM_BGK, "gmf": FLBM_GMF, "reg": FLBM_REG, "learned": FLBM_LEARNED}
PRECISIONS = {"fp64": FLBM_FP64, "fp32": FLBM_FP32, "fp16": FLBM_FP16}
FLBM_STATE_POPULATIONS, FLBM_STATE_MOMENTS = 0, 1
STATE_FORMS = {"populations": FLBM_STATE_POPULATIONS, "moments": FLBM_STATE_MOMENTS}
Q = 27


class flbm_params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("scheme", C.c_int32), ("precision", C.c_int32),
                ("noise_rho0", C.c_int32), ("stats_every", C.c_int32),
                ("noise_stream", C.c_int32), ("state_form", C.c_int32),
                ("tau", C.c_double), ("kT", C.c_double),
                ("rho0", C.c_double), ("seed", C.c_uint64)]


class flbm_stats_t(C.Structure):
    _fields_ = [("step", C.c_int64), ("n_samples", C.c_int64), ("mass", C.c_double),
                ("mom", C.c_double * 3), ("u2", C.c_double * 3), ("u2_avg", C.c_double * 3),
                ("m_mean", C.c_double * 4), ("m_var", C.c_double * 4), ("er", C.c_double * 4)]

    def as_dict(self):
        return {"step": self.step, "n_samples": self.n_samples, "mass": self.mass,
                "mom": list(self.mom), "u2": list(self.u2), "u2_avg": list(self.u2_avg),
                "m_mean": list(self.m_mean), "m_var": list(self.m_var), "er": list(self.er)}


class flbm_ensemble_tuning(C.Structure):
    _fields_ = [("item_nodes", C.c_int32), ("stages", C.c_int32), ("compute_warps", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("ms_per_step", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class FlbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("flbm error %d: %s" % (code, msg))
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libflbm.so is not built (run __graft_entry__.build() or "
                          "python paper_2601_03806_gb300/build.py); there is no CPU fallback")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, u64, d = C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_double
    P = C.POINTER
    sig = {
        "flbm_params_init": ([P(flbm_params), i32, i32, i32, d, d, d, u64, i32], i32),
        "flbm_state_bytes": ([P(flbm_params)], C.c_size_t),
        "flbm_create": ([i32, i32, i32, d, d, d, u64, i32, P(vp)], i32),
        "flbm_create_ex": ([P(flbm_params), vp, C.c_size_t, vp, P(vp)], i32),
        "flbm_step": ([vp, i64], i32),
        "flbm_moments": ([vp, vp, vp, vp], i32),
        "flbm_stats": ([vp, P(flbm_stats_t)], i32),
        "flbm_stats_reset": ([vp], i32),
        "flbm_structure_factor": ([vp, i32, i32, vp, vp], i32),
        "flbm_spectral_er": ([vp, i32, i32, vp, vp], i32),
        "flbm_get_populations": ([vp, vp], i32),
        "flbm_set_populations": ([vp, vp], i32),
        "flbm_probe": ([vp, vp, i64, vp], i32),
        "flbm_init_thermal": ([vp, u64], i32),
        "flbm_get_state": ([vp, vp], i32),
        "flbm_set_state": ([vp, vp], i32),
        "flbm_timing_enable": ([vp, i32], i32),
        "flbm_timing_read": ([vp, vp, vp], i32),
        "flbm_get_step": ([vp], i64),
        "flbm_set_step": ([vp, i64], i32),
        "flbm_get_params": ([vp, P(flbm_params)], i32),
        "flbm_last_error": ([vp], C.c_char_p),
        "flbm_destroy": ([vp], None),
        "flbm_step_noalloc": ([P(flbm_params), vp, i64, i32, vp, vp], i32),
        "flbm_ensemble_create": ([P(flbm_params), i32, vp, P(vp)], i32),
        "flbm_ensemble_replica": ([vp, i32, P(vp)], i32),
        "flbm_ensemble_step": ([vp, i64], i32),
        "flbm_ensemble_graph": ([vp, i32], i32),
        "flbm_ensemble_set_tuning": ([vp, P(flbm_ensemble_tuning)], i32),
        "flbm_ensemble_get_tuning": ([vp, P(flbm_ensemble_tuning)], i32),
        "flbm_ensemble_autotune": ([vp, i32, P(flbm_ensemble_tuning)], i32),
        "flbm_ensemble_count": ([vp], i32),
        "flbm_ensemble_get_step": ([vp], i64),
        "flbm_ensemble_last_error": ([vp], C.c_char_p),
        "flbm_ensemble_destroy": ([vp], None),
        "flbm_mlp_infer": ([vp, vp, i64, vp], i32),
        "flbm_mlp_pairs": ([vp, vp, vp], i32),
        "flbm_set_mlp": ([vp, vp], i32),
        "flbm_mlp_grad": ([vp, vp, vp, i64, vp, vp], i32),
        "flbm_mlp_train": ([vp, vp, vp, i64, i32, i32, d, u64, vp], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    return L


lib = _load()

# Same-name module-level functions (raw C ABI).
flbm_params_init = lib.flbm_params_init
flbm_state_bytes = lib.flbm_state_bytes
flbm_create = lib.flbm_create
flbm_create_ex = lib.flbm_create_ex
flbm_step = lib.flbm_step
flbm_moments = lib.flbm_moments
flbm_stats = lib.flbm_stats
flbm_stats_reset = lib.flbm_stats_reset
flbm_structure_factor = lib.flbm_structure_factor
flbm_spectral_er = lib.flbm_spectral_er
flbm_get_populations = lib.flbm_get_populations
flbm_set_populations = lib.flbm_set_populations
flbm_probe = lib.flbm_probe
flbm_init_thermal = lib.flbm_init_thermal
flbm_get_state = lib.flbm_get_state
flbm_set_state = lib.flbm_set_state
flbm_timing_enable = lib.flbm_timing_enable
flbm_timing_read = lib.flbm_timing_read
flbm_get_step = lib.flbm_get_step
flbm_set_step = lib.flbm_set_step
flbm_get_params = lib.flbm_get_params
flbm_last_error = lib.flbm_last_error
flbm_destroy = lib.flbm_destroy
flbm_step_noalloc = lib.flbm_step_noalloc
flbm_ensemble_create = lib.flbm_ensemble_create
flbm_ensemble_replica = lib.flbm_ensemble_replica
flbm_ensemble_step = lib.flbm_ensemble_step
flbm_ensemble_graph = lib.flbm_ensemble_graph
flbm_ensemble_set_tuning = lib.flbm_ensemble_set_tuning
flbm_ensemble_get_tuning = lib.flbm_ensemble_get_tuning
flbm_ensemble_autotune = lib.flbm_ensemble_autotune
flbm_ensemble_count = lib.flbm_ensemble_count
flbm_ensemble_get_step = lib.flbm_ensemble_get_step
flbm_ensemble_last_error = lib.flbm_ensemble_last_error
flbm_ensemble_destroy = lib.flbm_ensemble_destroy
flbm_mlp_infer = lib.flbm_mlp_infer
flbm_mlp_pairs = lib.flbm_mlp_pairs
flbm_set_mlp = lib.flbm_set_mlp
flbm_mlp_grad = lib.flbm_mlp_grad
flbm_mlp_train = lib.flbm_mlp_train
MLP_NPARAM = 7771


def _dev(t):
    """Device address of a CUDA torch tensor (float32, contiguous)."""
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def mlp_grad(params, dev_x, dev_t):
    """(gradient[7771], loss) of the mean squared error on device samples."""
    p = np.ascontiguousarray(params, np.float32)
    g = np.empty(MLP_NPARAM, np.float32)
    loss = C.c_double()
    n = dev_x.shape[0]
    rc = lib.flbm_mlp_grad(_ptr(p), _dev(dev_x), _dev(dev_t), n, _ptr(g), C.byref(loss))
    if rc != FLBM_OK:
        raise FlbmError(rc, lib.flbm_last_error(None).decode())
    return g, loss.value


def mlp_train(params, dev_x, dev_t, epochs, batch=1024, lr=3e-3, seed=0):
    """Adam-trained copy of params and the per-epoch mean losses."""
    p = np.array(params, np.float32)
    losses = np.zeros(int(epochs))
    rc = lib.flbm_mlp_train(_ptr(p), _dev(dev_x), _dev(dev_t), dev_x.shape[0], int(epochs), int(batch),
                            float(lr), int(seed), _ptr(losses))
    if rc != FLBM_OK:
        raise FlbmError(rc, lib.flbm_last_error(None).decode())
    return p, losses


def mlp_infer(params, x) -> np.ndarray:
    """Network outputs y[n, 27] of features x[n, 28] on the tensor cores."""
    p = np.ascontiguousarray(params, np.float32)
    if p.size != MLP_NPARAM:
        raise ValueError("params must hold %d values" % MLP_NPARAM)
    xx = np.ascontiguousarray(x, np.float32).reshape(-1, 28)
    y = np.empty((xx.shape[0], 27), np.float32)
    rc = lib.flbm_mlp_infer(_ptr(p), _ptr(xx), xx.shape[0], _ptr(y))
    if rc != FLBM_OK:
        raise FlbmError(rc, lib.flbm_last_error(None).decode())
    return y


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def make_params(nx, ny, nz, tau, kT, rho0=1.0, seed=0, scheme=FLBM_GMF, precision=FLBM_FP32,
                noise_rho0=False, stats_every=1, noise_stream=0, state_form=0) -> flbm_params:
    p = flbm_params()
    lib.flbm_params_init(C.byref(p), nx, ny, nz, tau, kT, rho0, seed,
                         SCHEMES.get(scheme, scheme) if isinstance(scheme, str) else scheme)
    p.precision = PRECISIONS.get(precision, precision) if isinstance(precision, str) else precision
    p.noise_rho0 = int(bool(noise_rho0))
    p.stats_every = int(stats_every)
    p.noise_stream = int(noise_stream)
    p.state_form = STATE_FORMS.get(state_form, state_form) if isinstance(state_form, str) else int(state_form)
    return p


class _CtxOps:
    """Calls on one flbm_ctx (self._h, self.params, self.nx/ny/nz)."""

    def _check(self, rc):
        if rc != FLBM_OK:
            raise FlbmError(rc, lib.flbm_last_error(self._h).decode())

    @property
    def handle(self):
        return self._h

    @property
    def step_count(self) -> int:
        return int(lib.flbm_get_step(self._h))

    def set_step(self, t: int) -> None:
        self._check(lib.flbm_set_step(self._h, int(t)))

    def step(self, n: int = 1) -> None:
        self._check(lib.flbm_step(self._h, int(n)))

    def timing_enable(self, on: bool = True) -> None:
        self._check(lib.flbm_timing_enable(self._h, int(bool(on))))

    def timing_read(self):
        """(summed step-kernel milliseconds, launches) since the last read."""
        ms = C.c_double()
        cnt = C.c_int64()
        self._check(lib.flbm_timing_read(self._h, C.byref(ms), C.byref(cnt)))
        return ms.value, cnt.value

    def moments(self):
        shape = (self.nz, self.ny, self.nx)
        rho = np.empty(shape)
        j = np.empty((3,) + shape)
        pi = np.empty((6,) + shape)
        self._check(lib.flbm_moments(self._h, _ptr(rho), _ptr(j), _ptr(pi)))
        return rho, j, pi

    def stats(self) -> dict:
        s = flbm_stats_t()
        self._check(lib.flbm_stats(self._h, C.byref(s)))
        return s.as_dict()

    def stats_reset(self) -> None:
        self._check(lib.flbm_stats_reset(self._h))

    def set_mlp(self, params) -> None:
        """Network of a learned-scheme context (7771 float parameters)."""
        p = np.ascontiguousarray(params, np.float32)
        if p.size != MLP_NPARAM:
            raise ValueError("params must hold %d values" % MLP_NPARAM)
        self._check(lib.flbm_set_mlp(self._h, _ptr(p)))

    def mlp_pairs(self, dev_x, dev_t) -> None:
        """Training pairs of every node into CUDA tensors x[N, 28], t[N, 27]."""
        self._check(lib.flbm_mlp_pairs(self._h, _dev(dev_x), _dev(dev_t)))

    def structure_factor(self, observable: int, nshell: int):
        S = np.zeros(nshell)
        cnt = np.zeros(nshell, np.int64)
        self._check(lib.flbm_structure_factor(self._h, int(observable), int(nshell), _ptr(S), _ptr(cnt)))
        return S, cnt

    def spectral_er(self, observable: int, nshell: int):
        """ER_m per shell of the current state and the shell populations
        (see flbm_spectral_er)."""
        er = np.zeros(nshell)
        cnt = np.zeros(nshell, np.int64)
        self._check(lib.flbm_spectral_er(self._h, int(observable), int(nshell), _ptr(er), _ptr(cnt)))
        return er, cnt

    def get_populations(self) -> np.ndarray:
        f = np.empty((Q, self.nz, self.ny, self.nx))
        self._check(lib.flbm_get_populations(self._h, _ptr(f)))
        return f

    def set_populations(self, f) -> None:
        ff = np.ascontiguousarray(f, np.float64).reshape(Q, self.nz, self.ny, self.nx)
        self._check(lib.flbm_set_populations(self._h, _ptr(ff)))

    def init_thermal(self, seed: int) -> None:
        """Sample the lattice invariant measure (see flbm_init_thermal)."""
        self._check(lib.flbm_init_thermal(self._h, int(seed)))

    def probe(self, nodes) -> np.ndarray:
        """Absolute f_i at the listed node indices, shape (len(nodes), 27)."""
        nn = np.ascontiguousarray(nodes, np.int64)
        out = np.empty((nn.size, Q))
        self._check(lib.flbm_probe(self._h, _ptr(nn), nn.size, _ptr(out)))
        return out

    def state_dtype(self):
        return {FLBM_FP64: np.float64, FLBM_FP32: np.float32, FLBM_FP16: np.float16}[
            self.params.precision]

    def get_state(self, out=None) -> np.ndarray:
        if out is None:
            out = np.empty((Q, self.nz, self.ny, self.nx), self.state_dtype())
        self._check(lib.flbm_get_state(self._h, _ptr(out) if isinstance(out, np.ndarray)
                                       else C.c_void_p(out.data_ptr())))
        return out

    def set_state(self, g) -> None:
        if isinstance(g, np.ndarray):
            gg = np.ascontiguousarray(g, self.state_dtype())
            self._check(lib.flbm_set_state(self._h, _ptr(gg)))
        else:  # a pinned torch tensor
            self._check(lib.flbm_set_state(self._h, C.c_void_p(g.data_ptr())))


class Lattice(_CtxOps):
    """Owning wrapper of one flbm_ctx.

    torch_memory=True: the population buffer is a torch CUDA tensor and the
    work is ordered on torch's current stream (``self.stream``).
    state_form="moments" (FP32, GMF or Reg): the box keeps ten numbers per
    node between steps instead of the populations (FLBM_STATE_MOMENTS)."""

    def __init__(self, nx, ny, nz, tau, kT, rho0=1.0, seed=0, scheme=FLBM_GMF,
                 precision=FLBM_FP32, noise_rho0=False, stats_every=1, torch_memory=False,
                 stream=None, noise_stream=0, state_form=0):
        self.params = make_params(nx, ny, nz, tau, kT, rho0, seed, scheme, precision,
                                  noise_rho0, stats_every, noise_stream, state_form)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.n = nx * ny * nz
        self._h = C.c_void_p()
        self._buf = None
        self.stream = stream
        dev, nbytes, sp = None, 0, None
        if torch_memory:
            import torch
            nbytes = int(lib.flbm_state_bytes(C.byref(self.params)))
            if nbytes == 0:
                raise FlbmError(FLBM_E_INVALID, "invalid parameters")
            self._buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            dev = self._buf.data_ptr()
            if self.stream is None:
                self.stream = torch.cuda.current_stream()
        if self.stream is not None:
            sp = self.stream.cuda_stream if hasattr(self.stream, "cuda_stream") else int(self.stream)
        rc = lib.flbm_create_ex(C.byref(self.params), dev, nbytes, sp, C.byref(self._h))
        if rc != FLBM_OK:
            raise FlbmError(rc, lib.flbm_last_error(None).decode())

    def close(self):
        if self._h:
            lib.flbm_destroy(self._h)
            self._h = C.c_void_p()
        self._buf = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Replica(_CtxOps):
    """Borrowed context of one replica of an Ensemble (not destroyed here)."""

    def __init__(self, ens: "Ensemble", index: int, params: flbm_params):
        self._ens = ens            # keeps the ensemble alive
        self.index = index
        self.params = params
        self.nx, self.ny, self.nz = params.nx, params.ny, params.nz
        self.n = self.nx * self.ny * self.nz
        self._h = C.c_void_p()
        rc = lib.flbm_ensemble_replica(ens._e, int(index), C.byref(self._h))
        if rc != FLBM_OK:
            raise FlbmError(rc, lib.flbm_ensemble_last_error(ens._e).decode())


class Ensemble:
    """Owning wrapper of one flbm_ensemble: many replica boxes advanced by one
    persistent kernel per step (see flbm_ensemble_create)."""

    def __init__(self, params, stream=None):
        self.params = list(params)
        arr = (flbm_params * len(self.params))(*self.params)
        self._e = C.c_void_p()
        self.stream = stream
        sp = None
        if stream is not None:
            sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        rc = lib.flbm_ensemble_create(arr, len(self.params), sp, C.byref(self._e))
        if rc != FLBM_OK:
            raise FlbmError(rc, lib.flbm_ensemble_last_error(None).decode())
        self.replicas = [Replica(self, r, p) for r, p in enumerate(self.params)]
        self.nodes = sum(r.n for r in self.replicas)

    def _check(self, rc):
        if rc != FLBM_OK:
            raise FlbmError(rc, lib.flbm_ensemble_last_error(self._e).decode())

    def __len__(self):
        return len(self.replicas)

    def __getitem__(self, i) -> Replica:
        return self.replicas[i]

    @property
    def step_count(self) -> int:
        return int(lib.flbm_ensemble_get_step(self._e))

    def step(self, n: int = 1) -> None:
        self._check(lib.flbm_ensemble_step(self._e, int(n)))

    def graph(self, enable: bool = True) -> None:
        self._check(lib.flbm_ensemble_graph(self._e, int(bool(enable))))

    @property
    def tuning(self) -> dict:
        t = flbm_ensemble_tuning()
        self._check(lib.flbm_ensemble_get_tuning(self._e, C.byref(t)))
        return t.as_dict()

    def set_tuning(self, item_nodes=256, stages=2, compute_warps=8, ctas_per_sm=2) -> None:
        t = flbm_ensemble_tuning(int(item_nodes), int(stages), int(compute_warps), int(ctas_per_sm), 0.0)
        self._check(lib.flbm_ensemble_set_tuning(self._e, C.byref(t)))

    def autotune(self, steps_per_trial: int = 4) -> dict:
        t = flbm_ensemble_tuning()
        self._check(lib.flbm_ensemble_autotune(self._e, int(steps_per_trial), C.byref(t)))
        return t.as_dict()

    def close(self):
        if self._e:
            for r in getattr(self, "replicas", []):
                r._h = C.c_void_p()
            lib.flbm_ensemble_destroy(self._e)
            self._e = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
