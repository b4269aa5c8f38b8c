"""ctypes binding of the plain-C FP64 oracle (``flbm_oracle.c``).

Test infrastructure only (see the package docstring).  ``build()`` compiles
the C source with gcc; the binding loads ``liboracle.so`` beside it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "flbm_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

Q = 27
BGK, GMF, REG = 0, 1, 2

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no FMA contraction so that
    x86 and Arm hosts give the same results)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "flbm_oracle.h"))
    ):
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-std=c99", "-o", tmp, SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        P = C.POINTER
        d, i32, i64, u64, vp = C.c_double, C.c_int, C.c_int64, C.c_uint64, C.c_void_p
        L.oracle_tables.argtypes = [vp, vp, vp, vp, vp, vp]
        L.oracle_philox4x32_10.argtypes = [vp, vp, vp]
        L.oracle_normals.argtypes = [u64, u64, u64, vp]
        L.oracle_normals_stream.argtypes = [u64, C.c_uint32, u64, u64, vp]
        L.oracle_set_stream.argtypes = [vp, C.c_uint32]
        L.oracle_feq2.argtypes = [d, vp, vp]
        L.oracle_noise_term.argtypes = [i32, d, d, d, vp, vp]
        L.oracle_collide_node.argtypes = [i32, d, d, d, i32, u64, u64, u64, vp, vp]
        L.oracle_create.argtypes = [i32, i32, i32, d, d, d, u64, i32, i32]
        L.oracle_create.restype = vp
        L.oracle_destroy.argtypes = [vp]
        L.oracle_set_populations.argtypes = [vp, vp]
        L.oracle_get_populations.argtypes = [vp, vp]
        L.oracle_get_step.argtypes = [vp]
        L.oracle_get_step.restype = i64
        L.oracle_set_step.argtypes = [vp, i64]
        L.oracle_step.argtypes = [vp, i64]
        L.oracle_trajectory_node0.argtypes = [vp, i64, vp]
        L.oracle_moments.argtypes = [vp, vp, vp, vp]
        L.oracle_structure_factor.argtypes = [vp, i32, i32, i32, i32, vp, vp]
        L.oracle_set_threads.argtypes = [i32]
        L.oracle_get_threads.restype = i32
        del P
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def tables():
    """Return dict with c (27x3), w (27), E (27x27, E[k,i]=e_ki), b, nk, muk."""
    c = np.zeros((Q, 3), np.int32)
    w = np.zeros(Q)
    E = np.zeros((Q, Q))
    b = np.zeros(Q)
    nk = np.zeros(Q, np.int32)
    mu = np.zeros(Q, np.int32)
    lib().oracle_tables(_p(c), _p(w), _p(E), _p(b), _p(nk), _p(mu))
    return {"c": c, "w": w, "E": E, "b": b, "nk": nk, "muk": mu}


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    lib().oracle_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def normals(seed: int, node: int, step: int, stream: int = 0) -> np.ndarray:
    r = np.zeros(Q)
    lib().oracle_normals_stream(seed, stream, node, step, _p(r))
    return r


def feq2(rho: float, u) -> np.ndarray:
    uu = np.ascontiguousarray(u, np.float64)
    f = np.zeros(Q)
    lib().oracle_feq2(rho, _p(uu), _p(f))
    return f


def noise_term(scheme: int, tau: float, kT: float, rho: float, r) -> np.ndarray:
    rr = np.ascontiguousarray(r, np.float64)
    xi = np.zeros(Q)
    lib().oracle_noise_term(scheme, tau, kT, rho, _p(rr), _p(xi))
    return xi


def collide_node(scheme, tau, kT, f, *, seed=0, node=0, step=0, rho0=1.0, noise_rho0=False):
    ff = np.ascontiguousarray(f, np.float64)
    out = np.zeros(Q)
    lib().oracle_collide_node(scheme, tau, kT, rho0, int(noise_rho0), seed, node, step,
                              _p(ff), _p(out))
    return out


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(lib().oracle_get_threads())


def structure_factor(m: np.ndarray, nshell: int):
    """m: real array shaped (nz, ny, nx).  Returns (S[nshell], count[nshell])."""
    mm = np.ascontiguousarray(m, np.float64)
    nz, ny, nx = mm.shape
    S = np.zeros(nshell)
    cnt = np.zeros(nshell, np.int64)
    lib().oracle_structure_factor(_p(mm), nx, ny, nz, nshell, _p(S), _p(cnt))
    return S, cnt


class Box:
    """A periodic nx*ny*nz box advanced by the oracle (two arrays, push)."""

    def __init__(self, nx, ny, nz, tau, kT, rho0=1.0, seed=0, scheme=GMF, noise_rho0=False,
                 stream=0):
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz
        self.nx, self.ny, self.nz = nx, ny, nz
        self.tau, self.kT, self.rho0, self.seed, self.scheme = tau, kT, rho0, seed, scheme
        h = lib().oracle_create(nx, ny, nz, tau, kT, rho0, seed, scheme, int(noise_rho0))
        if not h:
            raise ValueError("oracle_create failed")
        self._h = C.c_void_p(h)
        if stream:
            lib().oracle_set_stream(self._h, int(stream))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.oracle_destroy(h)
            self._h = None

    def step(self, n: int = 1) -> None:
        lib().oracle_step(self._h, int(n))

    @property
    def t(self) -> int:
        return int(lib().oracle_get_step(self._h))

    @t.setter
    def t(self, v: int) -> None:
        lib().oracle_set_step(self._h, int(v))

    def get_f(self) -> np.ndarray:
        f = np.zeros((Q,) + self.shape)
        lib().oracle_get_populations(self._h, _p(f))
        return f

    def set_f(self, f) -> None:
        ff = np.ascontiguousarray(f, np.float64).reshape((Q,) + self.shape)
        lib().oracle_set_populations(self._h, _p(ff))

    def moments(self):
        rho = np.zeros(self.shape)
        j = np.zeros((3,) + self.shape)
        pi = np.zeros((6,) + self.shape)
        lib().oracle_moments(self._h, _p(rho), _p(j), _p(pi))
        return rho, j, pi

    def trajectory_node0(self, n: int) -> np.ndarray:
        out = np.zeros((n, Q))
        lib().oracle_trajectory_node0(self._h, int(n), _p(out))
        return out
