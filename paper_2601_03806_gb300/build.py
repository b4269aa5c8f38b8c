"""Build libflbm.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked with the CUDA
runtime (shared, so a process that also loads PyTorch holds one runtime) and
cuFFT.  Objects go to ``_build/`` at the repository root.
"""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "libflbm.so")
BUILD = os.path.join(ROOT, "_build")
SOURCES = ["capi.cu", "aux.cu", "step_f32.cu", "step_f64.cu", "step_f16.cu", "step_f16_nx512.cu",
           "step_f32_paced.cu", "noalloc.cu",
           "ens_f32.cu", "ens_f16.cu", "ens_f32p.cu", "ens_f16p.cu", "ensemble.cu", "mlp_infer.cu",
           "mlp_train.cu", "step_learned.cu", "mstate.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "-ftz=true", "-I" + os.path.join(ROOT, "include")]
# extra nvcc flags, e.g. FLBM_NVCC_FLAGS="-DFLBM_MIN_BLOCKS=5" (register bound
# of the step kernel); the default build uses none
EXTRA = os.environ.get("FLBM_NVCC_FLAGS", "").split()


def _nvcc() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = os.path.join(home, "bin", "nvcc")
    return p if os.path.exists(p) else "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    stamp = os.path.join(BUILD, "flags")
    if os.path.exists(stamp) and open(stamp).read() != " ".join(EXTRA):
        return float("inf")
    files.append(os.path.join(ROOT, "include", "flbm.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= _deps():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, *EXTRA, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose:
            print(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = OUT + ".tmp%d" % os.getpid()
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs, "-lcufft"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, OUT)
    with open(os.path.join(BUILD, "flags"), "w") as fh:
        fh.write(" ".join(EXTRA))
    return OUT


if __name__ == "__main__":
    print(build(force=True, verbose=True))
