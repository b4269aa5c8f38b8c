"""The oracle's Philox4x32-10 against an independent implementation: the
cuRAND device API's Philox4_32_10 generator, run on the GPU (a library
call; nothing of it is reproduced here).

cuRAND's state for (seed, subsequence, offset) is key = (seed lo, seed hi)
and 128-bit counter = offset / 4 (low 64 bits) + subsequence (high 64
bits); curand4() then returns the block function of that counter.  So the
block of counter (c0, c1, c2, c3) is curand4 after
curand_init(seed, c2 | c3 << 32, 4 (c0 | c1 << 32)).
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SRC = r'''
#include <cstdio>
#include <cstdint>
#include <curand_kernel.h>
__global__ void k(const unsigned long long *in, unsigned int *out, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long seed = in[3 * i], sub = in[3 * i + 1], off = in[3 * i + 2];
    curandStatePhilox4_32_10_t st;
    curand_init(seed, sub, off, &st);
    const uint4 r = curand4(&st);
    out[4 * i] = r.x; out[4 * i + 1] = r.y; out[4 * i + 2] = r.z; out[4 * i + 3] = r.w;
}
int main()
{
    int n = 0;
    if (scanf("%d", &n) != 1 || n < 1 || n > 4096) return 2;
    unsigned long long h[3 * 4096];
    for (int i = 0; i < 3 * n; ++i) if (scanf("%llu", &h[i]) != 1) return 2;
    unsigned long long *din; unsigned int *dout; unsigned int o[4 * 4096];
    if (cudaMalloc(&din, sizeof(unsigned long long) * 3 * n) != cudaSuccess) return 3;
    if (cudaMalloc(&dout, sizeof(unsigned int) * 4 * n) != cudaSuccess) return 3;
    cudaMemcpy(din, h, sizeof(unsigned long long) * 3 * n, cudaMemcpyHostToDevice);
    k<<<(n + 127) / 128, 128>>>(din, dout, n);
    if (cudaMemcpy(o, dout, sizeof(unsigned int) * 4 * n, cudaMemcpyDeviceToHost) != cudaSuccess) return 4;
    for (int i = 0; i < 4 * n; ++i) printf("%u\n", o[i]);
    cudaFree(din); cudaFree(dout);
    return 0;
}
'''


def test_oracle_philox_matches_curand(oracle_mod, tmp_path):
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc") or pytest.skip("nvcc not found")
    src = tmp_path / "curand_philox.cu"
    src.write_text(SRC)
    exe = tmp_path / "curand_philox"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", str(src), "-o", str(exe)],
                   check=True)
    rng = np.random.default_rng(12)
    cases = []
    for _ in range(200):
        key = [int(v) for v in rng.integers(0, 2 ** 32, size=2)]
        ctr = [int(v) for v in rng.integers(0, 2 ** 32, size=4)]
        ctr[1] &= 0x3FFFFFFF          # offset = 4 (c0 | c1 << 32) must fit 64 bits
        cases.append((ctr, key))
    cases.append(([0, 0, 0, 0], [0, 0]))
    cases.append(([7, 0, 3, 0], [1234, 0]))              # (node 7, step 0, block 3), seed 1234
    lines = [str(len(cases))]
    for ctr, key in cases:
        seed = key[0] | (key[1] << 32)
        sub = ctr[2] | (ctr[3] << 32)
        off = 4 * (ctr[0] | (ctr[1] << 32))
        lines.append("%d %d %d" % (seed, sub, off))
    out = subprocess.run([str(exe)], input="\n".join(lines), capture_output=True, text=True, check=True).stdout
    got = np.array([int(v) for v in out.split()], dtype=np.uint64).reshape(-1, 4)
    for (ctr, key), g in zip(cases, got):
        o = oracle_mod.philox4x32_10(ctr, key)
        assert np.array_equal(o.astype(np.uint64), g), (ctr, key, o, g)
