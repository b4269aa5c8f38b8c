"""CPU check of the FP32 reduction error bound in reduction_sums.py: the
13 sums evaluated in plain FP32 (sequential 27-term moments, per-thread
FP32 accumulation over m nodes, an FP32 pairwise tree over 32 threads, FP64
above) stay within the bound of the oracle's FP64 sums, and the bound is far
below the sums' own scale."""
import numpy as np
import pytest

import reduction_sums as R
from synth import inputs


def fp32_sums(f, w, c, rho0, m):
    g = (f - w[:, None, None, None] * rho0).reshape(27, -1).astype(np.float32)
    c = c.astype(np.float32)
    one = np.float32(1)
    drho = np.zeros(g.shape[1], np.float32)
    j = np.zeros((3, g.shape[1]), np.float32)
    m3 = np.zeros(g.shape[1], np.float32)
    m4 = np.zeros(g.shape[1], np.float32)
    for i in range(27):                       # sequential FP32 moments
        drho = drho + g[i]
        for a in range(3):
            j[a] = j[a] + g[i] * c[i, a]
        m3 = m3 + g[i] * np.float32((c[i] ** 2).sum())
        m4 = m4 + g[i] * np.float32(c[i, 0] * c[i, 1] + c[i, 0] * c[i, 2] + c[i, 1] * c[i, 2])
    rho = np.float32(rho0) + drho
    irho = one / rho
    u = j * irho
    m2 = (j[0] + j[1]) + j[2]
    x = [drho, j[0], j[1], j[2], u[0] * u[0], u[1] * u[1], u[2] * u[2], m3, m4,
         drho * drho, m2 * m2, m3 * m3, m4 * m4]
    out = []
    for t in x:
        n = t.size
        pad = (-n) % (32 * m)
        t = np.concatenate([t, np.zeros(pad, np.float32)]).reshape(-1, 32, m)
        acc = np.zeros(t.shape[:2], np.float32)
        for k in range(m):                    # per-thread FP32 accumulation
            acc = acc + t[:, :, k]
        while acc.shape[1] > 1:               # warp tree in FP32
            h = acc.shape[1] // 2
            acc = acc[:, :h] + acc[:, h:]
        out.append(acc[:, 0].astype(np.float64).sum())
    return np.array(out)


@pytest.mark.parametrize("shape,m,amp", [((16, 16, 16), 1, 0.02), ((40, 12, 10), 12, 0.02),
                                         ((64, 32, 8), 64, 0.005)])
def test_fp32_sums_within_bound(oracle_mod, shape, m, amp):
    T = oracle_mod.tables()
    w, c = T["w"], T["c"]
    nx, ny, nz = shape
    rho0 = 1.0
    f = w[:, None, None, None] * (rho0 + amp * inputs.population_perturbation(nx, ny, nz, 41))
    S, B = R.sums_and_bounds(oracle_mod, f, rho0, m)
    G = fp32_sums(f, w, c, rho0, m)
    x, _ = R.node_terms(oracle_mod, f, rho0)
    scale = np.abs(x).sum(1)
    assert np.all(np.abs(G - S) <= B), (np.abs(G - S) / B)
    # the bound has teeth: well below the sums' own scale
    assert np.all(B <= 2e-4 * scale + 1e-300), B / scale
