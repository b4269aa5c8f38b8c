"""GPU parity of the fused reductions (row a9) at the storage precisions the
throughput runs use: every flbm_stats field of a reduced FP32 or FP16 step
against the same sums taken in FP64 by the oracle's moments of the GPU's own
pre-collision populations (flbm_get_populations), step by step.

Tolerance: the bound of reduction_sums.py, derived from the FP32 arithmetic
of the per-node terms and the FP32 part of the accumulation; it is checked on
the CPU against a plain FP32 evaluation (test_reduction_bound.py).  The
observed ratios |gpu - oracle| / bound are printed.
"""
import numpy as np
import pytest

import reduction_sums as R

pytestmark = pytest.mark.gpu

FIELDS = ["mass", "mom", "u2", "m_mean", "m_var", "er"]


@pytest.fixture(scope="module")
def F():
    from paper_2601_03806_gb300 import flbm
    return flbm


def _check_steps(F, O, g, nsteps, rho0, kT):
    nx, ny, nz = g.nx, g.ny, g.nz
    n = nx * ny * nz
    m = R.nodes_per_thread_bound(nx, ny, nz)
    worst = {k: 0.0 for k in FIELDS}
    for _ in range(nsteps):
        f = g.get_populations()
        S, B = R.sums_and_bounds(O, f, rho0, m)
        ref = R.stats_from_sums(S, n, rho0, kT)
        bnd = R.stats_bounds(S, B, n, rho0, kT)
        g.stats_reset()
        g.step(1)
        st = g.stats()
        assert st["n_samples"] == 1
        for k in FIELDS:
            d = np.abs(np.asarray(st[k], float) - np.asarray(ref[k], float))
            b = np.asarray(bnd[k], float)
            assert np.all(d <= b), (k, d, b)
            worst[k] = max(worst[k], float(np.max(d / np.maximum(b, 1e-300))))
    return worst


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("shape", [(16, 16, 16), (130, 3, 2), (64, 12, 10), (128, 64, 64),
                                   (512, 16, 8)])
def test_reductions_match_oracle_sums(F, oracle_mod, precision, shape):
    """16^3 and 130x3x2 run the direct kernel, the others the row pipeline
    (128x64x64: up to 27 rows per thread; 512 wide: two nodes per thread and
    row).  Thermal start, tau 0.7, kT 1e-4, 5 reduced steps."""
    nx, ny, nz = shape
    rho0, kT = 1.0, 1e-4
    g = F.Lattice(nx, ny, nz, 0.7, kT, rho0=rho0, seed=21, precision=precision, stats_every=1)
    g.init_thermal(7)
    worst = _check_steps(F, oracle_mod, g, 5, rho0, kT)
    print("precision", precision, shape, "max |gpu - oracle| / bound:", worst)
    g.close()


@pytest.mark.parametrize("precision", [1, 2])
def test_reductions_match_oracle_sums_256cube(F, oracle_mod, precision):
    """A 256^3 box (16.7 M nodes; the row pipeline gives each thread one node
    of about 216 rows per step, folded into FP64 every 8 rows): one reduced
    step against the oracle's FP64 sums."""
    n, rho0, kT = 256, 1.0, 1e-5
    g = F.Lattice(n, n, n, 0.6, kT, rho0=rho0, seed=3, precision=precision, stats_every=1)
    g.init_thermal(11)
    worst = _check_steps(F, oracle_mod, g, 1, rho0, kT)
    print("precision", precision, "256^3 max |gpu - oracle| / bound:", worst)
    g.close()
