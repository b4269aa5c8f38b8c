"""The single large box at full size: 512^3 GMF-FLBM, tau 0.6, kT 1e-5,
rho0 1, 2000 steps with the FP64 reductions every step, in FP32 deviation
storage and in FP16 storage.  Started from the lattice invariant measure
(flbm_init_thermal), the time averages must meet the equipartition gate:
<u_a^2> within 1 % of kT/rho0 on every axis, the four ER ratios within 1 %
of one, and the total mass conserved to the rounding of the FP64 sums
(FP32) or of the half-precision deviations (FP16)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2601_03806_gb300 import flbm
    return flbm


@pytest.mark.parametrize("precision,mass_tol", [(1, 1e-9), (2, 1e-6)])
def test_config3_2000_steps_equipartition(F, precision, mass_tol):
    n, tau, kT, rho0 = 512, 0.6, 1e-5, 1.0
    with F.Lattice(n, n, n, tau, kT, rho0=rho0, seed=2026, precision=precision) as g:
        g.init_thermal(2027)
        g.step(1)
        m0 = g.stats()["mass"]
        g.stats_reset()
        g.step(1999)
        s = g.stats()
    u2 = np.array(s["u2_avg"]) / (kT / rho0)
    er = np.array(s["er"])
    print("precision", precision, "u2/(kT/rho0)", u2, "ER", er, "mass drift", s["mass"] / m0 - 1)
    assert s["n_samples"] == 1999
    assert np.all(np.abs(u2 - 1) < 0.01), u2
    assert np.all(np.abs(er - 1) < 0.01), er
    assert abs(s["mass"] / m0 - 1) < mass_tol
