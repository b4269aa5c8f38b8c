"""The three collision schemes the paper compares (Sec. III: BGK-FLBM,
GMF-FLBM, Reg-FLBM) on the equilibrium-fluctuation box of config C2:
periodic 128^3, FP32 deviation storage, rho0 = 1, kT = 1e-5, tau in {0.55,
1, 2, 5}, seeds 1..4, 20 000 steps from a sample of the lattice invariant
measure (so no thermalisation transient), fused reductions every step.

Per scheme and tau the test reports <u_a^2>/(kT/rho0) and the four
equilibration ratios ER(rho, sum j, sum Pi_aa, sum_{a<b} Pi_ab) (Sec. III,
time-space variances over their invariant-measure values 3, 3, 5, 1 rho0
kT), as seed means with the standard error over the four seeds.

At kT = 1e-5 the dynamics are linear to O(kT) and the invariant measure is
exact for every scheme at every tau, so all three hold equipartition and
ER = 1; GMF and Reg are held to 1 %, BGK to 1 % as well.  C2' repeats the
sweep at the paper's kT = 1/3000 (two seeds, 5 000 steps), where the scheme
differences are nonlinear: GMF and Reg are held to 3 % ("close to unity for
all tau" in Sec. III), BGK is reported (a run that turns unstable is
reported as such, as the paper reports unstable BGK runs).
"""
import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SCHEMES = {0: "BGK", 1: "GMF", 2: "Reg"}
TAUS = [0.55, 1.0, 2.0, 5.0]


@pytest.fixture(scope="module")
def F():
    from paper_2601_03806_gb300 import flbm
    return flbm


def run_box(F, scheme, tau, kT, seed, steps, n=128, rho0=1.0, warm=200):
    """(u2 ratios [3], ER [4]) of one run, or None if it turned unstable."""
    g = F.Lattice(n, n, n, tau, kT, rho0=rho0, seed=seed, scheme=scheme, precision=F.FLBM_FP32,
                  stats_every=1)
    try:
        g.init_thermal(1000 + seed)
        g.step(warm)
        g.stats_reset()
        g.step(steps)
        s = g.stats()
    except F.FlbmError as e:
        if e.code == F.FLBM_E_UNSTABLE:
            return None
        raise
    finally:
        g.close()
    return np.array(s["u2_avg"]) / (kT / rho0), np.array(s["er"])


def sweep(F, kT, seeds, steps):
    table = {}
    for scheme in SCHEMES:
        for tau in TAUS:
            runs = [run_box(F, scheme, tau, kT, seed, steps) for seed in seeds]
            ok = [r for r in runs if r is not None]
            if len(ok) < len(runs):
                table[(scheme, tau)] = None
                print("kT=%g %s tau=%g: unstable in %d of %d runs" % (kT, SCHEMES[scheme], tau,
                                                                     len(runs) - len(ok), len(runs)))
                continue
            u2 = np.array([r[0].mean() for r in ok])
            er = np.array([r[1] for r in ok])
            sem = lambda a: a.std(axis=0, ddof=1) / np.sqrt(len(a)) if len(a) > 1 else a * 0
            row = {"u2": u2.mean(), "u2_se": sem(u2), "er": er.mean(0), "er_se": sem(er)}
            table[(scheme, tau)] = row
            print("kT=%g %s tau=%g: <u^2>/(kT/rho0) = %.5f +- %.5f; ER = %s +- %s"
                  % (kT, SCHEMES[scheme], tau, row["u2"], row["u2_se"],
                     np.array2string(row["er"], precision=5), np.array2string(row["er_se"], precision=5)))
    return table


def test_c2_three_schemes_kT_1e5(F):
    table = sweep(F, 1e-5, seeds=[1, 2, 3, 4], steps=20000)
    for (scheme, tau), row in table.items():
        assert row is not None, (SCHEMES[scheme], tau)
        assert abs(row["u2"] - 1) < 0.01, (SCHEMES[scheme], tau, row["u2"])
        assert np.all(np.abs(row["er"] - 1) < 0.01), (SCHEMES[scheme], tau, row["er"])


def test_c2prime_three_schemes_paper_kT(F):
    """Besides the 3 % band, the ordering Sec. III reports at the smallest
    tau: BGK's equilibration ratios depart from 1 further than GMF's, and
    GMF and Reg agree (here within 1e-3)."""
    table = sweep(F, 1.0 / 3000.0, seeds=[1, 2], steps=5000)
    for (scheme, tau), row in table.items():
        if scheme == 0:
            continue                      # reported, not held (Sec. III: BGK departs)
        assert row is not None, (SCHEMES[scheme], tau)
        assert abs(row["u2"] - 1) < 0.03, (SCHEMES[scheme], tau, row["u2"])
        assert np.all(np.abs(row["er"] - 1) < 0.03), (SCHEMES[scheme], tau, row["er"])
    bgk, gmf, reg = table[(0, 0.55)], table[(1, 0.55)], table[(2, 0.55)]
    assert np.abs(gmf["er"] - reg["er"]).max() < 1e-3, (gmf["er"], reg["er"])
    if bgk is not None:
        excess = (bgk["er"] - 1).mean() - (gmf["er"] - 1).mean()
        se = np.sqrt((bgk["er_se"] ** 2).mean() + (gmf["er_se"] ** 2).mean())
        assert excess > 5 * se and excess > 0, (bgk["er"], gmf["er"])
