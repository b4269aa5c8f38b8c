"""GPU statistics against what the paper and the oracle's pinned theory fix:
equipartition <u_a^2> = kT/rho0, equilibration ratios ER(m) = 1 and a flat
S_m(|k|) for GMF-FLBM over tau (Sec. III), and the noise-off shear-wave
viscosity nu = c_s^2 (tau - 1/2) (Sec. II).

Inputs: FP32 deviation storage, rho0 = 1, kT = 1e-5 (the config-2/3 thermal
energy), started from a seeded sample of the lattice invariant measure
<dg_i dg_j> = (rho0 kT / c_s^2) w_i delta_ij so no warm-up is needed."""
import numpy as np
import pytest

from synth import inputs

pytestmark = pytest.mark.gpu

CS2 = 1.0 / 3.0


@pytest.fixture(scope="module")
def F():
    from paper_2601_03806_gb300 import flbm
    return flbm


def thermal_state(O, n, kT, rho0, seed):
    w = O.tables()["w"]
    sd = np.sqrt(rho0 * kT * w / CS2)[:, None, None, None]
    return (sd * inputs.population_perturbation(n, n, n, seed)).astype(np.float32)


@pytest.mark.parametrize("tau", [0.51, 0.55, 0.6, 1.0, 2.0, 5.0, 20.0, 100.0])
def test_gmf_equipartition_and_er(F, oracle_mod, tau):
    n, kT, rho0 = 128, 1e-5, 1.0
    g = F.Lattice(n, n, n, tau, kT, rho0=rho0, seed=int(tau * 1000), precision=1)
    g.set_state(thermal_state(oracle_mod, n, kT, rho0, seed=int(tau * 100)))
    g.step(200)
    g.stats_reset()
    g.step(2000)
    s = g.stats()
    u2 = np.array(s["u2_avg"]) / (kT / rho0)
    assert np.all(np.abs(u2 - 1) < 0.01), u2
    er = np.array(s["er"])
    assert np.all(np.abs(er - 1) < 0.02), er


@pytest.mark.parametrize("tau", [0.51, 0.55, 1.0, 5.0])
def test_gmf_equipartition_fp16_storage(F, tau):
    """FP16 deviation storage keeps equipartition and ER within the 1 % gate
    of FP32 (measured at 128^3: within 0.05 %, equal to FP32's values to
    five digits on the same noise stream)."""
    n, kT, rho0 = 128, 1e-5, 1.0
    g = F.Lattice(n, n, n, tau, kT, rho0=rho0, seed=31, precision=2)
    g.init_thermal(32)
    g.step(200)
    g.stats_reset()
    g.step(2000)
    s = g.stats()
    u2 = np.array(s["u2_avg"]) / (kT / rho0)
    assert np.all(np.abs(u2 - 1) < 0.01), u2
    assert np.all(np.abs(np.array(s["er"]) - 1) < 0.01), s["er"]


def test_gmf_flat_structure_factor(F, oracle_mod):
    n, kT, rho0, tau = 64, 1e-5, 1.0, 0.8
    g = F.Lattice(n, n, n, tau, kT, rho0=rho0, seed=31, precision=1, stats_every=0)
    g.set_state(thermal_state(oracle_mod, n, kT, rho0, seed=32))
    theory = np.array([3, 3, 5, 1]) * rho0 * kT
    acc = np.zeros((4, 40))
    snaps = 60
    for s in range(snaps):
        g.step(25)
        for obs in range(4):
            S, cnt = g.structure_factor(obs, 40)
            acc[obs] += S
    acc /= snaps
    for obs in range(4):
        er_k = acc[obs, 4:32] / theory[obs]
        assert abs(er_k.mean() - 1) < 0.02, (obs, er_k.mean())
        assert np.all(np.abs(er_k - 1) < 0.08), (obs, er_k)


def shear_fit(make, feq, tau, ny):
    """Decay rate of the noise-off shear wave u_x = 1e-3 sin(2 pi y / ny) on
    the box `make(ny)` returns (GPU lattice or oracle box)."""
    k = 2 * np.pi / ny
    nu = CS2 * (tau - 0.5)
    ux = inputs.sine_profile(ny, 1e-3)
    box, nx = make(ny)
    f0 = np.zeros((27, 1, ny, nx))
    for y in range(ny):
        f0[:, 0, y, :] = feq(1.0, [ux[y], 0.0, 0.0])[:, None]
    if hasattr(box, "set_populations"):
        box.set_populations(f0)
        jx = lambda: box.moments()[1][0, 0, :, 0]
    else:
        box.set_f(f0)
        jx = lambda: box.moments()[1][0, 0, :, 0]
    sin = np.sin(k * np.arange(ny))
    t0, t1 = 20, int(min(4000, 1.5 / (nu * k * k)))
    box.step(t0)
    a0 = (jx() * sin).sum()
    box.step(t1 - t0)
    a1 = (jx() * sin).sum()
    return -np.log(a1 / a0) / ((t1 - t0) * k * k)


@pytest.mark.parametrize("scheme", [1, 0, 2])
@pytest.mark.parametrize("tau", [0.55, 1.0, 2.0, 5.0])
def test_shear_wave_viscosity_gpu(F, oracle_mod, scheme, tau):
    """Noise-off shear wave, amplitude 1e-3, k = 2 pi / ny (Sec. II: nu =
    c_s^2 (tau - 1/2)).  FP64 storage: the hydrodynamic limit (Richardson over
    ny = 128, 256) within 1 % of nu and each fit equal to the oracle's.  FP32
    storage: the ny = 128 fit within 1 % of the oracle's (FP32 deviations
    resolve a decay of 1e-5 per step only to ~0.6 % at ny = 256, tau = 0.55)."""
    nu = CS2 * (tau - 0.5)
    feq = oracle_mod.feq2

    def gpu(prec):
        return lambda ny: (F.Lattice(2, ny, 1, tau, 0.0, scheme=scheme, precision=prec,
                                     stats_every=0), 2)

    def orc(ny):
        return oracle_mod.Box(1, ny, 1, tau, 0.0, scheme=scheme), 1

    g128, g256 = shear_fit(gpu(0), feq, tau, 128), shear_fit(gpu(0), feq, tau, 256)
    o128, o256 = shear_fit(orc, feq, tau, 128), shear_fit(orc, feq, tau, 256)
    assert abs(g128 / o128 - 1) < 1e-9 and abs(g256 / o256 - 1) < 1e-9
    assert abs((4 * g256 - g128) / 3 / nu - 1) < 0.01
    s128 = shear_fit(gpu(1), feq, tau, 128)
    assert abs(s128 / o128 - 1) < 0.01


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_init_thermal_samples_invariant_measure(F, oracle_mod, precision):
    """flbm_init_thermal: per-population variance rho0 kT w_i / c_s^2 (weights
    from the oracle's Table I), zero mean, per-node moment variances
    (3, 3, 5, 1) rho0 kT, and the same state for the same seed."""
    n, kT, rho0 = 32, 1e-4, 1.3
    w = oracle_mod.tables()["w"]
    g = F.Lattice(n, n, n, 0.8, kT, rho0=rho0, precision=precision)
    g.init_thermal(77)
    dev = (g.get_populations() - rho0 * w[:, None, None, None]).reshape(27, -1)
    var = dev.var(axis=1) / (rho0 * kT * w / CS2)
    assert np.all(np.abs(var - 1) < 0.05), var
    assert np.all(np.abs(dev.mean(axis=1)) < 5 * np.sqrt(rho0 * kT * w / CS2 / n ** 3))
    rho, j, pi = g.moments()
    obs = [rho, j.sum(0), pi[:3].sum(0), pi[3:].sum(0)]
    er = np.array([o.var() for o in obs]) / (np.array([3, 3, 5, 1]) * rho0 * kT)
    assert np.all(np.abs(er - 1) < 0.05), er
    h = F.Lattice(n, n, n, 0.8, kT, rho0=rho0, precision=precision)
    h.init_thermal(77)
    assert np.array_equal(g.get_state(), h.get_state())


@pytest.mark.parametrize("tau", [0.55, 100.0])
def test_spectral_er_gmf_vs_reg_same_noise(F, oracle_mod, tau):
    """Scaled form of the Sec. III comparison (Fig. 3): GMF-FLBM and Reg-FLBM
    driven by the same noise realisation (same seed; the noise keying is
    scheme independent) at the paper's kT = 1/3000, at a small viscosity and
    at the paper's largest tau (strong under-relaxation).  Both spectral
    equilibration ratios stay near 1 over the resolved shells and the two
    curves overlap."""
    from paper_2601_03806_gb300 import analysis
    n, kT, rho0 = 48, 1.0 / 3000.0, 1.0
    curves = {}
    for scheme in (1, 2):
        g = F.Lattice(n, n, n, tau, kT, rho0=rho0, seed=2601, scheme=scheme, precision=1,
                      stats_every=0)
        g.set_state(thermal_state(oracle_mod, n, kT, rho0, seed=5))
        g.step(100)
        curves[scheme] = analysis.er_spectrum(g, 28, snapshots=30, every=10)
    for m in analysis.PAPER_OBSERVABLES:
        er_g, cnt = curves[1][m]
        er_r, _ = curves[2][m]
        lo, hi = analysis.window_extrema(er_g, cnt, 4, 20)
        assert 0.85 < lo and hi < 1.15, (m, lo, hi)
        sel = slice(4, 21)
        assert np.abs(er_g[sel] - er_r[sel]).max() < 0.03, (m, er_g[sel], er_r[sel])


def test_smallest_viscosity_bgk_fails_gmf_and_reg_hold(F, oracle_mod):
    """Sec. III at the paper's smallest viscosity, tau = 0.5001, and its
    kT = 1/3000 (scaled to 48^3): BGK-FLBM, whose ghost modes relax with
    omega close to 2, goes unstable within a few hundred steps, while
    GMF-FLBM and Reg-FLBM stay stable.  Driven by the same noise, their
    spectral ER curves coincide (max difference < 0.01 on shells 4..20) and
    stay near 1 with the mild overestimation the paper reports at the
    smallest viscosities (observed 0.90..1.24)."""
    from paper_2601_03806_gb300 import analysis
    n, kT, rho0, tau = 48, 1.0 / 3000.0, 1.0, 0.5001
    g = F.Lattice(n, n, n, tau, kT, rho0=rho0, seed=2601, scheme=0, precision=1, stats_every=0)
    g.set_state(thermal_state(oracle_mod, n, kT, rho0, seed=5))
    with pytest.raises(F.FlbmError) as ei:
        g.step(400)
    assert ei.value.code == F.FLBM_E_UNSTABLE
    assert 0 < g.step_count < 400
    g.close()
    curves = {}
    for scheme in (1, 2):
        g = F.Lattice(n, n, n, tau, kT, rho0=rho0, seed=2601, scheme=scheme, precision=1,
                      stats_every=0)
        g.set_state(thermal_state(oracle_mod, n, kT, rho0, seed=5))
        g.step(100)
        curves[scheme] = analysis.er_spectrum(g, 28, snapshots=30, every=10)
        assert g.step_count == 400
        g.close()
    for m in analysis.PAPER_OBSERVABLES:
        er_g, cnt = curves[1][m]
        er_r, _ = curves[2][m]
        lo, hi = analysis.window_extrema(er_g, cnt, 4, 20)
        assert 0.85 < lo and hi < 1.3, (m, lo, hi)
        sel = slice(4, 21)
        assert np.abs(er_g[sel] - er_r[sel]).max() < 0.01, (m, er_g[sel], er_r[sel])


def test_spectral_er_abi(F):
    """flbm_spectral_er returns flbm_structure_factor's S_m(|k|) over the flat
    invariant-measure value (3, 3, 5, 1, 1, 1, 1) rho0 kT of each observable,
    and rejects kT = 0."""
    n, kT, rho0 = 32, 1e-4, 1.3
    g = F.Lattice(n, n, n, 0.8, kT, rho0=rho0, seed=5, precision=1)
    g.init_thermal(6)
    g.step(10)
    th = np.array([3, 3, 5, 1, 1, 1, 1]) * rho0 * kT
    for obs in range(7):
        er, cnt = g.spectral_er(obs, 24)
        S, cnt2 = g.structure_factor(obs, 24)
        assert np.array_equal(cnt, cnt2)
        assert np.allclose(er[cnt > 0], S[cnt > 0] / th[obs], rtol=1e-15, atol=0)
        assert np.all(er[cnt == 0] == 0)
        assert abs(er[2:16].mean() - 1) < 0.1          # a thermal sample: flat, near 1
    g.close()
    z = F.Lattice(8, 8, 8, 0.8, 0.0, precision=1)
    with pytest.raises(F.FlbmError) as ei:
        z.spectral_er(0, 8)
    assert ei.value.code == F.FLBM_E_INVALID
    z.close()
