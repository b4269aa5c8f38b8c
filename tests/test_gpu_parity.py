"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (written here, derived from the arithmetic):
* FP64 storage: populations within 1e-12 absolute after 1000 steps (the
  paths differ only in rounding order: sum-factorised vs dense transforms,
  sincospi vs cos(2 pi u)); stats within 1e-12 relative.
* FP32 storage: moments within 1e-5 rho0 after 1000 steps; single-step
  populations within 2e-6 (FP32 rounding of O(1e-2) deviations plus the
  2^-21.4 absolute error of the hardware sin/cos in Box-Muller).
* FP16 storage: single-step populations within 2e-5 (half-precision rounding,
  2^-12 relative, of O(1e-2) deviations on load and store); after 1000 steps
  the rounding noise (~6e-6 per node and step in rho) random-walks in the
  conserved modes, so moments are bounded by 3e-3 rho0 (observed values are
  printed by the test).
"""
import numpy as np
import pytest

from synth import inputs

pytestmark = pytest.mark.gpu

CS2 = 1.0 / 3.0


@pytest.fixture(scope="module")
def F():
    from paper_2601_03806_gb300 import flbm
    return flbm


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def gpu(F, nx, ny, nz, tau, kT, seed=1234, scheme=1, precision=0, noise_rho0=False,
        stats_every=1, rho0=1.0):
    return F.Lattice(nx, ny, nz, tau, kT, rho0=rho0, seed=seed, scheme=scheme,
                     precision=precision, noise_rho0=noise_rho0, stats_every=stats_every)


def perturbed(O, nx, ny, nz, seed, amp=0.01, rho0=1.0):
    w = O.tables()["w"]
    return w[:, None, None, None] * (rho0 + amp * inputs.population_perturbation(nx, ny, nz, seed))


# ---------------------------------------------------------------------------
# Config 1: 16^3, FP64, rho0=1, u=0 equilibrium start, kT=1e-4, tau=0.8,
# 1000 steps, seed 1234.


def test_fp64_gmf_config1_populations_and_stats(F, O):
    n, tau, kT, seed = 16, 0.8, 1e-4, 1234
    g = gpu(F, n, n, n, tau, kT, seed=seed)
    o = O.Box(n, n, n, tau, kT, seed=seed)
    # odd step count first: exercises the AA odd form in get_populations
    g.step(7)
    o.step(7)
    assert np.abs(g.get_populations() - o.get_f()).max() < 1e-12
    # per-step oracle statistics for the time averages
    u2, m, m2 = [], [], []
    def record():
        rho, j, pi = o.moments()
        u2.append(((j / rho) ** 2).mean(axis=(1, 2, 3)))
        obs = [rho - 1.0, j.sum(0), pi[:3].sum(0) - 1.0, pi[3:].sum(0)]
        m.append([x.mean() for x in obs])
        m2.append([(x * x).mean() for x in obs])
    g.stats_reset()
    for _ in range(992):
        record()
        o.step(1)
    g.step(992)
    record()
    rho, j, pi = o.moments()
    s = g.stats()
    g.step(1)
    o.step(1)
    assert g.step_count == o.t == 1000
    assert np.abs(g.get_populations() - o.get_f()).max() < 1e-12
    s = g.stats()
    assert s["step"] == 999 and s["n_samples"] == 993
    N = n ** 3
    assert abs(s["mass"] - rho.sum()) < 1e-12 * N
    assert abs(s["mass"] - N) < 1e-12 * N                     # conservation
    assert np.allclose(s["mom"], j.sum(axis=(1, 2, 3)), atol=1e-12 * N, rtol=0)
    assert np.allclose(s["u2"], u2[-1], rtol=1e-10, atol=0)
    assert np.allclose(s["u2_avg"], np.mean(u2, 0), rtol=1e-10, atol=0)
    mm, mm2 = np.mean(m, 0), np.mean(m2, 0)
    # the oracle stores absolute f, so its mean density carries its own FP64
    # roundoff drift (~3e-14 after 1000 steps); the library stores deviations
    assert np.allclose(s["m_mean"], mm, rtol=0, atol=1e-12)
    assert np.allclose(s["m_var"], mm2 - mm * mm, rtol=1e-9, atol=0)
    er = (mm2 - mm * mm) / (np.array([3, 3, 5, 1]) * kT)
    assert np.allclose(s["er"], er, rtol=1e-9, atol=0)


@pytest.mark.parametrize("scheme", [0, 1, 2])
@pytest.mark.parametrize("shape", [(130, 3, 2), (5, 4, 3), (1, 1, 1), (1, 7, 1), (2, 1, 3)])
def test_fp64_schemes_ragged_boxes(F, O, scheme, shape):
    nx, ny, nz = shape
    tau, kT = 0.7, 1e-3
    f0 = perturbed(O, nx, ny, nz, seed=nx * 100 + ny * 10 + nz)
    g = gpu(F, nx, ny, nz, tau, kT, seed=77, scheme=scheme)
    o = O.Box(nx, ny, nz, tau, kT, seed=77, scheme=scheme)
    g.set_populations(f0)
    o.set_f(f0)
    for nsteps in (1, 4, 15):
        g.step(nsteps)
        o.step(nsteps)
        assert np.abs(g.get_populations() - o.get_f()).max() < 1e-12, nsteps


@pytest.mark.parametrize("noise_rho0", [False, True])
def test_fp64_noise_density_reading(F, O, noise_rho0):
    nx, ny, nz = 6, 5, 4
    f0 = perturbed(O, nx, ny, nz, seed=5, amp=0.05, rho0=1.3)
    g = gpu(F, nx, ny, nz, 0.9, 1e-3, seed=11, noise_rho0=noise_rho0, rho0=1.3)
    o = O.Box(nx, ny, nz, 0.9, 1e-3, rho0=1.3, seed=11, noise_rho0=noise_rho0)
    g.set_populations(f0)
    o.set_f(f0)
    g.step(9)
    o.step(9)
    assert np.abs(g.get_populations() - o.get_f()).max() < 1e-12


def test_fp32_gmf_config1_moments(F, O):
    n, tau, kT, seed = 16, 0.8, 1e-4, 1234
    g = gpu(F, n, n, n, tau, kT, seed=seed, precision=1)
    o = O.Box(n, n, n, tau, kT, seed=seed)
    g.step(1000)
    o.step(1000)
    for a, b in zip(g.moments(), o.moments()):
        assert np.abs(a - b).max() < 1e-5
    s = g.stats()
    assert abs(s["mass"] - n ** 3) < 1e-9 * n ** 3


def test_fp16_config1_moments(F, O):
    n, tau, kT, seed = 16, 0.8, 1e-4, 1234
    g = gpu(F, n, n, n, tau, kT, seed=seed, precision=2)
    o = O.Box(n, n, n, tau, kT, seed=seed)
    g.step(1000)
    o.step(1000)
    errs = [float(np.abs(a - b).max()) for a, b in zip(g.moments(), o.moments())]
    print("fp16 max |moment error| after 1000 steps (rho, j, Pi):", errs)
    assert max(errs) < 3e-3
    s = g.stats()
    assert abs(s["mass"] / n ** 3 - 1) < 1e-5


@pytest.mark.parametrize("scheme", [0, 1, 2])
@pytest.mark.parametrize("shape", [(130, 3, 2), (7, 5, 3), (64, 3, 2)])
def test_fp16_populations_short(F, O, scheme, shape):
    nx, ny, nz = shape
    f0 = perturbed(O, nx, ny, nz, seed=3, amp=0.02)
    g = gpu(F, nx, ny, nz, 0.6, 1e-4, seed=5, scheme=scheme, precision=2)
    o = O.Box(nx, ny, nz, 0.6, 1e-4, seed=5, scheme=scheme)
    g.set_populations(f0)
    o.set_f(f0)
    g.step(1)
    o.step(1)
    assert np.abs(g.get_populations() - o.get_f()).max() < 2e-5


@pytest.mark.parametrize("scheme", [0, 1, 2])
@pytest.mark.parametrize("shape", [(130, 3, 2), (7, 5, 3), (1, 1, 1)])
def test_fp32_populations_short(F, O, scheme, shape):
    nx, ny, nz = shape
    f0 = perturbed(O, nx, ny, nz, seed=3, amp=0.02)
    g = gpu(F, nx, ny, nz, 0.6, 1e-4, seed=5, scheme=scheme, precision=1)
    o = O.Box(nx, ny, nz, 0.6, 1e-4, seed=5, scheme=scheme)
    g.set_populations(f0)
    o.set_f(f0)
    g.step(1)
    o.step(1)
    assert np.abs(g.get_populations() - o.get_f()).max() < 2e-6
    g.step(6)
    o.step(6)
    assert np.abs(g.get_populations() - o.get_f()).max() < 1e-5


# ---------------------------------------------------------------------------
# State handling: checkpoints, AA parity, probes


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("k", [4, 5])
def test_resume_is_bit_exact(F, precision, k):
    a = gpu(F, 9, 8, 7, 0.75, 1e-4, seed=99, precision=precision)
    a.step(2 * k)
    b = gpu(F, 9, 8, 7, 0.75, 1e-4, seed=99, precision=precision)
    b.step(k)
    st = b.get_state()
    c = gpu(F, 9, 8, 7, 0.75, 1e-4, seed=99, precision=precision)
    c.set_state(st)
    c.set_step(k)
    c.step(k)
    assert np.array_equal(a.get_state(), c.get_state())
    assert np.array_equal(a.get_populations(), c.get_populations())


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_set_get_and_probe_roundtrip(F, O, precision):
    nx, ny, nz = 10, 6, 3
    f0 = perturbed(O, nx, ny, nz, seed=8)
    g = gpu(F, nx, ny, nz, 0.8, 1e-4, precision=precision)
    g.step(3)                         # odd AA form in storage
    g.set_populations(f0)             # natural form again
    tol = {0: 0.0, 1: 1e-8, 2: 5e-6}[precision]
    assert np.abs(g.get_populations() - f0).max() <= tol
    g.step(1)
    f1 = g.get_populations()
    nodes = np.array([0, 5, 17, nx * ny * nz - 1, 33])
    pr = g.probe(nodes)
    assert np.array_equal(pr, f1.reshape(27, -1)[:, nodes].T)
    g.set_step(10)
    assert np.array_equal(g.get_populations(), f1)


def test_unstable_state_is_reported(F, O):
    f0 = perturbed(O, 6, 6, 6, seed=2)
    f0[3, 2, 2, 2] = np.nan
    g = gpu(F, 6, 6, 6, 0.8, 1e-5, precision=1)
    g.step(4)
    g.set_populations(f0)
    with pytest.raises(F.FlbmError) as ei:
        g.step(3)
    assert ei.value.code == F.FLBM_E_UNSTABLE
    assert g.step_count == 4


# ---------------------------------------------------------------------------
# S(k)


@pytest.mark.parametrize("precision,rtol", [(0, 1e-10), (1, 2e-4)])
def test_structure_factor_parity(F, O, precision, rtol):
    nx, ny, nz = 12, 10, 8
    g = gpu(F, nx, ny, nz, 0.8, 1e-4, seed=4, precision=precision)
    o = O.Box(nx, ny, nz, 0.8, 1e-4, seed=4)
    g.step(40)
    o.step(40)
    rho, j, pi = o.moments()
    fields = [rho, j.sum(0), pi[:3].sum(0), pi[3:].sum(0), j[0], j[1], j[2]]
    for obs, m in enumerate(fields):
        S, cnt = g.structure_factor(obs, 12)
        So, cnto = O.structure_factor(m, 12)
        assert np.array_equal(cnt, cnto)
        assert np.allclose(S, So, rtol=rtol, atol=1e-30), obs


# ---------------------------------------------------------------------------
# Full-size launch configuration of the benchmark (512^3 GMF, tau=0.6,
# kT=1e-5; FP32 storage, and the FP16 storage variant): sampled nodes checked
# one by one against the oracle's collision of the probed inputs.


# mom_tol: total momentum starts at 0 and the collision conserves it; what
# remains is storage rounding: about 1e-10 per node and step in FP32, about
# 2e-6 in FP16 (half ulp of deviations of ~3e-3), random-walking over N =
# 1.3e8 nodes and 4 steps to ~2e-6 (FP32) and ~0.05 (FP16)
@pytest.mark.parametrize("precision,tol,mom_tol", [(1, 2e-6, 1e-3), (2, 2e-5, 0.2)])
def test_full_size_sampled_nodes(F, O, precision, tol, mom_tol):
    n, tau, kT, seed = 512, 0.6, 1e-5, 2024
    g = gpu(F, n, n, n, tau, kT, seed=seed, precision=precision)
    T = O.tables()
    c = T["c"]
    rng = np.random.default_rng(0)
    pts = rng.integers(0, n, size=(48, 3))
    pts[0] = (0, 0, 0)
    pts[1] = (n - 1, n - 1, n - 1)
    for t_check in (2, 3):
        g.step(t_check - g.step_count)
        src = []
        for (x, y, z) in pts:
            for i in range(27):
                xs, ys, zs = (x - c[i, 0]) % n, (y - c[i, 1]) % n, (z - c[i, 2]) % n
                src.append(xs + n * (ys + n * zs))
        src = np.array(src)
        fin = g.probe(src)
        g.step(1)
        dst = np.array([x + n * (y + n * z) for (x, y, z) in pts])
        fout = g.probe(dst)
        for p in range(len(pts)):
            for i in range(27):
                fs = O.collide_node(1, tau, kT, fin[p * 27 + i], seed=seed,
                                    node=int(src[p * 27 + i]), step=t_check)
                assert abs(fout[p, i] - fs[i]) < tol, (p, i, fout[p, i], fs[i])
    s = g.stats()
    assert abs(s["mass"] / n ** 3 - 1) < 1e-9
    assert np.abs(s["mom"]).max() < mom_tol


# ---------------------------------------------------------------------------
# TMA row pipeline (rows whose length is a multiple of 32): parity with the
# oracle, degenerate row neighbourhoods (ny, nz in {1, 2}), and bitwise
# agreement with the direct kernel on the same inputs.


@pytest.mark.parametrize("scheme", [0, 1, 2])
@pytest.mark.parametrize("shape", [(32, 3, 2), (64, 5, 4), (96, 2, 1), (32, 1, 1), (64, 1, 2),
                                   # two nodes per thread (FP32 / FP16 rows of 256 and more):
                                   # degenerate neighbourhoods, and 144 pairs over 96 threads
                                   (256, 1, 1), (256, 2, 1), (512, 1, 2), (288, 3, 2)])
def test_row_pipeline_parity(F, O, scheme, shape):
    nx, ny, nz = shape
    f0 = perturbed(O, nx, ny, nz, seed=ny * 7 + nz, amp=0.02)
    for precision, tol in ((0, 1e-12), (1, 2e-6), (2, 2e-5)):
        g = gpu(F, nx, ny, nz, 0.7, 1e-4, seed=13, scheme=scheme, precision=precision)
        o = O.Box(nx, ny, nz, 0.7, 1e-4, seed=13, scheme=scheme)
        g.set_populations(f0)
        o.set_f(f0)
        for nsteps in (1, 2, 5):
            g.step(nsteps)
            o.step(nsteps)
            assert np.abs(g.get_populations() - o.get_f()).max() < tol * nsteps, (precision, nsteps)


@pytest.mark.parametrize("scheme", [0, 1, 2])
@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("shape", [(64, 6, 5), (256, 3, 2), (512, 3, 2)])
def test_row_pipeline_matches_direct_kernel(F, O, precision, shape, scheme, monkeypatch):
    """Same inputs through the TMA row pipeline with two nodes per thread
    (packed FP32 pairs; rows of 256 and more in FP32 / FP16; rows of 512 run
    the kernel whose row length is a compile-time constant), with one node
    per thread, and through the direct kernel (FP64 512-rows fall back to it
    in every case): identical populations, bit for bit, as every kernel runs
    the same sequence of singly rounded operations per node."""
    nx, ny, nz = shape
    f0 = perturbed(O, nx, ny, nz, seed=4, amp=0.02)
    out = []
    for rows, pairs in (("1", "1"), ("1", "0"), ("0", "1")):
        monkeypatch.setenv("FLBM_ROWS", rows)
        monkeypatch.setenv("FLBM_ROW_PAIRS", pairs)
        g = gpu(F, nx, ny, nz, 0.6, 1e-4, seed=21, scheme=scheme, precision=precision)
        g.set_populations(f0)
        g.step(7)
        out.append((g.get_state(), g.stats()))
    for o in out[1:]:
        assert np.array_equal(out[0][0], o[0])
    # the sums are added in different orders (per-thread, per-warp, per-CTA)
    rtol = 1e-12 if precision == 0 else 1e-5
    for o in out[1:]:
        for k in ("mass", "u2", "m_var"):
            assert np.allclose(out[0][1][k], o[1][k], rtol=rtol, atol=1e-300)
