"""Batched ensemble (flbm_ensemble_*): many replica boxes advanced by one
persistent kernel per step.

* Every replica evolves as the single box of the same parameters (same
  noise stream): after 7 steps the states are identical, bit for bit (FP32
  or FP16; both kernels run the same singly rounded operations per node).
  Within the ensemble the results are bit for bit independent of the launch
  shape and of the CUDA graph.
* Against the FP64 oracle (a Box on the replica's noise stream): single-step
  populations within 2e-6 (FP32; the tolerance of the single-box parity
  tests) and moments within 1e-5 rho0 after 200 steps.
* The mixed-size workload of 256 x 32^3 + 64 x 64^3 + 8 x 128^3 replicas
  (tau uniform in [0.51, 3.0], kT = 1e-5, one stream per replica), in the
  launch shape the benchmark times: sampled replicas against the oracle.
* Statistics per replica, the autotuner's reset, the replica restrictions,
  and failure reports naming the replica.
* The full config-4 run (the mixed workload, 5000 steps): equipartition and
  ER of every replica within 1 %, and flat class-averaged structure factors.
"""
import time

import numpy as np
import pytest

from synth import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2601_03806_gb300 import flbm
    return flbm


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


SEED = 77

# (nx, ny, nz, tau, kT, rho0, noise_stream): ragged mixes of row lengths,
# rows per item (ny prime, ny < rows an item wants), thin boxes (ny, nz in
# {1, 2}) and densities
MIX = [
    (32, 8, 4, 0.7, 1e-4, 1.0, 1),
    (64, 6, 3, 1.3, 2e-4, 1.0, 2),
    (32, 5, 2, 0.55, 1e-4, 0.8, 7),
    (96, 4, 2, 2.5, 5e-5, 1.2, 3),
    (32, 1, 1, 0.9, 1e-4, 1.0, 11),
    (128, 2, 3, 0.6, 1e-4, 1.0, 12),
]


def make_params(F, mix, precision=1, scheme=1, stats_every=1):
    return [F.make_params(nx, ny, nz, tau, kT, rho0=rho0, seed=SEED, scheme=scheme,
                          precision=precision, stats_every=stats_every, noise_stream=s)
            for (nx, ny, nz, tau, kT, rho0, s) in mix]


def thermal(ens):
    for r, rep in enumerate(ens.replicas):
        rep.init_thermal(1000 + r)


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_replicas_match_single_boxes(F, precision, scheme):
    params = make_params(F, MIX, precision=precision, scheme=scheme)
    ens = F.Ensemble(params)
    thermal(ens)
    ens.step(7)                       # 3 graph periods + 1 eager step
    for r, (nx, ny, nz, tau, kT, rho0, s) in enumerate(MIX):
        box = F.Lattice(nx, ny, nz, tau, kT, rho0=rho0, seed=SEED, scheme=scheme,
                        precision=precision, noise_stream=s)
        box.init_thermal(1000 + r)
        box.step(7)
        assert ens[r].step_count == 7
        # the same singly rounded operations per node as the single-box
        # kernels: identical populations, bit for bit
        assert np.array_equal(ens[r].get_state(), box.get_state()), r
        sa, sb = ens[r].stats(), box.stats()
        assert sa["step"] == sb["step"] == 6 and sa["n_samples"] == sb["n_samples"] == 7
        assert np.allclose(sa["u2_avg"], sb["u2_avg"], rtol=1e-5, atol=0)
        assert np.allclose(sa["m_var"], sb["m_var"], rtol=1e-4, atol=0)
        assert abs(sa["mass"] - sb["mass"]) < 1e-6 * nx * ny * nz
        box.close()
    ens.close()


@pytest.mark.parametrize("shape", [dict(item_nodes=128, stages=4, compute_warps=4, ctas_per_sm=1),
                                   dict(item_nodes=512, stages=3, compute_warps=8, ctas_per_sm=1),
                                   dict(item_nodes=32, stages=2, compute_warps=1, ctas_per_sm=2)])
def test_launch_shape_and_graph_do_not_change_results(F, shape):
    params = make_params(F, MIX, stats_every=3)
    ref = F.Ensemble(params)
    ref.graph(False)
    thermal(ref)
    ref.step(12)
    ens = F.Ensemble(params)
    ens.set_tuning(**shape)
    t = ens.tuning
    assert all(t[k] == v for k, v in shape.items() if k != "ctas_per_sm")
    thermal(ens)
    ens.step(4)                        # eager steps 0..3, then 4, 5 eager and
    ens.step(8)                        # 6..11 from the graph (period 6)
    for r in range(len(MIX)):
        assert np.array_equal(ref[r].get_state(), ens[r].get_state()), r
        sa, sb = ref[r].stats(), ens[r].stats()
        assert sa["n_samples"] == sb["n_samples"] == 4
        assert np.allclose(sa["u2_avg"], sb["u2_avg"], rtol=1e-5, atol=0)


@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_replicas_against_oracle(F, O, scheme):
    mix = MIX[:4]
    params = make_params(F, mix, scheme=scheme)
    ens = F.Ensemble(params)
    boxes = []
    for r, (nx, ny, nz, tau, kT, rho0, s) in enumerate(mix):
        w = O.tables()["w"]
        f0 = w[:, None, None, None] * (rho0 + 0.02 * inputs.population_perturbation(nx, ny, nz, 40 + r))
        ens[r].set_populations(f0)
        o = O.Box(nx, ny, nz, tau, kT, rho0=rho0, seed=SEED, scheme=scheme, stream=s)
        o.set_f(f0)
        boxes.append(o)
    ens.step(1)
    for r, o in enumerate(boxes):
        o.step(1)
        assert np.abs(ens[r].get_populations() - o.get_f()).max() < 2e-6, r
    ens.step(199)
    for r, o in enumerate(boxes):
        o.step(199)
        rho, j, _ = ens[r].moments()
        orho, oj, _ = o.moments()
        rho0 = mix[r][5]
        assert np.abs(rho - orho).max() < 1e-5 * rho0, r
        assert np.abs(j - oj).max() < 1e-5 * rho0, r


def test_stats_per_replica_and_equipartition(F):
    mix = [(32, 32, 32, tau, 1e-5, 1.0, r) for r, tau in enumerate((0.51, 0.8, 1.5, 3.0))]
    ens = F.Ensemble(make_params(F, mix))
    thermal(ens)
    mass0 = [rep.moments()[0].sum() for rep in ens.replicas]   # the sample's own mass
    ens.step(20)
    for rep in ens.replicas:
        rep.stats_reset()
    ens.step(200)
    for r, rep in enumerate(ens.replicas):
        s = rep.stats()
        assert s["n_samples"] == 200 and s["step"] == 219
        # <u_a^2> = kT / rho0 (Sec. III); 200 steps of 32^3 nodes: ~1% noise
        assert np.all(np.abs(np.array(s["u2_avg"]) / 1e-5 - 1) < 0.05), (r, s["u2_avg"])
        assert abs(s["mass"] / mass0[r] - 1) < 1e-7


def test_autotune_resets_to_rest(F):
    ens = F.Ensemble(make_params(F, MIX))
    best = ens.autotune(steps_per_trial=2)
    assert best["ms_per_step"] > 0
    assert 2 <= best["stages"] <= 4 and best["item_nodes"] in (128, 256, 512)
    assert ens.step_count == 0
    for rep in ens.replicas:
        assert rep.step_count == 0
        assert not np.any(rep.get_state())
        assert rep.stats()["n_samples"] == 0
    # the tuned ensemble reproduces an untuned one
    ref = F.Ensemble(make_params(F, MIX))
    for e in (ens, ref):
        thermal(e)
        e.step(5)
    for r in range(len(MIX)):
        assert np.array_equal(ens[r].get_state(), ref[r].get_state()), r
    with pytest.raises(F.FlbmError) as ei:
        ens.autotune(1)                # only at step 0
    assert ei.value.code == F.FLBM_E_INVALID


def test_replica_restrictions(F):
    ens = F.Ensemble(make_params(F, MIX[:2]))
    rep = ens[0]
    with pytest.raises(F.FlbmError) as ei:
        rep.step(1)
    assert ei.value.code == F.FLBM_E_INVALID
    with pytest.raises(F.FlbmError):
        rep.set_step(4)
    g = rep.get_state()
    ens.step(1)
    with pytest.raises(F.FlbmError) as ei:       # odd step: AA-shifted storage
        rep.set_state(g)
    assert ei.value.code == F.FLBM_E_INVALID
    ens.step(1)
    rep.set_state(g)                             # even step: allowed
    assert np.array_equal(rep.get_state(), g)
    F.flbm_destroy(rep.handle)                   # a replica is not destroyed alone
    assert rep.step_count == 2


def test_instability_names_the_replica(F, O):
    mix = MIX[:3]
    ens = F.Ensemble(make_params(F, mix))
    nx, ny, nz = mix[2][:3]
    f = np.tile(O.tables()["w"][:, None, None, None], (1, nz, ny, nx))
    f[:, 1, 2, 5] = -0.1                         # rho < 0 at one node of replica 2
    ens[2].set_populations(f)
    with pytest.raises(F.FlbmError) as ei:
        ens.step(2)
    assert ei.value.code == F.FLBM_E_UNSTABLE
    assert "replica 2" in str(ei.value)


def test_bounded_wait_runs_out(F, monkeypatch):
    monkeypatch.setenv("FLBM_INJECT_STARVE", "1")
    ens = F.Ensemble(make_params(F, MIX[:2]))
    monkeypatch.delenv("FLBM_INJECT_STARVE")
    t0 = time.time()
    with pytest.raises(F.FlbmError) as ei:
        ens.step(1)
    assert ei.value.code == F.FLBM_E_TIMEOUT
    assert time.time() - t0 < 30
    ens.close()
    ok = F.Ensemble(make_params(F, MIX[:2]))
    ok.step(3)
    assert ok.step_count == 3


# ---------------------------------------------------------------------------
# The mixed-size ensemble in the benchmark's launch shape


def mixed_workload(F, precision=1, seed=20260101):
    rng = np.random.default_rng(seed)
    sizes = [32] * 256 + [64] * 64 + [128] * 8
    taus = rng.uniform(0.51, 3.0, size=len(sizes))
    return [F.make_params(n, n, n, float(t), 1e-5, seed=seed, precision=precision, noise_stream=r)
            for r, (n, t) in enumerate(zip(sizes, taus))]


def test_mixed_workload_sampled_replicas(F, O):
    params = mixed_workload(F)
    ens = F.Ensemble(params)
    assert len(ens) == 328 and ens.nodes == 256 * 32 ** 3 + 64 * 64 ** 3 + 8 * 128 ** 3
    thermal(ens)
    sample = [0, 255, 256, 319, 320, 327]
    f0 = {r: ens[r].get_populations() for r in sample}
    mass0 = {r: f0[r].sum() for r in sample}
    ens.step(3)
    for r in sample:
        p = params[r]
        o = O.Box(p.nx, p.ny, p.nz, p.tau, p.kT, seed=p.seed, stream=r)
        o.set_f(f0[r])
        o.step(3)
        d = np.abs(ens[r].get_populations() - o.get_f()).max()
        assert d < 6e-6, (r, d)
        s = ens[r].stats()
        assert s["n_samples"] == 3 and abs(s["mass"] / mass0[r] - 1) < 1e-7


def test_fp16_replicas_against_oracle(F, O):
    """FP16 deviation storage: one step of every replica against the oracle
    within 2e-5 (the single-box FP16 tolerance: half rounding on load and
    store of O(1e-2) deviations)."""
    mix = MIX[:3]
    ens = F.Ensemble(make_params(F, mix, precision=2))
    boxes = []
    for r, (nx, ny, nz, tau, kT, rho0, s) in enumerate(mix):
        w = O.tables()["w"]
        f0 = w[:, None, None, None] * (rho0 + 0.02 * inputs.population_perturbation(nx, ny, nz, 60 + r))
        ens[r].set_populations(f0)
        o = O.Box(nx, ny, nz, tau, kT, rho0=rho0, seed=SEED, stream=s)
        o.set_f(ens[r].get_populations())   # the oracle starts from the stored (half-rounded) state
        boxes.append(o)
    ens.step(1)
    for r, o in enumerate(boxes):
        o.step(1)
        assert np.abs(ens[r].get_populations() - o.get_f()).max() < 2e-5, r


def test_replica_structure_factor_matches_single_box(F):
    """S(k) of a replica (its borrowed context) against the single box of the
    same parameters and noise stream: the states agree to a few units in the
    last place, so the spectra agree to 1e-5 relative."""
    nx = ny = nz = 32
    params = [F.make_params(nx, ny, nz, 0.8, 1e-4, seed=SEED, noise_stream=s) for s in (4, 9)]
    ens = F.Ensemble(params)
    for r, rep in enumerate(ens.replicas):
        rep.init_thermal(70 + r)
    ens.step(6)
    box = F.Lattice(nx, ny, nz, 0.8, 1e-4, seed=SEED, noise_stream=9)
    box.init_thermal(71)
    box.step(6)
    for obs in range(7):
        Sa, ca = ens[1].structure_factor(obs, 16)
        Sb, cb = box.structure_factor(obs, 16)
        assert np.array_equal(ca, cb)
        assert np.allclose(Sa, Sb, rtol=1e-5, atol=1e-30), obs
    box.close()
    ens.close()


def test_config4_5000_steps_statistics(F):
    """The mixed ensemble over the full run (5000 steps after an invariant-
    measure start, statistics every step): every replica meets the 1 %
    equipartition gate and keeps its four ER ratios within 1 %, and the
    structure factors of each size class, averaged over its replicas (one
    snapshot each), are flat at their Sec. III values (3, 3, 5, 1) rho0 kT:
    the class mean over shells within 1 %, every shell within five standard
    errors of a mean of cnt/2 independent exponential variables per replica
    (the squared modulus of a Gaussian Fourier amplitude, k and -k paired)."""
    params = mixed_workload(F)
    ens = F.Ensemble(params)
    thermal(ens)
    ens.step(1)
    for rep in ens.replicas:
        rep.stats_reset()
    ens.step(5000)
    sizes = np.array([p.nx for p in params])
    for r, rep in enumerate(ens.replicas):
        s = rep.stats()
        assert s["n_samples"] == 5000
        u2 = np.array(s["u2_avg"]) / 1e-5
        assert np.all(np.abs(u2 - 1) < 0.01), (r, u2)
        assert np.all(np.abs(np.array(s["er"]) - 1) < 0.01), (r, s["er"])
    theory = np.array([3, 3, 5, 1]) * 1e-5
    for n in (32, 64, 128):
        idx = np.where(sizes == n)[0]
        nsh = n // 2
        acc = np.zeros((4, nsh))
        for r in idx:
            for obs in range(4):
                S, cnt = ens[r].structure_factor(obs, nsh)
                acc[obs] += S
        acc /= len(idx)
        shells = slice(2, nsh - 2)
        for obs in range(4):
            ratio = acc[obs, shells] / theory[obs]
            assert abs(ratio.mean() - 1) < 0.01, (n, obs, ratio.mean())
            bound = 5.0 / np.sqrt(0.5 * cnt[shells] * len(idx))
            assert np.all(np.abs(ratio - 1) < bound), (n, obs, ratio, bound)
    ens.close()
