"""The moment-state form (FLBM_STATE_MOMENTS, the paper's thread-safe
formulation at the end of Sec. II): ten numbers per node between steps,
populations rebuilt from the neighbours' numbers and regenerated noise.

* Against the population form on the same inputs: bit for bit.  Both forms
  hand the same rounded amplitudes and the same regenerated normals to the
  same reconstruction code, and collide the same FP32 populations; shapes
  cover several 30 x 14 columns with ragged edges, several z segments, and
  boxes smaller than a column (the halo wraps onto itself).
* Against the FP64 oracle: single-step populations within 2e-6 and moments
  within 1e-5 rho0 after 200 steps (the FP32 population-form tolerances).
* Reads between steps (populations rebuilt into the population buffer) do
  not perturb the run; checkpoints resume bit-exactly; instability is
  reported at the failing step.
* Full size (512^3, tau 0.6, kT 1e-5, the benchmark's launch): sampled nodes
  against the oracle's collision of the probed upstream populations.
"""
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


def box(F, shape, scheme, form, tau=0.8, kT=1e-4, seed=31, stats_every=1, stream=0):
    nx, ny, nz = shape
    return F.Lattice(nx, ny, nz, tau, kT, seed=seed, scheme=scheme, precision=F.FLBM_FP32,
                     stats_every=stats_every, noise_stream=stream, state_form=form)


SHAPES = [(37, 19, 5), (30, 14, 3), (32, 13, 3), (1, 1, 1), (64, 2, 9), (5, 31, 70), (61, 29, 2),
          (96, 27, 130)]


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("shape", SHAPES)
def test_matches_population_form_bit_for_bit(F, scheme, shape):
    a = box(F, shape, scheme, F.FLBM_STATE_POPULATIONS, stream=5)
    b = box(F, shape, scheme, F.FLBM_STATE_MOMENTS, stream=5)
    for lat in (a, b):
        lat.init_thermal(77)
    for k in (1, 1, 5):                    # boot, first moment step, then a run
        a.step(k)
        b.step(k)
        assert np.array_equal(a.get_state(), b.get_state()), (shape, a.step_count)
    sa, sb = a.stats(), b.stats()
    assert sa["step"] == sb["step"] and sa["n_samples"] == sb["n_samples"] == 7
    assert np.allclose(sa["u2_avg"], sb["u2_avg"], rtol=1e-6, atol=0)
    assert np.allclose(sa["m_var"], sb["m_var"], rtol=1e-5, atol=0)
    assert abs(sa["mass"] - sb["mass"]) < 1e-9 * np.prod(shape)
    a.close()
    b.close()


@pytest.mark.parametrize("kw", [dict(noise_rho0=True), dict(stats_every=3), dict(kT=0.0),
                                dict(torch_memory=True), dict(rho0=1.3, tau=2.5)])
def test_variants_match_population_form(F, kw):
    """Local or reference density in the noise amplitude, reductions every
    third step, no noise, a torch-owned population buffer, another density
    and viscosity."""
    shape = (34, 16, 7)
    args = dict(tau=0.9, kT=2e-4, seed=12, scheme=1, precision=F.FLBM_FP32, noise_stream=3)
    args.update(kw)
    a = F.Lattice(*shape, state_form=F.FLBM_STATE_POPULATIONS, **args)
    b = F.Lattice(*shape, state_form=F.FLBM_STATE_MOMENTS, **args)
    for lat in (a, b):
        lat.init_thermal(4)
    a.step(8)
    b.step(8)
    assert np.array_equal(a.get_state(), b.get_state())
    sa, sb = a.stats(), b.stats()
    assert sa["n_samples"] == sb["n_samples"]
    assert np.allclose(sa["u2_avg"], sb["u2_avg"], rtol=1e-6, atol=1e-30)


def test_reads_between_steps_do_not_change_the_run(F):
    shape = (45, 17, 12)
    ref = box(F, shape, 1, F.FLBM_STATE_POPULATIONS)
    m = box(F, shape, 1, F.FLBM_STATE_MOMENTS)
    for lat in (ref, m):
        lat.init_thermal(5)
    ref.step(9)
    m.step(3)
    m.get_populations()                    # rebuilt into the population buffer
    m.moments()
    m.step(2)
    m.structure_factor(0, 8)
    m.probe(np.array([0, 7, 100]))
    m.step(4)
    assert m.step_count == 9
    assert np.array_equal(ref.get_state(), m.get_state())


def test_checkpoint_resumes_bit_exactly(F):
    shape = (33, 15, 6)
    a = box(F, shape, 2, F.FLBM_STATE_MOMENTS, seed=8)
    a.step(10)
    b = box(F, shape, 2, F.FLBM_STATE_MOMENTS, seed=8)
    b.step(5)
    st = b.get_state()
    c = box(F, shape, 2, F.FLBM_STATE_MOMENTS, seed=8)
    c.set_state(st)
    c.set_step(5)
    c.step(5)
    assert np.array_equal(a.get_state(), c.get_state())
    b.set_step(5)                          # back to the populations, same step: no change
    b.step(5)
    assert np.array_equal(a.get_state(), b.get_state())


@pytest.mark.parametrize("scheme", [1, 2])
def test_against_oracle(F, O, scheme):
    nx, ny, nz = 31, 15, 9
    w = O.tables()["w"]
    f0 = w[:, None, None, None] * (1.0 + 0.02 * inputs.population_perturbation(nx, ny, nz, 12))
    g = box(F, (nx, ny, nz), scheme, F.FLBM_STATE_MOMENTS, tau=0.7, kT=1e-4, seed=3, stream=2)
    o = O.Box(nx, ny, nz, 0.7, 1e-4, seed=3, scheme=scheme, stream=2)
    g.set_populations(f0)
    o.set_f(f0)
    g.step(1)
    o.step(1)
    assert np.abs(g.get_populations() - o.get_f()).max() < 2e-6
    g.step(2)                              # two moment-form steps
    o.step(2)
    assert np.abs(g.get_populations() - o.get_f()).max() < 4e-6
    g.step(197)
    o.step(197)
    rho, j, _ = g.moments()
    orho, oj, _ = o.moments()
    assert np.abs(rho - orho).max() < 1e-5
    assert np.abs(j - oj).max() < 1e-5


def test_instability_is_reported(F, O):
    shape = (12, 9, 4)
    w = O.tables()["w"]
    f0 = np.tile(w[:, None, None, None], (1, shape[2], shape[1], shape[0]))
    g = box(F, shape, 1, F.FLBM_STATE_MOMENTS, kT=1e-5)
    g.step(3)
    f0[5, 1, 2, 3] = np.nan
    g.set_populations(f0)
    with pytest.raises(F.FlbmError) as ei:
        g.step(2)
    assert ei.value.code == F.FLBM_E_UNSTABLE
    assert g.step_count == 3


def test_full_size_sampled_nodes(F, O):
    """512^3 FP32 GMF, tau 0.6, kT 1e-5: the nodes' populations after a
    moment-form step against the oracle's collision of the probed upstream
    populations (probing rebuilds the populations of the current step)."""
    n, tau, kT, seed = 512, 0.6, 1e-5, 2024
    g = box(F, (n, n, n), 1, F.FLBM_STATE_MOMENTS, tau=tau, kT=kT, seed=seed)
    g.init_thermal(9)
    T = O.tables()
    c = T["c"]
    rng = np.random.default_rng(1)
    pts = rng.integers(0, n, size=(40, 3))
    pts[0] = (0, 0, 0)
    pts[1] = (n - 1, n - 1, n - 1)
    pts[2] = (29, 13, 127)                 # a column corner and a z-segment end
    pts[3] = (30, 14, 128)
    g.step(2)                              # boot + one moment step
    s1 = g.stats()                         # reductions of step 1
    for t_check in (2, 3):
        src = []
        for (x, y, z) in pts:
            for i in range(27):
                xs, ys, zs = (x - c[i, 0]) % n, (y - c[i, 1]) % n, (z - c[i, 2]) % n
                src.append(xs + n * (ys + n * zs))
        src = np.array(src)
        fin = g.probe(src)
        g.step(1)
        assert g.step_count == t_check + 1
        dst = np.array([x + n * (y + n * z) for (x, y, z) in pts])
        fout = g.probe(dst)
        for p in range(len(pts)):
            for i in range(27):
                fs = O.collide_node(1, tau, kT, fin[p * 27 + i], seed=seed,
                                    node=int(src[p * 27 + i]), step=t_check)
                assert abs(fout[p, i] - fs[i]) < 2e-6, (p, i, fout[p, i], fs[i])
    s = g.stats()
    assert s["n_samples"] == 4 and s["step"] == 3
    # a thermal sample has its own mass and momentum; the steps conserve them
    # (FP32 per-thread partial sums over ~2000 nodes each: ~1e-4 absolute)
    assert abs(s["mass"] / s1["mass"] - 1) < 1e-9
    assert np.abs(np.array(s["mom"]) - np.array(s1["mom"])).max() < 1e-2
