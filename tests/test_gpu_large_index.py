"""Boxes whose population index 27 N passes 2^32 (544^3: 27 N = 4.35e9), so
every kernel runs its 64-bit index instantiation: the TMA row pipeline (FP32,
FP16), the direct kernel (FP32, FP64), the moment-state step and the learned
step.  Sampled nodes, including the last plane's, against the oracle's
collision of the probed upstream populations (within the single-step
tolerances of the storage type: 2e-6 FP32, 2e-5 FP16, 1e-12 FP64) or the
oracle's network correction (learned step, within the propagated bf16
bound of test_gpu_mlp)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N3 = 544
TAU, KT, SEED = 0.6, 1e-5, 77


@pytest.fixture(scope="module")
def F():
    from paper_2601_03806_gb300 import flbm
    return flbm


def sample_points(n):
    rng = np.random.default_rng(5)
    pts = rng.integers(0, n, size=(24, 3))
    pts[0] = (0, 0, 0)
    pts[1] = (n - 1, n - 1, n - 1)
    pts[2] = (n - 1, 0, n - 1)          # node indices near N - 1 (27 N > 2^32)
    pts[3] = (3, n - 2, n - 1)
    return pts


def check_steps(lat, O, n, t_checks, tol=2e-6):
    c = O.tables()["c"]
    pts = sample_points(n)
    for t in t_checks:
        lat.step(t - lat.step_count)
        src = np.array([((x - c[i, 0]) % n) + n * (((y - c[i, 1]) % n) + n * ((z - c[i, 2]) % n))
                        for (x, y, z) in pts for i in range(27)])
        fin = lat.probe(src)
        lat.step(1)
        fout = lat.probe(np.array([x + n * (y + n * z) for (x, y, z) in pts]))
        for p in range(len(pts)):
            for i in range(27):
                fs = O.collide_node(1, TAU, KT, fin[p * 27 + i], seed=SEED, node=int(src[p * 27 + i]), step=t)
                assert abs(fout[p, i] - fs[i]) < tol, (t, p, i, fout[p, i], fs[i])


@pytest.mark.parametrize("rows,precision,tol", [
    ("1", 1, 2e-6),      # FP32 TMA row pipeline
    ("0", 1, 2e-6),      # FP32 direct kernel
    ("1", 2, 2e-5),      # FP16 storage, row pipeline (half rounding on load and store)
    ("1", 0, 1e-12),     # FP64: rows of 544 exceed the row pipeline's shared memory -> direct
])
def test_population_form_64bit_index(F, oracle_mod, rows, precision, tol, monkeypatch):
    monkeypatch.setenv("FLBM_ROWS", rows)
    lat = F.Lattice(N3, N3, N3, TAU, KT, seed=SEED, precision=precision)
    lat.init_thermal(2)
    check_steps(lat, oracle_mod, N3, (1, 2), tol)
    lat.close()


def test_moment_form_64bit_index(F, oracle_mod):
    lat = F.Lattice(N3, N3, N3, TAU, KT, seed=SEED, state_form=F.FLBM_STATE_MOMENTS)
    lat.init_thermal(2)
    lat.step(1)                                        # the first collision, from populations
    check_steps(lat, oracle_mod, N3, (1, 2))           # moment-form steps
    lat.close()


def test_learned_step_64bit_index(F, oracle_mod):
    from oracle import mlp as M
    O = oracle_mod
    n, tau, kT, rho0 = N3, 0.8, 1e-3, 1.0
    rng = np.random.default_rng(9)
    theta = M.init_params(9)
    p = M.unpack(theta)
    for b in ("b1", "b2", "b3"):
        p[b] = p[b] + 0.3 * rng.normal(size=p[b].shape)
    theta = M.pack(p).astype(np.float32).astype(np.float64)
    c, w = O.tables()["c"], O.tables()["w"]
    pts = sample_points(n)
    node = lambda x, y, z: int(x % n + n * ((y % n) + n * (z % n)))
    post = {}
    pre = None
    for scheme in (F.FLBM_GMF, F.FLBM_LEARNED):
        b = F.Lattice(n, n, n, tau, kT, rho0=rho0, seed=21, scheme=scheme)
        b.init_thermal(5)
        if scheme == F.FLBM_LEARNED:
            b.set_mlp(theta)
            pre = b.probe([node(*q) for q in pts])
        b.step(1)
        dst = [node(x + c[i, 0], y + c[i, 1], z + c[i, 2]) for (x, y, z) in pts for i in range(27)]
        post[scheme] = b.probe(dst).reshape(len(pts), 27, 27)
        b.close()
    idx = np.arange(27)
    D = post[F.FLBM_LEARNED][:, idx, idx] - post[F.FLBM_GMF][:, idx, idx]
    corr = M.correction(theta, pre, rho0, kT, 1.0 / tau, bf16=True)
    # the propagated bound of test_gpu_mlp (bf16 flips, hardware tanh, FP32)
    q = M.unpack(theta)
    r = M.bf16_round
    x = M.features(pre, rho0, kT, 1.0 / tau)
    y, (_, z1, h1, z2, h2) = M.forward(theta, x, bf16=True)
    e1 = 2.0 ** -7 * np.abs(h1) + 2.0 ** -11.9 * np.abs(z1)
    e2 = 1.1 * e1 @ np.abs(r(q["W2"])).T + 2.0 ** -7 * np.abs(h2) + 2.0 ** -11.9 * np.abs(z2)
    ey = e2 @ np.abs(r(q["W3"])).T + 1e-5 * (1 + np.abs(y))
    dlt = w * (kT / rho0) ** 1.5 * ey
    eb = dlt + w * (1 + 3 * np.abs(c).sum(1)) * dlt.sum(1, keepdims=True) + 1e-8
    assert np.all(np.abs(D - corr) <= eb), (np.abs(D - corr).max(), (np.abs(D - corr) / eb).max())
    assert np.abs(corr).max() > 1e-6
