"""Pins of the learned-collision oracle (oracle/mlp.py), no GPU.

* backward() against central finite differences of loss() (a mistake in any
  chain-rule factor, index or transpose fails it);
* closed forms: zero weights give y = b3, silu at 0 and far out;
* the projection: corrections of the form w (a + b.c / c_s^2) vanish, the
  projected correction carries no mass or momentum, projecting twice changes
  nothing;
* the training target equals the ghost equilibrium content
  w_i sum_{k>=10} e_ki rho u^(deg k) / b_k built from the Table II basis
  (the multi-index of each mode read off its polynomial), in units of
  w_i sigma^3;
* the learned collision conserves mass and momentum and reduces to GMF for
  a zero network.
"""
import numpy as np
import pytest

from synth import inputs


@pytest.fixture(scope="module")
def M(oracle_mod):
    from oracle import mlp
    return mlp


def small_batch(M, seed, B=6):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(B, M.NIN)), rng.normal(size=(B, M.NOUT))


def test_backward_matches_finite_differences(M):
    theta = M.init_params(1) + 0.05 * np.random.default_rng(2).normal(size=M.NPARAM)
    x, t = small_batch(M, 3)
    g = M.backward(theta, x, t)
    rng = np.random.default_rng(4)
    idx = np.concatenate([rng.choice(M.NPARAM, 300, replace=False),
                          [0, M.NPARAM - 1, 64 * 28, 64 * 28 + 64]])
    h = 1e-6
    for k in idx:
        e = np.zeros(M.NPARAM)
        e[k] = h
        fd = (M.loss(theta + e, x, t) - M.loss(theta - e, x, t)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(fd)), (k, fd, g[k])


def test_closed_forms(M):
    p = M.unpack(np.zeros(M.NPARAM))
    p["b3"] = np.arange(27.0)
    theta = M.pack(p)
    y, _ = M.forward(theta, np.random.default_rng(0).normal(size=(5, M.NIN)))
    assert np.array_equal(y, np.tile(np.arange(27.0), (5, 1)))
    assert M.silu(0.0) == 0.0
    assert abs(M.silu(40.0) - 40.0) < 1e-12 and abs(M.silu(-40.0)) < 1e-15
    assert M.NPARAM == 7771
    th = np.arange(float(M.NPARAM))
    assert np.array_equal(M.pack(M.unpack(th)), th)
    assert M.unpack(th)["W2"][0, 0] == 64 * 28 + 64


def test_bf16_rounding(M):
    assert M.bf16_round(1.0) == 1.0
    # 8 significant bits: ulp(1) = 2^-7; ties go to the even neighbour
    assert M.bf16_round(1.0 + 2 ** -8) == 1.0
    assert M.bf16_round(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6
    assert M.bf16_round(1.0 + 2 ** -8 + 2 ** -12) == 1.0 + 2 ** -7
    assert M.bf16_round(-3.0) == -3.0
    a = np.random.default_rng(1).normal(size=1000)
    assert np.all(np.abs(M.bf16_round(a) - a) <= 2 ** -8 * np.abs(a))


def test_projection(M, oracle_mod):
    T = oracle_mod.tables()
    w, c = T["w"], T["c"].astype(float)
    rng = np.random.default_rng(5)
    d = rng.normal(size=(10, 27))
    pd = M.project(d)
    assert np.abs(pd.sum(-1)).max() < 1e-13
    assert np.abs(pd @ c).max() < 1e-13
    assert np.abs(M.project(pd) - pd).max() < 1e-13
    a, b = rng.normal(size=10), rng.normal(size=(10, 3))
    conserved = w * (a[:, None] + (b @ c.T) / M.CS2)
    assert np.abs(M.project(conserved)).max() < 1e-13
    # a correction orthogonal (in the w-weighted sense) to 1 and c is kept
    q = w * (c[:, 0] ** 2 - M.CS2)
    assert np.abs(M.project(q) - q).max() < 1e-15


def mode_exponents(T):
    """(n_x, n_y, n_z) of each Table II mode, read off its polynomial values:
    independent of c_a -> 0, odd in c_a -> 1, even and varying -> 2."""
    c, E = T["c"], T["E"]
    idx = {tuple(v): i for i, v in enumerate(c)}
    out = []
    for k in range(27):
        ex = []
        for a in range(3):
            def val(s):
                v = [0, 0, 0]
                v[a] = s
                # pick a velocity with a nonzero value on the other axes too
                best = []
                for other in ((1, 1), (1, -1), (0, 1), (1, 0), (0, 0)):
                    vv = list(v)
                    o = [b for b in range(3) if b != a]
                    vv[o[0]], vv[o[1]] = other
                    best.append(E[k, idx[tuple(vv)]])
                return np.array(best)
            p, z, m = val(1), val(0), val(-1)
            if np.allclose(p, z) and np.allclose(m, z):
                ex.append(0)
            elif np.allclose(p, -m):
                ex.append(1)
            else:
                ex.append(2)
        out.append(ex)
    return np.array(out)


def test_target_is_ghost_equilibrium_content(M, oracle_mod):
    T = oracle_mod.tables()
    w, c, E, b, nk = T["w"], T["c"].astype(float), T["E"], T["b"], T["nk"]
    ex = mode_exponents(T)
    assert np.array_equal(ex.sum(1), nk)
    rho0, kT, tau = 1.0, 1e-5, 0.7
    rng = np.random.default_rng(6)
    for trial in range(5):
        f = w * rho0 + np.sqrt(rho0 * kT * w / M.CS2) * rng.normal(size=27) * 3
        rho = f.sum()
        u = (f @ c) / rho
        aeq = rho * np.prod(u[None, :] ** ex, axis=1)
        ghost = nk >= 3
        expect = w * ((E[ghost] * (aeq[ghost] / b[ghost])[:, None]).sum(0))
        y = M.target(f, tau, rho0, kT)
        sig3 = np.sqrt(kT / rho0) ** 3
        assert np.abs(y * w * sig3 - expect).max() < 1e-15, trial
        assert np.abs(y).max() > 1e-3           # order-one in units of sigma^3


def test_learned_collision_conserves_and_reduces_to_gmf(M, oracle_mod):
    w = oracle_mod.tables()["w"]
    c = oracle_mod.tables()["c"].astype(float)
    rho0, kT, tau = 1.0, 1e-4, 0.8
    f = w * (rho0 + 0.05 * inputs.population_perturbation(1, 1, 1, 9)[:, 0, 0, 0])
    theta = M.init_params(7)
    fs = M.learned_collide_node(theta, tau, kT, f, seed=3, node=0, step=2)
    assert abs(fs.sum() - f.sum()) < 1e-14
    assert np.abs(fs @ c - f @ c).max() < 1e-14
    zero = np.zeros(M.NPARAM)
    g = oracle_mod.collide_node(oracle_mod.GMF, tau, kT, f, seed=3, node=0, step=2)
    assert np.array_equal(M.learned_collide_node(zero, tau, kT, f, seed=3, node=0, step=2), g)


def test_features_invert(M, oracle_mod):
    w = oracle_mod.tables()["w"]
    rho0, kT = 1.2, 3e-5
    rng = np.random.default_rng(8)
    f = w * rho0 + rng.normal(size=(4, 27)) * 1e-3
    x = M.features(f, rho0, kT, 1.25)
    assert np.allclose(x[:, 27], 0.25)
    assert np.abs(w * rho0 + x[:, :27] * np.sqrt(rho0 * kT * w / M.CS2) - f).max() < 1e-15
