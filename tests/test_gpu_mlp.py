"""The learned-collision network on the GPU against the oracle (oracle/mlp.py).

Tensor-core forward (flbm_mlp_infer, the tcgen05 kernel the learned step
uses) against the oracle's forward with the same bfloat16 roundings.  The
two differ by FP32 vs exact accumulation (about 1e-7 relative), by the
hardware tanh in silu (absolute error <= 2^-10.9 in tanh, so
|d silu(z)| <= 2^-11.9 |z|), and therefore by bfloat16 rounding decisions of
the hidden activations, each at most one unit in the last place (2^-7 |h|).
Propagated through the layers (|silu'| <= 1.1):
  e_h1 = 2^-7 |h1| + 2^-11.9 |z1|
  e_h2 = 1.1 |W2| e_h1 + 2^-7 |h2| + 2^-11.9 |z2|
  e_y  = |W3| e_h2 + 1e-5 (1 + |y|)
with |W| the elementwise absolute bf16 weights and the activations of the
oracle; the test holds every output to that bound and the bulk to 1 %.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2601_03806_gb300 import flbm
    return flbm


@pytest.fixture(scope="module")
def M(oracle_mod):
    from oracle import mlp
    return mlp


def random_net(M, seed):
    rng = np.random.default_rng(seed)
    theta = M.init_params(seed)
    p = M.unpack(theta)
    for b in ("b1", "b2", "b3"):
        p[b] = p[b] + 0.3 * rng.normal(size=p[b].shape)
    return M.pack(p).astype(np.float32).astype(np.float64)


def bound(M, theta, x):
    p = M.unpack(theta)
    r = M.bf16_round
    y, (xb, z1, h1, z2, h2) = M.forward(theta, x, bf16=True)
    e1 = 2.0 ** -7 * np.abs(h1) + 2.0 ** -11.9 * np.abs(z1)
    e2 = 1.1 * e1 @ np.abs(r(p["W2"])).T + 2.0 ** -7 * np.abs(h2) + 2.0 ** -11.9 * np.abs(z2)
    return y, e2 @ np.abs(r(p["W3"])).T + 1e-5 * (1 + np.abs(y))


@pytest.mark.parametrize("n", [1, 127, 128, 1000, 70000])
def test_tensor_core_forward_matches_oracle(F, M, n):
    theta = random_net(M, 11)
    rng = np.random.default_rng(n)
    x = rng.normal(size=(n, 28))
    x[:, 27] = rng.uniform(-0.67, 0.96, size=n)
    x = x.astype(np.float32).astype(np.float64)
    yg = F.mlp_infer(theta, x).astype(np.float64)
    yo, b = bound(M, theta, x)
    err = np.abs(yg - yo)
    assert np.all(err <= b), (err.max(), np.argmax(err - b))
    scale = np.sqrt(np.mean(yo ** 2))
    assert np.median(err) < 0.01 * scale


def test_tensor_core_forward_zero_and_bias_only(F, M):
    p = M.unpack(np.zeros(M.NPARAM))
    p["b3"] = np.arange(27.0) / 8
    x = np.random.default_rng(1).normal(size=(300, 28))
    y = F.mlp_infer(M.pack(p), x)
    assert np.array_equal(y, np.tile(np.arange(27.0, dtype=np.float32) / 8, (300, 1)))


# ---------------------------------------------------------------------------
# Training: pairs, gradient, Adam


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    return torch


def device(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32)).cuda()


def test_pairs_match_oracle(F, M, oracle_mod, torch_cuda):
    """Features and targets of every node against the oracle's, from the
    same stored state (FP32 storage: the oracle reads the stored values).
    Both are computed in FP64 and stored in FP32 (relative 2^-24)."""
    torch = torch_cuda
    nx, ny, nz, kT, tau, rho0 = 32, 6, 5, 1e-5, 0.7, 1.1
    box = F.Lattice(nx, ny, nz, tau, kT, rho0=rho0, seed=4, scheme=F.FLBM_REG)
    box.init_thermal(9)
    box.step(3)                                   # odd step: AA-shifted storage
    f = box.get_populations().reshape(27, -1).T   # [N, 27], node order
    N = f.shape[0]
    X = torch.empty((N, 28), dtype=torch.float32, device="cuda")
    T = torch.empty((N, 27), dtype=torch.float32, device="cuda")
    box.mlp_pairs(X, T)
    X, T = X.cpu().numpy().astype(float), T.cpu().numpy().astype(float)
    xo = M.features(f, rho0, kT, 1.0 / tau)
    assert np.abs(X - xo).max() <= 1e-6 * (1 + np.abs(xo).max())
    to = np.array([M.target(f[n], tau, rho0, kT) for n in range(0, N, 7)])
    scale = np.abs(to).max()
    assert scale > 1e-2
    assert np.abs(T[::7] - to).max() <= 2e-6 * scale


def test_gradient_matches_oracle(F, M, torch_cuda):
    """FP32 gradient of the mean squared error against the oracle's exact
    backward on 1000 samples (8 tiles, the last ragged)."""
    torch = torch_cuda
    rng = np.random.default_rng(3)
    theta = (M.init_params(5) + 0.05 * rng.normal(size=M.NPARAM)).astype(np.float32).astype(float)
    x = rng.normal(size=(1000, 28)).astype(np.float32).astype(float)
    t = rng.normal(size=(1000, 27)).astype(np.float32).astype(float)
    g, loss = F.mlp_grad(theta, device(torch, x), device(torch, t))
    go = M.backward(theta, x, t)
    assert abs(loss - M.loss(theta, x, t)) <= 1e-6 * M.loss(theta, x, t)
    assert np.linalg.norm(g - go) <= 1e-5 * np.linalg.norm(go)
    assert np.abs(g - go).max() <= 1e-4 * np.abs(go).max()


def reg_pairs(F, torch, taus, n=32, steps=40, seed=1):
    """Training pairs from Reg-FLBM boxes (one per tau) after `steps` steps
    from the invariant measure at kT = 1e-5."""
    xs, ts = [], []
    for r, tau in enumerate(taus):
        box = F.Lattice(n, n, n, tau, 1e-5, seed=seed, scheme=F.FLBM_REG, noise_stream=r)
        box.init_thermal(100 + r + 10 * seed)
        box.step(steps)
        X = torch.empty((n ** 3, 28), dtype=torch.float32, device="cuda")
        T = torch.empty((n ** 3, 27), dtype=torch.float32, device="cuda")
        box.mlp_pairs(X, T)
        xs.append(X)
        ts.append(T)
        box.close()
    return torch.cat(xs), torch.cat(ts)


def test_training_learns_the_regularized_correction(F, M, torch_cuda):
    """Trained on Reg-FLBM pairs (four 32^3 boxes, tau in [0.51, 3.0]), the
    network recovers the Reg-minus-GMF collision residual on a held-out box
    at another tau through the tensor-core forward: plain GMF misses all of
    it (relative error 1); the trained network about 3 % of it."""
    torch = torch_cuda
    X, T = reg_pairs(F, torch, [0.51, 0.9, 1.7, 3.0])
    theta0 = M.init_params(2).astype(np.float32)
    theta, losses = F.mlp_train(theta0, X, T, epochs=120, batch=1024, lr=1e-2, seed=7)
    assert losses[-1] < 0.01 * losses[0], losses[[0, -1]]
    Xh, Th = reg_pairs(F, torch, [1.2], seed=5)
    y = F.mlp_infer(theta, Xh.cpu().numpy())
    t = Th.cpu().numpy()
    rel = np.linalg.norm(y - t) / np.linalg.norm(t)
    print("held-out relative error of the learned correction: %.4f (GMF: 1)" % rel)
    assert rel < 0.06


# ---------------------------------------------------------------------------
# The learned step (scheme FLBM_LEARNED): GMF collision + network correction


def streamed(O, field):
    """f_i(x) <- field_i(x - c_i) on the periodic box, field[27, nz, ny, nx]."""
    c = O.tables()["c"]
    out = np.empty_like(field)
    for i in range(27):
        out[i] = np.roll(field[i], shift=(c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2))
    return out


@pytest.mark.parametrize("shape", [(130, 4, 3), (64, 2, 1), (32, 3, 2)])
def test_learned_step_correction_matches_oracle(F, M, oracle_mod, shape):
    """One learned step minus one GMF step from the same state with the same
    noise leaves the network correction P(w sigma^3 y), streamed; it must
    match the oracle's within the propagated bf16/tanh bound of y (plus the
    FP32 rounding of two stored states, 1e-8).  kT = 1e-3 puts the
    correction well above that rounding."""
    O = oracle_mod
    nx, ny, nz = shape
    tau, kT, rho0 = 0.8, 1e-3, 1.0
    theta = random_net(M, 21)
    boxes = {}
    for scheme in (F.FLBM_GMF, F.FLBM_LEARNED):
        b = F.Lattice(nx, ny, nz, tau, kT, rho0=rho0, seed=8, scheme=scheme)
        b.init_thermal(3)
        boxes[scheme] = b
    boxes[F.FLBM_LEARNED].set_mlp(theta)
    f0 = boxes[F.FLBM_LEARNED].get_populations()
    for b in boxes.values():
        b.step(1)
    D = boxes[F.FLBM_LEARNED].get_populations() - boxes[F.FLBM_GMF].get_populations()
    fn = f0.reshape(27, -1).T
    corr = M.correction(theta, fn, rho0, kT, 1.0 / tau, bf16=True)
    # bound on the correction error from the bound on y
    w = O.tables()["w"]
    c = O.tables()["c"]
    _, ey = bound(M, theta, M.features(fn, rho0, kT, 1.0 / tau))
    dlt = w * (kT / rho0) ** 1.5 * ey
    eb = dlt + w * (1 + 3 * np.abs(c).sum(1)) * dlt.sum(1, keepdims=True) + 1e-8
    expect = streamed(O, corr.T.reshape(27, nz, ny, nx))
    ebound = streamed(O, eb.T.reshape(27, nz, ny, nx))
    err = np.abs(D - expect)
    assert np.all(err <= ebound), (err.max(), (err / ebound).max())
    assert np.abs(expect).max() > 100 * 1e-8


def test_learned_step_conserves_and_needs_its_network(F, M):
    nx, ny, nz, tau, kT = 64, 4, 4, 0.7, 1e-4
    b = F.Lattice(nx, ny, nz, tau, kT, seed=2, scheme=F.FLBM_LEARNED)
    b.init_thermal(1)
    with pytest.raises(F.FlbmError) as ei:
        b.step(1)
    assert ei.value.code == F.FLBM_E_INVALID
    b.set_mlp(random_net(M, 4))
    rho, j, _ = b.moments()
    b.step(6)
    rho2, j2, _ = b.moments()
    assert abs(rho2.sum() - rho.sum()) < 1e-6 * rho.size * 1e-3
    assert np.abs(j2.sum(axis=(1, 2, 3)) - j.sum(axis=(1, 2, 3))).max() < 1e-6
    for kw in (dict(precision=F.FLBM_FP16), dict(precision=F.FLBM_FP64)):
        with pytest.raises(F.FlbmError):
            F.Lattice(nx, ny, nz, tau, kT, scheme=F.FLBM_LEARNED, **kw)
    with pytest.raises(F.FlbmError):
        F.Lattice(nx, ny, nz, tau, 0.0, scheme=F.FLBM_LEARNED)
    g = F.Lattice(nx, ny, nz, tau, kT, scheme=F.FLBM_GMF)
    with pytest.raises(F.FlbmError):
        g.set_mlp(random_net(M, 4))


def test_learned_equipartition_and_flat_spectrum(F, M, torch_cuda):
    """Config-5 statistics on a 64^3 box (tau 0.8, kT 1e-5) with a network
    trained on Reg-FLBM pairs: <u_a^2> = kT/rho0 and S_jx(k) = rho0 kT,
    within the sampling noise, as for plain GMF-FLBM."""
    torch = torch_cuda
    X, T = reg_pairs(F, torch, [0.51, 0.9, 1.7, 3.0])
    theta, _ = F.mlp_train(M.init_params(2).astype(np.float32), X, T, epochs=60, batch=1024, lr=1e-2, seed=7)
    out = {}
    for scheme in (F.FLBM_GMF, F.FLBM_LEARNED):
        b = F.Lattice(64, 64, 64, 0.8, 1e-5, seed=12, scheme=scheme)
        if scheme == F.FLBM_LEARNED:
            b.set_mlp(theta)
        b.init_thermal(6)
        b.step(20)
        b.stats_reset()
        b.step(200)
        S, cnt = b.structure_factor(F.FLBM_OBS_JX, 32)
        m = cnt > 0
        out[scheme] = (np.array(b.stats()["u2_avg"]) / 1e-5,
                       np.sum(S[m] * cnt[m]) / np.sum(cnt[m]) / 1e-5)
    for scheme, (u2, s) in out.items():
        print(scheme, u2, s)
        assert np.all(np.abs(u2 - 1) < 0.02), (scheme, u2)
        assert abs(s - 1) < 0.03, (scheme, s)
    assert np.all(np.abs(out[F.FLBM_LEARNED][0] - out[F.FLBM_GMF][0]) < 0.01)


def test_learned_step_full_size_sampled_nodes(F, M, oracle_mod):
    """The 256^3 learned box in the benchmark's launch shape: one learned step
    minus one GMF step from the same state and noise, at 48 sampled nodes
    (all 27 directions, read where streaming put them) against the oracle's
    correction of the probed pre-collision populations.  kT = 1e-3 keeps the
    correction above FP32 rounding; the bound is the propagated one."""
    O = oracle_mod
    n, tau, kT, rho0 = 256, 0.8, 1e-3, 1.0
    theta = random_net(M, 33)
    boxes = {}
    for scheme in (F.FLBM_GMF, F.FLBM_LEARNED):
        b = F.Lattice(n, n, n, tau, kT, rho0=rho0, seed=21, scheme=scheme)
        b.init_thermal(5)
        boxes[scheme] = b
    boxes[F.FLBM_LEARNED].set_mlp(theta)
    c = O.tables()["c"]
    w = O.tables()["w"]
    rng = np.random.default_rng(0)
    pts = rng.integers(0, n, size=(48, 3))
    pts[0] = (0, 0, 0)
    pts[1] = (n - 1, n - 1, n - 1)
    node = lambda x, y, z: int(x % n + n * ((y % n) + n * (z % n)))
    pre = boxes[F.FLBM_LEARNED].probe([node(*p) for p in pts])          # [48, 27]
    for b in boxes.values():
        b.step(1)
    dst = [node(x + c[i, 0], y + c[i, 1], z + c[i, 2]) for (x, y, z) in pts for i in range(27)]
    post = {s: b.probe(dst).reshape(48, 27, 27) for s, b in boxes.items()}
    idx = np.arange(27)
    D = post[F.FLBM_LEARNED][:, idx, idx] - post[F.FLBM_GMF][:, idx, idx]
    corr = M.correction(theta, pre, rho0, kT, 1.0 / tau, bf16=True)
    _, ey = bound(M, theta, M.features(pre, rho0, kT, 1.0 / tau))
    dlt = w * (kT / rho0) ** 1.5 * ey
    eb = dlt + w * (1 + 3 * np.abs(c).sum(1)) * dlt.sum(1, keepdims=True) + 1e-8
    assert np.all(np.abs(D - corr) <= eb), (np.abs(D - corr).max(), (np.abs(D - corr) / eb).max())
    assert np.abs(corr).max() > 1e-6
