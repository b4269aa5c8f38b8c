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
