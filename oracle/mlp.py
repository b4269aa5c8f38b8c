"""FP64 oracle of the learned collision (test infrastructure only).

The learned collision replaces the costly high-order part of the regularized
collision (Reg-FLBM, Sec. III) by a small per-node network on top of the
GMF-FLBM collision (Eq. flbe2):

    f*_learned = f*_GMF + P(dF),   dF_i = w_i sigma^3 y_i(x),

* x (28 features): the pre-collision deviations g_i = f_i - w_i rho0 in units
  of their equilibrium standard deviation sqrt(rho0 kT w_i / c_s^2) (the
  lattice invariant measure), i = 0..26, and omega - 1;
* y = W3 h2 + b3, h2 = silu(W2 h1 + b2), h1 = silu(W1 x + b1): 28-64-64-27,
  silu(z) = z / (1 + e^-z);
* sigma = sqrt(kT / rho0), the thermal velocity scale: the quantity learned is
  of order u^3 (the lowest ghost equilibrium content rho u^3);
* P: the w-orthogonal projection that removes mass and momentum,
  P(d)_i = d_i - w_i (sum_j d_j + c_i . sum_j d_j c_j / c_s^2), so the
  correction conserves rho and rho u exactly.

Training pairs: pre-collision states of a Reg-FLBM run and the target
y_target = (f*_Reg - f*_GMF) / (w sigma^3) of their deterministic (kT = 0)
collisions, which in this implementation's reading of Reg-FLBM is the ghost
equilibrium content w_i sum_{k >= 10} e_ki rho u^(deg k) / b_k.

Parity status: ``forward``/``backward`` pinned by central finite differences
and closed forms; ``project`` by the conservation identities; ``target`` by
the closed-form ghost synthesis from the Table II basis (it inherits the
Reg-FLBM reading, whose implementation is pinned but which the paper's text
does not define).

Parameter vector (float, this order): W1[64][28], b1[64], W2[64][64],
b2[64], W3[27][64], b3[27] -- 7771 values.
"""
from __future__ import annotations

import numpy as np

from . import oracle as _o

NIN, NH, NOUT = 28, 64, 27
CS2 = 1.0 / 3.0
SHAPES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)),
          ("W3", (NOUT, NH)), ("b3", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    theta = np.asarray(theta, np.float64)
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = theta[k:k + n].reshape(shape)
        k += n
    return out


def pack(p) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SHAPES])


def init_params(seed: int) -> np.ndarray:
    """He-style random initialisation (the training starting point)."""
    rng = np.random.default_rng(seed)
    p = {"W1": rng.normal(0, np.sqrt(1.0 / NIN), (NH, NIN)), "b1": np.zeros(NH),
         "W2": rng.normal(0, np.sqrt(1.0 / NH), (NH, NH)), "b2": np.zeros(NH),
         "W3": rng.normal(0, np.sqrt(1.0 / NH), (NOUT, NH)), "b3": np.zeros(NOUT)}
    return pack(p)


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def features(f, rho0, kT, omega):
    """x[..., 28] of absolute populations f[..., 27]."""
    w = _o.tables()["w"]
    f = np.asarray(f, np.float64)
    x = np.empty(f.shape[:-1] + (NIN,))
    x[..., :27] = (f - w * rho0) / np.sqrt(rho0 * kT * w / CS2)
    x[..., 27] = omega - 1.0
    return x


def forward(theta, x, bf16=False):
    """y[..., 27] and the cache for backward.  bf16=True rounds what the
    tensor-core path rounds: the weights, the input features and both hidden
    activations (accumulation and biases stay exact)."""
    p = unpack(theta)
    r = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
    x = r(x)
    z1 = x @ r(p["W1"]).T + p["b1"]
    h1 = r(silu(z1))
    z2 = h1 @ r(p["W2"]).T + p["b2"]
    h2 = r(silu(z2))
    y = h2 @ r(p["W3"]).T + p["b3"]
    return y, (x, z1, h1, z2, h2)


def loss(theta, x, t):
    """Mean squared error over samples and outputs."""
    y, _ = forward(theta, x)
    return float(np.mean((y - t) ** 2))


def backward(theta, x, t):
    """Gradient of loss() with respect to theta (exact arithmetic, no bf16)."""
    p = unpack(theta)
    y, (x, z1, h1, z2, h2) = forward(theta, x)
    B = x.shape[0]
    dy = 2.0 * (y - t) / (B * NOUT)
    g = {"W3": dy.T @ h2, "b3": dy.sum(0)}
    dz2 = (dy @ p["W3"]) * dsilu(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * dsilu(z1)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(0)
    return pack(g)


def project(d):
    """Remove mass and momentum from population-space corrections d[..., 27]."""
    T = _o.tables()
    w, c = T["w"], T["c"].astype(np.float64)
    d = np.asarray(d, np.float64)
    alpha = d.sum(-1)
    beta = d @ c
    return d - w * (alpha[..., None] + (beta @ c.T) / CS2)


def target(f, tau, rho0, kT):
    """y_target of one node: (f*_Reg - f*_GMF) / (w sigma^3), deterministic."""
    w = _o.tables()["w"]
    freg = _o.collide_node(_o.REG, tau, 0.0, f, rho0=rho0)
    fgmf = _o.collide_node(_o.GMF, tau, 0.0, f, rho0=rho0)
    return (freg - fgmf) / (w * np.sqrt(kT / rho0) ** 3)


def correction(theta, f, rho0, kT, omega, bf16=True):
    """P(dF) of populations f[..., 27] (absolute)."""
    w = _o.tables()["w"]
    y, _ = forward(theta, features(f, rho0, kT, omega), bf16=bf16)
    return project(w * np.sqrt(kT / rho0) ** 3 * y)


def learned_collide_node(theta, tau, kT, f, *, seed=0, node=0, step=0, rho0=1.0, bf16=True):
    """Post-collision populations of one node under the learned collision: the
    GMF collision with its noise, plus the projected network correction."""
    fs = _o.collide_node(_o.GMF, tau, kT, f, seed=seed, node=node, step=step, rho0=rho0)
    return fs + correction(theta, f, rho0, kT, 1.0 / tau, bf16=bf16)
