"""The 13 sums of the fused reductions (row a9), computed in FP64 from a
state's populations with the oracle's moments, and a bound on how far the
FP32 kernels' sums may lie from them.

The sums run over the nodes of the pre-collision state (Eqs. rho, u; the ER
observables of Sec. III): drho, j_x, j_y, j_z, u_x^2, u_y^2, u_z^2, m3, m4,
drho^2, (sum_a j_a)^2, m3^2, m4^2 with drho = rho - rho0, m3 = sum_a Pi_aa -
rho0, m4 = sum_{a<b} Pi_ab.

Error model of the FP32 path (unit roundoff u = 2^-24; the stored FP32 or
FP16 deviations g_i = f_i - w_i rho0 are read exactly):
* a linear moment x (drho, j_a, m3, m4) is a sum of the 27 deviations with
  coefficients of magnitude <= 1 (|c|^2 <= 3 for m3, taken as 3): in any
  evaluation with at most 32 roundings on a path, each of a partial sum
  bounded by 3 sigma, sigma = sum_i |g_i|, |dx| <= E = 96 u sigma (the
  kernels' three sum-factorised passes use fewer roundings and smaller
  partial sums); sum_a j_a adds two roundings: 3 E + 2 u |m2|;
* a square x^2 (one rounding): 2 |x| E + E^2 + u (|x| + E)^2;
* u_a = j_a (1/rho) with rho = rho0 + drho (one rounding) and the hardware
  reciprocal (within 2 ulp): |du| <= (E + |u| (E + u rho)) / rho + 6 u |u|,
  and u_a^2 as a square;
* accumulation: every thread adds its nodes' terms in FP32 (a two-node
  thread in two lanes, added once at the end), at most m of them before its
  warp adds the 32 threads' sums in five FP32 levels into its slot (every 8
  rows of the row pipeline, every 8 chunks of the direct kernel), a slot
  kept exactly as an unevaluated pair of FP32 numbers (TwoSum); blocks and
  the grid add in FP64: gamma(m + 7) sum_n (|x_n| + e_n),
  gamma(k) = k u / (1 - k u).
The bound is sum_n e_n + gamma(m + 7) sum_n (|x_n| + e_n).
"""
import numpy as np

U32 = 2.0 ** -24
NAMES = ["drho", "jx", "jy", "jz", "ux2", "uy2", "uz2", "m3", "m4",
         "drho2", "m2sq", "m3sq", "m4sq"]


def _gamma(k):
    return k * U32 / (1 - k * U32)


def node_terms(oracle_mod, f, rho0):
    """Per-node FP64 terms x[13, N] and their FP32 error bounds e[13, N] for
    absolute populations f (27, nz, ny, nx)."""
    _, nz, ny, nx = f.shape
    w = oracle_mod.tables()["w"]
    box = oracle_mod.Box(nx, ny, nz, tau=0.8, kT=0.0, rho0=rho0)
    box.set_f(f)
    rho, j, pi = box.moments()
    rho, j, pi = rho.ravel(), j.reshape(3, -1), pi.reshape(6, -1)
    sigma = np.abs(f - w[:, None, None, None] * rho0).reshape(27, -1).sum(0)
    E = 96 * U32 * sigma
    drho = rho - rho0
    m2 = j.sum(0)
    m3 = pi[:3].sum(0) - rho0
    m4 = pi[3:].sum(0)
    uu = j / rho
    du = (E + np.abs(uu) * (E + U32 * rho)) / rho + 6 * U32 * np.abs(uu)
    E2 = 3 * E + 2 * U32 * np.abs(m2)

    def sq(x, e):
        return 2 * np.abs(x) * e + e * e + U32 * (np.abs(x) + e) ** 2

    x = np.array([drho, j[0], j[1], j[2], uu[0] ** 2, uu[1] ** 2, uu[2] ** 2, m3, m4,
                  drho ** 2, m2 ** 2, m3 ** 2, m4 ** 2])
    e = np.array([E, E, E, E, sq(uu[0], du[0]), sq(uu[1], du[1]), sq(uu[2], du[2]), E, E,
                  sq(drho, E), sq(m2, E2), sq(m3, E), sq(m4, E)])
    return x, e


def sums_and_bounds(oracle_mod, f, rho0, m_per_thread):
    """FP64 sums S[13] of the per-node terms and the bound B[13] on the FP32
    path's |S_gpu - S| when no thread adds more than m_per_thread nodes."""
    x, e = node_terms(oracle_mod, f, rho0)
    g = _gamma(m_per_thread + 7)
    return x.sum(1), e.sum(1) + g * (np.abs(x) + e).sum(1)


FLUSH_EVERY = 8


def nodes_per_thread_bound(nx, ny, nz):
    """Nodes any thread (or lane) of the step kernels adds in FP32 at most
    before its warp folds the sums, for a GB300's 152 SMs: the row pipeline
    gives each CTA ceil(rows / grid) rows, each thread ceil(nx / 256) nodes
    of a row (one-node kernel) or ceil(nx / 256) pairs, one node of each per
    lane (two-node kernel), and flushes every 8 rows; the direct kernel one
    node per 128-node chunk, ceil(chunks / grid) chunks, flushed every 8
    chunks; every grid holds at least min(work, 152) CTAs."""
    rows = ny * nz
    chunks = -(-nx // 128) * rows
    row_kernel = min(-(-rows // min(rows, 152)), FLUSH_EVERY) * -(-nx // 256)
    direct = min(-(-chunks // min(chunks, 152)), FLUSH_EVERY)
    return max(row_kernel, direct)


def stats_from_sums(S, n, rho0, kT):
    """The flbm_stats fields that one reduced step (after flbm_stats_reset)
    gives for the sums S[13] over n nodes."""
    th = np.array([3.0, 3.0, 5.0, 1.0]) * rho0 * kT
    mean = np.array([S[0], S[1] + S[2] + S[3], S[7], S[8]]) / n
    var = np.array([S[9], S[10], S[11], S[12]]) / n - mean ** 2
    return {"mass": n * rho0 + S[0], "mom": S[1:4], "u2": S[4:7] / n, "m_mean": mean,
            "m_var": var, "er": var / th if kT > 0 else np.zeros(4)}


def stats_bounds(S, B, n, rho0, kT):
    """Bounds on the flbm_stats fields derived from per-sum bounds B."""
    th = np.array([3.0, 3.0, 5.0, 1.0]) * rho0 * kT
    mean = np.abs(np.array([S[0], S[1] + S[2] + S[3], S[7], S[8]])) / n
    bmean = np.array([B[0], B[1] + B[2] + B[3], B[7], B[8]]) / n
    bvar = np.array([B[9], B[10], B[11], B[12]]) / n + 2 * mean * bmean + bmean ** 2
    return {"mass": B[0] + 1e-15 * n * rho0, "mom": B[1:4], "u2": B[4:7] / n, "m_mean": bmean,
            "m_var": bvar, "er": bvar / th if kT > 0 else np.zeros(4)}
