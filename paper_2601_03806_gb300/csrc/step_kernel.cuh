// step_kernel.cuh -- fused D3Q27 fluctuating-LB stream-and-collide kernel.
//
// One thread updates one node per loop iteration; a CTA owns a chunk of
// kBlock consecutive x of one (y, z) row, so every population plane is read
// and written as contiguous 4/8-byte-per-lane warp accesses.  The grid is a
// persistent multiple of the SM count that strides over row chunks.
//
// Storage: deviations g_i = f_i - w_i rho0, SoA planes g[i*N + n], updated
// in place with the AA pattern (no second array):
//   even form (natural): node x reads f_i from slot i at x and writes the
//     post-collision f*_i to slot opp(i) at x;
//   odd form: node x reads f_i from slot opp(i) at x - c_i and writes f*_i to
//     slot i at x + c_i.
// Both forms realise f_i(x + c_i, t+1) = f*_i(x, t) (LHS of Eq. flbe2) on a
// periodic box, and each thread reads exactly the locations it writes.
//
// Per node (Eq. flbe2 in mode space):
//   a2  forward Hermite projection (three 1-D passes): drho, j_a, m_ab
//   a3  a2neq_ab = m_ab - rho u_a u_b (equal to Eq. moments2 because the
//       second-order f^eq has second Hermite moment rho u_a u_b)
//   a4  M_ab = rho u_a u_b + (1 - omega) a2neq_ab          (k = 4..9)
//   a5  ghost modes k = 10..26: no deterministic content (GMF); (1-omega) m_k
//       for BGK-FLBM (Eq. flbe); rho u^(deg) for Reg-FLBM
//   a6  M_k += phi_k r_k  (Eqs. fluct_phi / fluct_phig), r_k from
//       Philox4x32-10 keyed on (seed; node, step, block) + Box-Muller
//   a7  f*_i = w_i sum_k e_ki M_k / b_k (three 1-D passes), minus w_i rho0
//   a8  AA store
//   a9  optional per-thread partial sums for the FP64 reductions
#pragma once

#include "internal.h"
#include "lattice.cuh"

namespace flbm {

template <typename S, typename R> struct Conv;
template <> struct Conv<double, double> {
    static __device__ __forceinline__ double ld(const double *p) { return *p; }
    static __device__ __forceinline__ void st(double *p, double v) { *p = v; }
};
template <> struct Conv<float, float> {
    static __device__ __forceinline__ float ld(const float *p) { return *p; }
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};

template <typename R> __device__ __forceinline__ R rcp_(R v);
template <> __device__ __forceinline__ double rcp_<double>(double v) { return 1.0 / v; }
template <> __device__ __forceinline__ float rcp_<float>(float v) { return __frcp_rn(v); }
template <typename R> __device__ __forceinline__ R sqrt_(R v);
template <> __device__ __forceinline__ double sqrt_<double>(double v) { return sqrt(v); }
template <> __device__ __forceinline__ float sqrt_<float>(float v) { return sqrtf(v); }

// 1-D Hermite analysis of a 3-point line (values at c = -1, 0, +1):
// (sum v, sum v c, sum v (c^2 - 1/3)).
template <typename R>
__device__ __forceinline__ void analyse(R &m, R &o, R &p)
{
    const R s = m + p;
    const R d = p - m;
    const R h0 = s + o;
    const R h2 = R(2.0 / 3.0) * s - R(1.0 / 3.0) * o;
    m = h0;
    o = d;
    p = h2;
}

// 1-D synthesis with the weights folded in: value at c of
// w1(c) (q0 + q1 c + q2 (c^2 - 1/3)), written back as (c = -1, 0, +1).
template <typename R>
__device__ __forceinline__ void synthesise(R &q0, R &q1, R &q2)
{
    const R t = R(1.0 / 6.0) * q0 + R(1.0 / 9.0) * q2;    // w1(+-1) (q0 + 2/3 q2)
    const R s = R(1.0 / 6.0) * q1;                         // w1(+-1) q1
    const R z = R(2.0 / 3.0) * q0 - R(2.0 / 9.0) * q2;    // w1(0) (q0 - 1/3 q2)
    q0 = t - s;
    q1 = z;
    q2 = t + s;
}

template <typename R>
__device__ __forceinline__ R warp_sum(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename R>
__device__ __forceinline__ void block_reduce_store(const R (&acc)[NSTAT], double *out)
{
    __shared__ double sh[kBlock / 32][NSTAT];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < NSTAT; ++s) {
        const R v = warp_sum(acc[s]);
        if (lane == 0) sh[warp][s] = double(v);
    }
    __syncthreads();
    if (threadIdx.x < NSTAT) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < kBlock / 32; ++w) t += sh[w][threadIdx.x];
        out[threadIdx.x] = t;
    }
}

template <typename S, typename R, int SCHEME, bool ODD, bool STATS>
__device__ __forceinline__ void node_update(S *__restrict__ g, const StepArgs<R> &a, uint32_t x,
                                            uint32_t y, uint32_t z, R (&acc)[NSTAT])
{
    const uint32_t nx = a.nx, ny = a.ny, nz = a.nz;
    const uint64_t N = a.n;
    const uint32_t xs[3] = {x ? x - 1 : nx - 1, x, (x + 1 < nx) ? x + 1 : 0};
    const uint32_t ys[3] = {y ? y - 1 : ny - 1, y, (y + 1 < ny) ? y + 1 : 0};
    const uint32_t zs[3] = {z ? z - 1 : nz - 1, z, (z + 1 < nz) ? z + 1 : 0};
    const uint64_t n = xs[1] + uint64_t(nx) * (ys[1] + uint64_t(ny) * zs[1]);

    // a1: load the 27 incoming populations, v[cx+1][cy+1][cz+1]
    R v[3][3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                uint64_t idx;
                if (!ODD) {
                    idx = uint64_t(slot_of(i - 1, j - 1, k - 1)) * N + n;
                } else {
                    const uint64_t nb = xs[2 - i] + uint64_t(nx) * (ys[2 - j] + uint64_t(ny) * zs[2 - k]);
                    idx = uint64_t(slot_of(1 - i, 1 - j, 1 - k)) * N + nb;
                }
                v[i][j][k] = Conv<S, R>::ld(g + idx);
            }

    // a2: forward Hermite projection, three 1-D passes
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) analyse(v[0][j][k], v[1][j][k], v[2][j][k]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) analyse(v[i][0][k], v[i][1][k], v[i][2][k]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) analyse(v[i][j][0], v[i][j][1], v[i][j][2]);

    const R drho = v[0][0][0];
    const R rho = a.rho0 + drho;
    const R jx = v[1][0][0], jy = v[0][1][0], jz = v[0][0][1];
    const R irho = rcp_(rho);
    const R ux = jx * irho, uy = jy * irho, uz = jz * irho;

    if (!(rho > R(0)) || !(rho < R(INFINITY))) {
        *a.flag = 1u;
        atomicMin(a.bad_step, (unsigned long long)a.step);
    }

    if (STATS) {
        const R m2 = jx + jy + jz;
        const R m3 = v[2][0][0] + v[0][2][0] + v[0][0][2] + drho;
        const R m4 = v[1][1][0] + v[1][0][1] + v[0][1][1];
        acc[S_DRHO] += drho;
        acc[S_JX] += jx;
        acc[S_JY] += jy;
        acc[S_JZ] += jz;
        acc[S_UX2] += ux * ux;
        acc[S_UY2] += uy * uy;
        acc[S_UZ2] += uz * uz;
        acc[S_M2] += m2;
        acc[S_M3] += m3;
        acc[S_M4] += m4;
        acc[S_M1SQ] += drho * drho;
        acc[S_M2SQ] += m2 * m2;
        acc[S_M3SQ] += m3 * m3;
        acc[S_M4SQ] += m4 * m4;
    }

    // a3-a5: post-collision mode amplitudes M, then Q = M / b_k
    const R lam = a.lambda;
    R qm[3][3][3];
    const R uu[3] = {ux, uy, uz};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int ord = mode_order(i, j, k);
                R post;
                if (ord == 0) {
                    post = drho;                      // deviation of M_0 = rho
                } else if (ord == 1) {
                    post = v[i][j][k];                // momentum, conserved
                } else {
                    // Maxwell-Boltzmann Hermite coefficient rho u_x^i u_y^j u_z^k
                    R aeq = rho;
#pragma unroll
                    for (int e = 0; e < i; ++e) aeq *= uu[0];
#pragma unroll
                    for (int e = 0; e < j; ++e) aeq *= uu[1];
#pragma unroll
                    for (int e = 0; e < k; ++e) aeq *= uu[2];
                    if (ord == 2) {
                        post = aeq + lam * (v[i][j][k] - aeq);
                    } else if (SCHEME == 0) {             // BGK: 2nd-order f^eq
                        post = lam * v[i][j][k];
                    } else if (SCHEME == 2) {             // Reg: full-order f^eq
                        post = aeq;
                    } else {                              // GMF: filtered
                        post = R(0);
                    }
                }
                qm[i][j][k] = post * R(1.0 / b_of(i, j, k));
            }

    // a6: FDT noise, M_k += phi_k r_k for k = 4..26 (in Q units: / b_k)
    {
        const R sr = a.noise_rho0 ? a.sqrt_rho0 : sqrt_(rho);
        R r[28];
#pragma unroll
        for (int blk = 0; blk < 6; ++blk) {
            const u32x4 o = philox4x32_10(
                u32x4{uint32_t(n), uint32_t(a.step), uint32_t(blk), uint32_t(a.step >> 32)},
                a.key0, a.key1);
            box_muller(o.x, o.y, r[4 + 4 * blk], r[5 + 4 * blk]);
            box_muller(o.z, o.w, r[6 + 4 * blk], r[7 + 4 * blk]);
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const int mk = mode_of(i, j, k);
                    if (mk >= 4) qm[i][j][k] += (sr * a.nc[mk]) * r[mk];
                }
    }

    // a7: reconstruction f*_i - w_i rho0 = w_i sum_k e_ki Q_k (Q_0 = drho)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) synthesise(qm[i][j][0], qm[i][j][1], qm[i][j][2]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) synthesise(qm[i][0][k], qm[i][1][k], qm[i][2][k]);
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) synthesise(qm[0][j][k], qm[1][j][k], qm[2][j][k]);

    // a8: AA store
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                uint64_t idx;
                if (!ODD) {
                    idx = uint64_t(slot_of(1 - i, 1 - j, 1 - k)) * N + n;
                } else {
                    const uint64_t nb = xs[i] + uint64_t(nx) * (ys[j] + uint64_t(ny) * zs[k]);
                    idx = uint64_t(slot_of(i - 1, j - 1, k - 1)) * N + nb;
                }
                Conv<S, R>::st(g + idx, qm[i][j][k]);
            }
}

template <typename S, typename R, int SCHEME, bool ODD, bool STATS>
__global__ void __launch_bounds__(kBlock) k_step(S *__restrict__ g, const StepArgs<R> a)
{
    R acc[NSTAT];
#pragma unroll
    for (int s = 0; s < NSTAT; ++s) acc[s] = R(0);
    for (uint64_t ch = blockIdx.x; ch < a.nchunks; ch += gridDim.x) {
        const uint32_t xc = uint32_t(ch % a.cpr);
        const uint64_t r = ch / a.cpr;
        const uint32_t y = uint32_t(r % a.ny);
        const uint32_t z = uint32_t(r / a.ny);
        const uint32_t x = xc * kBlock + threadIdx.x;
        if (x < a.nx) node_update<S, R, SCHEME, ODD, STATS>(g, a, x, y, z, acc);
    }
    if (STATS) block_reduce_store(acc, a.partials + size_t(blockIdx.x) * NSTAT);
}

template <typename S, typename R>
cudaError_t launch_step_t(S *g, const StepArgs<R> &a, int scheme, bool odd, bool stats, int grid,
                          cudaStream_t s)
{
#define FLBM_LAUNCH(SC, OD, ST) \
    k_step<S, R, SC, OD, ST><<<grid, kBlock, 0, s>>>(g, a)
    if (scheme == 0) {
        if (odd) { if (stats) FLBM_LAUNCH(0, true, true); else FLBM_LAUNCH(0, true, false); }
        else     { if (stats) FLBM_LAUNCH(0, false, true); else FLBM_LAUNCH(0, false, false); }
    } else if (scheme == 1) {
        if (odd) { if (stats) FLBM_LAUNCH(1, true, true); else FLBM_LAUNCH(1, true, false); }
        else     { if (stats) FLBM_LAUNCH(1, false, true); else FLBM_LAUNCH(1, false, false); }
    } else {
        if (odd) { if (stats) FLBM_LAUNCH(2, true, true); else FLBM_LAUNCH(2, true, false); }
        else     { if (stats) FLBM_LAUNCH(2, false, true); else FLBM_LAUNCH(2, false, false); }
    }
#undef FLBM_LAUNCH
    return cudaGetLastError();
}

template <typename S, typename R>
int step_occupancy_t(int scheme, bool stats)
{
    int nb = 0;
    cudaError_t e;
    // the odd form has the larger register footprint; use it for both
    if (scheme == 0)
        e = stats ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step<S, R, 0, true, true>, kBlock, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step<S, R, 0, true, false>, kBlock, 0);
    else if (scheme == 1)
        e = stats ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step<S, R, 1, true, true>, kBlock, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step<S, R, 1, true, false>, kBlock, 0);
    else
        e = stats ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step<S, R, 2, true, true>, kBlock, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step<S, R, 2, true, false>, kBlock, 0);
    return (e == cudaSuccess && nb > 0) ? nb : 1;
}

}  // namespace flbm
