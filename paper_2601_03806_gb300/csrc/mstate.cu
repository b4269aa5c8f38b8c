// mstate.cu -- the moment-state form of the GMF / Reg step: the paper's
// "thread-safe" formulation (end of Sec. II), in which a node reads its
// neighbours' macroscopic fields and writes only its own.
//
// Between steps a node keeps ten numbers: the deterministic part of its last
// collision's output, (rho - rho0, j_x, j_y, j_z) and the six relaxed
// second-order amplitudes Q_ab = syn_scale (rho u_a u_b + (1 - omega)
// a2neq_ab) of Eq. flbe2.  Everything else the post-collision populations
// need is either zero (GMF ghosts), a function of rho and j (Reg ghosts,
// rho u^deg), or the node's noise, which the counter-keyed generator
// regenerates from (node, step).  So the populations f(x, t+1) = f*(x - c,
// t) are rebuilt where they are pulled: 80 B of state traffic per node and
// step (40 read, 40 written) instead of 216.  BGK's ghosts keep a memory of
// their own and have no such form.
//
// k_ms_step: a CTA owns a column of 30 x 14 (x, y) nodes and marches along
// z.  Each of its 512 threads owns one node of the column's 32 x 16 halo
// footprint (warp w = footprint row w): per plane it loads that node's ten
// numbers, adds its noise and reconstructs its 27 post-collision populations
// (collide_core's second half, the same code) into a ring of four planes in
// shared memory.  The 420 interior threads then pull their 27 incoming
// populations from the ring and collide (collide_core's first half) into
// the next state; the two all-halo warps skip the pull.  The halo is
// recomputed by the neighbouring columns (512 / 420 = 1.22 times the
// reconstruction work); the ten loads per halo node mostly hit L2.  With
// four planes in the ring, the plane a thread overwrites was last pulled two
// planes earlier, before the previous barrier, so one barrier per plane
// suffices and warps run from one plane's pull straight into the next
// plane's reconstruction.
//
// k_ms_boot: the first collision from a population state (any state,
// including one with ghost content); k_ms_step<EXPORT>: the populations of
// the current step rebuilt into population storage (natural AA form), for
// every call that reads populations.
#include "../../include/flbm.h"
#include "internal.h"
#include "step_kernel.cuh"

namespace flbm {

namespace {

constexpr int kMsTX = 30, kMsTY = 14;                      // interior of a column
constexpr int kMsHX = kMsTX + 2, kMsHY = kMsTY + 2;        // with the halo: 32 x 16
constexpr int kMsThreads = kMsHX * kMsHY;                  // 512: one halo node per thread
constexpr int kMsSlots = 4;                                // planes in the ring
constexpr size_t kMsRingBytes = size_t(kMsSlots) * kQ * kMsThreads * sizeof(float);   // 221,184 B

// the six second-order modes in state order: xx, yy, zz, xy, xz, yz
__host__ __device__ constexpr int ord2_deg(int r, int ax)
{
    return r < 3 ? (ax == r ? 2 : 0) : (r == 3 ? (ax < 2) : (r == 4 ? (ax != 1) : (ax > 0)));
}

// Store the ten state numbers of node n.
template <typename I>
__device__ __forceinline__ void store_state(float *__restrict__ ms, I N, I n, const float (&qm)[3][3][3],
                                            const float (&dj)[4])
{
#pragma unroll
    for (int s = 0; s < 4; ++s) __stcs(ms + I(s) * N + n, dj[s]);
#pragma unroll
    for (int r = 0; r < 6; ++r) __stcs(ms + I(4 + r) * N + n, qm[ord2_deg(r, 0)][ord2_deg(r, 1)][ord2_deg(r, 2)]);
}

template <typename I>
__device__ __forceinline__ void load_state(const float *__restrict__ ms, I N, I n, float (&st)[kMsVals])
{
#pragma unroll
    for (int s = 0; s < kMsVals; ++s) st[s] = __ldcg(ms + I(s) * N + n);
}

// The post-collision deviations of node n from its state st (noise of the
// step the noise arguments an name) -- the same amplitudes, in the same
// rounding, as collide_core hands to its reconstruction.
template <int SCHEME>
__device__ __forceinline__ void rebuild(const float (&st)[kMsVals], uint32_t node, const StepArgs<float> &an,
                                        float (&v)[3][3][3])
{
    const float drho = st[0];
    const float rho = an.rho0 + drho;
    const float jj[3] = {st[1], st[2], st[3]};
    const float irho = rcp_(rho);
    const float uu[3] = {jj[0] * irho, jj[1] * irho, jj[2] * irho};
    float qm[3][3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int ord = mode_order(i, j, k);
                const float syn = float(syn_scale(i, j, k));
                float q = 0.0f;
                if (ord == 0) q = drho * syn;
                else if (ord == 1) q = jj[i ? 0 : (j ? 1 : 2)] * syn;
                else if (ord > 2 && SCHEME == FLBM_REG) q = mul_rn(syn, aeq_coef(i, j, k, jj, uu));
                qm[i][j][k] = q;
            }
#pragma unroll
    for (int r = 0; r < 6; ++r) qm[ord2_deg(r, 0)][ord2_deg(r, 1)][ord2_deg(r, 2)] = st[4 + r];
    float nzd[kNoise];   // unused: drawn inside
    // scalar passes (the same bits as the paired ones; faster in this
    // kernel's register budget, measured)
    noise_synthesise<float, false, false>(qm, rho, an, nzd, node, v);
}

template <bool ODD, int SCHEME, bool STATS, typename I>
__global__ void __launch_bounds__(kBlock) k_ms_boot(const float *__restrict__ g, float *__restrict__ ms,
                                                    const StepArgs<float> a)
{
    float acc[NSTAT];
#pragma unroll
    for (int s = 0; s < NSTAT; ++s) acc[s] = 0.0f;
    const I N = I(a.n), NS = I(a.ns);   // moment-state stride, population slab stride
    for (uint64_t ch = blockIdx.x; ch < a.nchunks; ch += gridDim.x) {
        const uint32_t xc = uint32_t(ch % a.cpr);
        const uint64_t r = ch / a.cpr;
        const uint32_t y = uint32_t(r % a.ny), z = uint32_t(r / a.ny);
        const uint32_t x = xc * kBlock + threadIdx.x;
        if (x >= a.nx) continue;
        const Nbr<I> nb(x, y, z, a.nx, a.ny, a.nz);
        const I n = nb.node();
        float v[3][3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    I idx;
                    if (!ODD) idx = I(slot_of(i - 1, j - 1, k - 1)) * NS + n;
                    else idx = I(slot_of(1 - i, 1 - j, 1 - k)) * NS + (nb.xs[2 - i] + nb.ry[2 - j] + nb.rz[2 - k]);
                    v[i][j][k] = __ldcg(g + idx);
                }
        float qm[3][3][3], rho, dj[4];
        collide_modes<float, SCHEME, STATS>(v, a, acc, qm, rho, dj);
        store_state(ms, N, n, qm, dj);
    }
    if (STATS) block_reduce_store(acc, a.partials + size_t(blockIdx.x) * NSTAT);
}

struct MsGeom {
    uint32_t ntx, nty, nzs, zseg;   // columns along x and y, z segments of zseg planes
    uint64_t items;
};

// EXPORT = false: one step, state ms_in (collision t - 1) -> out = state of
// collision t (noise arguments an of step t - 1, collision arguments ac of
// step t).  EXPORT = true: out = population storage, natural form, of step t.
template <int SCHEME, bool STATS, bool EXPORT, typename I>
__global__ void __launch_bounds__(kMsThreads, 1) k_ms_step(const float *__restrict__ ms_in, float *__restrict__ out,
                                                           const StepArgs<float> an, const StepArgs<float> ac,
                                                           const MsGeom geo)
{
    extern __shared__ __align__(16) float ring[];   // [4][27][512]
    float acc[NSTAT];
#pragma unroll
    for (int s = 0; s < NSTAT; ++s) acc[s] = 0.0f;
    const I N = I(an.n), NS = I(an.ns);   // moment-state stride, population slab stride
    const uint32_t nx = an.nx, ny = an.ny, nz = an.nz;
    const uint32_t hx = threadIdx.x % kMsHX, hy = threadIdx.x / kMsHX;
    for (uint64_t item = blockIdx.x; item < geo.items; item += gridDim.x) {
        const uint32_t tx = uint32_t(item % geo.ntx);
        const uint64_t rest = item / geo.ntx;
        const uint32_t ty = uint32_t(rest % geo.nty), zs = uint32_t(rest / geo.nty);
        const uint32_t x0 = tx * kMsTX, y0 = ty * kMsTY, z0 = zs * geo.zseg;
        const uint32_t z1 = min(z0 + geo.zseg, nz);
        // this thread's halo node (periodic) and whether it is an interior node
        const uint32_t xg = (x0 + hx + nx - 1) % nx, yg = (y0 + hy + ny - 1) % ny;
        const bool inner = hx >= 1 && hx <= kMsTX && hy >= 1 && hy <= kMsTY && x0 + hx - 1 < nx &&
                           y0 + hy - 1 < ny;
        const I col = I(xg) + I(nx) * I(yg);
        const I plane = I(nx) * I(ny);
        // plane m of the march is z0 - 1 + m (periodic), held in ring slot m
        // % 4; its state is loaded one plane ahead (in flight during the
        // previous plane's pull) into st
        const uint32_t last = z1 - z0 + 1;
        auto node_of = [&](uint32_t m) { return col + I((z0 + m + nz - 1) % nz) * plane; };
        float st[kMsVals];
        auto build = [&](uint32_t m) {
            float v[3][3][3];
            rebuild<SCHEME>(st, uint32_t(node_of(m)), an, v);
            float *slot = ring + size_t(m % kMsSlots) * kQ * kMsThreads + threadIdx.x;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int k = 0; k < 3; ++k) slot[(9 * i + 3 * j + k) * kMsThreads] = v[i][j][k];
        };
        load_state(ms_in, N, node_of(0), st);
        build(0);
        load_state(ms_in, N, node_of(1), st);
        build(1);
        load_state(ms_in, N, node_of(2), st);
        for (uint32_t m = 1; m < last; ++m) {
            build(m + 1);
            if (m + 2 <= last) load_state(ms_in, N, node_of(m + 2), st);
            __syncthreads();
            if (inner) {
                // a1: f_c(x) = f*_c(x - c) from the ring
                float v[3][3][3];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j)
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const uint32_t src = (m + 1 - k) % kMsSlots;   // plane m - (k - 1)
                            const uint32_t pos = (hy + 1 - j) * kMsHX + (hx + 1 - i);
                            v[i][j][k] = ring[(size_t(src) * kQ + 9 * i + 3 * j + k) * kMsThreads + pos];
                        }
                const I n = col + I((z0 + m - 1) % nz) * plane;
                if (EXPORT) {
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int j = 0; j < 3; ++j)
#pragma unroll
                            for (int k = 0; k < 3; ++k) out[I(slot_of(i - 1, j - 1, k - 1)) * NS + n] = v[i][j][k];
                } else {
                    float qm[3][3][3], rho, dj[4];
                    collide_modes<float, SCHEME, STATS, false>(v, ac, acc, qm, rho, dj);
                    store_state(out, N, n, qm, dj);
                }
            }
        }
        __syncthreads();   // the next item's first planes reuse the ring
    }
    if (STATS) block_reduce_store(acc, ac.partials + size_t(blockIdx.x) * NSTAT);
}

bool fits32(uint64_t n) { return n * kQ < (1ull << 32); }

MsGeom geometry(const StepArgs<float> &a, int zseg)
{
    MsGeom g;
    g.ntx = (a.nx + kMsTX - 1) / kMsTX;
    g.nty = (a.ny + kMsTY - 1) / kMsTY;
    g.zseg = uint32_t(zseg);
    g.nzs = (a.nz + g.zseg - 1) / g.zseg;
    g.items = uint64_t(g.ntx) * g.nty * g.nzs;
    return g;
}

template <int SCHEME, bool STATS, bool EXPORT>
cudaError_t launch_ms_t(const float *ms, float *out, const StepArgs<float> &an, const StepArgs<float> &ac,
                        int grid, int zseg, cudaStream_t s)
{
    const MsGeom geo = geometry(an, zseg);
    const int g = int(std::min<uint64_t>(geo.items, uint64_t(grid)));
    if (fits32(an.ns))   // ns >= n: covers the 10 n moment-state indices too
        k_ms_step<SCHEME, STATS, EXPORT, uint32_t><<<g, kMsThreads, kMsRingBytes, s>>>(ms, out, an, ac, geo);
    else
        k_ms_step<SCHEME, STATS, EXPORT, uint64_t><<<g, kMsThreads, kMsRingBytes, s>>>(ms, out, an, ac, geo);
    return cudaGetLastError();
}

template <int SCHEME>
cudaError_t set_attrs()
{
    const int b = int(kMsRingBytes);
    cudaError_t e = cudaSuccess;
#define FLBM_MS_ATTR(ST, EX, I)                                                                              \
    if (e == cudaSuccess)                                                                                    \
        e = cudaFuncSetAttribute(k_ms_step<SCHEME, ST, EX, I>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    FLBM_MS_ATTR(false, false, uint32_t)
    FLBM_MS_ATTR(true, false, uint32_t)
    FLBM_MS_ATTR(false, true, uint32_t)
    FLBM_MS_ATTR(false, false, uint64_t)
    FLBM_MS_ATTR(true, false, uint64_t)
    FLBM_MS_ATTR(false, true, uint64_t)
#undef FLBM_MS_ATTR
    return e;
}

template <bool ODD, int SCHEME, bool STATS>
cudaError_t launch_boot_t(const float *g, float *ms, const StepArgs<float> &a, int grid, cudaStream_t s)
{
    if (fits32(a.ns)) k_ms_boot<ODD, SCHEME, STATS, uint32_t><<<grid, kBlock, 0, s>>>(g, ms, a);
    else k_ms_boot<ODD, SCHEME, STATS, uint64_t><<<grid, kBlock, 0, s>>>(g, ms, a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t ms_prepare(int scheme, int nsm, const StepArgs<float> &a, int &grid, int &zseg)
{
    const cudaError_t e = scheme == FLBM_REG ? set_attrs<FLBM_REG>() : set_attrs<FLBM_GMF>();
    if (e != cudaSuccess) return e;
    // z segments: long enough that the two extra halo planes per segment cost
    // little (<= 128 planes: 1.6 %), short enough for about eight
    // column segments per CTA
    const uint64_t cols = uint64_t((a.nx + kMsTX - 1) / kMsTX) * ((a.ny + kMsTY - 1) / kMsTY);
    const uint64_t want = uint64_t(8) * uint64_t(nsm);
    uint64_t z = (cols * a.nz + want - 1) / want;
    zseg = int(std::max<uint64_t>(8, std::min<uint64_t>(128, z)));
    zseg = int(std::min<uint64_t>(uint64_t(zseg), a.nz));
    grid = int(std::min<uint64_t>(geometry(a, zseg).items, uint64_t(nsm)));   // one CTA per SM (shared ring)
    if (grid < 1) grid = 1;
    return cudaSuccess;
}

cudaError_t launch_ms_boot(const float *g, float *ms, const StepArgs<float> &a, int scheme, bool odd, bool stats,
                           int grid, cudaStream_t s)
{
    if (scheme == FLBM_REG) {
        if (odd) return stats ? launch_boot_t<true, FLBM_REG, true>(g, ms, a, grid, s)
                              : launch_boot_t<true, FLBM_REG, false>(g, ms, a, grid, s);
        return stats ? launch_boot_t<false, FLBM_REG, true>(g, ms, a, grid, s)
                     : launch_boot_t<false, FLBM_REG, false>(g, ms, a, grid, s);
    }
    if (odd) return stats ? launch_boot_t<true, FLBM_GMF, true>(g, ms, a, grid, s)
                          : launch_boot_t<true, FLBM_GMF, false>(g, ms, a, grid, s);
    return stats ? launch_boot_t<false, FLBM_GMF, true>(g, ms, a, grid, s)
                 : launch_boot_t<false, FLBM_GMF, false>(g, ms, a, grid, s);
}

cudaError_t launch_ms_step(const float *ms_in, float *ms_out, const StepArgs<float> &an, const StepArgs<float> &ac,
                           int scheme, bool stats, int grid, int zseg, cudaStream_t s)
{
    if (scheme == FLBM_REG)
        return stats ? launch_ms_t<FLBM_REG, true, false>(ms_in, ms_out, an, ac, grid, zseg, s)
                     : launch_ms_t<FLBM_REG, false, false>(ms_in, ms_out, an, ac, grid, zseg, s);
    return stats ? launch_ms_t<FLBM_GMF, true, false>(ms_in, ms_out, an, ac, grid, zseg, s)
                 : launch_ms_t<FLBM_GMF, false, false>(ms_in, ms_out, an, ac, grid, zseg, s);
}

cudaError_t launch_ms_export(const float *ms, float *g, const StepArgs<float> &an, int scheme, int grid, int zseg,
                             cudaStream_t s)
{
    if (scheme == FLBM_REG) return launch_ms_t<FLBM_REG, false, true>(ms, g, an, an, grid, zseg, s);
    return launch_ms_t<FLBM_GMF, false, true>(ms, g, an, an, grid, zseg, s);
}

}  // namespace flbm
