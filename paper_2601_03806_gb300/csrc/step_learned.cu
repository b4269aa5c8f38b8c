// step_learned.cu -- the learned-collision step: GMF-FLBM (Eq. flbe2) plus
// the network correction, fused in one kernel.
//
// A CTA of 512 threads (one per SM: it allocates tensor memory) takes four
// row chunks of 128 consecutive x-nodes (the chunking of the direct step
// kernel) at a time, one per network sub-tile; threads past a row end or
// past the last chunk only take part in the tile.  Each thread's node's 27
// incoming populations (AA pattern) arrive in its own column of a shared
// staging buffer by 4-byte cp.async, issued one round ahead, so the global
// latency hides behind the previous node's work; no other thread touches
// that column, so the thread's own wait suffices.  The thread writes the
// node's features to the network tile, and, while the first layer's
// tensor-core MMAs run, starts the next round's copies and collides the node
// with the GMF collision (collide_core, noise included).  Then it adds
// P(w_i sigma^3 y_i), the network output mapped to populations with mass and
// momentum projected out, and stores (AA pattern).  The network runs on the
// tcgen05 path of mlp_tc.cuh.
//
// Early reads are safe in place: under the AA pattern the locations a node
// reads are exactly those it writes, so no other node's store can land on a
// staged value.
#include "../../include/flbm.h"
#include "internal.h"
#include "mlp_tc.cuh"

namespace flbm {

namespace {

constexpr size_t kStageBytes = size_t(kQ) * kMlpThreads * sizeof(float);   // [27][512] floats
constexpr size_t kLearnSmemBytes = kMlpSmemBytes + kStageBytes;

// Position (x-chunk, y, z) of this thread's row chunk; chunk ch = (z ny + y)
// cpr + xc.  Across the rounds a thread's chunk advances by 4 x gridDim.x,
// decomposed once in the same mixed radix, so a round costs two carries
// instead of two divisions.
struct Walk {
    uint32_t xc, y, z;
};
__device__ __forceinline__ Walk walk_of(const StepArgs<float> &a, uint64_t ch)
{
    const uint64_t r = ch / a.cpr;
    return Walk{uint32_t(ch % a.cpr), uint32_t(r % a.ny), uint32_t(r / a.ny)};
}
__device__ __forceinline__ Walk advance(Walk w, const Walk &d, const StepArgs<float> &a)
{
    w.xc += d.xc;
    w.y += d.y;
    w.z += d.z;
    if (w.xc >= a.cpr) {
        w.xc -= a.cpr;
        ++w.y;
    }
    if (w.y >= a.ny) {
        w.y -= a.ny;
        ++w.z;
    }
    return w;
}

// This thread's node at walk position w (x = 0 when inactive: past a row's
// end, or z past the box for chunks beyond the last).
struct Site {
    uint32_t x, y, z;
    bool active;
};
__device__ __forceinline__ Site site_of(const Walk &w, const StepArgs<float> &a)
{
    Site s;
    s.x = w.xc * 128 + (threadIdx.x & 127u);
    s.y = w.y;
    s.z = w.z;
    s.active = w.z < a.nz && s.x < a.nx;
    if (!s.active) s.x = s.y = s.z = 0;
    return s;
}

__device__ __forceinline__ void cp_async4(float *dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Population c = (i-1, j-1, k-1) of node (x, y, z) as the AA pattern reads it.
template <typename I, bool ODD>
__device__ __forceinline__ I load_index(const Nbr<I> &nb, I N, int i, int j, int k)
{
    if (!ODD) return I(slot_of(i - 1, j - 1, k - 1)) * N + nb.node();
    return I(slot_of(1 - i, 1 - j, 1 - k)) * N + (nb.xs[2 - i] + nb.ry[2 - j] + nb.rz[2 - k]);
}

// Start the copies of this thread's node at site s into its column.
template <typename I, bool ODD>
__device__ __forceinline__ void stage_node(const float *g, float *stage, const StepArgs<float> &a, const Site &s)
{
    if (s.active) {
        const Nbr<I> nb(s.x, s.y, s.z, a.nx, a.ny, a.nz);
        const I N = I(a.ns);   // slab stride
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    cp_async4(stage + (9 * i + 3 * j + k) * kMlpThreads + threadIdx.x,
                              g + load_index<I, ODD>(nb, N, i, j, k));
    }
    cp_async_commit();
}

template <typename I, bool ODD, bool STATS>
__global__ void __launch_bounds__(kMlpThreads, 1) k_step_learned(float *__restrict__ g, const StepArgs<float> a,
                                                         const LearnArgs L)
{
    extern __shared__ __align__(1024) unsigned char smraw[];
    MlpSmem &sm = *reinterpret_cast<MlpSmem *>(smraw);
    float *stage = reinterpret_cast<float *>(smraw + kMlpSmemBytes);
    const uint64_t nsuper = (a.nchunks + kMlpSub - 1) / kMlpSub;
    Walk w = walk_of(a, uint64_t(blockIdx.x) * kMlpSub + (threadIdx.x >> 7));
    const Walk step = walk_of(a, uint64_t(gridDim.x) * kMlpSub);
    if (blockIdx.x < nsuper) stage_node<I, ODD>(g, stage, a, site_of(w, a));
    mlp_setup(sm, L.img);
    uint32_t phase = 0;
    float acc[NSTAT];
#pragma unroll
    for (int s = 0; s < NSTAT; ++s) acc[s] = 0.0f;
    const I N = I(a.ns);   // slab stride
    for (uint64_t sc = blockIdx.x; sc < nsuper; sc += gridDim.x) {
        const Site cur = site_of(w, a);
        w = advance(w, step, a);
        cp_async_wait_all();
        float v[3][3][3];
        float xf[kMlpIn];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    v[i][j][k] = cur.active ? stage[(9 * i + 3 * j + k) * kMlpThreads + threadIdx.x] : 0.0f;
                    // feature of population c = (i-1, j-1, k-1): g_c / sqrt(rho0 kT w_c / c_s^2)
                    xf[slot_of(i - 1, j - 1, k - 1)] = v[i][j][k] * L.inv_s[(i != 1) + (j != 1) + (k != 1)];
                }
        xf[27] = cur.active ? L.x27 : 0.0f;
        float yv[kMlpOut];
        float nzd[kNoise];   // unused: the collision draws its normals inside
        const uint64_t next = sc + gridDim.x;
        const bool ok = mlp_tile(sm, phase, xf, yv, [&] {
            if (next < nsuper) stage_node<I, ODD>(g, stage, a, site_of(w, a));
            if (cur.active) {
                const Nbr<I> nb(cur.x, cur.y, cur.z, a.nx, a.ny, a.nz);
                collide_core<float, 1, STATS, false>(v, a, nzd, uint32_t(nb.node()), acc);
            }
        }, L.starve != 0);
        if (!ok) {
            if ((threadIdx.x & 127u) == 0) atomicOr(a.flag, 2u);   // one report per group
            break;
        }
        if (!cur.active) continue;
        const Nbr<I> nb(cur.x, cur.y, cur.z, a.nx, a.ny, a.nz);
        const I n = nb.node();
        // correction d_c = w_c sigma^3 y_c minus its mass and momentum:
        // P(d)_c = d_c - w_c (alpha + 3 c . beta), alpha = sum d, beta = sum c d,
        // with the sums and the 27 offsets taken axis by axis
        float d[3][3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    d[i][j][k] = (float(w1(i - 1) * w1(j - 1) * w1(k - 1)) * L.sig3) * yv[slot_of(i - 1, j - 1, k - 1)];
        float T[3][3], bz = 0.0f;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                T[i][j] = (d[i][j][0] + d[i][j][2]) + d[i][j][1];
                bz += d[i][j][2] - d[i][j][0];
            }
        float Sx[3], by = 0.0f;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            Sx[i] = (T[i][0] + T[i][2]) + T[i][1];
            by += T[i][2] - T[i][0];
        }
        const float alpha = (Sx[0] + Sx[2]) + Sx[1];
        const float bx = Sx[2] - Sx[0];
        const float b3[3] = {3.0f * bx, 3.0f * by, 3.0f * bz};
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float ti = i == 1 ? alpha : (i == 2 ? alpha + b3[0] : alpha - b3[0]);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float tij = j == 1 ? ti : (j == 2 ? ti + b3[1] : ti - b3[1]);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float t = k == 1 ? tij : (k == 2 ? tij + b3[2] : tij - b3[2]);
                    const float w = float(w1(i - 1) * w1(j - 1) * w1(k - 1));
                    v[i][j][k] += __fmaf_rn(-w, t, d[i][j][k]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    I idx;
                    if (!ODD) idx = I(slot_of(1 - i, 1 - j, 1 - k)) * N + n;
                    else idx = I(slot_of(i - 1, j - 1, k - 1)) * N + (nb.xs[i] + nb.ry[j] + nb.rz[k]);
                    __stcs(g + idx, v[i][j][k]);
                }
    }
    cp_async_wait_all();   // no copy may land after the CTA has left
    mlp_teardown(sm);
    if (STATS) block_reduce_store(acc, a.partials + size_t(blockIdx.x) * NSTAT);
}

template <typename I>
cudaError_t launch_t(float *g, const StepArgs<float> &a, const LearnArgs &L, bool odd, bool stats, int grid,
                     cudaStream_t s)
{
    if (odd) {
        if (stats) k_step_learned<I, true, true><<<grid, kMlpThreads, kLearnSmemBytes, s>>>(g, a, L);
        else k_step_learned<I, true, false><<<grid, kMlpThreads, kLearnSmemBytes, s>>>(g, a, L);
    } else {
        if (stats) k_step_learned<I, false, true><<<grid, kMlpThreads, kLearnSmemBytes, s>>>(g, a, L);
        else k_step_learned<I, false, false><<<grid, kMlpThreads, kLearnSmemBytes, s>>>(g, a, L);
    }
    return cudaGetLastError();
}

bool fits32(uint64_t n) { return n * kQ < (1ull << 32); }

}  // namespace

cudaError_t launch_step_learned(float *g, const StepArgs<float> &a, const LearnArgs &L, bool odd, bool stats,
                                int grid, cudaStream_t s)
{
    if (fits32(a.ns)) return launch_t<uint32_t>(g, a, L, odd, stats, grid, s);
    return launch_t<uint64_t>(g, a, L, odd, stats, grid, s);
}

int learned_occupancy(uint64_t n)
{
    // the sub-tile buffers exceed the 48 KB default
    const int sm = int(kLearnSmemBytes);
    cudaFuncSetAttribute(k_step_learned<uint32_t, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_step_learned<uint32_t, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_step_learned<uint32_t, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_step_learned<uint32_t, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_step_learned<uint64_t, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_step_learned<uint64_t, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_step_learned<uint64_t, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_step_learned<uint64_t, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    int nb = 0;
    const cudaError_t e = fits32(n)
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_learned<uint32_t, true, true>, kMlpThreads,
                                                        kLearnSmemBytes)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_learned<uint64_t, true, true>, kMlpThreads,
                                                        kLearnSmemBytes);
    (void)nb;
    (void)e;
    return 1;   // a CTA holds all 512 tensor-memory columns of its SM
}

}  // namespace flbm
