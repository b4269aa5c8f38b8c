// ens_kernel.cuh -- one persistent kernel advancing many independent boxes.
//
// Work decomposition.  Replica r is cut into items of rpi_r whole x-rows of
// one z-plane (rpi_r divides ny_r, so an item never crosses a plane); the
// items of all replicas, replica after replica, form one global sequence.
// CTA b owns the contiguous chunk [b K + min(b, rem), ...) of it (K = items /
// grid), so every CTA moves the same number of items whatever the mix of box
// sizes, and a CTA meets only a few replicas, in order.
//
// Per item the CTA runs the same warp-specialised pipeline as the single-box
// row kernel (step_kernel.cuh): the copy warp's lanes 0..26 each move one of
// the 27 plane segments of the item between HBM and a shared-memory stage
// with bulk copies (cp.async.bulk) completing on a "full" mbarrier; the
// compute warps apply the periodic x-shift in shared memory, collide
// (collide_core, the same code as the single-box kernels, so a replica's
// populations equal its single box's bit for bit; with NP = 2 a thread
// collides two adjacent nodes of a row at once), overwrite the
// segments and release the stage through an "empty" mbarrier, after which
// the copy warp stores the segments back.  In the odd AA form a segment that
// starts or ends on the periodic y-seam of the plane takes two copies.
//
// Statistics: each compute warp keeps FP32 per-thread sums (per lane with
// NP = 2) of the replica it is on and, when the CTA leaves that replica,
// writes its warp totals to
// partial slot (cta + replica, warp); along the chunk order the pairs
// (cta, replica) met are distinct, so slot cta + replica is unique.  No
// barrier is involved, so a wait that runs out cannot hang the others.  The
// post kernel adds a replica's slots in a fixed order (deterministic FP64
// totals) into its context's DevStats and advances the device step counter,
// which the next step kernel reads, so that a captured CUDA graph replays
// correctly.
#pragma once

#include "step_kernel.cuh"
#include "stats.cuh"

namespace flbm {

// The per-replica scalars collide_core and draw_noise read (the member
// names of StepArgs).
template <typename R>
struct EnsView {
    const uint32_t (&rk)[20];
    uint64_t step;
    uint32_t ctr2;
    int32_t noise_rho0;
    R rho0, sqrt_rho0, lambda, omega, amp_h, amp_g;
    unsigned int *flag;
    unsigned long long *bad_step;
};

// Philox block blk of node for a replica: round 0's product of counter word
// 2 = blk | stream << 8 is formed here (philox4x32_10_r0).  Forming all
// launch-uniform words of rounds 0-1 instead (as the single-box kernels read
// them) lets the compiler hoist 19 values per item out of the node loop,
// which spills at this kernel's register cap.
template <typename R>
__device__ __forceinline__ u32x4 noise_block(const EnsView<R> &v, uint32_t node, int blk)
{
    const uint64_t m = uint64_t(0xCD9E8D57u) * (uint32_t(blk) | v.ctr2);
    return philox4x32_10_r0(node, uint32_t(v.step), uint32_t(v.step >> 32), uint32_t(m >> 32) ^ v.rk[0],
                            uint32_t(m), v.rk);
}

// Index of the replica holding global item i (replicas ordered by item0).
__device__ __forceinline__ uint32_t ens_find(const EnsReplica *reps, uint32_t nrep, uint64_t i)
{
    uint32_t lo = 0, hi = nrep - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (reps[mid].item0 <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Advance the replica cursor `cur` to the replica holding item i (i never
// decreases along a CTA's chunk).
__device__ __forceinline__ void ens_advance(const EnsReplica *reps, uint32_t nrep, uint64_t i, uint32_t &cur)
{
    while (cur + 1 < nrep && reps[cur + 1].item0 <= i) ++cur;
}

// The contiguous copies (at most two) that move segment d = 9 (cx+1) +
// 3 (cy+1) + (cz+1) of the item at rows y0 .. y0 + rpi - 1 of plane z:
// element offset in the replica's planes, element offset inside the staged
// segment, element count.  Even form: slot c of the item's own rows.  Odd
// form: slot opp(c) of rows y - cy of plane z - cz, periodic, so a segment
// whose rows cross the y-seam is split in two.
template <bool ODD>
__device__ __forceinline__ int ens_pieces(const EnsReplica &r, uint32_t z, uint32_t y0, int d,
                                          uint64_t (&go)[2], uint32_t (&lo)[2], uint32_t (&cnt)[2])
{
    const int cx = d / 9 - 1, cy = (d / 3) % 3 - 1, cz = d % 3 - 1;
    const uint32_t nx = r.nx, ny = r.ny, rpi = r.rpi;
    uint32_t zz = z;
    int slot = slot_of(cx, cy, cz);
    if (ODD) {
        slot = slot_of(-cx, -cy, -cz);
        if (cz > 0) zz = z ? z - 1 : r.nz - 1;
        if (cz < 0) zz = (z + 1 < r.nz) ? z + 1 : 0;
    }
    const uint64_t base = uint64_t(slot) * r.n + uint64_t(zz) * ny * nx;
    lo[0] = 0;
    cnt[0] = rpi * nx;
    if (!ODD || cy == 0) {                       // rows y0 .. y0 + rpi - 1
        go[0] = base + uint64_t(y0) * nx;
        return 1;
    }
    if (cy > 0) {                                // rows y0 - 1 .. y0 + rpi - 2
        if (y0 > 0) {
            go[0] = base + uint64_t(y0 - 1) * nx;
            return 1;
        }
        go[0] = base + uint64_t(ny - 1) * nx;    // row ny - 1 -> local row 0
        cnt[0] = nx;
        if (rpi == 1) return 1;
        go[1] = base;                            // rows 0 .. rpi - 2 -> local rows 1 ..
        lo[1] = nx;
        cnt[1] = (rpi - 1) * nx;
        return 2;
    }
    if (y0 + rpi < ny) {                         // rows y0 + 1 .. y0 + rpi
        go[0] = base + uint64_t(y0 + 1) * nx;
        return 1;
    }
    go[0] = base;                                // row 0 -> local row rpi - 1
    lo[0] = (rpi - 1) * nx;
    cnt[0] = nx;
    if (rpi == 1) return 1;
    go[1] = base + uint64_t(y0 + 1) * nx;        // rows y0 + 1 .. ny - 1 -> local rows 0 ..
    lo[1] = 0;
    cnt[1] = (rpi - 1) * nx;
    return 2;
}

// Item i of replica rp: its plane z and first row y0.
// (A replica has fewer than 2^31 nodes, so its item index fits 32 bits.)
__device__ __forceinline__ void ens_item(const EnsReplica &rp, uint64_t i, uint32_t &z, uint32_t &y0)
{
    const uint32_t j = uint32_t(i - rp.item0);
    z = j / rp.items_per_plane;
    y0 = (j - z * rp.items_per_plane) * rp.rpi;
}

// NP = 1: one node per compute thread, at most 112 registers a thread (the
// collision spills little at that cap; registers are split over the SM's four
// sub-partitions, so two CTAs fit an SM up to 7 compute warps each).  NP = 2:
// two adjacent nodes of a row per thread as packed FP32 pairs (row lengths
// are even: a replica's rows are 16-byte aligned), at most 168 registers, so
// two CTAs of up to 4 compute warps fit an SM.
// STRIDE: the stage stride as a compile-time constant (256 or 512 nodes, the
// common tunings), which folds the 27 segment offsets of a node's shared
// loads and stores into their immediates; 0 reads it from the arguments.
template <typename S, typename R, int SCHEME, bool ODD, bool STATS, int STRIDE = 0, int NP = 1>
__global__ void __maxnreg__(NP == 2 ? 168 : 112) k_step_ens(const __grid_constant__ EnsArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kEnsMaxStages], empty[kEnsMaxStages];
    S *const stage = reinterpret_cast<S *>(smem_raw);
    const EnsReplica *__restrict__ reps = a.reps;
    const uint32_t nc = blockDim.x - 32;                 // compute threads
    const uint32_t stages = a.stages;
    const uint32_t stride = STRIDE ? uint32_t(STRIDE) : a.stride;
    const uint32_t stage_elems = uint32_t(kQ) * stride;
    const uint32_t lane = threadIdx.x & 31;
    uint64_t begin, end;
    ens_chunk(a.nitems, blockIdx.x, gridDim.x, begin, end);

    if (threadIdx.x == 0) {
        for (uint32_t s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], nc / 32);
        }
        mbar_init_fence();
    }
    __syncthreads();
    if (begin >= end) return;
    const uint32_t nk = uint32_t(end - begin);
    const uint32_t r0 = ens_find(reps, a.nrep, begin);

    if (threadIdx.x >= nc) {
        // ---------------- copy warp ----------------
        const int d = int(lane);
        uint32_t r_load = r0, r_store = r0;
        bool ok = true;
        auto move = [&](uint32_t k, uint32_t s, uint32_t &cur, bool load, uint64_t *bar) {
            const uint64_t i = begin + k;
            ens_advance(reps, a.nrep, i, cur);
            const EnsReplica &rp = reps[cur];
            uint32_t z, y0;
            ens_item(rp, i, z, y0);
            uint64_t go[2];
            uint32_t lo[2], cnt[2];
            const int np = ens_pieces<ODD>(rp, z, y0, d, go, lo, cnt);
            S *gp = static_cast<S *>(rp.g);
            S *sp = stage + size_t(s) * stage_elems + size_t(d) * stride;
            for (int q = 0; q < np; ++q) {
                if (load) bulk_g2s(sp + lo[q], gp + go[q], cnt[q] * uint32_t(sizeof(S)), bar);
                else bulk_s2g(gp + go[q], sp + lo[q], cnt[q] * uint32_t(sizeof(S)));
            }
        };
        // stage and mbarrier phase of the next store (ss, sph) and load (s)
        uint32_t ss = 0, sph = 0;
        auto store_item = [&](uint32_t kk) {
            ok = mbar_wait(&empty[ss], sph);
            if (!ok) return;
            if (d < kQ) {
                move(kk, ss, r_store, false, nullptr);
                bulk_commit();
                bulk_wait_read_all();
            }
            __syncwarp();
            if (++ss == stages) {
                ss = 0;
                sph ^= 1u;
            }
        };
        uint32_t k = 0, s = 0;
        for (; k < nk; ++k) {
            if (k >= stages) {
                store_item(k - stages);
                if (!ok) break;
            }
            ens_advance(reps, a.nrep, begin + k, r_load);
            if (lane == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&full[s], uint32_t(kQ) * reps[r_load].item_nodes * uint32_t(sizeof(S)) +
                                                    a.tx_pad);
            }
            __syncwarp();
            if (d < kQ) move(k, s, r_load, true, &full[s]);
            if (++s == stages) s = 0;
        }
        for (uint32_t kk = (k > stages ? k - stages : 0); ok && kk < k; ++kk) store_item(kk);
        if (!ok && lane == 0) atomicOr(a.flag, 2u);
        if (d < kQ) bulk_wait_all();
    } else {
        // ---------------- compute warps ----------------
        using V = typename std::conditional<NP == 2, float2, R>::type;
        const uint64_t step = *a.dstep;
        const uint32_t warp = threadIdx.x >> 5;
        V acc[NSTAT];
#pragma unroll
        for (int s = 0; s < NSTAT; ++s) acc[s] = vset<V>(0.0);
        uint32_t r = r0;
        uint32_t s = 0, ph = 0;   // stage and mbarrier phase of item k
        for (uint32_t k = 0; k < nk; ++k) {
            const uint64_t i = begin + k;
            ens_advance(reps, a.nrep, i, r);
            const EnsReplica &rp = reps[r];
            const EnsView<R> v{a.rk, step, rp.ctr2, rp.noise_rho0, R(rp.rho0), R(rp.sqrt_rho0),
                               R(rp.lambda), R(rp.omega), R(rp.amp_h), R(rp.amp_g), a.flag, rp.bad_step};
            const uint32_t nx = rp.nx, item_nodes = rp.item_nodes;
            uint32_t z, y0;
            ens_item(rp, i, z, y0);
            const uint32_t base = (z * rp.ny + y0) * nx;   // first node of the item
            // row of local node l: (l + 1/2) / nx in FP32 is within 128 x 2^-23
            // of its exact value and at least 1/(2 nx) >= 5.6e-4 from an
            // integer (l < 4096, nx <= 896), so truncation gives l / nx exactly
            const float inv_nx = __frcp_rn(float(nx));
            if constexpr (NP == 2) {
                if (!mbar_wait(&full[s], ph)) {
                    if (lane == 0) atomicOr(a.flag, 2u);
                    break;
                }
                S *st = stage + size_t(s) * stage_elems;
                for (uint32_t l = 2 * threadIdx.x; l < item_nodes; l += 2 * nc) {
                    // nodes l (lane .x) and l + 1 (lane .y) of one row: l and nx are even
                    const uint32_t t = uint32_t((float(l) + 0.5f) * inv_nx), x = l - t * nx, rb = t * nx;
                    const uint32_t xa[3] = {rb + (x ? x - 1 : nx - 1), l, l + 1};
                    const uint32_t xb[3] = {l, l + 1, rb + ((x + 2 < nx) ? x + 2 : 0)};
                    V vv[3][3][3];
#pragma unroll
                    for (int ci = 0; ci < 3; ++ci)
#pragma unroll
                        for (int cj = 0; cj < 3; ++cj)
#pragma unroll
                            for (int ck = 0; ck < 3; ++ck) {
                                const S *seg = st + (9 * ci + 3 * cj + ck) * stride;
                                if (!ODD || ci == 1) vv[ci][cj][ck] = ld_pair(seg + l);
                                else vv[ci][cj][ck] = make_float2(stage_ld(seg[xa[2 - ci]]), stage_ld(seg[xb[2 - ci]]));
                            }
                    V nzp[kNoise];   // unused: the normals are drawn inside, pair by pair
                    collide_core<V, SCHEME, STATS, false>(vv, v, nzp, base + l, acc);
#pragma unroll
                    for (int ci = 0; ci < 3; ++ci)
#pragma unroll
                        for (int cj = 0; cj < 3; ++cj)
#pragma unroll
                            for (int ck = 0; ck < 3; ++ck) {
                                S *seg = st + (9 * (2 - ci) + 3 * (2 - cj) + (2 - ck)) * stride;
                                if (!ODD || ci == 1) st_pair(seg + l, vv[ci][cj][ck]);
                                else {
                                    seg[xa[ci]] = stage_st<S>(vv[ci][cj][ck].x);
                                    seg[xb[ci]] = stage_st<S>(vv[ci][cj][ck].y);
                                }
                            }
                }
            } else {
                R nz[kNoise];
                if (threadIdx.x < item_nodes) draw_noise(v, base + threadIdx.x, nz);
                if (!mbar_wait(&full[s], ph)) {
                    if (lane == 0) atomicOr(a.flag, 2u);
                    break;
                }
                S *st = stage + size_t(s) * stage_elems;
                for (uint32_t l = threadIdx.x; l < item_nodes; l += nc) {
                    if (l != threadIdx.x) draw_noise(v, base + l, nz);
                    const uint32_t t = uint32_t((float(l) + 0.5f) * inv_nx), x = l - t * nx, rb = t * nx;
                    const uint32_t xsh[3] = {rb + (x ? x - 1 : nx - 1), l, rb + ((x + 1 < nx) ? x + 1 : 0)};
                    R vv[3][3][3];
#pragma unroll
                    for (int ci = 0; ci < 3; ++ci)
#pragma unroll
                        for (int cj = 0; cj < 3; ++cj)
#pragma unroll
                            for (int ck = 0; ck < 3; ++ck) {
                                const uint32_t pos = ODD ? xsh[2 - ci] : l;
                                vv[ci][cj][ck] = R(stage_ld(st[(9 * ci + 3 * cj + ck) * stride + pos]));
                            }
                    collide_core<R, SCHEME, STATS, true>(vv, v, nz, base + l, acc);
#pragma unroll
                    for (int ci = 0; ci < 3; ++ci)
#pragma unroll
                        for (int cj = 0; cj < 3; ++cj)
#pragma unroll
                            for (int ck = 0; ck < 3; ++ck) {
                                const uint32_t pos = ODD ? xsh[ci] : l;
                                st[(9 * (2 - ci) + 3 * (2 - cj) + (2 - ck)) * stride + pos] =
                                    stage_st<S>(vv[ci][cj][ck]);
                            }
                }
            }
            fence_proxy_async_smem();   // generic-proxy writes before the bulk store reads
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            if (++s == stages) {
                s = 0;
                ph ^= 1u;
            }
            if (STATS) {
                const bool leaving = (k + 1 == nk) || (r + 1 < a.nrep && reps[r + 1].item0 <= i + 1);
                if (leaving) {
                    double *out = a.partials + ((size_t(blockIdx.x) + r) * kEnsMaxWarps + warp) * NSTAT;
#pragma unroll
                    for (int q = 0; q < NSTAT; ++q) {
                        const R tot = warp_sum(lane_total(acc[q]));
                        if (lane == 0) out[q] = double(tot);
                        acc[q] = vset<V>(0.0);
                    }
                }
            }
        }
    }
}

// Per replica (one CTA each, stats steps): FP64 totals of its partial slots
// in (cta, warp) order into its DevStats; then the last CTA to finish
// advances the step counter.  Non-stats steps launch one CTA that only
// advances it.
template <bool STATS>
__global__ void k_ens_post(const __grid_constant__ EnsArgs a, uint32_t cwarps, unsigned int *done,
                           unsigned long long *dstep)
{
    if (STATS) {
        __shared__ double tot[NSTAT];
        const uint32_t r = blockIdx.x;
        const EnsReplica &rp = a.reps[r];
        if (threadIdx.x < NSTAT) {
            double t = 0.0;
            for (int b = rp.cta_lo; b <= rp.cta_hi; ++b)
                for (uint32_t w = 0; w < cwarps; ++w)
                    t += a.partials[((size_t(b) + r) * kEnsMaxWarps + w) * NSTAT + threadIdx.x];
            tot[threadIdx.x] = t;
        }
        __syncthreads();
        if (threadIdx.x == 0) stats_update(rp.st, tot, (long long)(*dstep), double(rp.n));
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int prev = atomicAdd(done, 1u);
        if (prev == gridDim.x - 1) {
            *dstep += 1ull;
            *done = 0u;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------------------
// launchers

template <typename S, typename R, int NP>
cudaError_t launch_ens_step_t(const EnsArgs &a, int scheme, bool odd, bool stats, int grid, int threads,
                              size_t smem, cudaStream_t s)
{
#define FLBM_LAUNCH_ENS(SC, OD, ST) k_step_ens<S, R, SC, OD, ST, 0, NP><<<grid, threads, smem, s>>>(a)
#define FLBM_LAUNCH_ENS_W(W, OD, ST) k_step_ens<S, R, 1, OD, ST, W, NP><<<grid, threads, smem, s>>>(a)
    if (scheme == 1 && (a.stride == 512 || a.stride == 256)) {   // GMF at a compile-time stride
        if (a.stride == 512) {
            if (odd) { if (stats) FLBM_LAUNCH_ENS_W(512, true, true); else FLBM_LAUNCH_ENS_W(512, true, false); }
            else     { if (stats) FLBM_LAUNCH_ENS_W(512, false, true); else FLBM_LAUNCH_ENS_W(512, false, false); }
        } else {
            if (odd) { if (stats) FLBM_LAUNCH_ENS_W(256, true, true); else FLBM_LAUNCH_ENS_W(256, true, false); }
            else     { if (stats) FLBM_LAUNCH_ENS_W(256, false, true); else FLBM_LAUNCH_ENS_W(256, false, false); }
        }
    } else if (scheme == 0) {
        if (odd) { if (stats) FLBM_LAUNCH_ENS(0, true, true); else FLBM_LAUNCH_ENS(0, true, false); }
        else     { if (stats) FLBM_LAUNCH_ENS(0, false, true); else FLBM_LAUNCH_ENS(0, false, false); }
    } else if (scheme == 1) {
        if (odd) { if (stats) FLBM_LAUNCH_ENS(1, true, true); else FLBM_LAUNCH_ENS(1, true, false); }
        else     { if (stats) FLBM_LAUNCH_ENS(1, false, true); else FLBM_LAUNCH_ENS(1, false, false); }
    } else {
        if (odd) { if (stats) FLBM_LAUNCH_ENS(2, true, true); else FLBM_LAUNCH_ENS(2, true, false); }
        else     { if (stats) FLBM_LAUNCH_ENS(2, false, true); else FLBM_LAUNCH_ENS(2, false, false); }
    }
#undef FLBM_LAUNCH_ENS
#undef FLBM_LAUNCH_ENS_W
    return cudaGetLastError();
}

template <typename S, typename R, int SC, int NP>
int ens_occupancy_scheme(int threads, size_t smem)
{
    // the attribute is per kernel and process-wide: the largest staging any
    // ensemble may use (occupancy below is for this shape's smem)
    const int sm = int(kRowMaxSmem);
    cudaFuncSetAttribute(k_step_ens<S, R, SC, false, false, 0, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_step_ens<S, R, SC, false, true, 0, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_step_ens<S, R, SC, true, false, 0, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_step_ens<S, R, SC, true, true, 0, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (SC == 1) {
        cudaFuncSetAttribute(k_step_ens<S, R, 1, false, false, 256, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaFuncSetAttribute(k_step_ens<S, R, 1, false, true, 256, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaFuncSetAttribute(k_step_ens<S, R, 1, true, false, 256, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaFuncSetAttribute(k_step_ens<S, R, 1, true, true, 256, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaFuncSetAttribute(k_step_ens<S, R, 1, false, false, 512, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaFuncSetAttribute(k_step_ens<S, R, 1, false, true, 512, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaFuncSetAttribute(k_step_ens<S, R, 1, true, false, 512, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaFuncSetAttribute(k_step_ens<S, R, 1, true, true, 512, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_ens<S, R, SC, true, true, 0, NP>, threads, smem) !=
        cudaSuccess)
        return 0;
    return nb;
}

template <typename S, typename R, int NP>
int ens_occupancy_t(int scheme, int threads, size_t smem)
{
    if (scheme == 0) return ens_occupancy_scheme<S, R, 0, NP>(threads, smem);
    if (scheme == 1) return ens_occupancy_scheme<S, R, 1, NP>(threads, smem);
    return ens_occupancy_scheme<S, R, 2, NP>(threads, smem);
}

}  // namespace flbm
