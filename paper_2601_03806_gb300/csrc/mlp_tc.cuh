// mlp_tc.cuh -- the learned-collision network (28-64-64-27, SiLU, BF16
// weights, FP32 accumulation) on the tcgen05 tensor cores, one tile of 128
// nodes per CTA at a time.
//
// A kernel that allocates tensor memory gets one CTA per SM, so a CTA runs
// four independent sub-tiles of 128 rows at once: 512 threads, thread t owns
// row t % 128 of sub-tile t / 128 (warp w reads tensor-memory lanes
// 32 (w % 4) .. + 31, its rows), and sub-tile q owns tensor-memory columns
// 128 q .. 128 q + 127 (all 512 columns of the SM).  Per sub-tile
//   A1[128 x 32]  bf16 features, then 1, 1, 1, 0            -> shared memory
//   D1 = A1 W1'^T (M 128, N 64, K 32: two MMAs)             -> tensor memory cols 0..63
//   h1 = silu(z1) = hz (1 + tanh hz), hz = D1, as bf16       -> A2 (shared)
//   D2 = [h1 | U] W2'^T  (N 64, K 64 + 16: five MMAs)        -> cols 64..127
//   h2 = silu(z2), hz = D2, as bf16                          -> A2 again
//   y  = [h2 | U] W3'^T  (N 32, K 64 + 16: five MMAs; rows 27..31 zero) -> cols 0..31
// The biases ride in the MMAs: each is split into three bf16 parts
// b = b_hi + b_mid + b_lo (exact to FP32) that multiply constant-one
// columns -- A1's padding columns 28..30 for layer 1, the shared block U
// (128 x 16, columns 0..2 one) for layers 2 and 3 -- and W1, b1, W2, b2 are
// stored halved (exact in bf16), so the accumulators hold z / 2 and SiLU
// costs one tanh and one FMA per activation.
// Each sub-tile is an independent group of 4 warps (128 threads) with its
// own named barrier (id 1 + group), its own mbarrier and its own MMA issuer,
// so the groups drift out of phase and one group's epilogue fills another's
// MMA latency -- what separate CTAs would do if the SM granted them.  Every
// wait is bounded, and its outcome is made uniform over the group.  The weight
// image (bf16, already in the operand layout of umma.cuh) and the FP32
// biases are copied into shared memory once per CTA.
#pragma once

#include <cuda_bf16.h>

#include "step_kernel.cuh"
#include "umma.cuh"

namespace flbm {

constexpr int kMlpIn = 28, kMlpHidden = 64, kMlpOut = 27;
constexpr uint32_t kSbo16 = 2 * 128;          // SBO of a K = 16 operand
constexpr uint32_t kSbo32 = 4 * 128;          // SBO of a K = 32 operand
constexpr uint32_t kSbo64 = 8 * 128;          // SBO of a K = 64 operand
// image: W1' [64 x 32] | W2' [64 x 64] | W3 [32 x 64] | B2' [64 x 16] |
// B3 [32 x 16] | U [128 x 16], all bf16 in the operand layout of umma.cuh
constexpr uint32_t kW1Off = 0, kW2Off = 4096, kW3Off = 12288, kB2Off = 16384, kB3Off = 18432, kOnesOff = 19456;
constexpr uint32_t kMlpImageBytes = kOnesOff + 128 * 16 * 2;   // 23,552 B
constexpr uint32_t kMlpSub = 4;                 // sub-tiles of 128 rows per CTA
constexpr uint32_t kMlpThreads = 128 * kMlpSub;  // CTA size
constexpr uint32_t kMlpTmemCols = 128 * kMlpSub; // the whole tensor memory of an SM

struct MlpSmem {
    __align__(128) unsigned char w[kMlpImageBytes];    // the network image
    __align__(128) unsigned char a1[kMlpSub][128 * 32 * 2];
    __align__(128) unsigned char a2[kMlpSub][128 * 64 * 2];
    uint64_t bar[kMlpSub];
    uint32_t tmem;
};
constexpr size_t kMlpSmemBytes = (sizeof(MlpSmem) + 1023) / 1024 * 1024;

// silu(z) = z sigmoid(z) = hz (1 + tanh(hz)) with hz = z / 2, from hz, with
// the hardware tanh (absolute error about 2^-11, below the bf16 rounding of
// the activations); two activations at a time, the FMA as one packed FP32
// pair (each lane rounded as the scalar FMA would be).
__device__ __forceinline__ void silu_half2(float &a, float &b)
{
    float ta, tb;
    asm("tanh.approx.f32 %0, %1;\n" : "=f"(ta) : "f"(a));
    asm("tanh.approx.f32 %0, %1;\n" : "=f"(tb) : "f"(b));
    const float2 h = make_float2(a, b);
    const float2 r = __ffma2_rn(h, make_float2(ta, tb), h);
    a = r.x;
    b = r.y;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// Write 16 consecutive columns k0..k0+15 of row r of a K-major operand.
__device__ __forceinline__ void store_row16(unsigned char *base, uint32_t sbo, uint32_t r, uint32_t k0,
                                            const float (&v)[16])
{
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        uint4 q;
        q.x = pack_bf16x2(v[8 * half + 0], v[8 * half + 1]);
        q.y = pack_bf16x2(v[8 * half + 2], v[8 * half + 3]);
        q.z = pack_bf16x2(v[8 * half + 4], v[8 * half + 5]);
        q.w = pack_bf16x2(v[8 * half + 6], v[8 * half + 7]);
        *reinterpret_cast<uint4 *>(base + core_offset(r, k0 + 8 * half, sbo)) = q;
    }
}

// CTA set-up: network image to shared memory, mbarriers, tensor memory.
__device__ __forceinline__ void mlp_setup(MlpSmem &sm, const unsigned char *__restrict__ img)
{
    const uint4 *src = reinterpret_cast<const uint4 *>(img);
    uint4 *dst = reinterpret_cast<uint4 *>(sm.w);
    for (uint32_t i = threadIdx.x; i < kMlpImageBytes / 16; i += blockDim.x) dst[i] = src[i];
    if (threadIdx.x == 0) {
        for (uint32_t q = 0; q < kMlpSub; ++q) mbar_init(&sm.bar[q], 1);
        mbar_init_fence();
    }
    if (threadIdx.x < 32) tmem_alloc(&sm.tmem, kMlpTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// CTA tear-down: every tensor-memory read done, then free the columns.
__device__ __forceinline__ void mlp_teardown(MlpSmem &sm)
{
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(sm.tmem, kMlpTmemCols);
}

// Barrier of the 128 threads of group q (named barrier 1 + q).
__device__ __forceinline__ void group_sync(uint32_t q)
{
    asm volatile("bar.sync %0, 128;\n" ::"r"(1u + q) : "memory");
}
// The same barrier, returning whether pred held on every thread of the group.
__device__ __forceinline__ bool group_all(uint32_t q, bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, o;\n setp.ne.u32 p, %1, 0;\n"
        " bar.red.and.pred o, %2, 128, p;\n selp.u32 %0, 1, 0, o;\n}\n"
        : "=r"(r)
        : "r"(uint32_t(pred)), "r"(1u + q)
        : "memory");
    return r != 0;
}

// Wait for the MMAs committed to the group's mbarrier; the outcome is made
// uniform over the group so that no thread leaves the loop alone.
__device__ __forceinline__ bool mlp_wait(MlpSmem &sm, uint32_t q, uint32_t &phase)
{
    const bool ok = mbar_wait(&sm.bar[q], phase);
    phase ^= 1u;
    const bool all = group_all(q, ok);
    tc_fence_after();
    return all;
}

__device__ __forceinline__ void mlp_sync_for_mma(uint32_t q)
{
    fence_proxy_async_smem();   // generic-proxy operand writes before the MMAs read them
    tc_fence_before();          // earlier tensor-memory reads before the MMAs overwrite
    group_sync(q);
}

// One round: x = this thread's 28 features (row t % 128 of sub-tile t / 128),
// y = its 27 outputs.  work() runs while the first layer's MMAs are in flight.  Returns
// false (on every thread) if a wait ran out; the MMAs are then drained with
// one more bounded wait before returning.  starve (failure injection, tests
// only): the issuer issues none of the first layer's MMAs and commits
// nothing, so the group's wait runs out with no tensor-core work in flight
// when the tensor memory is later released.
template <typename Work>
__device__ __forceinline__ bool mlp_tile(MlpSmem &sm, uint32_t &phase, const float (&x)[kMlpIn],
                                         float (&y)[kMlpOut], Work &&work, bool starve = false)
{
    const uint32_t t = threadIdx.x & 127u, q = threadIdx.x >> 7;
    const uint32_t tmem = sm.tmem + 128u * q;                 // this sub-tile's columns
    const uint32_t lane_base = ((threadIdx.x >> 5) & 3u) << 21;   // (32 (warp % 4)) << 16
    const uint32_t w = smem_u32(sm.w);
    unsigned char *a1p = sm.a1[q], *a2p = sm.a2[q];
    constexpr uint32_t idesc64 = umma_idesc_bf16(128, 64), idesc32 = umma_idesc_bf16(128, 32);
    {
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = x[i];
        store_row16(a1p, kSbo32, t, 0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = (16 + i < kMlpIn) ? x[16 + i] : (16 + i < kMlpIn + 3 ? 1.0f : 0.0f);
        store_row16(a1p, kSbo32, t, 16, v);
    }
    mlp_sync_for_mma(q);
    if (t == 0 && !starve) {
        tc_fence_after();
        const uint32_t a1 = smem_u32(a1p);
#pragma unroll
        for (uint32_t s = 0; s < 2; ++s)
            umma_bf16(tmem, umma_smem_desc(a1 + 256 * s, 128, kSbo32),
                      umma_smem_desc(w + kW1Off + 256 * s, 128, kSbo32), idesc64, s > 0);
        umma_commit(&sm.bar[q]);
    }
    work();
    bool ok = mlp_wait(sm, q, phase);
    if (ok) {
#pragma unroll
        for (uint32_t ch = 0; ch < 4; ++ch) {
            float z[16];
            tmem_ld16(tmem + lane_base + 16 * ch, z);
#pragma unroll
            for (int i = 0; i < 16; i += 2) silu_half2(z[i], z[i + 1]);
            store_row16(a2p, kSbo64, t, 16 * ch, z);
        }
        mlp_sync_for_mma(q);
        if (t == 0) {
            tc_fence_after();
            const uint32_t a2 = smem_u32(a2p);
#pragma unroll
            for (uint32_t s = 0; s < 4; ++s)
                umma_bf16(tmem + 64, umma_smem_desc(a2 + 256 * s, 128, kSbo64),
                          umma_smem_desc(w + kW2Off + 256 * s, 128, kSbo64), idesc64, s > 0);
            umma_bf16(tmem + 64, umma_smem_desc(w + kOnesOff, 128, kSbo16),
                      umma_smem_desc(w + kB2Off, 128, kSbo16), idesc64, true);
            umma_commit(&sm.bar[q]);
        }
        ok = mlp_wait(sm, q, phase);
    }
    if (ok) {
#pragma unroll
        for (uint32_t ch = 0; ch < 4; ++ch) {
            float z[16];
            tmem_ld16(tmem + lane_base + 64 + 16 * ch, z);
#pragma unroll
            for (int i = 0; i < 16; i += 2) silu_half2(z[i], z[i + 1]);
            store_row16(a2p, kSbo64, t, 16 * ch, z);
        }
        mlp_sync_for_mma(q);
        if (t == 0) {
            tc_fence_after();
            const uint32_t a2 = smem_u32(a2p);
#pragma unroll
            for (uint32_t s = 0; s < 4; ++s)
                umma_bf16(tmem, umma_smem_desc(a2 + 256 * s, 128, kSbo64),
                          umma_smem_desc(w + kW3Off + 256 * s, 128, kSbo64), idesc32, s > 0);
            umma_bf16(tmem, umma_smem_desc(w + kOnesOff, 128, kSbo16),
                      umma_smem_desc(w + kB3Off, 128, kSbo16), idesc32, true);
            umma_commit(&sm.bar[q]);
        }
        ok = mlp_wait(sm, q, phase);
    }
    if (ok) {
#pragma unroll
        for (uint32_t ch = 0; ch < 2; ++ch) {
            float z[16];
            tmem_ld16(tmem + lane_base + 16 * ch, z);
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (16 * ch + i < kMlpOut) y[16 * ch + i] = z[i];
        }
        return true;
    }
    // a wait ran out: give the MMAs in flight one more bounded wait (none
    // are when starving)
    if (!starve) mbar_wait(&sm.bar[q], phase);
    return false;
}

}  // namespace flbm
