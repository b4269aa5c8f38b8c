// step_kernel.cuh -- fused D3Q27 fluctuating-LB stream-and-collide kernels.
//
// Storage: deviations g_i = f_i - w_i rho0, SoA planes g[i*N + n] (node
// n = x + nx (y + ny z)), updated in place with the AA pattern:
//   even form (natural): node x reads f_i from slot i at x and writes the
//     post-collision f*_i to slot opp(i) at x;
//   odd form: node x reads f_i from slot opp(i) at x - c_i and writes f*_i to
//     slot i at x + c_i.
// Both forms realise f_i(x + c_i, t+1) = f*_i(x, t) (LHS of Eq. flbe2) on a
// periodic box, and the set of locations a node reads is the set it writes.
//
// Per node (Eq. flbe2 in mode space), collide_core (collide_modes +
// noise_synthesise), on one node (lane type float or double) or on two nodes
// at once (float2, one node per lane, as packed FP32 instructions); every
// operation is one explicitly rounded IEEE operation, so every kernel gives
// the same bits:
//   a2  forward Hermite projection (three 1-D passes): drho, j_a, m_ab
//   a3  a2neq_ab = m_ab - rho u_a u_b (equal to Eq. moments2 because the
//       second-order f^eq has second Hermite moment rho u_a u_b)
//   a4  M_ab = rho u_a u_b + (1 - omega) a2neq_ab          (k = 4..9)
//   a5  ghost modes k = 10..26: no deterministic content (GMF); (1-omega) m_k
//       for BGK-FLBM (Eq. flbe); rho u^(deg) for Reg-FLBM
//   a6  M_k += phi_k r_k  (Eqs. fluct_phi / fluct_phig), r_k from
//       Philox4x32-10 keyed on (seed; node, step, block | stream << 8) +
//       Box-Muller
//   a7  f*_i = w_i sum_k e_ki M_k / b_k (three 1-D passes), minus w_i rho0
//   a9  optional per-thread partial sums of the reductions, folded per warp
//       every 8 rows into exact (hi, lo) slots and summed per CTA in FP64
//
// Two kernels move the data (a1 load, a8 store):
//   k_step_rows  (rows whose x-extent is a multiple of 32 and fits shared
//                memory): a persistent, warp-specialised CTA owns whole
//                x-rows.  Its producer warp moves, per row, the 27 aligned
//                plane segments the row reads -- from the 9 neighbouring rows
//                in the odd form -- into shared memory with TMA bulk copies
//                (cp.async.bulk, one lane per segment) completing on a "full"
//                mbarrier, stages ahead of the compute warps.  The compute
//                warps apply the periodic +-1 x-shift inside shared memory,
//                collide, overwrite the same segments (a node's read set is
//                its write set) and release the stage on an "empty"
//                mbarrier; the producer then bulk-stores the segments back.
//                All HBM traffic is aligned bulk transfers and no CTA-wide
//                barrier sits in the loop.  FP32 / FP16 rows of 256 nodes
//                and more: a compute thread collides two adjacent nodes at
//                once (NP = 2); otherwise one (NP = 1).
//   k_step       (any box): one thread per node, a CTA per 128-node chunk of
//                a row, direct coalesced loads and stores.
#pragma once

#include <cuda_fp16.h>

#include <type_traits>

#include "internal.h"
#include "lattice.cuh"

namespace flbm {

// ---------------------------------------------------------------------------
// element access

template <typename S, typename R> struct Conv;
template <> struct Conv<double, double> {
    static __device__ __forceinline__ double ld(const double *p) { return *p; }
    static __device__ __forceinline__ void st(double *p, double v) { *p = v; }
};
template <> struct Conv<float, float> {
    // L2-only loads and evict-first stores: the populations are streamed once
    // per step (cache-policy choice measured on the 512^3 workload).
    static __device__ __forceinline__ float ld(const float *p) { return __ldcg(p); }
    static __device__ __forceinline__ void st(float *p, float v) { __stcs(p, v); }
};
template <> struct Conv<__half, float> {
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(__ldcg(p)); }
    static __device__ __forceinline__ void st(__half *p, float v) { __stcs(p, __float2half_rn(v)); }
};
// Shared-memory staging element conversions of the row pipeline.
__device__ __forceinline__ float stage_ld(const float &v) { return v; }
__device__ __forceinline__ double stage_ld(const double &v) { return v; }
__device__ __forceinline__ float stage_ld(const __half &v) { return __half2float(v); }
template <typename S> __device__ __forceinline__ S stage_st(float v);
template <> __device__ __forceinline__ float stage_st<float>(float v) { return v; }
template <> __device__ __forceinline__ __half stage_st<__half>(float v) { return __float2half_rn(v); }
template <typename S> __device__ __forceinline__ S stage_st(double v);
template <> __device__ __forceinline__ double stage_st<double>(double v) { return v; }

// ---------------------------------------------------------------------------
// Lane arithmetic.  A thread collides one node in V = float or double, or
// two nodes in V = float2, one per lane, as Blackwell's packed FP32
// instructions (FADD2 / FMUL2 / FFMA2: one instruction for both nodes).
// Every operation below is one IEEE operation rounded once (no contraction
// left to the compiler), so a float2 lane computes bit for bit what the
// float code computes for that node.

__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double vadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double vsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double vmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as fma(b, -1, a): the product is exact, so one rounding of a - b
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Scalar of the lane type's precision, one copy per lane.
template <typename V> struct Lane { using T = V; };
template <> struct Lane<float2> { using T = float; };
template <typename V> __device__ __forceinline__ V vset(double c) { return V(c); }
template <> __device__ __forceinline__ float2 vset<float2>(double c) { return make_float2(float(c), float(c)); }
__device__ __forceinline__ float vbc(float c, float) { return c; }
__device__ __forceinline__ double vbc(double c, double) { return c; }
__device__ __forceinline__ float2 vbc(float c, float2) { return make_float2(c, c); }

// Reciprocal and square root of the density: IEEE in FP64, the hardware
// approximations (relative error ~1e-7) in FP32, per lane.
__device__ __forceinline__ double rcp_(double v) { return 1.0 / v; }
__device__ __forceinline__ float rcp_(float v) { return __fdividef(1.0f, v); }
__device__ __forceinline__ float2 rcp_(float2 v) { return make_float2(rcp_(v.x), rcp_(v.y)); }
__device__ __forceinline__ double sqrt_(double v) { return sqrt(v); }
__device__ __forceinline__ float sqrt_(float v) { return __fmul_rn(v, rsqrtf(v)); }
__device__ __forceinline__ float2 sqrt_(float2 v)
{
    return vmul(v, make_float2(rsqrtf(v.x), rsqrtf(v.y)));
}
// Whether any lane's density fails rho > 0 and rho finite.
__device__ __forceinline__ bool bad_density(float r) { return !(r > 0.0f) || !(r < INFINITY); }
__device__ __forceinline__ bool bad_density(double r) { return !(r > 0.0) || !(r < INFINITY); }
__device__ __forceinline__ bool bad_density(float2 r) { return bad_density(r.x) || bad_density(r.y); }

// ---------------------------------------------------------------------------
// 1-D transforms (see lattice.cuh for the scales)

// Hermite analysis of a 3-point line (values at c = -1, 0, +1):
// (sum v, sum v c, -3 sum v (c^2 - 1/3)); the factor -3 is undone through
// the mode coefficients (fwd_scale).  Four operations: s = m + p,
// d = p - m, h0 = s + o, h2 = o - 2 s (an FMA).
template <typename V>
__device__ __forceinline__ void analyse(V &m, V &o, V &p)
{
    const V s = vadd(m, p);
    const V d = vsub(p, m);
    const V h0 = vadd(s, o);
    const V h2 = vfma(s, vset<V>(-2.0), o);
    m = h0;
    o = d;
    p = h2;
}

// Synthesis of prescaled amplitudes (syn_scale, degree 0 carrying 4): the
// values at c = -1, 0, +1 of w1(c) (q0 + q1 c + q2 (c^2 - 1/3)) for the
// unscaled q.  t = p0 / 4 + p2 and p0 - 2 p2 are single FMAs whose exact
// products make them equal to p0/4 + p2 and 4 (p0/4) - 2 p2 rounded once.
template <typename V>
__device__ __forceinline__ void synthesise(V &p0, V &p1, V &p2)
{
    const V t = vfma(p0, vset<V>(0.25), p2);
    const V z = vfma(p2, vset<V>(-2.0), p0);
    p0 = vsub(t, p1);
    p2 = vadd(t, p1);
    p1 = z;
}

// The same two transforms on two lines of one node at once (lines a and
// b).  In FP32 they run as packed FP32 pairs: four instructions for two
// lines instead of eight, each lane rounded exactly as the scalar code.
template <typename V>
__device__ __forceinline__ void analyse_pair(V &ma, V &mb, V &oa, V &ob, V &pa, V &pb)
{
    analyse(ma, oa, pa);
    analyse(mb, ob, pb);
}
template <>
__device__ __forceinline__ void analyse_pair<float>(float &ma, float &mb, float &oa, float &ob, float &pa,
                                                    float &pb)
{
    float2 m = make_float2(ma, mb), o = make_float2(oa, ob), p = make_float2(pa, pb);
    analyse(m, o, p);
    ma = m.x;
    mb = m.y;
    oa = o.x;
    ob = o.y;
    pa = p.x;
    pb = p.y;
}
template <typename V>
__device__ __forceinline__ void synthesise_pair(V &p0a, V &p0b, V &p1a, V &p1b, V &p2a, V &p2b)
{
    synthesise(p0a, p1a, p2a);
    synthesise(p0b, p1b, p2b);
}
template <>
__device__ __forceinline__ void synthesise_pair<float>(float &p0a, float &p0b, float &p1a, float &p1b,
                                                       float &p2a, float &p2b)
{
    float2 p0 = make_float2(p0a, p0b), p1 = make_float2(p1a, p1b), p2 = make_float2(p2a, p2b);
    synthesise(p0, p1, p2);
    p0a = p0.x;
    p0b = p0.y;
    p1a = p1.x;
    p1b = p1.y;
    p2a = p2.x;
    p2b = p2.y;
}

// ---------------------------------------------------------------------------
// reductions

template <typename R>
__device__ __forceinline__ R warp_sum(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Fused-reduction totals of a CTA, one slot per warp and sum (blockDim.x a
// multiple of 32, at most 32 warps).  Threads add their nodes' terms in R;
// every kFlushEvery rows (row pipeline) or chunks (direct kernel) each warp
// adds its threads' partial sums (a warp_sum in R) to its slots and restarts
// them, so that in FP32 no sum spans more than kFlushEvery rows of a
// thread's nodes.  A slot is an unevaluated pair hi + lo kept by Knuth's
// error-free TwoSum (no FP64 arithmetic in the loop: the FP64 pipe is slow),
// and block_store_totals adds the slots in fixed warp order in FP64.
constexpr int kFlushEvery = 8;

template <typename R> struct TotSlot { R hi, lo; };

// s + e = a + b exactly (round to nearest, no underflow).
__device__ __forceinline__ float two_sum(float a, float b, float &e)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}
__device__ __forceinline__ double two_sum(double a, double b, double &e)
{
    const double s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
    return s;
}

template <typename R>
__device__ __forceinline__ void totals_init(TotSlot<R> (*tot)[NSTAT])
{
    for (int i = threadIdx.x; i < 32 * NSTAT; i += blockDim.x) tot[i / NSTAT][i % NSTAT] = TotSlot<R>{R(0), R(0)};
}

// A thread's partial sum of both lanes.
__device__ __forceinline__ float lane_total(float v) { return v; }
__device__ __forceinline__ double lane_total(double v) { return v; }
__device__ __forceinline__ float lane_total(float2 v) { return __fadd_rn(v.x, v.y); }

// All 32 lanes of the warp take part; lane s < NSTAT updates slot s.
template <typename V, typename R>
__device__ __forceinline__ void warp_flush(V (&acc)[NSTAT], TotSlot<R> (*tot)[NSTAT])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    R mine = R(0);
#pragma unroll
    for (int s = 0; s < NSTAT; ++s) {
        const R v = warp_sum(lane_total(acc[s]));
        if (lane == s) mine = v;
        acc[s] = vset<V>(0.0);
    }
    if (lane < NSTAT) {
        TotSlot<R> t = tot[warp][lane];
        R e;
        t.hi = two_sum(t.hi, mine, e);
        t.lo += e;
        tot[warp][lane] = t;
    }
}

// Every thread of the CTA calls this once, after its last warp_flush.
template <typename R>
__device__ __forceinline__ void block_store_totals(TotSlot<R> (*tot)[NSTAT], double *out)
{
    __syncthreads();
    if (threadIdx.x < NSTAT) {
        const int nw = blockDim.x >> 5;
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += double(tot[w][threadIdx.x].hi) + double(tot[w][threadIdx.x].lo);
        out[threadIdx.x] = t;
    }
}

// Per-CTA FP64 partials of the per-thread sums (blockDim.x a multiple of 32,
// at most 32 warps).
template <typename R>
__device__ __forceinline__ void block_reduce_store(const R (&acc)[NSTAT], double *out)
{
    __shared__ double sh[32][NSTAT];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int s = 0; s < NSTAT; ++s) {
        const R v = warp_sum(acc[s]);
        if (lane == 0) sh[warp][s] = double(v);
    }
    __syncthreads();
    if (threadIdx.x < NSTAT) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += sh[w][threadIdx.x];
        out[threadIdx.x] = t;
    }
}

// ---------------------------------------------------------------------------
// a6, first half: the node's 23 standard normals r_k (k = 4..26), drawn from
// Philox4x32-10 keyed on (seed; node, step, block) + Box-Muller and scaled by
// the compile-time syn_scale_k sqrt(b_k / c_s^2): nz[k - 4].  They depend
// only on (node, step), so the kernels can draw them while the populations
// are still in flight.

constexpr int kNoise = kQ - 4;

// Philox block blk of node at the step: counter (node, step lo, blk | stream
// << 8, step hi).  One box: the launch-uniform words of rounds 0-1 come
// precomputed from the host (philox4x32_10_r2).  An ensemble replica has its
// own overload (ens_kernel.cuh).
template <typename R>
__device__ __forceinline__ u32x4 noise_block(const StepArgs<R> &a, uint32_t node, int blk)
{
    return philox4x32_10_r2(node, a.ph_zk, a.ph_u1[blk], a.ph_u2[blk], a.ph_u3[blk], a.rk);
}

// Box-Muller (1958) on the uniforms of words (w1, w2), returned as a
// radius rad = sqrt(-2 ln u1) >= 0 and (ca, sa) = -(cos, sin)(2 pi u2): the
// standard normals are -rad ca and -rad sa, and the sign is folded into the
// mode scale (noise_scale).  FP32: hardware log2 (absolute error <= 2^-22
// on [0.5, 1), <= 2 ulp below), so the radius has absolute error <= ln2
// 2^-22 / rad (~1.7e-7 / rad: below 1e-6 for u1 <= 0.986, 98.6 % of draws,
// at most 4.7e-4 at the smallest radius 3.5e-4, u1 = 1 - 2^-24); the angle
// is taken as 2 pi u2 - pi in (-pi, pi), where the hardware sin/cos hold
// their 2^-21.4 absolute error bound.
__device__ __forceinline__ void normal_pair(uint32_t w1, uint32_t w2, float &rad, float &ca, float &sa)
{
    const float u1 = uniform23f(w1);
    const float u2 = uniform23f(w2);
    const float t = __fmul_rn(-1.3862943611198906f, __log2f(u1));   // -2 ln u1
    rad = __fmul_rn(t, rsqrtf(t));
    __sincosf(__fmaf_rn(u2, 6.2831853071795865f, -3.1415926535897932f), &sa, &ca);
}
__device__ __forceinline__ void normal_pair(uint32_t w1, uint32_t w2, double &rad, double &ca, double &sa)
{
    const double u1 = uniform23d(w1);
    const double u2 = uniform23d(w2);
    rad = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    ca = -c;
    sa = -s;
}
// Two nodes, one per lane (words of node a in .x, of node b in .y).
__device__ __forceinline__ void normal_pair(uint2 w1, uint2 w2, float2 &rad, float2 &ca, float2 &sa)
{
    const float2 c1 = make_float2(-(1.0f - 0x1p-24f), -(1.0f - 0x1p-24f));
    const float2 u1 = __fadd2_rn(make_float2(__uint_as_float(0x3f800000u | (w1.x >> 9)),
                                             __uint_as_float(0x3f800000u | (w1.y >> 9))), c1);
    const float2 u2 = __fadd2_rn(make_float2(__uint_as_float(0x3f800000u | (w2.x >> 9)),
                                             __uint_as_float(0x3f800000u | (w2.y >> 9))), c1);
    const float2 t = __fmul2_rn(make_float2(-1.3862943611198906f, -1.3862943611198906f),
                                make_float2(__log2f(u1.x), __log2f(u1.y)));
    rad = __fmul2_rn(t, make_float2(rsqrtf(t.x), rsqrtf(t.y)));
    const float2 ang = __ffma2_rn(u2, make_float2(6.2831853071795865f, 6.2831853071795865f),
                                  make_float2(-3.1415926535897932f, -3.1415926535897932f));
    __sincosf(ang.x, &sa.x, &ca.x);
    __sincosf(ang.y, &sa.y, &ca.y);
}

// The four normals of Philox block blk as (rad0, c0, s0, rad1, c1, s1):
// r_{4+4 blk + m} = -(rad0 c0, rad0 s0, rad1 c1, rad1 s1)[m].  V = float2:
// nodes node and node + 1.
template <typename V, typename A>
__device__ __forceinline__ void block_normals(const A &a, uint32_t node, int blk, V &rad0, V &c0, V &s0, V &rad1,
                                              V &c1, V &s1)
{
    if constexpr (std::is_same<V, float2>::value) {
        const u32x4 oa = noise_block(a, node, blk), ob = noise_block(a, node + 1, blk);
        normal_pair(make_uint2(oa.x, ob.x), make_uint2(oa.y, ob.y), rad0, c0, s0);
        normal_pair(make_uint2(oa.z, ob.z), make_uint2(oa.w, ob.w), rad1, c1, s1);
    } else {
        const u32x4 o = noise_block(a, node, blk);
        normal_pair(o.x, o.y, rad0, c0, s0);
        normal_pair(o.z, o.w, rad1, c1, s1);
    }
}

// Scale of mode mk's normal in the reconstruction's units: syn_scale
// sqrt(b_k / c_s^2), negated (normal_pair returns -r / rad).
__host__ __device__ constexpr double noise_scale(int mk)
{
    return -syn_scale(mode_deg(mk) % 3, (mode_deg(mk) / 3) % 3, mode_deg(mk) / 9) *
           sqrt_b_over_cs2(mode_deg(mk) % 3, (mode_deg(mk) / 3) % 3, mode_deg(mk) / 9);
}

// A is the step's scalar set: StepArgs<R> for one box, or a per-replica view
// with the same member names (rk, step, ctr2, rho0, ...) for an ensemble.
template <typename V, typename A>
__device__ __forceinline__ void draw_noise(const A &a, uint32_t node, V (&nz)[kNoise])
{
#pragma unroll
    for (int blk = 0; blk < 6; ++blk) {
        V rad0, c0, s0, rad1, c1, s1;
        block_normals(a, node, blk, rad0, c0, s0, rad1, c1, s1);
        const V trig[4] = {c0, s0, c1, s1};
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int mk = 4 + 4 * blk + m;
            if (mk < kQ) nz[mk - 4] = vmul(vmul(m < 2 ? rad0 : rad1, vset<V>(noise_scale(mk))), trig[m]);
        }
    }
}

// ---------------------------------------------------------------------------
// Maxwell-Boltzmann coefficient rho u_x^i u_y^j u_z^k of mode (i, j, k),
// order >= 1, as j_first * (the remaining u factors).
template <typename V>
__device__ __forceinline__ V aeq_coef(int i, int j, int k, const V (&jj)[3], const V (&uu)[3])
{
    const int first = i ? 0 : (j ? 1 : 2);
    V aeq = jj[first];
    const int rest[3] = {i - (first == 0), j - (first == 1), k - (first == 2)};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax)
#pragma unroll
        for (int e = 0; e < rest[ax]; ++e) aeq = vmul(aeq, uu[ax]);
    return aeq;
}

// A product rounded on its own (never fused into a following add), so that a
// relaxed amplitude has one value whether it stays in registers or is stored
// and reloaded before its noise is added.
__device__ __forceinline__ float mul_rn(float x, float y) { return __fmul_rn(x, y); }
__device__ __forceinline__ double mul_rn(double x, double y) { return __dmul_rn(x, y); }

// a2-a5: forward projection of the incoming deviations v (destroyed), the
// instability check, the fused reductions, and the deterministic
// post-collision amplitudes qm in the reconstruction's units, Q = syn_scale
// * M (noise not yet added); rho is the node's density, dj = (rho - rho0,
// j_x, j_y, j_z) as projected.  V = float2 collides two nodes, one per lane.
// PAIRS (V = float): the x and y passes take the lines k = 0 and k = 2 as
// packed pairs (the same bits either way; the faster choice depends on the
// kernel's register budget).
template <typename V, int SCHEME, bool STATS, bool PAIRS = true, typename A>
__device__ __forceinline__ void collide_modes(V (&v)[3][3][3], const A &a, V (&acc)[NSTAT], V (&qm)[3][3][3],
                                              V &rho, V (&dj)[4])
{
    using T = typename Lane<V>::T;
    // a2: forward Hermite projection, three 1-D passes
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (PAIRS) analyse_pair(v[0][j][0], v[0][j][2], v[1][j][0], v[1][j][2], v[2][j][0], v[2][j][2]);
        else {
            analyse(v[0][j][0], v[1][j][0], v[2][j][0]);
            analyse(v[0][j][2], v[1][j][2], v[2][j][2]);
        }
        analyse(v[0][j][1], v[1][j][1], v[2][j][1]);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (PAIRS) analyse_pair(v[i][0][0], v[i][0][2], v[i][1][0], v[i][1][2], v[i][2][0], v[i][2][2]);
        else {
            analyse(v[i][0][0], v[i][1][0], v[i][2][0]);
            analyse(v[i][0][2], v[i][1][2], v[i][2][2]);
        }
        analyse(v[i][0][1], v[i][1][1], v[i][2][1]);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) analyse(v[i][j][0], v[i][j][1], v[i][j][2]);

    const V drho = v[0][0][0];
    rho = vadd(vbc(a.rho0, drho), drho);
    const V jx = v[1][0][0], jy = v[0][1][0], jz = v[0][0][1];
    const V irho = rcp_(rho);
    const V ux = vmul(jx, irho), uy = vmul(jy, irho), uz = vmul(jz, irho);

    if (bad_density(rho)) {
        atomicOr(a.flag, 1u);
        atomicMin(a.bad_step, (unsigned long long)a.step);
    }

    if (STATS) {
        // the degree-2 projections carry fwd_scale -3
        const V m2 = vadd(vadd(jx, jy), jz);
        const V m3 = vfma(vset<V>(-1.0 / 3.0), vadd(vadd(v[2][0][0], v[0][2][0]), v[0][0][2]), drho);
        const V m4 = vadd(vadd(v[1][1][0], v[1][0][1]), v[0][1][1]);
        acc[S_DRHO] = vadd(acc[S_DRHO], drho);
        acc[S_JX] = vadd(acc[S_JX], jx);
        acc[S_JY] = vadd(acc[S_JY], jy);
        acc[S_JZ] = vadd(acc[S_JZ], jz);
        acc[S_UX2] = vfma(ux, ux, acc[S_UX2]);
        acc[S_UY2] = vfma(uy, uy, acc[S_UY2]);
        acc[S_UZ2] = vfma(uz, uz, acc[S_UZ2]);
        acc[S_M3] = vadd(acc[S_M3], m3);
        acc[S_M4] = vadd(acc[S_M4], m4);
        acc[S_M1SQ] = vfma(drho, drho, acc[S_M1SQ]);
        acc[S_M2SQ] = vfma(m2, m2, acc[S_M2SQ]);
        acc[S_M3SQ] = vfma(m3, m3, acc[S_M3SQ]);
        acc[S_M4SQ] = vfma(m4, m4, acc[S_M4SQ]);
    }

    // a3-a5: post-collision amplitudes in the reconstruction's units,
    // Q = syn_scale * M.  The pre-collision moments v carry fwd_scale.
    const V jj[3] = {jx, jy, jz};
    const V uu[3] = {ux, uy, uz};
    const V lam = vbc(a.lambda, drho), om = vbc(a.omega, drho);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int ord = mode_order(i, j, k);
                const V syn = vset<V>(syn_scale(i, j, k));
                const V unfwd = vset<V>(1.0 / fwd_scale(i, j, k));
                V q;
                if (ord == 0) {
                    q = vmul(drho, syn);                        // deviation of M_0 = rho
                } else if (ord == 1) {
                    q = vmul(v[i][j][k], syn);                  // momentum, conserved
                } else if (ord == 2 || SCHEME == 2) {
                    const V aeq = aeq_coef(i, j, k, jj, uu);
                    if (ord == 2)   // a_eq + (1 - omega)(m - a_eq) = omega a_eq + lambda m
                        q = vmul(syn, vfma(lam, vmul(v[i][j][k], unfwd), vmul(om, aeq)));
                    else            // Reg ghosts: a_eq (unit relaxation)
                        q = vmul(syn, aeq);
                } else if (SCHEME == 0) {                       // BGK ghosts
                    q = vmul(vset<V>(T(syn_scale(i, j, k)) * T(1.0 / fwd_scale(i, j, k))), vmul(lam, v[i][j][k]));
                } else {
                    q = vset<V>(0.0);                           // GMF: filtered
                }
                qm[i][j][k] = q;
            }
    dj[0] = drho;
    dj[1] = jx;
    dj[2] = jy;
    dj[3] = jz;
}

// a6-a7: the node's noise added to the amplitudes qm (destroyed), then the
// reconstruction into post-collision deviations v (PAIRS as collide_modes).
template <typename V, bool PREDRAWN, bool PAIRS = true, typename A>
__device__ __forceinline__ void noise_synthesise(V (&qm)[3][3][3], V rho, const A &a, const V (&nz)[kNoise],
                                                 uint32_t node, V (&v)[3][3][3])
{
    // a6: M_k += phi_k r_k for k = 4..26 with phi_k = sqrt(rho) amp
    // sqrt(b_k / c_s^2) (amp_h for k = 4..9, amp_g for the ghosts)
    {
        const V sr = a.noise_rho0 ? vbc(a.sqrt_rho0, rho) : sqrt_(rho);
        const V sh = vmul(sr, vbc(a.amp_h, rho)), sg = vmul(sr, vbc(a.amp_g, rho));
        if (PREDRAWN) {
#pragma unroll
            for (int mk = 4; mk < kQ; ++mk) {
                const int d = mode_deg(mk);
                V &q = qm[d % 3][(d / 3) % 3][d / 9];
                q = vfma(mk <= 9 ? sh : sg, nz[mk - 4], q);
            }
        } else {
            // pairs never mix hydrodynamic and ghost modes
#pragma unroll
            for (int blk = 0; blk < 6; ++blk) {
                V rad0, c0, s0, rad1, c1, s1;
                block_normals(a, node, blk, rad0, c0, s0, rad1, c1, s1);
                const V trig[4] = {c0, s0, c1, s1};
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const int mk = 4 + 4 * blk + m;
                    if (mk < kQ) {
                        const int d = mode_deg(mk);
                        // same rounding order as draw_noise + the PREDRAWN branch
                        const V t = vmul(vmul(m < 2 ? rad0 : rad1, vset<V>(noise_scale(mk))), trig[m]);
                        V &q = qm[d % 3][(d / 3) % 3][d / 9];
                        q = vfma(mk <= 9 ? sh : sg, t, q);
                    }
                }
            }
        }
    }

    // a7: reconstruction f*_i - w_i rho0 = w_i sum_k e_ki M_k / b_k (M_0 -> drho)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) synthesise(qm[i][j][0], qm[i][j][1], qm[i][j][2]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (PAIRS) synthesise_pair(qm[i][0][0], qm[i][0][2], qm[i][1][0], qm[i][1][2], qm[i][2][0], qm[i][2][2]);
        else {
            synthesise(qm[i][0][0], qm[i][1][0], qm[i][2][0]);
            synthesise(qm[i][0][2], qm[i][1][2], qm[i][2][2]);
        }
        synthesise(qm[i][0][1], qm[i][1][1], qm[i][2][1]);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (PAIRS) synthesise_pair(qm[0][j][0], qm[0][j][2], qm[1][j][0], qm[1][j][2], qm[2][j][0], qm[2][j][2]);
        else {
            synthesise(qm[0][j][0], qm[1][j][0], qm[2][j][0]);
            synthesise(qm[0][j][2], qm[1][j][2], qm[2][j][2]);
        }
        synthesise(qm[0][j][1], qm[1][j][1], qm[2][j][1]);
    }

#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) v[i][j][k] = qm[i][j][k];
}

// a2-a7, a9: collision of one node (V = float2: of nodes node and node + 1,
// one per lane).  v[cx+1][cy+1][cz+1] holds the incoming deviations on entry
// and the post-collision deviations on exit.  PREDRAWN: nz holds the node's
// scaled normals (draw_noise, drawn before the populations arrived);
// otherwise the normals of `node` are drawn here pair by pair and folded in
// at once (fewer live registers).
template <typename V, int SCHEME, bool STATS, bool PREDRAWN, typename A>
__device__ __forceinline__ void collide_core(V (&v)[3][3][3], const A &a,
                                             const V (&nz)[kNoise], uint32_t node, V (&acc)[NSTAT])
{
    V qm[3][3][3];
    V rho, dj[4];
    collide_modes<V, SCHEME, STATS, !std::is_same<V, float2>::value>(v, a, acc, qm, rho, dj);
    noise_synthesise<V, PREDRAWN, !std::is_same<V, float2>::value>(qm, rho, a, nz, node, v);
}

// ---------------------------------------------------------------------------
// k_step: one thread per node, direct loads/stores (general boxes)

// Periodic neighbour offsets of node (x,y,z): xs[d], ry[d], rz[d] for the
// displacements d-1 = -1, 0, +1 along each axis (node index = xs + ry + rz).
template <typename I>
struct Nbr {
    I xs[3], ry[3], rz[3];
    __device__ __forceinline__ Nbr(uint32_t x, uint32_t y, uint32_t z, uint32_t nx, uint32_t ny,
                                   uint32_t nz)
    {
        const I plane = I(nx) * I(ny);
        xs[0] = I(x ? x - 1 : nx - 1);
        xs[1] = I(x);
        xs[2] = I((x + 1 < nx) ? x + 1 : 0);
        ry[0] = I(y ? y - 1 : ny - 1) * I(nx);
        ry[1] = I(y) * I(nx);
        ry[2] = I((y + 1 < ny) ? y + 1 : 0) * I(nx);
        rz[0] = I(z ? z - 1 : nz - 1) * plane;
        rz[1] = I(z) * plane;
        rz[2] = I((z + 1 < nz) ? z + 1 : 0) * plane;
    }
    __device__ __forceinline__ I node() const { return xs[1] + ry[1] + rz[1]; }
};

template <typename S, typename R, typename I, int SCHEME, bool ODD, bool STATS>
__global__ void __launch_bounds__(kBlock, FLBM_MIN_BLOCKS) k_step(S *__restrict__ g, const StepArgs<R> a)
{
    __shared__ TotSlot<R> tot[32][NSTAT];
    R acc[NSTAT];
#pragma unroll
    for (int s = 0; s < NSTAT; ++s) acc[s] = R(0);
    if (STATS) {
        totals_init(tot);
        __syncthreads();
    }
    const I N = I(a.ns);   // slab stride
    uint32_t it = 0;
    for (uint64_t ch = blockIdx.x; ch < a.nchunks; ch += gridDim.x, ++it) {
        // CTA-uniform: every thread walks the same chunks
        if (STATS && it % kFlushEvery == kFlushEvery - 1) warp_flush(acc, tot);
        const uint32_t xc = uint32_t(ch % a.cpr);
        const uint64_t r = ch / a.cpr;
        const uint32_t y = uint32_t(r % a.ny);
        const uint32_t z = uint32_t(r / a.ny);
        const uint32_t x = xc * kBlock + threadIdx.x;
        if (x >= a.nx) continue;
        const Nbr<I> nb(x, y, z, a.nx, a.ny, a.nz);
        const I n = nb.node();
        // a1: load
        R v[3][3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    I idx;
                    if (!ODD) idx = I(slot_of(i - 1, j - 1, k - 1)) * N + n;
                    else idx = I(slot_of(1 - i, 1 - j, 1 - k)) * N + (nb.xs[2 - i] + nb.ry[2 - j] + nb.rz[2 - k]);
                    v[i][j][k] = Conv<S, R>::ld(g + idx);
                }
        R nz[kNoise];   // unused: the direct kernel draws the normals inside
        collide_core<R, SCHEME, STATS, false>(v, a, nz, uint32_t(n), acc);
        // a8: AA store
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    I idx;
                    if (!ODD) idx = I(slot_of(1 - i, 1 - j, 1 - k)) * N + n;
                    else idx = I(slot_of(i - 1, j - 1, k - 1)) * N + (nb.xs[i] + nb.ry[j] + nb.rz[k]);
                    Conv<S, R>::st(g + idx, v[i][j][k]);
                }
    }
    if (STATS) {
        warp_flush(acc, tot);
        block_store_totals(tot, a.partials + size_t(blockIdx.x) * NSTAT);
    }
}

// ---------------------------------------------------------------------------
// k_step_rows: TMA bulk-copy row pipeline

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// Bounded wait for the phase with the given parity: a poll that finds the
// phase open sleeps before the next one, 64 ns doubling to 512 ns (a warp
// that waits burns few issue slots of its sub-partition), and the wait gives
// up after 2^21 polls (at least half a second) and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t addr = smem_u32(bar);
    uint32_t ns = 64;
    for (uint32_t it = 0; it < (1u << 21); ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n"
            " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        __nanosleep(ns);
        ns = ns < 512 ? 2 * ns : 512;
    }
    return false;
}
// global -> shared bulk copy completing on an mbarrier (16-byte aligned
// addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst),
                 "r"(smem_u32(src)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all()
{
    asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// max compute threads of a row CTA (build option; 256 = 8 warps)
#ifndef FLBM_ROW_COMPUTE
#define FLBM_ROW_COMPUTE 256
#endif
constexpr int kRowCompute = FLBM_ROW_COMPUTE;
constexpr int kRowStages = 2;      // shared-memory stages (rows in flight), one node per thread
// Two nodes per thread (FP32 and FP16 storage): CTAs of 4 compute warps,
// several per SM (so that one CTA's row waits overlap the others' work),
// each with 4 shared-memory stages where they fit its share of the SM, else 2.
constexpr int kRowPairCompute = 128;
constexpr int kRowMaxStages = 4;
// CTAs per SM of the two-node kernel: 3 for FP16 storage (128 registers), 2
// for FP32 (whose 512-wide rows leave shared memory for two); the stages of
// one CTA share an equal part of two stages of a 512-wide FP32 row per CTA
// of a pair of CTAs.
template <typename S> constexpr int row_pair_ctas() { return sizeof(S) == 2 ? 3 : 2; }
constexpr size_t kRowPairSmSmem = size_t(4) * 27 * 512 * 4;

// Adjacent pair (x, x+1) of a staged segment (x even): one 64-bit or 32-bit
// shared access.
__device__ __forceinline__ float2 ld_pair(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ float2 ld_pair(const __half *p)
{
    return __half22float2(*reinterpret_cast<const __half2 *>(p));
}
__device__ __forceinline__ void st_pair(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
__device__ __forceinline__ void st_pair(__half *p, float2 v)
{
    *reinterpret_cast<__half2 *>(p) = __float22half2_rn(v);
}

// Shared staging of a row CTA per stage: 27 segments of nx elements.
template <typename S>
__host__ __device__ constexpr size_t row_stage_bytes(uint32_t nx) { return size_t(kQ) * nx * sizeof(S); }

// Global segment (plane slot, row) of segment index d = 9 (cx+1) + 3 (cy+1) +
// (cz+1) for the row (y, z): the even form reads slot c of the row itself,
// the odd form slot opp(c) of row (y - cy, z - cz).  The same segment later
// receives the post-collision values of direction -c.
// A copy lane moves the same segment d of every row: its slot's offset and
// its row shift are fixed for the launch.
struct SegLane {
    uint64_t slot_off;   // slot * ns
    int cy, cz;          // the odd form's row shift (0 in the even form)
};
template <typename R, bool ODD>
__device__ __forceinline__ SegLane seg_lane(const StepArgs<R> &a, int d)
{
    const int cx = d / 9 - 1, cy = (d / 3) % 3 - 1, cz = d % 3 - 1;
    SegLane L;
    L.slot_off = uint64_t(ODD ? slot_of(-cx, -cy, -cz) : slot_of(cx, cy, cz)) * a.ns;
    L.cy = ODD ? cy : 0;
    L.cz = ODD ? cz : 0;
    return L;
}
template <typename S, typename R>
__device__ __forceinline__ S *row_segment(S *g, const StepArgs<R> &a, const SegLane &L, uint32_t y, uint32_t z)
{
    uint32_t yy = y, zz = z;
    if (L.cy > 0) yy = y ? y - 1 : a.ny - 1;
    if (L.cy < 0) yy = (y + 1 < a.ny) ? y + 1 : 0;
    if (L.cz > 0) zz = z ? z - 1 : a.nz - 1;
    if (L.cz < 0) zz = (z + 1 < a.nz) ? z + 1 : 0;
    return g + (L.slot_off + (uint64_t(zz) * a.ny + yy) * a.nx);
}

// The same address from the row index (y = row % ny, z = row / ny) and the
// segment index d, decoded on every call: the copy warp of a PACED kernel.
template <typename S, typename R, bool ODD>
__device__ __forceinline__ S *row_segment_paced(S *g, const StepArgs<R> &a, int d, uint64_t row)
{
    return row_segment<S, R>(g, a, seg_lane<R, ODD>(a, d), uint32_t(row % a.ny), uint32_t(row / a.ny));
}

// (y, z) of a CTA's rows blockIdx.x + k gridDim.x, k = 0, 1, ..., stepped
// without a division per row; the rows end at z >= nz.
struct RowWalk {
    uint32_t y, z, dy, dz;
    __device__ __forceinline__ explicit RowWalk(uint32_t ny)
        : y(blockIdx.x % ny), z(blockIdx.x / ny), dy(gridDim.x % ny), dz(gridDim.x / ny) {}
    __device__ __forceinline__ void next(uint32_t ny)
    {
        y += dy;
        z += dz;
        if (y >= ny) {
            y -= ny;
            ++z;
        }
    }
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// Warp-specialised row pipeline.  Warps 0..nc/32-1 collide; the last warp
// is the producer: its lanes 0..26 each move one of the 27 segments of a row
// (bulk load into stage k % nst, completing on full[s]; after the compute
// warps release the stage through empty[s], bulk store back to HBM).  Every
// wait is bounded; a wait that runs out sets flag bit 1 and stops.
// NP = 1: a compute thread collides one node at a time, its normals drawn
// while the row lands; NP = 2 (FP32 arithmetic): it collides the adjacent
// nodes (x, x+1) at once as packed FP32 pairs, and moves each unshifted
// segment value pair with one shared access.
// NXC = 0: the row length is a.nx.  NXC > 0 (NP = 2 only): the row length
// is the constant NXC = a.nx and the CTA has kRowPairCompute compute
// threads, so every segment offset in the stage is an immediate of the
// shared-memory access instead of an address computed per access.
// PACED: the copy warp derives every copy's address from the row index
// (row_segment_paced) instead of walking the rows (RowWalk): the same
// addresses, issued more slowly.  Launched for the FP32 two-node rows
// staged twice (288-512 nodes; the HBM-bound 512^3 step), where walking made
// the step 1.5-2.1 % slower; everywhere else walking is faster (256^3 FP32
// +10.8 %, 128^3 FP32 +8.3 %, 512^3 FP16 +2.5 %).
template <typename S, typename R, int SCHEME, bool ODD, bool STATS, int NP, uint32_t NXC = 0, bool PACED = false>
__global__ void __launch_bounds__(NP == 2 ? kRowPairCompute + 32 : kRowCompute + 32,
                                  NP == 2 ? row_pair_ctas<S>() : (sizeof(S) <= 4 ? 2 : 1))
    k_step_rows(S *__restrict__ g, const StepArgs<R> a, uint32_t nst_log2)
{
    static_assert(NXC == 0 || (NP == 2 && NXC % 32 == 0), "a fixed row length needs two nodes per thread");
    using V = typename std::conditional<NP == 2, float2, R>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kRowMaxStages], empty[kRowMaxStages];
    // stages: a power of two, nst = 1 << nst_log2 <= kRowMaxStages
    const uint32_t nst = 1u << nst_log2, st_mask = nst - 1;
    __shared__ TotSlot<R> tot[32][NSTAT];
    S *const stage = reinterpret_cast<S *>(smem_raw);
    const uint32_t nx = NXC ? NXC : a.nx;
    const uint32_t nc = NXC ? uint32_t(kRowPairCompute) : blockDim.x - 32;   // compute threads
    const uint32_t stage_elems = uint32_t(kQ) * nx;
    const uint32_t seg_bytes = nx * uint32_t(sizeof(S));
    const uint32_t lane = threadIdx.x & 31;
    V acc[NSTAT];
#pragma unroll
    for (int s = 0; s < NSTAT; ++s) acc[s] = vset<V>(0.0);

    if (threadIdx.x == 0) {
        for (uint32_t s = 0; s < nst; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], nc / 32);
        }
        mbar_init_fence();
    }
    if (STATS) totals_init(tot);
    __syncthreads();

    if (threadIdx.x >= nc) {
        // ---------------- producer warp ----------------
        const int d = int(lane);
        const SegLane L = seg_lane<R, ODD>(a, d < kQ ? d : 0);
        RowWalk wl(a.ny), ws(a.ny);   // the rows loaded / stored next
        // PACED: (y, z) from the row index by a division, and the lane's
        // slot and shift decoded again, before every copy (row_segment_paced)
        uint64_t k = 0;
        bool ok = true;
        // store of row number kk (this CTA's kk-th row) out of its stage;
        // called for kk = 0, 1, 2, ... in turn (ws walks along)
        auto store_row = [&](uint64_t kk) {
            const int s = int(kk & st_mask);
            ok = mbar_wait(&empty[s], uint32_t((kk >> nst_log2) & 1));
            if (!ok) return;
            if (d < kQ) {
                S *gp = PACED ? row_segment_paced<S, R, ODD>(g, a, d, blockIdx.x + kk * gridDim.x)
                              : row_segment<S, R>(g, a, L, ws.y, ws.z);
                bulk_s2g(gp, stage + size_t(s) * stage_elems + d * nx, seg_bytes);
                bulk_commit();
                bulk_wait_read_all();
            }
            ws.next(a.ny);
            __syncwarp();
        };
        for (;; ++k, wl.next(a.ny)) {
            if (wl.z >= a.nz) break;
            const int s = int(k & st_mask);
            if (k >= nst) {
                store_row(k - nst);
                if (!ok) break;
            }
            if (lane == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&full[s], uint32_t(kQ) * seg_bytes + a.tx_pad);
            }
            __syncwarp();
            if (d < kQ) {
                S *gp = PACED ? row_segment_paced<S, R, ODD>(g, a, d, blockIdx.x + k * gridDim.x)
                              : row_segment<S, R>(g, a, L, wl.y, wl.z);
                bulk_g2s(stage + size_t(s) * stage_elems + d * nx, gp, seg_bytes, &full[s]);
            }
        }
        // drain the last stages
        for (uint64_t kk = (k > nst ? k - nst : 0); ok && kk < k; ++kk) store_row(kk);
        if (!ok && lane == 0) atomicOr(a.flag, 2u);
        if (d < kQ) bulk_wait_all();
    } else if constexpr (NP == 2) {
        // ---------------- compute warps, two nodes per thread ----------------
        RowWalk w(a.ny);
        for (uint64_t k = 0;; ++k, w.next(a.ny)) {
            if (w.z >= a.nz) break;
            const int s = int(k & st_mask);
            const uint32_t rowbase = nx * (w.y + a.ny * w.z);
            // the outcome is made warp-uniform: warp_flush needs every lane
            if (!__all_sync(0xffffffffu, mbar_wait(&full[s], uint32_t((k >> nst_log2) & 1)))) {
                if (lane == 0) atomicOr(a.flag, 2u);
                break;
            }
            S *st = stage + size_t(s) * stage_elems;
#pragma unroll 1
            for (uint32_t x = 2 * threadIdx.x; x < nx; x += 2 * nc) {
                // periodic x-1, x, x+1 of the nodes x (lane .x) and x+1 (lane .y);
                // x is even and nx a multiple of 32, so x+1 < nx
                const uint32_t xa[3] = {x ? x - 1 : nx - 1, x, x + 1};
                const uint32_t xb[3] = {x, x + 1, (x + 2 < nx) ? x + 2 : 0};
                // a1: incoming f_c from segment d(c) at x (even) / x - c_x (odd)
                V v[3][3][3];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j)
#pragma unroll
                        for (int kk = 0; kk < 3; ++kk) {
                            const S *seg = st + (9 * i + 3 * j + kk) * nx;
                            if (!ODD || i == 1) v[i][j][kk] = ld_pair(seg + x);
                            else v[i][j][kk] = make_float2(stage_ld(seg[xa[2 - i]]), stage_ld(seg[xb[2 - i]]));
                        }
                V nz[kNoise];   // unused: the normals are drawn inside, pair by pair
                collide_core<V, SCHEME, STATS, false>(v, a, nz, rowbase + x, acc);
                // a8: f*_c to segment d(-c) at x (even) / x + c_x (odd)
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j)
#pragma unroll
                        for (int kk = 0; kk < 3; ++kk) {
                            S *seg = st + (9 * (2 - i) + 3 * (2 - j) + (2 - kk)) * nx;
                            if (!ODD || i == 1) st_pair(seg + x, v[i][j][kk]);
                            else {
                                seg[xa[i]] = stage_st<S>(v[i][j][kk].x);
                                seg[xb[i]] = stage_st<S>(v[i][j][kk].y);
                            }
                        }
            }
            fence_proxy_async_smem();   // generic-proxy writes before the bulk store reads
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            if (STATS && k % kFlushEvery == kFlushEvery - 1) warp_flush(acc, tot);
        }
    } else {
        // ---------------- compute warps, one node per thread ----------------
        RowWalk w(a.ny);
        for (uint64_t k = 0;; ++k, w.next(a.ny)) {
            if (w.z >= a.nz) break;
            const int s = int(k & st_mask);
            const uint32_t rowbase = nx * (w.y + a.ny * w.z);
            // the first node's normals are drawn while the row's segments land
            R nz[kNoise];
            if (threadIdx.x < nx) draw_noise(a, rowbase + threadIdx.x, nz);
            // the outcome is made warp-uniform: warp_flush needs every lane
            if (!__all_sync(0xffffffffu, mbar_wait(&full[s], uint32_t((k >> nst_log2) & 1)))) {
                if (lane == 0) atomicOr(a.flag, 2u);
                break;
            }
            S *st = stage + size_t(s) * stage_elems;
            for (uint32_t x = threadIdx.x; x < nx; x += nc) {
                if (x != threadIdx.x) draw_noise(a, rowbase + x, nz);
                const uint32_t xsh[3] = {x ? x - 1 : nx - 1, x, (x + 1 < nx) ? x + 1 : 0};
                // a1: incoming f_c(x) from segment d(c) at x (even) / x - c_x (odd)
                R v[3][3][3];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j)
#pragma unroll
                        for (int kk = 0; kk < 3; ++kk) {
                            const uint32_t pos = ODD ? xsh[2 - i] : x;
                            v[i][j][kk] = R(stage_ld(st[(9 * i + 3 * j + kk) * nx + pos]));
                        }
                collide_core<R, SCHEME, STATS, true>(v, a, nz, rowbase + x, acc);
                // a8: f*_c(x) to segment d(-c) at x (even) / x + c_x (odd)
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j)
#pragma unroll
                        for (int kk = 0; kk < 3; ++kk) {
                            const uint32_t pos = ODD ? xsh[i] : x;
                            st[(9 * (2 - i) + 3 * (2 - j) + (2 - kk)) * nx + pos] = stage_st<S>(v[i][j][kk]);
                        }
            }
            fence_proxy_async_smem();   // generic-proxy writes before the bulk store reads
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            if (STATS && k % kFlushEvery == kFlushEvery - 1) warp_flush(acc, tot);
        }
    }
    if (STATS) {
        warp_flush(acc, tot);
        block_store_totals(tot, a.partials + size_t(blockIdx.x) * NSTAT);
    }
}

// ---------------------------------------------------------------------------
// launchers

// Dynamic shared memory of a row-pipeline CTA at most.
constexpr size_t kRowMaxSmem = 200 * 1024;

// Whether the row pipeline serves a box of row length nx, and its CTA shape:
// np nodes per compute thread, 1 << stages_log2 shared-memory stages.
struct RowPlan {
    bool use = false;
    int threads = 0;
    size_t smem = 0;
    int np = 1;
    uint32_t stages_log2 = 1;
};
template <typename S>
inline RowPlan row_plan(uint32_t nx)
{
    RowPlan p;
    if (nx % 32 != 0 || nx < 32) return p;
    const size_t sb = row_stage_bytes<S>(nx);
    uint32_t cmax = kRowCompute;
    // pairs from rows of 256 nodes (a full CTA of 4 compute warps); narrower
    // rows run faster with one node per thread (measured at 128^3)
    const size_t cta_smem = kRowPairSmSmem / size_t(row_pair_ctas<S>());
    if (!std::is_same<S, double>::value && row_pairs_enabled() && nx >= 2 * kRowPairCompute &&
        2 * sb <= cta_smem) {
        p.np = 2;
        p.stages_log2 = (size_t(kRowMaxStages) * sb <= cta_smem) ? 2 : 1;
        cmax = kRowPairCompute;
    }
    const size_t smem = (size_t(1) << p.stages_log2) * sb;
    if (smem > kRowMaxSmem) return p;
    const uint32_t units = nx / uint32_t(p.np);       // nodes or node pairs of a row
    const uint32_t npt = (units + cmax - 1) / cmax;
    uint32_t thr = (units + npt - 1) / npt;
    thr = (thr + 31) / 32 * 32;
    p.use = true;
    p.threads = int(thr) + 32;   // compute warps + the producer warp
    p.smem = smem;
    return p;
}

// One launch of the row kernel variant that plan rp picks.
template <typename S, typename R, int SC, bool OD, bool ST>
void launch_rows(S *g, const StepArgs<R> &a, const RowPlan &rp, int row_grid, cudaStream_t s)
{
    if constexpr (!std::is_same<S, double>::value) {
        if (rp.np == 2) {
            k_step_rows<S, R, SC, OD, ST, 2><<<row_grid, rp.threads, rp.smem, s>>>(g, a, rp.stages_log2);
            return;
        }
    }
    k_step_rows<S, R, SC, OD, ST, 1><<<row_grid, rp.threads, rp.smem, s>>>(g, a, rp.stages_log2);
}

template <typename S, typename R, typename I>
cudaError_t launch_step_t(S *g, const StepArgs<R> &a, int scheme, bool odd, bool stats, int grid,
                          int row_grid, cudaStream_t s)
{
    const RowPlan rp = row_plan<S>(a.nx);
    if (rp.use && row_grid > 0) {
#define FLBM_LAUNCH_ROWS(SC, OD, ST) launch_rows<S, R, SC, OD, ST>(g, a, rp, row_grid, s)
        if (scheme == 0) {
            if (odd) { if (stats) FLBM_LAUNCH_ROWS(0, true, true); else FLBM_LAUNCH_ROWS(0, true, false); }
            else     { if (stats) FLBM_LAUNCH_ROWS(0, false, true); else FLBM_LAUNCH_ROWS(0, false, false); }
        } else if (scheme == 1) {
            if (odd) { if (stats) FLBM_LAUNCH_ROWS(1, true, true); else FLBM_LAUNCH_ROWS(1, true, false); }
            else     { if (stats) FLBM_LAUNCH_ROWS(1, false, true); else FLBM_LAUNCH_ROWS(1, false, false); }
        } else {
            if (odd) { if (stats) FLBM_LAUNCH_ROWS(2, true, true); else FLBM_LAUNCH_ROWS(2, true, false); }
            else     { if (stats) FLBM_LAUNCH_ROWS(2, false, true); else FLBM_LAUNCH_ROWS(2, false, false); }
        }
#undef FLBM_LAUNCH_ROWS
        return cudaGetLastError();
    }
#define FLBM_LAUNCH(SC, OD, ST) k_step<S, R, I, SC, OD, ST><<<grid, kBlock, 0, s>>>(g, a)
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

// Opts the four row kernels of one variant into kRowMaxSmem bytes of dynamic
// shared memory and returns the resident CTAs per SM of the larger
// (reducing, odd-form) one for plan rp.
template <typename S, typename R, int SC, int NP, uint32_t NXC = 0, bool PACED = false>
int prepare_rows(const RowPlan &rp, bool stats)
{
    const int dmax = int(kRowMaxSmem);
    cudaFuncSetAttribute(k_step_rows<S, R, SC, false, false, NP, NXC, PACED>, cudaFuncAttributeMaxDynamicSharedMemorySize, dmax);
    cudaFuncSetAttribute(k_step_rows<S, R, SC, false, true, NP, NXC, PACED>, cudaFuncAttributeMaxDynamicSharedMemorySize, dmax);
    cudaFuncSetAttribute(k_step_rows<S, R, SC, true, false, NP, NXC, PACED>, cudaFuncAttributeMaxDynamicSharedMemorySize, dmax);
    cudaFuncSetAttribute(k_step_rows<S, R, SC, true, true, NP, NXC, PACED>, cudaFuncAttributeMaxDynamicSharedMemorySize, dmax);
    int nb = 0;
    const cudaError_t e = stats
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_rows<S, R, SC, true, true, NP, NXC, PACED>, rp.threads, rp.smem)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_rows<S, R, SC, true, false, NP, NXC, PACED>, rp.threads, rp.smem);
    return (e == cudaSuccess && nb > 0) ? nb : 0;
}

// Whether a box of row length nx runs the PACED two-node row kernel under
// plan rp: FP32 storage, two nodes per thread, two stages.
template <typename S>
inline bool rows_paced(const RowPlan &rp)
{
    return std::is_same<S, float>::value && rp.use && rp.np == 2 && rp.stages_log2 == 1;
}

// Whether a box of row length nx runs the fixed-length two-node row kernel
// of length NXC under plan rp (the plan it would take anyway: two nodes per
// thread and kRowPairCompute compute threads).
template <uint32_t NXC>
inline bool rows_fixed(const RowPlan &rp, uint32_t nx)
{
    return rp.use && rp.np == 2 && nx == NXC && rp.threads == kRowPairCompute + 32;
}

// One launch of a fixed-length (NXC) or PACED two-node row kernel; the
// caller has checked rows_fixed<NXC> / rows_paced<S> on row_plan<S>(a.nx).
template <typename S, typename R, uint32_t NXC, bool PACED = false>
cudaError_t launch_rows_fixed(S *g, const StepArgs<R> &a, int scheme, bool odd, bool stats, int row_grid,
                              cudaStream_t s)
{
    const RowPlan rp = row_plan<S>(a.nx);
#define FLBM_LAUNCH_FIXED(SC, OD, ST) \
    k_step_rows<S, R, SC, OD, ST, 2, NXC, PACED><<<row_grid, rp.threads, rp.smem, s>>>(g, a, rp.stages_log2)
    if (scheme == 0) {
        if (odd) { if (stats) FLBM_LAUNCH_FIXED(0, true, true); else FLBM_LAUNCH_FIXED(0, true, false); }
        else     { if (stats) FLBM_LAUNCH_FIXED(0, false, true); else FLBM_LAUNCH_FIXED(0, false, false); }
    } else if (scheme == 1) {
        if (odd) { if (stats) FLBM_LAUNCH_FIXED(1, true, true); else FLBM_LAUNCH_FIXED(1, true, false); }
        else     { if (stats) FLBM_LAUNCH_FIXED(1, false, true); else FLBM_LAUNCH_FIXED(1, false, false); }
    } else {
        if (odd) { if (stats) FLBM_LAUNCH_FIXED(2, true, true); else FLBM_LAUNCH_FIXED(2, true, false); }
        else     { if (stats) FLBM_LAUNCH_FIXED(2, false, true); else FLBM_LAUNCH_FIXED(2, false, false); }
    }
#undef FLBM_LAUNCH_FIXED
    return cudaGetLastError();
}

// prepare_rows for the fixed-length or PACED kernels of one scheme (rows of nx).
template <typename S, typename R, uint32_t NXC, bool PACED = false>
int prepare_rows_fixed(int scheme, bool stats, uint32_t nx = NXC)
{
    const RowPlan rp = row_plan<S>(nx);
    if (scheme == 0) return prepare_rows<S, R, 0, 2, NXC, PACED>(rp, stats);
    if (scheme == 1) return prepare_rows<S, R, 1, 2, NXC, PACED>(rp, stats);
    return prepare_rows<S, R, 2, 2, NXC, PACED>(rp, stats);
}

// Resident CTAs per SM of the larger (reducing, odd-form) variant of each
// kernel; also opts the row kernels into their shared memory on the current
// device.  rows = 0 when the row pipeline does not serve the box.
template <typename S, typename R, typename I, int SC>
void prepare_scheme(uint32_t nx, bool stats, int &direct, int &rows)
{
    direct = 1;
    rows = 0;
    int nb = 0;
    cudaError_t e = stats
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step<S, R, I, SC, true, true>, kBlock, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step<S, R, I, SC, true, false>, kBlock, 0);
    if (e == cudaSuccess && nb > 0) direct = nb;
    const RowPlan rp = row_plan<S>(nx);
    if (!rp.use) return;
    // the attribute is per kernel, shared by every context of the process:
    // set it to the largest staging any box may use, not to this box's
    if constexpr (!std::is_same<S, double>::value) {
        if (rp.np == 2) {
            rows = prepare_rows<S, R, SC, 2>(rp, stats);
            return;
        }
    }
    rows = prepare_rows<S, R, SC, 1>(rp, stats);
}

template <typename S, typename R, typename I>
void step_occupancy_t(int scheme, uint32_t nx, bool stats, int &direct, int &rows)
{
    if (scheme == 0) prepare_scheme<S, R, I, 0>(nx, stats, direct, rows);
    else if (scheme == 1) prepare_scheme<S, R, I, 1>(nx, stats, direct, rows);
    else prepare_scheme<S, R, I, 2>(nx, stats, direct, rows);
}

}  // namespace flbm
