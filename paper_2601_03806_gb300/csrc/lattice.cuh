// lattice.cuh -- D3Q27 lattice, tensor-product Hermite basis and the
// counter-based noise source, as compile-time device code.
//
// Everything here folds to immediates inside fully unrolled loops; there are
// no run-time tables.
//
// Basis (Table II).  Every Table II vector is a tensor product
//   e_k(c) = p_a(c_x) p_b(c_y) p_c(c_z),  p_0 = 1, p_1 = c, p_2 = c^2 - c_s^2,
// with per-axis degrees (a,b,c) read off its Hermite symbol (H_{x^2 y} ->
// (2,1,0)), and b_k = beta_a beta_b beta_c with beta = (1, 1/3, 2/9); the
// weights factor as w_i = w1(c_x) w1(c_y) w1(c_z), w1(0) = 2/3, w1(+-1) = 1/6
// (Table I).  The library therefore evaluates the forward projection and the
// reconstruction f_i = w_i sum_k e_ki M_k / b_k (Eqs. expeq/expneq) as three
// 1-D passes over 3-point lines instead of a dense 27x27 product.
#pragma once

#include <cstdint>

namespace flbm {

constexpr int Q = 27;

// Velocity slot of c = (cx,cy,cz) in the ABI order (Table I groups):
// rest; +x -x +y -y +z -z; xy, xz, yz planes as (++,--,+-,-+); corners
// (+++),(---),(++-),(--+),(+-+),(-+-),(-++),(+--).
__host__ __device__ constexpr int slot_of(int cx, int cy, int cz)
{
    const int s = cx * cx + cy * cy + cz * cz;
    if (s == 0) return 0;
    if (s == 1) {
        const int axis = cx ? 0 : (cy ? 1 : 2);
        const int v = cx + cy + cz;
        return 1 + 2 * axis + (v < 0 ? 1 : 0);
    }
    if (s == 2) {
        const int plane = (cz == 0) ? 0 : ((cy == 0) ? 1 : 2);
        const int u = (plane == 2) ? cy : cx;
        const int v = (plane == 0) ? cy : cz;
        const int pat = (u > 0 && v > 0) ? 0 : (u < 0 && v < 0) ? 1 : (u > 0) ? 2 : 3;
        return 7 + 4 * plane + pat;
    }
    // corners: a "first" member has at most one negative component; its
    // opposite follows it.
    const int neg = (cx < 0) + (cy < 0) + (cz < 0);
    const bool first = neg <= 1;
    const int ax = first ? cx : -cx, ay = first ? cy : -cy, az = first ? cz : -cz;
    const int q = (ax > 0 && ay > 0 && az > 0) ? 0 : (az < 0) ? 1 : (ay < 0) ? 2 : 3;
    return 19 + 2 * q + (first ? 0 : 1);
}

// 1-D weights and Hermite polynomial values (c in {-1,0,1}, d in {0,1,2}).
__host__ __device__ constexpr double w1(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
__host__ __device__ constexpr double p1d(int d, int c)
{
    return d == 0 ? 1.0 : (d == 1 ? double(c) : double(c * c) - 1.0 / 3.0);
}
__host__ __device__ constexpr double beta1d(int d)
{
    return d == 0 ? 1.0 : (d == 1 ? 1.0 / 3.0 : 2.0 / 9.0);
}

// Table II mode index k of the tensor-product degrees (a,b,c).
__host__ __device__ constexpr int mode_of(int a, int b, int c)
{
    // listing order of Table II
    return (a == 0 && b == 0 && c == 0) ? 0 :
           (a == 1 && b == 0 && c == 0) ? 1 :
           (a == 0 && b == 1 && c == 0) ? 2 :
           (a == 0 && b == 0 && c == 1) ? 3 :
           (a == 2 && b == 0 && c == 0) ? 4 :
           (a == 0 && b == 2 && c == 0) ? 5 :
           (a == 0 && b == 0 && c == 2) ? 6 :
           (a == 1 && b == 1 && c == 0) ? 7 :
           (a == 1 && b == 0 && c == 1) ? 8 :
           (a == 0 && b == 1 && c == 1) ? 9 :
           (a == 2 && b == 1 && c == 0) ? 10 :   // x^2 y
           (a == 2 && b == 0 && c == 1) ? 11 :   // x^2 z
           (a == 1 && b == 2 && c == 0) ? 12 :   // y^2 x
           (a == 1 && b == 0 && c == 2) ? 13 :   // z^2 x
           (a == 0 && b == 2 && c == 1) ? 14 :   // y^2 z
           (a == 0 && b == 1 && c == 2) ? 15 :   // z^2 y
           (a == 1 && b == 1 && c == 1) ? 16 :   // xyz
           (a == 2 && b == 2 && c == 0) ? 17 :   // x^2 y^2
           (a == 2 && b == 0 && c == 2) ? 18 :   // x^2 z^2
           (a == 0 && b == 2 && c == 2) ? 19 :   // y^2 z^2
           (a == 1 && b == 1 && c == 2) ? 20 :   // x y z^2
           (a == 1 && b == 2 && c == 1) ? 21 :   // x z y^2
           (a == 2 && b == 1 && c == 1) ? 22 :   // y z x^2
           (a == 2 && b == 1 && c == 2) ? 23 :   // x^2 y z^2
           (a == 2 && b == 2 && c == 1) ? 24 :   // x^2 z y^2
           (a == 1 && b == 2 && c == 2) ? 25 :   // y^2 x z^2
                                          26;    // x^2 y^2 z^2
}

// Inverse of mode_of: per-axis degrees of Table II mode k, packed a + 3b + 9c.
__host__ __device__ constexpr int mode_deg(int k)
{
    for (int c = 0; c < 3; ++c)
        for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a)
                if (mode_of(a, b, c) == k) return a + 3 * b + 9 * c;
    return -1;
}

__host__ __device__ constexpr int mode_order(int a, int b, int c) { return a + b + c; }
__host__ __device__ constexpr double b_of(int a, int b, int c)
{
    return beta1d(a) * beta1d(b) * beta1d(c);
}

// Scales of the kernel's transforms.  The forward pass returns
// fwd_scale * M_abc: its degree-2 line sum is o - 2 s = -3 sum v p_2(c) (one
// FMA with no negated operand), so each degree-2 axis contributes -3.  The
// reconstruction consumes Q_abc = syn_scale * M_abc with syn_scale =
// prod kappa(d), kappa = (4/6, 1/2, 1/2): per-axis w1-prescale / beta, times 4
// on the degree-0 amplitude, which makes every 1-D synthesis pass
// (t - p1, p0 - 2 p2, t + p1) with t = p0 / 4 + p2 (two FMAs and two adds;
// the values at c = -1, 0, +1 of w1(c) (q0 + q1 c + q2 (c^2 - 1/3))).  Every
// factor is exact in binary, so the scales change no rounding.
__host__ __device__ constexpr double fwd_scale(int a, int b, int c)
{
    return (a == 2 ? -3.0 : 1.0) * (b == 2 ? -3.0 : 1.0) * (c == 2 ? -3.0 : 1.0);
}
__host__ __device__ constexpr double kappa1d(int d) { return d == 0 ? 2.0 / 3.0 : 0.5; }

// sqrt(b_k / c_s^2) of mode (a,b,c): sqrt(3) prod sqrt(beta_d), with
// sqrt(beta) = (1, 1/sqrt(3), sqrt(2)/3) written as literals so the product
// folds to an immediate.
__host__ __device__ constexpr double sqrt_beta1d(int d)
{
    return d == 0 ? 1.0 : (d == 1 ? 0.57735026918962576451 : 0.47140452079103168293);
}
__host__ __device__ constexpr double sqrt_b_over_cs2(int a, int b, int c)
{
    return 1.7320508075688772935 * sqrt_beta1d(a) * sqrt_beta1d(b) * sqrt_beta1d(c);
}
__host__ __device__ constexpr double syn_scale(int a, int b, int c)
{
    return kappa1d(a) * kappa1d(b) * kappa1d(c);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 block function (Salmon, Moraes, Dror, Shaw, SC'11): ten
// rounds of two 32x32->64 multiplies with a Weyl-sequence key schedule.
struct u32x4 { uint32_t x, y, z, w; };

// rk holds the round keys (k0, k1) of rounds 0..9: the key, bumped by the
// Weyl constants 0x9E3779B9 / 0xBB67AE85 before every round after the first
// (precomputed on the host, so the kernel reads them as constants).
__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, const uint32_t (&rk)[20])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = uint64_t(0xD2511F53u) * c.x;
        const uint64_t p1 = uint64_t(0xCD9E8D57u) * c.z;
        c = u32x4{uint32_t(p1 >> 32) ^ c.y ^ rk[2 * r], uint32_t(p1),
                  uint32_t(p0 >> 32) ^ c.w ^ rk[2 * r + 1], uint32_t(p0)};
    }
    return c;
}

// The block function with round 0's product of counter word 2 supplied by
// the caller (h2k = hi(M1 c2) ^ k0(0), l2 = lo(M1 c2)) and rounds 1..9 as
// usual: for callers whose c2 is uniform but not known to the host.
__device__ __forceinline__ u32x4 philox4x32_10_r0(uint32_t c0, uint32_t c1, uint32_t c3, uint32_t h2k,
                                                  uint32_t l2, const uint32_t (&rk)[20])
{
    const uint64_t p0 = uint64_t(0xD2511F53u) * c0;
    u32x4 c{h2k ^ c1, l2, uint32_t(p0 >> 32) ^ c3 ^ rk[1], uint32_t(p0)};
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        const uint64_t q0 = uint64_t(0xD2511F53u) * c.x;
        const uint64_t q1 = uint64_t(0xCD9E8D57u) * c.z;
        c = u32x4{uint32_t(q1 >> 32) ^ c.y ^ rk[2 * r], uint32_t(q1),
                  uint32_t(q0 >> 32) ^ c.w ^ rk[2 * r + 1], uint32_t(q0)};
    }
    return c;
}

// The same block function for counter (c0, c1, c2, c3) when only c0 varies
// between the threads of a launch.  Rounds 0 and 1 then split into a part
// that depends on c0 alone and launch-uniform words the caller supplies:
//   zk = c3 ^ k1(0);  x0 = hi(M1 c2) ^ c1 ^ k0(0),  y0 = lo(M1 c2);
//   u1 = y0 ^ k0(1),  u2 = hi(M0 x0) ^ k1(1),  u3 = lo(M0 x0).
// Round 0 gives (x0, y0, hi(M0 c0) ^ zk, lo(M0 c0)) and round 1
// (hi(M1 z0) ^ u1, lo(M1 z0), u2 ^ w0, u3); rounds 2..9 follow as usual.
__device__ __forceinline__ u32x4 philox4x32_10_r2(uint32_t c0, uint32_t zk, uint32_t u1, uint32_t u2,
                                                  uint32_t u3, const uint32_t (&rk)[20])
{
    const uint64_t p0 = uint64_t(0xD2511F53u) * c0;
    const uint32_t z0 = uint32_t(p0 >> 32) ^ zk, w0 = uint32_t(p0);
    const uint64_t p1 = uint64_t(0xCD9E8D57u) * z0;
    u32x4 c{uint32_t(p1 >> 32) ^ u1, uint32_t(p1), u2 ^ w0, u3};
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        const uint64_t q0 = uint64_t(0xD2511F53u) * c.x;
        const uint64_t q1 = uint64_t(0xCD9E8D57u) * c.z;
        c = u32x4{uint32_t(q1 >> 32) ^ c.y ^ rk[2 * r], uint32_t(q1),
                  uint32_t(q0 >> 32) ^ c.w ^ rk[2 * r + 1], uint32_t(q0)};
    }
    return c;
}

// 23-bit uniform in (0,1): ((w >> 9) + 0.5) 2^-23, exact in float and double.
// FP32 builds it from the bits: (1 + m 2^-23) - (1 - 2^-24) is exact.
__device__ __forceinline__ float uniform23f(uint32_t w)
{
    return __uint_as_float(0x3f800000u | (w >> 9)) - (1.0f - 0x1p-24f);
}
__device__ __forceinline__ double uniform23d(uint32_t w)
{
    return __fma_rn(double(w >> 9), 0x1p-23, 0x1p-24);
}

// Box-Muller (1958) in polar form: r_a = rad * ca, r_b = rad * sa with
// r_a, r_b = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).
// FP32: hardware log2, whose absolute error is <= 2^-22 on [0.5, 1) and
// <= 2 ulp below 0.5.  The radius then has absolute error <= ln2 2^-22 / rad
// (~1.7e-7 / rad): below 1e-6 when u1 <= 0.986 (98.6 % of draws) and at most
// 4.7e-4 at the smallest radius 3.5e-4 (u1 = 1 - 2^-24).  The angle is taken
// as 2 pi u2 - pi in (-pi, pi), where the hardware sin/cos hold their
// 2^-21.4 absolute error bound; the half-turn is undone by the sign of rad.
__device__ __forceinline__ void box_muller(uint32_t w1u, uint32_t w2u, float &rad, float &ca,
                                           float &sa)
{
    const float u1 = uniform23f(w1u);
    const float u2 = uniform23f(w2u);
    const float t = -1.3862943611198906f * __log2f(u1);   // -2 ln u1
    rad = -(t * rsqrtf(t));
    __sincosf(__fmaf_rn(u2, 6.2831853071795865f, -3.1415926535897932f), &sa, &ca);
}
__device__ __forceinline__ void box_muller(uint32_t w1u, uint32_t w2u, double &rad, double &ca,
                                           double &sa)
{
    const double u1 = uniform23d(w1u);
    const double u2 = uniform23d(w2u);
    rad = sqrt(-2.0 * log(u1));
    sincospi(2.0 * u2, &sa, &ca);
}

}  // namespace flbm
