// aux.cu -- non-hot kernels: initial state, AA-aware gather/scatter of the
// populations, moment export (Eqs. rho/u and Pi), observable fields and the
// FP64 shell binning of S(k) (Sec. III), and the final pass of the fused
// reductions.
#include <cuda_fp16.h>

#include <type_traits>

#include "internal.h"
#include "stats.cuh"
#include "lattice.cuh"

namespace flbm {

namespace {

__device__ __forceinline__ void node_xyz(uint64_t n, const BoxDesc &b, uint32_t &x, uint32_t &y,
                                         uint32_t &z)
{
    x = uint32_t(n % b.nx);
    const uint64_t r = n / b.nx;
    y = uint32_t(r % b.ny);
    z = uint32_t(r / b.ny);
}

__device__ __forceinline__ uint32_t wrap(uint32_t v, int d, uint32_t L)
{
    if (d > 0) return (v + 1 < L) ? v + 1 : 0;
    if (d < 0) return v ? v - 1 : L - 1;
    return v;
}

// Storage index of f_i(x, t) for the current parity: natural form keeps it in
// slot i at x; the AA odd form keeps it in slot opp(i) at x - c_i.
__device__ __forceinline__ uint64_t storage_index(int cx, int cy, int cz, uint32_t x, uint32_t y,
                                                  uint32_t z, const BoxDesc &b)
{
    if (b.parity == 0) {
        const uint64_t n = x + uint64_t(b.nx) * (y + uint64_t(b.ny) * z);
        return uint64_t(slot_of(cx, cy, cz)) * b.ns + n;
    }
    const uint32_t xx = wrap(x, -cx, b.nx), yy = wrap(y, -cy, b.ny), zz = wrap(z, -cz, b.nz);
    const uint64_t n = xx + uint64_t(b.nx) * (yy + uint64_t(b.ny) * zz);
    return uint64_t(slot_of(-cx, -cy, -cz)) * b.ns + n;
}

// storage element <-> double
template <typename S>
__device__ __forceinline__ double to_d(S v) { return double(v); }
template <>
__device__ __forceinline__ double to_d<__half>(__half v) { return double(__half2float(v)); }
template <typename S>
__device__ __forceinline__ S from_d(double v) { return S(v); }
template <>
__device__ __forceinline__ __half from_d<__half>(double v) { return __float2half_rn(float(v)); }

template <typename S>
__device__ __forceinline__ double ldd(const S *g, uint64_t i) { return to_d(g[i]); }

// Arithmetic type of the auxiliary kernels: double for FP64 storage, float
// otherwise (the deviations are O(1e-2) and the storage is FP32 / FP16
// anyway; FP64 arithmetic is the slow pipe on this GPU).
template <typename S>
using Acc = typename std::conditional<std::is_same<S, double>::value, double, float>::type;

template <typename S>
__device__ __forceinline__ Acc<S> lda(const S *g, uint64_t i) { return Acc<S>(to_d(g[i])); }
template <>
__device__ __forceinline__ float lda<float>(const float *g, uint64_t i) { return g[i]; }
template <>
__device__ __forceinline__ float lda<__half>(const __half *g, uint64_t i) { return __half2float(g[i]); }



template <typename S>
__global__ void k_fill_zero(S *g, uint64_t count)
{
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < count;
         i += uint64_t(gridDim.x) * blockDim.x)
        g[i] = from_d<S>(0.0);
}

// out[i*cn + k] = f_i (absolute, or deviation) at node n0 + k
template <typename S>
__global__ void k_gather_f(const S *g, BoxDesc b, uint64_t n0, uint64_t cn, double *out, int dev)
{
    for (uint64_t k = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; k < cn;
         k += uint64_t(gridDim.x) * blockDim.x) {
        uint32_t x, y, z;
        node_xyz(n0 + k, b, x, y, z);
#pragma unroll
        for (int cx = -1; cx <= 1; ++cx)
#pragma unroll
            for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
                for (int cz = -1; cz <= 1; ++cz) {
                    const int i = slot_of(cx, cy, cz);
                    const double w = w1(cx) * w1(cy) * w1(cz);
                    const double gv = ldd(g, storage_index(cx, cy, cz, x, y, z, b));
                    out[uint64_t(i) * cn + k] = dev ? gv : gv + w * b.rho0;
                }
    }
}

template <typename S>
__global__ void k_gather_state(const S *g, BoxDesc b, uint64_t n0, uint64_t cn, S *out)
{
    for (uint64_t k = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; k < cn;
         k += uint64_t(gridDim.x) * blockDim.x) {
        uint32_t x, y, z;
        node_xyz(n0 + k, b, x, y, z);
#pragma unroll
        for (int cx = -1; cx <= 1; ++cx)
#pragma unroll
            for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
                for (int cz = -1; cz <= 1; ++cz)
                    out[uint64_t(slot_of(cx, cy, cz)) * cn + k] =
                        g[storage_index(cx, cy, cz, x, y, z, b)];
    }
}

// natural-form write of f_i - w_i rho0 from in[i*cn + k]
template <typename S>
__global__ void k_scatter_f(S *g, BoxDesc b, uint64_t n0, uint64_t cn, const double *in)
{
    for (uint64_t k = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; k < cn;
         k += uint64_t(gridDim.x) * blockDim.x) {
#pragma unroll
        for (int cx = -1; cx <= 1; ++cx)
#pragma unroll
            for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
                for (int cz = -1; cz <= 1; ++cz) {
                    const int i = slot_of(cx, cy, cz);
                    const double w = w1(cx) * w1(cy) * w1(cz);
                    g[uint64_t(i) * b.ns + n0 + k] = from_d<S>(in[uint64_t(i) * cn + k] - w * b.rho0);
                }
    }
}

// Natural-form thermal sample g_i = sqrt(rho0 kT w_i / c_s^2) xi_i.
template <typename S>
__global__ void k_init_thermal(S *g, BoxDesc b, double kT, uint32_t key0, uint32_t key1)
{
    uint32_t rk[20];
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = key0 + uint32_t(r) * 0x9E3779B9u;
        rk[2 * r + 1] = key1 + uint32_t(r) * 0xBB67AE85u;
    }
    using A = Acc<S>;
    const A base = A(sqrt(b.rho0 * kT * 3.0));   // sqrt(rho0 kT / c_s^2)
    for (uint64_t n = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; n < b.n;
         n += uint64_t(gridDim.x) * blockDim.x) {
        A xi[28];
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            const u32x4 o = philox4x32_10(u32x4{uint32_t(n), 0u, uint32_t(6 + j), 0u}, rk);
            A rad, c, sn;
            box_muller(o.x, o.y, rad, c, sn);
            xi[4 * j] = rad * c;
            xi[4 * j + 1] = rad * sn;
            box_muller(o.z, o.w, rad, c, sn);
            xi[4 * j + 2] = rad * c;
            xi[4 * j + 3] = rad * sn;
        }
#pragma unroll
        for (int cx = -1; cx <= 1; ++cx)
#pragma unroll
            for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
                for (int cz = -1; cz <= 1; ++cz) {
                    const int i = slot_of(cx, cy, cz);
                    // sqrt(w_i) = prod sqrt(w1): sqrt(2/3), sqrt(1/6)
                    const double sw = (cx ? 0.40824829046386302 : 0.81649658092772603) *
                                      (cy ? 0.40824829046386302 : 0.81649658092772603) *
                                      (cz ? 0.40824829046386302 : 0.81649658092772603);
                    g[uint64_t(i) * b.ns + n] = from_d<S>(double(base * A(sw) * xi[i]));
                }
    }
}

// out[k*27 + i] = f_i (absolute) at node nodes[k]
template <typename S>
__global__ void k_probe(const S *g, BoxDesc b, const long long *nodes, long long count, double *out)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
         k += (long long)gridDim.x * blockDim.x) {
        uint32_t x, y, z;
        node_xyz(uint64_t(nodes[k]), b, x, y, z);
#pragma unroll
        for (int cx = -1; cx <= 1; ++cx)
#pragma unroll
            for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
                for (int cz = -1; cz <= 1; ++cz) {
                    const int i = slot_of(cx, cy, cz);
                    const double w = w1(cx) * w1(cy) * w1(cz);
                    out[k * 27 + i] = ldd(g, storage_index(cx, cy, cz, x, y, z, b)) + w * b.rho0;
                }
    }
}

// Pre-collision moments: out planes rho, jx, jy, jz, Pxx, Pyy, Pzz, Pxy, Pxz,
// Pyz (FP64; Pi = sum f c c includes the rest part rho0 c_s^2 delta).
template <typename S>
__global__ void k_moments(const S *g, BoxDesc b, uint64_t n0, uint64_t cn, double *out)
{
    using A = Acc<S>;
    for (uint64_t k = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; k < cn;
         k += uint64_t(gridDim.x) * blockDim.x) {
        uint32_t x, y, z;
        node_xyz(n0 + k, b, x, y, z);
        A m[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int cx = -1; cx <= 1; ++cx)
#pragma unroll
            for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
                for (int cz = -1; cz <= 1; ++cz) {
                    const A gv = lda(g, storage_index(cx, cy, cz, x, y, z, b));
                    m[0] += gv;
                    if (cx) m[1] += cx * gv;
                    if (cy) m[2] += cy * gv;
                    if (cz) m[3] += cz * gv;
                    if (cx) m[4] += gv;
                    if (cy) m[5] += gv;
                    if (cz) m[6] += gv;
                    if (cx && cy) m[7] += (cx * cy) * gv;
                    if (cx && cz) m[8] += (cx * cz) * gv;
                    if (cy && cz) m[9] += (cy * cz) * gv;
                }
        const double pr = b.rho0 / 3.0;   // rest-state c_s^2 rho0 on the diagonal
        out[0 * cn + k] = b.rho0 + double(m[0]);
        out[1 * cn + k] = double(m[1]);
        out[2 * cn + k] = double(m[2]);
        out[3 * cn + k] = double(m[3]);
        out[4 * cn + k] = pr + double(m[4]);
        out[5 * cn + k] = pr + double(m[5]);
        out[6 * cn + k] = pr + double(m[6]);
        out[7 * cn + k] = double(m[7]);
        out[8 * cn + k] = double(m[8]);
        out[9 * cn + k] = double(m[9]);
    }
}

// Observable field m(x) (deviation from the rest state; the constant offset
// only affects the excluded n = 0 mode).
template <typename S, typename F>
__global__ void k_observable(const S *g, BoxDesc b, int obs, F *field)
{
    using A = Acc<S>;
    for (uint64_t n = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; n < b.n;
         n += uint64_t(gridDim.x) * blockDim.x) {
        uint32_t x, y, z;
        node_xyz(n, b, x, y, z);
        A acc = 0;
#pragma unroll
        for (int cx = -1; cx <= 1; ++cx)
#pragma unroll
            for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
                for (int cz = -1; cz <= 1; ++cz) {
                    int c;
                    switch (obs) {
                    case 0: c = 1; break;
                    case 1: c = cx + cy + cz; break;
                    case 2: c = cx * cx + cy * cy + cz * cz; break;
                    case 3: c = cx * cy + cx * cz + cy * cz; break;
                    case 4: c = cx; break;
                    case 5: c = cy; break;
                    default: c = cz; break;
                    }
                    if (c != 0) acc += A(c) * lda(g, storage_index(cx, cy, cz, x, y, z, b));
                }
        field[n] = F(acc);
    }
}

// Shell binning of the R2C spectrum [nz][ny][nx/2+1] (complex of T).
template <typename T>
__global__ void k_shells(const T *spec, BoxDesc b, int nshell, double *S, unsigned long long *cnt)
{
    extern __shared__ double smem[];
    double *sh_s = smem;
    unsigned long long *sh_c = reinterpret_cast<unsigned long long *>(smem + nshell);
    for (int s = threadIdx.x; s < nshell; s += blockDim.x) { sh_s[s] = 0.0; sh_c[s] = 0ull; }
    __syncthreads();
    const uint32_t nxh = b.nx / 2 + 1;
    const uint64_t total = uint64_t(nxh) * b.ny * b.nz;
    const double invN = 1.0 / double(b.n);
    for (uint64_t e = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; e < total;
         e += uint64_t(gridDim.x) * blockDim.x) {
        const uint32_t kx = uint32_t(e % nxh);
        const uint64_t r = e / nxh;
        const uint32_t ky = uint32_t(r % b.ny), kz = uint32_t(r / b.ny);
        const long long ax = kx;
        const long long ay = (2ull * ky < b.ny) ? (long long)ky : (long long)ky - (long long)b.ny;
        const long long az = (2ull * kz < b.nz) ? (long long)kz : (long long)kz - (long long)b.nz;
        const long long n2 = ax * ax + ay * ay + az * az;
        if (n2 == 0) continue;
        // round(|n|): s^2 - s < n2 <= s^2 + s for integer s (|n| is never a half-integer)
        long long s = llrint(sqrt(double(n2)));
        while (s * s - s >= n2) --s;
        while (s * s + s < n2) ++s;
        if (s >= nshell) continue;
        const double re = double(spec[2 * e]), im = double(spec[2 * e + 1]);
        // the conjugate half (kx -> -kx) has the same |n|; kx = 0 and the even
        // Nyquist plane are their own partners
        const unsigned wgt = (kx == 0 || (b.nx % 2 == 0 && kx == b.nx / 2)) ? 1u : 2u;
        atomicAdd(&sh_s[s], wgt * (re * re + im * im) * invN);
        atomicAdd(&sh_c[s], (unsigned long long)wgt);
    }
    __syncthreads();
    for (int s = threadIdx.x; s < nshell; s += blockDim.x) {
        if (sh_c[s]) {
            atomicAdd(&S[s], sh_s[s]);
            atomicAdd(&cnt[s], sh_c[s]);
        }
    }
}

__global__ void k_stats_finalize(const double *partials, int nblocks, DevStats *st, long long step,
                                 double n)
{
    __shared__ double red[NSTAT][256];
    double loc[NSTAT];
#pragma unroll
    for (int s = 0; s < NSTAT; ++s) loc[s] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int s = 0; s < NSTAT; ++s) loc[s] += partials[size_t(b) * NSTAT + s];
#pragma unroll
    for (int s = 0; s < NSTAT; ++s) red[s][threadIdx.x] = loc[s];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int s = 0; s < NSTAT; ++s) red[s][threadIdx.x] += red[s][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double tot[NSTAT];
        for (int s = 0; s < NSTAT; ++s) tot[s] = red[s][0];
        stats_update(st, tot, step, n);
    }
}

inline int grid_for(uint64_t work, int block)
{
    uint64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 65535ull * 16) g = 65535ull * 16;
    return int(g);
}

}  // namespace

// Calls f with a value of the storage type of precision code prec
// (0 double, 1 float, 2 half).
template <typename F>
void with_storage(int prec, F &&f)
{
    if (prec == 0) f(double{});
    else if (prec == 1) f(float{});
    else f(__half{});
}

cudaError_t launch_fill_rest(void *g, int prec, uint64_t count, cudaStream_t s)
{
    const int grid = grid_for(count, 256) > 4096 ? 4096 : grid_for(count, 256);
    with_storage(prec, [&](auto tag) {
        using S = decltype(tag);
        k_fill_zero<S><<<grid, 256, 0, s>>>(static_cast<S *>(g), count);
    });
    return cudaGetLastError();
}

cudaError_t launch_gather_f(const void *g, int prec, const BoxDesc &b, uint64_t n0, uint64_t cn,
                            double *out, bool deviations, cudaStream_t s)
{
    const int grid = grid_for(cn, 128);
    with_storage(prec, [&](auto tag) {
        using S = decltype(tag);
        k_gather_f<S><<<grid, 128, 0, s>>>(static_cast<const S *>(g), b, n0, cn, out, deviations);
    });
    return cudaGetLastError();
}

cudaError_t launch_gather_state(const void *g, int prec, const BoxDesc &b, uint64_t n0, uint64_t cn,
                                void *out, cudaStream_t s)
{
    const int grid = grid_for(cn, 128);
    with_storage(prec, [&](auto tag) {
        using S = decltype(tag);
        k_gather_state<S><<<grid, 128, 0, s>>>(static_cast<const S *>(g), b, n0, cn, static_cast<S *>(out));
    });
    return cudaGetLastError();
}

cudaError_t launch_scatter_f(void *g, int prec, const BoxDesc &b, uint64_t n0, uint64_t cn,
                             const double *in, cudaStream_t s)
{
    const int grid = grid_for(cn, 128);
    with_storage(prec, [&](auto tag) {
        using S = decltype(tag);
        k_scatter_f<S><<<grid, 128, 0, s>>>(static_cast<S *>(g), b, n0, cn, in);
    });
    return cudaGetLastError();
}

cudaError_t launch_init_thermal(void *g, int prec, const BoxDesc &b, double kT, uint64_t seed,
                                cudaStream_t s)
{
    const int grid = grid_for(b.n, 128) > 8192 ? 8192 : grid_for(b.n, 128);
    const uint32_t k0 = uint32_t(seed & 0xffffffffu), k1 = uint32_t(seed >> 32);
    with_storage(prec, [&](auto tag) {
        using S = decltype(tag);
        k_init_thermal<S><<<grid, 128, 0, s>>>(static_cast<S *>(g), b, kT, k0, k1);
    });
    return cudaGetLastError();
}

cudaError_t launch_probe(const void *g, int prec, const BoxDesc &b, const long long *nodes,
                         long long count, double *out, cudaStream_t s)
{
    const int grid = grid_for(uint64_t(count), 128);
    with_storage(prec, [&](auto tag) {
        using S = decltype(tag);
        k_probe<S><<<grid, 128, 0, s>>>(static_cast<const S *>(g), b, nodes, count, out);
    });
    return cudaGetLastError();
}

cudaError_t launch_moments(const void *g, int prec, const BoxDesc &b, uint64_t n0, uint64_t cn,
                           double *out, cudaStream_t s)
{
    const int grid = grid_for(cn, 128);
    with_storage(prec, [&](auto tag) {
        using S = decltype(tag);
        k_moments<S><<<grid, 128, 0, s>>>(static_cast<const S *>(g), b, n0, cn, out);
    });
    return cudaGetLastError();
}

// The observable field is double for FP64 storage and float otherwise.
cudaError_t launch_observable(const void *g, int prec, const BoxDesc &b, int obs, void *field,
                              cudaStream_t s)
{
    const int grid = grid_for(b.n, 256);
    with_storage(prec, [&](auto tag) {
        using S = decltype(tag);
        using F = typename std::conditional<std::is_same<S, double>::value, double, float>::type;
        k_observable<S, F><<<grid, 256, 0, s>>>(static_cast<const S *>(g), b, obs, static_cast<F *>(field));
    });
    return cudaGetLastError();
}

cudaError_t launch_shells(const void *spec, int prec, const BoxDesc &b, int nshell, double *S,
                          unsigned long long *cnt, cudaStream_t s)
{
    const uint64_t total = uint64_t(b.nx / 2 + 1) * b.ny * b.nz;
    int grid = grid_for(total, 256);
    if (grid > 2048) grid = 2048;
    const size_t sm = size_t(nshell) * (sizeof(double) + sizeof(unsigned long long));
    if (prec == 0)
        k_shells<double><<<grid, 256, sm, s>>>(static_cast<const double *>(spec), b, nshell, S, cnt);
    else
        k_shells<float><<<grid, 256, sm, s>>>(static_cast<const float *>(spec), b, nshell, S, cnt);
    return cudaGetLastError();
}

cudaError_t launch_stats_finalize(const double *partials, int nblocks, DevStats *st, long long step,
                                  double n, cudaStream_t s)
{
    k_stats_finalize<<<1, 256, 0, s>>>(partials, nblocks, st, step, n);
    return cudaGetLastError();
}

}  // namespace flbm
