// mlp_train.cu -- training of the learned-collision network on the GPU:
// training pairs from a lattice state, the loss gradient (forward and
// backward in FP32 on the CUDA cores), and Adam.
//
// Pairs: for every node, the features x (28) and the target
//   t_i = w_i sum_{k >= 10} e_ki rho u^(deg k) / b_k / (w_i sigma^3),
// the ghost equilibrium content by which the regularized collision
// (Reg-FLBM) differs from the GMF collision of the same pre-collision state.
// It is synthesised in FP64 with the same sum-factorised transform as the
// step kernels (only the ghost amplitudes non-zero).
//
// Gradient of L = mean over samples and outputs of (y - t)^2: a CTA of 128
// threads takes tiles of 128 samples; thread s runs sample s's forward and
// backward rows against the FP32 weights in shared memory and keeps the
// activations there (rows padded to odd strides, so the threads of a warp
// hit distinct banks); then thread p accumulates parameters p, p + 128, ...
// as sums over the tile's samples in registers, across all of its tiles.
// Each CTA writes its partial sums once; a second kernel adds them in CTA
// order (FP64), so the gradient does not depend on scheduling.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <random>
#include <string>
#include <vector>

#include "../../include/flbm.h"
#include "internal.h"
#include "lattice.cuh"
#include "step_kernel.cuh"

namespace flbm {

namespace {

constexpr int kNin = 28, kNh = 64, kNout = 27, kNp = 7771;
constexpr int kOffW1 = 0, kOffB1 = 1792, kOffW2 = 1856, kOffB2 = 5952, kOffW3 = 6016, kOffB3 = 7744;
constexpr int kTile = 128;
constexpr int kPerThread = (kNp + kTile - 1) / kTile;   // 61
constexpr int kSx = 29, kSh = 65, kSy = 28;              // padded row strides (floats)

struct GradSmem {
    float w[kNp];
    float x[kTile * kSx];
    float h1[kTile * kSh];
    float h2[kTile * kSh];
    float s1[kTile * kSh];   // silu'(z1), then dL/dz1
    float s2[kTile * kSh];   // silu'(z2), then dL/dz2
    float dy[kTile * kSy];
};

__device__ __forceinline__ float sigm(float z) { return 1.0f / (1.0f + expf(-z)); }

// Sample s of the epoch order: (mult s + off) mod n, a bijection of [0, n)
// for mult coprime to n (mult = 1, off = 0: the identity).  s < n < 2^32 and
// mult < n keep the product below 2^64.
__device__ __forceinline__ uint64_t sample_index(uint64_t s, uint64_t mult, uint64_t off, uint64_t n)
{
    return (mult * s + off) % n;
}

__global__ void __launch_bounds__(kTile) k_mlp_grad(const float *__restrict__ params, const float *__restrict__ X,
                                                    const float *__restrict__ T, uint64_t n, uint64_t start,
                                                    uint64_t count, uint64_t mult, uint64_t off, float inv_norm,
                                                    double *__restrict__ partials)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    GradSmem &sm = *reinterpret_cast<GradSmem *>(smraw);
    const uint32_t t = threadIdx.x;
    for (int i = t; i < kNp; i += kTile) sm.w[i] = params[i];
    float acc[kPerThread];
#pragma unroll
    for (int m = 0; m < kPerThread; ++m) acc[m] = 0.0f;
    double loss = 0.0;
    __syncthreads();
    const float *W1 = sm.w + kOffW1, *b1 = sm.w + kOffB1, *W2 = sm.w + kOffW2, *b2 = sm.w + kOffB2;
    const float *W3 = sm.w + kOffW3, *b3 = sm.w + kOffB3;
    const uint64_t ntiles = (count + kTile - 1) / kTile;
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t s = tile * kTile + t;
        const bool live = s < count;
        float *xr = sm.x + t * kSx, *h1 = sm.h1 + t * kSh, *h2 = sm.h2 + t * kSh;
        float *s1 = sm.s1 + t * kSh, *s2 = sm.s2 + t * kSh, *dy = sm.dy + t * kSy;
        uint64_t idx = 0;
        if (live) idx = sample_index(start + s, mult, off, n);
        for (int k = 0; k < kNin; ++k) xr[k] = live ? X[idx * kNin + k] : 0.0f;
        // forward rows
        for (int o = 0; o < kNh; ++o) {
            float z = b1[o];
            for (int k = 0; k < kNin; ++k) z = fmaf(W1[o * kNin + k], xr[k], z);
            const float g = sigm(z);
            h1[o] = live ? z * g : 0.0f;
            s1[o] = live ? g * (1.0f + z * (1.0f - g)) : 0.0f;
        }
        for (int o = 0; o < kNh; ++o) {
            float z = b2[o];
            for (int k = 0; k < kNh; ++k) z = fmaf(W2[o * kNh + k], h1[k], z);
            const float g = sigm(z);
            h2[o] = live ? z * g : 0.0f;
            s2[o] = live ? g * (1.0f + z * (1.0f - g)) : 0.0f;
        }
        for (int o = 0; o < kNout; ++o) {
            float y = b3[o];
            for (int k = 0; k < kNh; ++k) y = fmaf(W3[o * kNh + k], h2[k], y);
            const float d = live ? y - T[idx * kNout + o] : 0.0f;
            loss += double(d) * double(d);
            dy[o] = 2.0f * d * inv_norm;
        }
        // backward rows
        for (int k = 0; k < kNh; ++k) {
            float g = 0.0f;
            for (int o = 0; o < kNout; ++o) g = fmaf(dy[o], W3[o * kNh + k], g);
            s2[k] *= g;
        }
        for (int k = 0; k < kNh; ++k) {
            float g = 0.0f;
            for (int o = 0; o < kNh; ++o) g = fmaf(s2[o], W2[o * kNh + k], g);
            s1[k] *= g;
        }
        __syncthreads();
        // parameter sums over the tile's samples
#pragma unroll
        for (int m = 0; m < kPerThread; ++m) {
            const int p = int(t) + kTile * m;
            if (p >= kNp) break;
            float a = 0.0f;
            if (p < kOffB1) {
                const int o = p / kNin, k = p % kNin;
                for (int q = 0; q < kTile; ++q) a = fmaf(sm.s1[q * kSh + o], sm.x[q * kSx + k], a);
            } else if (p < kOffW2) {
                const int o = p - kOffB1;
                for (int q = 0; q < kTile; ++q) a += sm.s1[q * kSh + o];
            } else if (p < kOffB2) {
                const int o = (p - kOffW2) / kNh, k = (p - kOffW2) % kNh;
                for (int q = 0; q < kTile; ++q) a = fmaf(sm.s2[q * kSh + o], sm.h1[q * kSh + k], a);
            } else if (p < kOffW3) {
                const int o = p - kOffB2;
                for (int q = 0; q < kTile; ++q) a += sm.s2[q * kSh + o];
            } else if (p < kOffB3) {
                const int o = (p - kOffW3) / kNh, k = (p - kOffW3) % kNh;
                for (int q = 0; q < kTile; ++q) a = fmaf(sm.dy[q * kSy + o], sm.h2[q * kSh + k], a);
            } else {
                const int o = p - kOffB3;
                for (int q = 0; q < kTile; ++q) a += sm.dy[q * kSy + o];
            }
            acc[m] += a;
        }
        __syncthreads();
    }
    double *out = partials + size_t(blockIdx.x) * (kNp + 1);
#pragma unroll
    for (int m = 0; m < kPerThread; ++m) {
        const int p = int(t) + kTile * m;
        if (p < kNp) out[p] = double(acc[m]);
    }
    // the loss: a fixed-order block sum
    __shared__ double red[kTile];
    red[t] = loss;
    __syncthreads();
    if (t == 0) {
        double sum = 0.0;
        for (int i = 0; i < kTile; ++i) sum += red[i];
        out[kNp] = sum;
    }
}

// grad[p] = sum over CTAs of partial[cta][p] (p = kNp: the loss sum)
__global__ void k_mlp_reduce(const double *__restrict__ partials, int nblocks, double *__restrict__ grad)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kNp) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[size_t(b) * (kNp + 1) + p];
    grad[p] = s;
}

// Adam (Kingma & Ba 2015) with bias-corrected step size lr_t.
__global__ void k_mlp_adam(float *__restrict__ theta, float *__restrict__ m1, float *__restrict__ m2,
                           const double *__restrict__ grad, float lr_t, float beta1, float beta2, float eps)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kNp) return;
    const float g = float(grad[p]);
    const float a = beta1 * m1[p] + (1.0f - beta1) * g;
    const float b = beta2 * m2[p] + (1.0f - beta2) * g * g;
    m1[p] = a;
    m2[p] = b;
    theta[p] -= lr_t * a / (sqrtf(b) + eps);
}

// Training pairs of cn nodes from FP64 deviations g[27][cn] (SoA, ABI order).
__global__ void k_mlp_pairs(const double *__restrict__ g, uint64_t cn, double rho0, double inv_s_sqrt3,
                            double inv_sig3, float x27, float *__restrict__ X, float *__restrict__ T)
{
    for (uint64_t k = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; k < cn;
         k += uint64_t(gridDim.x) * blockDim.x) {
        double rho = rho0, j[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int i = slot_of(a - 1, b - 1, c - 1);
                    const double d = g[uint64_t(i) * cn + k];
                    rho += d;
                    j[0] += d * (a - 1);
                    j[1] += d * (b - 1);
                    j[2] += d * (c - 1);
                    // x_i = g_i / sqrt(rho0 kT w_i / c_s^2); w_i = w1 w1 w1
                    X[k * 28 + i] = float(d * inv_s_sqrt3 / sqrt(w1(a - 1) * w1(b - 1) * w1(c - 1)));
                }
        X[k * 28 + 27] = x27;
        const double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
        // ghost amplitudes Q = syn_scale * rho u^(deg), zero below order 3
        double q[3][3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    double m = 0.0;
                    if (mode_order(a, b, c) >= 3) {
                        m = rho;
                        for (int e = 0; e < a; ++e) m *= u[0];
                        for (int e = 0; e < b; ++e) m *= u[1];
                        for (int e = 0; e < c; ++e) m *= u[2];
                        m *= syn_scale(a, b, c);
                    }
                    q[a][b][c] = m;
                }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) synthesise(q[a][b][0], q[a][b][1], q[a][b][2]);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) synthesise(q[a][0][c], q[a][1][c], q[a][2][c]);
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) synthesise(q[0][b][c], q[1][b][c], q[2][b][c]);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int i = slot_of(a - 1, b - 1, c - 1);
                    T[k * 27 + i] = float(q[a][b][c] * inv_sig3 / (w1(a - 1) * w1(b - 1) * w1(c - 1)));
                }
    }
}

int grid_for_grad(uint64_t count, int nsm)
{
    const uint64_t tiles = (count + kTile - 1) / kTile;
    return int(std::max<uint64_t>(1, std::min<uint64_t>(tiles, uint64_t(nsm))));
}

struct Scratch {
    double *partials = nullptr;
    double *grad = nullptr;
    float *theta = nullptr, *m1 = nullptr, *m2 = nullptr;
    cudaStream_t s = nullptr;
    ~Scratch()
    {
        if (s) cudaStreamSynchronize(s);
        cudaFree(partials);
        cudaFree(grad);
        cudaFree(theta);
        cudaFree(m1);
        cudaFree(m2);
        if (s) cudaStreamDestroy(s);
    }
};

int fail(const std::string &m, int code)
{
    set_thread_error(m.c_str());
    return code;
}

// Whether p is device (or managed) memory; a host pointer handed to a
// kernel would fault instead of failing.
bool is_device_memory(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int prepare(Scratch &sc, const float *params, int &nsm, bool adam)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sc.s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   int(sizeof(GradSmem)));
    if (e != cudaSuccess) return fail(std::string("mlp: device set-up: ") + cudaGetErrorString(e), FLBM_E_CUDA);
    e = cudaMalloc(&sc.partials, size_t(nsm) * (kNp + 1) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&sc.grad, (kNp + 1) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&sc.theta, kNp * sizeof(float));
    if (e == cudaSuccess && adam) e = cudaMalloc(&sc.m1, kNp * sizeof(float));
    if (e == cudaSuccess && adam) e = cudaMalloc(&sc.m2, kNp * sizeof(float));
    if (e != cudaSuccess) return fail(std::string("mlp: cudaMalloc: ") + cudaGetErrorString(e), FLBM_E_NOMEM);
    e = cudaMemcpyAsync(sc.theta, params, kNp * sizeof(float), cudaMemcpyHostToDevice, sc.s);
    if (e == cudaSuccess && adam) e = cudaMemsetAsync(sc.m1, 0, kNp * sizeof(float), sc.s);
    if (e == cudaSuccess && adam) e = cudaMemsetAsync(sc.m2, 0, kNp * sizeof(float), sc.s);
    if (e != cudaSuccess) return fail(std::string("mlp: upload: ") + cudaGetErrorString(e), FLBM_E_CUDA);
    return FLBM_OK;
}

// gradient (and loss sum) of the samples start .. start + count - 1 of the
// epoch order into sc.grad
cudaError_t launch_grad(Scratch &sc, int nsm, const float *X, const float *T, uint64_t n, uint64_t start,
                        uint64_t count, uint64_t mult, uint64_t off)
{
    const int grid = grid_for_grad(count, nsm);
    const float inv_norm = float(1.0 / (double(count) * kNout));
    k_mlp_grad<<<grid, kTile, sizeof(GradSmem), sc.s>>>(sc.theta, X, T, n, start, count, mult, off, inv_norm,
                                                         sc.partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_mlp_reduce<<<(kNp + 1 + 255) / 256, 256, 0, sc.s>>>(sc.partials, grid, sc.grad);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mlp_pairs(const double *g, uint64_t cn, double rho0, double kT, double omega, float *X,
                             float *T, cudaStream_t s)
{
    const double inv_s_sqrt3 = 1.0 / std::sqrt(rho0 * kT * 3.0);   // 1 / sqrt(rho0 kT / c_s^2)
    const double sig = std::sqrt(kT / rho0);
    const int grid = int(std::min<uint64_t>((cn + 127) / 128, 65535ull * 8));
    k_mlp_pairs<<<std::max(grid, 1), 128, 0, s>>>(g, cn, rho0, inv_s_sqrt3, 1.0 / (sig * sig * sig),
                                                  float(omega - 1.0), X, T);
    return cudaGetLastError();
}

}  // namespace flbm

using namespace flbm;

extern "C" int flbm_mlp_grad(const float *params, const float *dev_x, const float *dev_t, int64_t n, float *grad,
                             double *loss)
{
    if (!params || !dev_x || !dev_t || !grad || n < 1 || n >= (int64_t(1) << 32))
        return fail("flbm_mlp_grad: NULL argument or n outside [1, 2^32)", FLBM_E_INVALID);
    if (!is_device_memory(dev_x) || !is_device_memory(dev_t))
        return fail("flbm_mlp_grad: dev_x and dev_t must be device (or managed) memory", FLBM_E_INVALID);
    Scratch sc;
    int nsm = 0;
    int rc = prepare(sc, params, nsm, false);
    if (rc) return rc;
    cudaError_t e = launch_grad(sc, nsm, dev_x, dev_t, uint64_t(n), 0, uint64_t(n), 1, 0);
    std::vector<double> h(kNp + 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), sc.grad, (kNp + 1) * sizeof(double), cudaMemcpyDeviceToHost, sc.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sc.s);
    if (e != cudaSuccess) return fail(std::string("flbm_mlp_grad: ") + cudaGetErrorString(e), FLBM_E_CUDA);
    for (int p = 0; p < kNp; ++p) grad[p] = float(h[p]);
    if (loss) *loss = h[kNp] / (double(n) * kNout);
    return FLBM_OK;
}

extern "C" int flbm_mlp_train(float *params, const float *dev_x, const float *dev_t, int64_t n, int epochs,
                              int batch, double lr, uint64_t seed, double *epoch_loss)
{
    if (!params || !dev_x || !dev_t || n < 1 || n >= (int64_t(1) << 32) || epochs < 1 || batch < 1 ||
        !(lr > 0.0) || !std::isfinite(lr))
        return fail("flbm_mlp_train: bad argument", FLBM_E_INVALID);
    if (!is_device_memory(dev_x) || !is_device_memory(dev_t))
        return fail("flbm_mlp_train: dev_x and dev_t must be device (or managed) memory", FLBM_E_INVALID);
    Scratch sc;
    int nsm = 0;
    int rc = prepare(sc, params, nsm, true);
    if (rc) return rc;
    const uint64_t N = uint64_t(n);
    const uint64_t B = std::min<uint64_t>(uint64_t(batch), N);
    const uint64_t nb = (N + B - 1) / B;
    const uint64_t total = uint64_t(epochs) * nb;
    std::mt19937_64 rng(seed);
    const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    double p1 = 1.0, p2 = 1.0;
    uint64_t it = 0;
    std::vector<double> losses(size_t(epochs), 0.0);
    double *dloss = nullptr;
    cudaError_t e = cudaMalloc(&dloss, sizeof(double) * size_t(nb));
    if (e != cudaSuccess) return fail(std::string("flbm_mlp_train: cudaMalloc: ") + cudaGetErrorString(e), FLBM_E_NOMEM);
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        // epoch order: an affine bijection of [0, n) with a random multiplier coprime to n
        uint64_t mult = 1, off = 0;
        if (N > 1) {
            do mult = 1 + rng() % (N - 1);
            while (std::gcd(mult, N) != 1);
            off = rng() % N;
        }
        for (uint64_t b = 0; b < nb && e == cudaSuccess; ++b, ++it) {
            const uint64_t start = b * B, count = std::min<uint64_t>(B, N - start);
            e = launch_grad(sc, nsm, dev_x, dev_t, N, start, count, mult, off);
            if (e != cudaSuccess) break;
            e = cudaMemcpyAsync(dloss + b, sc.grad + kNp, sizeof(double), cudaMemcpyDeviceToDevice, sc.s);
            // cosine decay of the step size to 5 % over the run
            const double frac = double(it) / double(std::max<uint64_t>(total - 1, 1));
            const double lr_it = lr * (0.05 + 0.95 * 0.5 * (1.0 + std::cos(3.141592653589793 * frac)));
            p1 *= beta1;
            p2 *= beta2;
            const float lr_t = float(lr_it * std::sqrt(1.0 - p2) / (1.0 - p1));
            k_mlp_adam<<<(kNp + 255) / 256, 256, 0, sc.s>>>(sc.theta, sc.m1, sc.m2, sc.grad, lr_t, beta1, beta2, eps);
            if (e == cudaSuccess) e = cudaGetLastError();
        }
        if (e != cudaSuccess) break;
        std::vector<double> h(nb);
        e = cudaMemcpyAsync(h.data(), dloss, sizeof(double) * nb, cudaMemcpyDeviceToHost, sc.s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(sc.s);
        double sum = 0.0;
        for (double v : h) sum += v;
        losses[size_t(ep)] = sum / (double(N) * kNout);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(params, sc.theta, kNp * sizeof(float), cudaMemcpyDeviceToHost, sc.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sc.s);
    cudaFree(dloss);
    if (e != cudaSuccess) return fail(std::string("flbm_mlp_train: ") + cudaGetErrorString(e), FLBM_E_CUDA);
    if (epoch_loss)
        for (int ep = 0; ep < epochs; ++ep) epoch_loss[ep] = losses[size_t(ep)];
    return FLBM_OK;
}
