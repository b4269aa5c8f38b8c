// mlp_infer.cu -- the learned-collision network on the tensor cores:
// flbm_mlp_infer (network outputs of caller-given features) and the weight
// image the tcgen05 path reads (mlp_tc.cuh).
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/flbm.h"
#include "internal.h"
#include "mlp_tc.cuh"

namespace flbm {

namespace {

// float -> bfloat16, round to nearest, ties to even
uint16_t bf16_rne(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return uint16_t((u >> 16) | 0x40u);   // quiet NaN
    u += 0x7fffu + ((u >> 16) & 1u);
    return uint16_t(u >> 16);
}

float bf16_value(uint16_t h)
{
    const uint32_t u = uint32_t(h) << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// b = hi + mid + lo with bf16 parts, each taken to nearest of what is left
// (8 significant bits a part: together the 24 of an FP32 b), then scaled by
// s, a power of two (exact).
void bias_parts(float b, float s, uint16_t (&out)[3])
{
    float r = b;
    for (int k = 0; k < 3; ++k) {
        const uint16_t h = bf16_rne(r);
        r -= bf16_value(h);   // exact: the rounding error of a representable r
        out[k] = bf16_rne(s * bf16_value(h));
    }
}

void put(std::vector<unsigned char> &img, uint32_t off, uint16_t v) { std::memcpy(&img[off], &v, 2); }

__global__ void __launch_bounds__(kMlpThreads, 1) k_mlp_infer(const float *__restrict__ x, float *__restrict__ y,
                                                   uint64_t n, const unsigned char *__restrict__ img,
                                                   unsigned int *flag)
{
    extern __shared__ __align__(1024) unsigned char smraw[];
    MlpSmem &sm = *reinterpret_cast<MlpSmem *>(smraw);
    mlp_setup(sm, img);
    uint32_t phase = 0;
    const uint64_t ntiles = (n + kMlpThreads - 1) / kMlpThreads;
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t row = tile * kMlpThreads + threadIdx.x;
        float xr[kMlpIn];
#pragma unroll
        for (int i = 0; i < kMlpIn; ++i) xr[i] = row < n ? x[row * kMlpIn + i] : 0.0f;
        float yr[kMlpOut];
        if (!mlp_tile(sm, phase, xr, yr, [] {})) {
            if ((threadIdx.x & 127u) == 0) atomicOr(flag, 2u);   // one report per group
            break;
        }
        if (row < n)
#pragma unroll
            for (int i = 0; i < kMlpOut; ++i) y[row * kMlpOut + i] = yr[i];
    }
    mlp_teardown(sm);
}

}  // namespace

void build_mlp_image(const float *p, std::vector<unsigned char> &img)
{
    img.assign(kMlpImageBytes, 0);
    const float *W1 = p, *b1 = p + 1792, *W2 = p + 1856, *b2 = p + 5952, *W3 = p + 6016, *b3 = p + 7744;
    // layers 1 and 2 halved (a power of two: exact in bf16), layer 3 as is;
    // the bias parts go to K columns 28..30 of W1' and 0..2 of B2' / B3
    for (uint32_t nrow = 0; nrow < 64; ++nrow) {
        uint16_t bp[3];
        bias_parts(b1[nrow], 0.5f, bp);
        for (uint32_t k = 0; k < 32; ++k) {
            const uint16_t v = k < 28 ? bf16_rne(0.5f * W1[nrow * 28 + k]) : (k < 31 ? bp[k - 28] : 0);
            put(img, kW1Off + core_offset(nrow, k, kSbo32), v);
        }
        for (uint32_t k = 0; k < 64; ++k)
            put(img, kW2Off + core_offset(nrow, k, kSbo64), bf16_rne(0.5f * W2[nrow * 64 + k]));
        bias_parts(b2[nrow], 0.5f, bp);
        for (uint32_t k = 0; k < 3; ++k) put(img, kB2Off + core_offset(nrow, k, kSbo16), bp[k]);
    }
    for (uint32_t nrow = 0; nrow < 27; ++nrow) {
        for (uint32_t k = 0; k < 64; ++k) put(img, kW3Off + core_offset(nrow, k, kSbo64), bf16_rne(W3[nrow * 64 + k]));
        uint16_t bp[3];
        bias_parts(b3[nrow], 1.0f, bp);
        for (uint32_t k = 0; k < 3; ++k) put(img, kB3Off + core_offset(nrow, k, kSbo16), bp[k]);
    }
    for (uint32_t row = 0; row < 128; ++row)
        for (uint32_t k = 0; k < 3; ++k) put(img, kOnesOff + core_offset(row, k, kSbo16), bf16_rne(1.0f));
}

}  // namespace flbm

using namespace flbm;

extern "C" int flbm_mlp_infer(const float *params, const float *x, int64_t n, float *y)
{
    if (!params || n < 0 || (n > 0 && (!x || !y))) {
        set_thread_error("flbm_mlp_infer: NULL argument or n < 0");
        return FLBM_E_INVALID;
    }
    if (n == 0) return FLBM_OK;
    std::vector<unsigned char> img;
    build_mlp_image(params, img);
    int dev = 0, nsm = 0;
    unsigned char *dimg = nullptr;
    float *dx = nullptr, *dy = nullptr;
    unsigned int *dflag = nullptr;
    cudaStream_t s = nullptr;
    unsigned int hflag = 0;
    auto done = [&](int code, const char *what, cudaError_t e) {
        if (code != FLBM_OK)
            set_thread_error((std::string("flbm_mlp_infer: ") + what + ": " +
                              (e != cudaSuccess ? cudaGetErrorString(e) : "")).c_str());
        if (s) cudaStreamSynchronize(s);
        cudaFree(dimg);
        cudaFree(dx);
        cudaFree(dy);
        cudaFree(dflag);
        if (s) cudaStreamDestroy(s);
        return code;
    };
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return done(FLBM_E_CUDA, "device", e);
    e = cudaMalloc(&dimg, img.size());
    if (e == cudaSuccess) e = cudaMalloc(&dx, size_t(n) * kMlpIn * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dy, size_t(n) * kMlpOut * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dflag, sizeof(unsigned int));
    if (e != cudaSuccess) return done(FLBM_E_NOMEM, "cudaMalloc", e);
    e = cudaMemcpyAsync(dimg, img.data(), img.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dx, x, size_t(n) * kMlpIn * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dflag, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return done(FLBM_E_CUDA, "upload", e);
    // one CTA per SM (a kernel that allocates tensor memory gets no more)
    const uint64_t ntiles = (uint64_t(n) + kMlpThreads - 1) / kMlpThreads;
    const int grid = int(std::min<uint64_t>(ntiles, uint64_t(nsm)));
    e = cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kMlpSmemBytes));
    if (e != cudaSuccess) return done(FLBM_E_CUDA, "shared-memory attribute", e);
    k_mlp_infer<<<grid, kMlpThreads, kMlpSmemBytes, s>>>(dx, dy, uint64_t(n), dimg, dflag);
    e = cudaGetLastError();
    if (e != cudaSuccess) return done(FLBM_E_CUDA, "launch", e);
    e = cudaMemcpyAsync(y, dy, size_t(n) * kMlpOut * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, dflag, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return done(FLBM_E_CUDA, "run", e);
    if (hflag & 2u) return done(FLBM_E_TIMEOUT, "a bounded tensor-core wait ran out", cudaSuccess);
    return done(FLBM_OK, "", cudaSuccess);
}
