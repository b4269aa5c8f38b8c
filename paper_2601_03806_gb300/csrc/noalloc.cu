// noalloc.cu -- flbm_step_noalloc: one fused step on caller-owned device
// memory with no device allocation at all.
//
// Some callers cannot let a library call cudaMalloc: applications whose
// framework owns every byte of device memory (a pooled or arena allocator
// sized at start-up, a host program embedding this solver as a plug-in under
// a fixed memory budget).  For them this entry point runs the same fused
// stream-and-collide kernels as flbm_step, but all the scratch it needs --
// the per-CTA FP64 partial sums of the reductions and the instability flags
// -- lives in the file-scope array below, which every GPU that loads the
// library holds until the process exits.  The caller passes the population
// state (updated in place) and a device buffer for the reduction results.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/flbm.h"
#include "ctx.h"
#include "internal.h"
#include "lattice.cuh"

namespace flbm {
namespace {

// Scratch capacity: partial sums of at most kNoallocMaxCtas CTAs (13 doubles
// each, 208 KiB) plus 16 bytes of flags, per device.
constexpr int kNoallocMaxCtas = 2048;

struct NoallocScratch {
    double partials[kNoallocMaxCtas * NSTAT];
    unsigned int flag;
    unsigned int pad;
    unsigned long long bad_step;
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
NoallocScratch *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (resolved once
// per device, with that device current, and kept: the library must not be
// used on a device across a cudaDeviceReset, which unloads the module that
// holds the array).
cudaError_t scratch_address(int dev, NoallocScratch **out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<NoallocScratch *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// Fixed-order sum of the per-CTA partials into the caller's 13 doubles.
__global__ void k_noalloc_sums(const NoallocScratch *sc, int nblocks, double *sums)
{
    __shared__ double red[NSTAT][256];
    double loc[NSTAT];
#pragma unroll
    for (int s = 0; s < NSTAT; ++s) loc[s] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int s = 0; s < NSTAT; ++s) loc[s] += sc->partials[size_t(b) * NSTAT + s];
#pragma unroll
    for (int s = 0; s < NSTAT; ++s) red[s][threadIdx.x] = loc[s];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int s = 0; s < NSTAT; ++s) red[s][threadIdx.x] += red[s][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < NSTAT) sums[threadIdx.x] = red[threadIdx.x][0];
}

// Errors are reported through flbm_last_error(NULL), like create-time ones.
int noalloc_fail(int code, const char *msg)
{
    set_thread_error(msg);
    return code;
}

}  // namespace
}  // namespace flbm

using namespace flbm;

extern "C" int flbm_step_noalloc(const flbm_params *p, void *dev_state, int64_t step, int parity,
                                 double *dev_sums, void *cuda_stream)
{
    if (!p || !dev_state || !dev_sums) return noalloc_fail(FLBM_E_INVALID, "NULL argument");
    // every parameter check of flbm_create (box size, finite tau / kT / rho0,
    // noise stream range, ...), then what this entry point adds
    const std::string why = validate_params(p);
    if (!why.empty()) return noalloc_fail(FLBM_E_INVALID, why.c_str());
    if (step < 0 || (parity != 0 && parity != 1))
        return noalloc_fail(FLBM_E_INVALID, "step must be >= 0 and parity 0 or 1");
    if (p->precision != FLBM_FP32)
        return noalloc_fail(FLBM_E_UNSUPPORTED, "flbm_step_noalloc serves FP32 storage only");
    if (p->state_form != FLBM_STATE_POPULATIONS)
        return noalloc_fail(FLBM_E_UNSUPPORTED, "flbm_step_noalloc steps population storage only");
    if (p->scheme == FLBM_LEARNED)
        return noalloc_fail(FLBM_E_UNSUPPORTED, "flbm_step_noalloc runs BGK-, GMF- or Reg-FLBM");
    if (reinterpret_cast<uintptr_t>(dev_state) % 256 != 0)
        return noalloc_fail(FLBM_E_INVALID, "dev_state must be 256-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return noalloc_fail(FLBM_E_CUDA, "no usable CUDA device");
    NoallocScratch *sc = nullptr;
    if (scratch_address(dev, &sc) != cudaSuccess)
        return noalloc_fail(FLBM_E_CUDA, "cudaGetSymbolAddress of the scratch array failed");

    // the launch shape flbm_create picks for this box (step_grids, with the
    // same environment knobs), so the populations and the order of the FP64
    // sums are those of flbm_step + flbm_stats
    const uint64_t n = uint64_t(p->nx) * uint64_t(p->ny) * uint64_t(p->nz);
    const uint64_t nchunks = uint64_t((p->nx + kBlock - 1) / kBlock) * p->ny * p->nz;
    int occ = 1, occ_rows = 0, grid = 0, row_grid = 0;
    step_occupancy_f32(p->scheme, uint32_t(p->nx), n, true, occ, occ_rows);
    step_grids(*p, nsm, occ, occ_rows, grid, row_grid);
    const int used = row_grid > 0 ? row_grid : grid;
    if (used > kNoallocMaxCtas)
        return noalloc_fail(FLBM_E_INVALID,
                            "launch needs more CTA partial slots than the 2048 the scratch array holds");

    // the step's arguments: same mode coefficients and key schedule as flbm_step
    StepArgs<float> a;
    std::memset(&a, 0, sizeof(a));
    a.nx = uint32_t(p->nx);
    a.ny = uint32_t(p->ny);
    a.nz = uint32_t(p->nz);
    a.cpr = uint32_t((p->nx + kBlock - 1) / kBlock);
    a.n = n;
    a.ns = n;   // the caller's state: 27 unpadded slabs
    a.nchunks = nchunks;
    a.step = uint64_t(step);
    fill_step_constants(*p, a);
    a.partials = sc->partials;
    a.flag = &sc->flag;
    a.bad_step = &sc->bad_step;

    // reset what the previous call left behind: the flags start at zero and
    // the first bad step at all-ones (every CTA overwrites its own partials)
    if (cudaMemsetAsync(&sc->flag, 0, 2 * sizeof(unsigned int), s) != cudaSuccess ||
        cudaMemsetAsync(&sc->bad_step, 0xff, sizeof(unsigned long long), s) != cudaSuccess)
        return noalloc_fail(FLBM_E_CUDA, "clearing the scratch flags failed");
    cudaError_t e = launch_step_f32(static_cast<float *>(dev_state), a, p->scheme, parity != 0, true,
                                    grid, row_grid, s);
    if (e == cudaSuccess) {
        k_noalloc_sums<<<1, 256, 0, s>>>(sc, used, dev_sums);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return noalloc_fail(FLBM_E_CUDA, cudaGetErrorString(e));
    unsigned int flag = 0;
    if (cudaMemcpyAsync(&flag, &sc->flag, sizeof(flag), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return noalloc_fail(FLBM_E_CUDA, "reading the step flags failed");
    if (flag & 2u) return noalloc_fail(FLBM_E_TIMEOUT, "a bounded device wait ran out");
    if (flag & 1u) return noalloc_fail(FLBM_E_UNSTABLE, "instability: rho <= 0 or non-finite");
    return FLBM_OK;
}
