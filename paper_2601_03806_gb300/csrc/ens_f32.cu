// ens_f32.cu -- FP32 instantiations of the ensemble step kernel, and the
// post-step kernel (statistics totals, step counter).
#include "ens_kernel.cuh"

namespace flbm {

cudaError_t launch_ens_step_f32(const EnsArgs &a, int scheme, bool odd, bool stats, int grid, int threads,
                                size_t smem, cudaStream_t s, int np)
{
    if (np == 2) return launch_ens_step_f32p(a, scheme, odd, stats, grid, threads, smem, s);
    return launch_ens_step_t<float, float, 1>(a, scheme, odd, stats, grid, threads, smem, s);
}

int ens_occupancy_f32(int scheme, int threads, size_t smem, int np)
{
    if (np == 2) return ens_occupancy_f32p(scheme, threads, smem);
    return ens_occupancy_t<float, float, 1>(scheme, threads, smem);
}

cudaError_t launch_ens_post(const EnsArgs &a, bool stats, uint32_t cwarps, unsigned int *done,
                            unsigned long long *dstep, cudaStream_t s)
{
    if (stats) k_ens_post<true><<<a.nrep, 32, 0, s>>>(a, cwarps, done, dstep);
    else k_ens_post<false><<<1, 32, 0, s>>>(a, cwarps, done, dstep);
    return cudaGetLastError();
}

}  // namespace flbm
