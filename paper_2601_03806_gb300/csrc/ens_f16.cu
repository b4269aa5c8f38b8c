// ens_f16.cu -- FP16-storage instantiations of the ensemble step kernel
// (half deviations, FP32 arithmetic).
#include "ens_kernel.cuh"

namespace flbm {

cudaError_t launch_ens_step_f16(const EnsArgs &a, int scheme, bool odd, bool stats, int grid, int threads,
                                size_t smem, cudaStream_t s, int np)
{
    if (np == 2) return launch_ens_step_f16p(a, scheme, odd, stats, grid, threads, smem, s);
    return launch_ens_step_t<__half, float, 1>(a, scheme, odd, stats, grid, threads, smem, s);
}

int ens_occupancy_f16(int scheme, int threads, size_t smem, int np)
{
    if (np == 2) return ens_occupancy_f16p(scheme, threads, smem);
    return ens_occupancy_t<__half, float, 1>(scheme, threads, smem);
}

}  // namespace flbm
