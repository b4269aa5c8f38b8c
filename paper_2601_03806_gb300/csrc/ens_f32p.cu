// ens_f32p.cu -- FP32-storage instantiations of the two-node ensemble step
// kernel (adjacent node pairs as packed FP32 lanes).
#include "ens_kernel.cuh"

namespace flbm {

cudaError_t launch_ens_step_f32p(const EnsArgs &a, int scheme, bool odd, bool stats, int grid, int threads,
                                 size_t smem, cudaStream_t s)
{
    return launch_ens_step_t<float, float, 2>(a, scheme, odd, stats, grid, threads, smem, s);
}

int ens_occupancy_f32p(int scheme, int threads, size_t smem)
{
    return ens_occupancy_t<float, float, 2>(scheme, threads, smem);
}

}  // namespace flbm
