// ens_f16p.cu -- FP16-storage instantiations of the two-node ensemble step
// kernel (adjacent node pairs as packed FP32 lanes).
#include "ens_kernel.cuh"

namespace flbm {

cudaError_t launch_ens_step_f16p(const EnsArgs &a, int scheme, bool odd, bool stats, int grid, int threads,
                                 size_t smem, cudaStream_t s)
{
    return launch_ens_step_t<__half, float, 2>(a, scheme, odd, stats, grid, threads, smem, s);
}

int ens_occupancy_f16p(int scheme, int threads, size_t smem)
{
    return ens_occupancy_t<__half, float, 2>(scheme, threads, smem);
}

}  // namespace flbm
