// step_f32.cu -- FP32 instantiations of the fused step kernel (throughput
// path: float deviations, float arithmetic, FP64 only in the reductions).
#include "step_kernel.cuh"

namespace flbm {

cudaError_t launch_step_f32(float *g, const StepArgs<float> &a, int scheme, bool odd, bool stats,
                            int grid, cudaStream_t s)
{
    return launch_step_t<float, float>(g, a, scheme, odd, stats, grid, s);
}

int step_occupancy_f32(int scheme, bool stats) { return step_occupancy_t<float, float>(scheme, stats); }

}  // namespace flbm
