// step_f64.cu -- FP64 instantiations of the fused step kernel (parity path:
// double deviations, double arithmetic, double-precision log/sqrt/sincospi).
#include "step_kernel.cuh"

namespace flbm {

cudaError_t launch_step_f64(double *g, const StepArgs<double> &a, int scheme, bool odd, bool stats,
                            int grid, cudaStream_t s)
{
    return launch_step_t<double, double>(g, a, scheme, odd, stats, grid, s);
}

int step_occupancy_f64(int scheme, bool stats) { return step_occupancy_t<double, double>(scheme, stats); }

}  // namespace flbm
