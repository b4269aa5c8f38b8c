// step_f64.cu -- FP64 instantiations of the fused step kernels (parity path:
// double deviations, double arithmetic, double-precision log/sqrt/sincospi).
#include "step_kernel.cuh"

namespace flbm {

cudaError_t launch_step_f64(double *g, const StepArgs<double> &a, int scheme, bool odd, bool stats,
                            int grid, int row_grid, cudaStream_t s)
{
    return launch_step_t<double, double, uint64_t>(g, a, scheme, odd, stats, grid, row_grid, s);
}

void step_occupancy_f64(int scheme, uint32_t nx, bool stats, int &direct, int &rows)
{
    step_occupancy_t<double, double, uint64_t>(scheme, nx, stats, direct, rows);
}

}  // namespace flbm
