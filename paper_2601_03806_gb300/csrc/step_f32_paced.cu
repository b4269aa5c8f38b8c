// step_f32_paced.cu -- the PACED two-node row kernels of the FP32 step: rows
// staged twice (288-512 nodes), whose copy warp derives each address from the
// row index instead of walking the rows (see k_step_rows).  Bit-identical to
// the walking kernel: the same rows, copies and arithmetic.
#include "step_kernel.cuh"

namespace flbm {

cudaError_t launch_rows_f32_paced(float *g, const StepArgs<float> &a, int scheme, bool odd, bool stats,
                                  int row_grid, cudaStream_t s)
{
    return launch_rows_fixed<float, float, 0, true>(g, a, scheme, odd, stats, row_grid, s);
}

int rows_occupancy_f32_paced(int scheme, bool stats, uint32_t nx)
{
    return prepare_rows_fixed<float, float, 0, true>(scheme, stats, nx);
}

}  // namespace flbm
