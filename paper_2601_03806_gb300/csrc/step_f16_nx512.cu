// step_f16_nx512.cu -- the two-node row kernels of the FP16-storage step for rows
// of exactly 512 nodes: the row length is a compile-time constant, so the 27
// segment offsets of a stage are immediates of the shared-memory accesses.
// Bit-identical to the general kernel (same arithmetic, same order).
#include <cuda_fp16.h>

#include "step_kernel.cuh"

namespace flbm {

cudaError_t launch_rows_f16_nx512(void *g, const StepArgs<float> &a, int scheme, bool odd, bool stats,
                                  int row_grid, cudaStream_t s)
{
    return launch_rows_fixed<__half, float, 512>(static_cast<__half *>(g), a, scheme, odd, stats, row_grid, s);
}

int rows_occupancy_f16_nx512(int scheme, bool stats)
{
    return prepare_rows_fixed<__half, float, 512>(scheme, stats);
}

}  // namespace flbm
