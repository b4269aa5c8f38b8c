// step_f16.cu -- FP16-storage instantiations of the fused step kernels:
// half-precision deviations g_i = f_i - w_i rho0 in HBM (108 B per lattice
// update instead of 216 B), FP32 arithmetic, FP64 reductions.
#include <cuda_fp16.h>

#include "step_kernel.cuh"

namespace flbm {

static bool fits32(uint64_t n) { return n * kQ < (1ull << 32); }

cudaError_t launch_step_f16(void *g, const StepArgs<float> &a, int scheme, bool odd, bool stats,
                            int grid, int row_grid, cudaStream_t s)
{
    __half *h = static_cast<__half *>(g);
    if (row_grid > 0 && rows_fixed<512>(row_plan<__half>(a.nx), a.nx))
        return launch_rows_f16_nx512(g, a, scheme, odd, stats, row_grid, s);
    if (fits32(a.ns))
        return launch_step_t<__half, float, uint32_t>(h, a, scheme, odd, stats, grid, row_grid, s);
    return launch_step_t<__half, float, uint64_t>(h, a, scheme, odd, stats, grid, row_grid, s);
}

void step_occupancy_f16(int scheme, uint32_t nx, uint64_t ns, bool stats, int &direct, int &rows)
{
    if (fits32(ns)) step_occupancy_t<__half, float, uint32_t>(scheme, nx, stats, direct, rows);
    else step_occupancy_t<__half, float, uint64_t>(scheme, nx, stats, direct, rows);
    if (rows > 0 && rows_fixed<512>(row_plan<__half>(nx), nx)) rows = rows_occupancy_f16_nx512(scheme, stats);
}

}  // namespace flbm
