// step_f32.cu -- FP32 instantiations of the fused step kernels (throughput
// path: float deviations, float arithmetic, FP64 only in the reductions).
// The direct kernel uses 32-bit node offsets when every population index
// fits (27 N < 2^32, e.g. up to 539^3), 64-bit otherwise.
#include "step_kernel.cuh"

namespace flbm {

static bool fits32(uint64_t n) { return n * kQ < (1ull << 32); }

cudaError_t launch_step_f32(float *g, const StepArgs<float> &a, int scheme, bool odd, bool stats,
                            int grid, int row_grid, cudaStream_t s)
{
    if (row_grid > 0 && rows_paced<float>(row_plan<float>(a.nx)))
        return launch_rows_f32_paced(g, a, scheme, odd, stats, row_grid, s);
    if (fits32(a.ns))
        return launch_step_t<float, float, uint32_t>(g, a, scheme, odd, stats, grid, row_grid, s);
    return launch_step_t<float, float, uint64_t>(g, a, scheme, odd, stats, grid, row_grid, s);
}

void step_occupancy_f32(int scheme, uint32_t nx, uint64_t ns, bool stats, int &direct, int &rows)
{
    if (fits32(ns)) step_occupancy_t<float, float, uint32_t>(scheme, nx, stats, direct, rows);
    else step_occupancy_t<float, float, uint64_t>(scheme, nx, stats, direct, rows);
    if (rows > 0 && rows_paced<float>(row_plan<float>(nx))) rows = rows_occupancy_f32_paced(scheme, stats, nx);
}

}  // namespace flbm
