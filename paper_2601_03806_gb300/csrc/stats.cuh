// stats.cuh -- accumulation of one reduced step into DevStats (row a9).
#pragma once

#include "internal.h"

namespace flbm {

// red: the NSTAT global sums of one step (StatSlot order) over n nodes.
__device__ __forceinline__ void stats_update(DevStats *st, const double *red, long long step, double n)
{
    for (int s = 0; s < NSTAT; ++s) st->last[s] = red[s];
    for (int a = 0; a < 3; ++a) st->acc_u2[a] += red[S_UX2 + a] / n;
    st->acc_m[0] += red[S_DRHO] / n;
    st->acc_m[1] += (red[S_JX] + red[S_JY] + red[S_JZ]) / n;
    st->acc_m[2] += red[S_M3] / n;
    st->acc_m[3] += red[S_M4] / n;
    for (int k = 0; k < 4; ++k) st->acc_m2[k] += red[S_M1SQ + k] / n;
    st->step = step;
    st->nsamp += 1;
}

}  // namespace flbm
