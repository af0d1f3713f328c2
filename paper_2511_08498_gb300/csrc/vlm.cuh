// Index-of-dispersion test of one 2x2 (2D) or 2x2x2 (3D) group of children
// (Section 2.2, Eq. IoD), shared by the static, Core-and-Voigt and 3D MIP builds.
#pragma once

#include "dex_internal.h"

namespace dex {

struct GroupStat {
    float val;
    float iod;
};

// value and IoD of a 2x2 group at voxel side ds (ln_ds = ln ds)
__device__ __forceinline__ GroupStat reduce_group(float g0, float g1, float g2, float g3, float ln_ds, bool log_mean)
{
    GroupStat r;
    const int npos = (g0 > 0.0f) + (g1 > 0.0f) + (g2 > 0.0f) + (g3 > 0.0f);
    const float lin = 0.25f * ((g0 + g1) + (g2 + g3));
    if (npos == 4) {
        const float L0 = logf(g0), L1 = logf(g1), L2 = logf(g2), L3 = logf(g3);
        const float mL = 0.25f * ((L0 + L1) + (L2 + L3));
        const float mu = mL + ln_ds;
        const float d0 = L0 - mL, d1 = L1 - mL, d2 = L2 - mL, d3 = L3 - mL;
        const float var = 0.25f * ((d0 * d0 + d1 * d1) + (d2 * d2 + d3 * d3));
        r.iod = var == 0.0f ? 0.0f : fabsf(var / mu);
        r.val = log_mean ? expf(mL) : lin;
    } else if (npos == 0) {
        r.iod = 0.0f;
        r.val = 0.0f;
    } else {
        r.iod = __int_as_float(0x7f800000);
        r.val = lin;
    }
    return r;
}

// value and IoD of a 2x2x2 group g[8] at voxel side ds (ln_ds = ln ds); the same
// rules as reduce_group, sums taken as a balanced tree
__device__ __forceinline__ GroupStat reduce_group8(const float* g, float ln_ds, bool log_mean)
{
    GroupStat r;
    int npos = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) npos += g[q] > 0.0f;
    const float lin = 0.125f * (((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])));
    if (npos == 8) {
        float L[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) L[q] = logf(g[q]);
        const float mL = 0.125f * (((L[0] + L[1]) + (L[2] + L[3])) + ((L[4] + L[5]) + (L[6] + L[7])));
        float d2[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) d2[q] = (L[q] - mL) * (L[q] - mL);
        const float var = 0.125f * (((d2[0] + d2[1]) + (d2[2] + d2[3])) + ((d2[4] + d2[5]) + (d2[6] + d2[7])));
        const float mu = mL + ln_ds;
        r.iod = var == 0.0f ? 0.0f : fabsf(var / mu);
        r.val = log_mean ? expf(mL) : lin;
    } else if (npos == 0) {
        r.iod = 0.0f;
        r.val = 0.0f;
    } else {
        r.iod = __int_as_float(0x7f800000);
        r.val = lin;
    }
    return r;
}

}  // namespace dex
