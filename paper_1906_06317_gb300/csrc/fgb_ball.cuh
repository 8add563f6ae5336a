// Ball-query candidate walk shared by the neighbor-list build and the fused Steinhardt
// forward pass.
#pragma once

#include "fgb_device.cuh"

namespace fgb {

struct BallArgs {
    Stencil S;
    BoxF bf;
    BoxD bd;
    const float4 *pts;          // sorted points (cell-local xyz, index bits)
    const uint32_t *cell_start;
    const float4 *qs;           // sorted query points
    const uint32_t *qcell;
    int64_t nq;
    const float *p_orig;        // (n,3) caller coordinates
    const float *q_orig;        // (nq,3)
    Band band;                  // FP32 band around T
    double T;                   // r < r_max  <=>  r2 < T (exact)
    int exclude;                // exclude_ii
    unsigned long long *esc;    // FP64 re-decisions
    int *err;                   // internal consistency flag
};

// Visits every neighbor (exactly decided) of one sorted query: fn(j, d, r2f, e) with the
// FP32 displacement d, its FP32 r2 and the FP64 r2 when the pair was re-decided (else -1).
template <class F>
__device__ __forceinline__ int ball_visit(const BallArgs &a, float4 q, uint32_t qc, int i, F &&fn) {
    int cx, cy, cz;
    cell_coords(qc, a.S.nc, cx, cy, cz);
    const int excl = a.exclude ? i : -1;
    int nesc = 0;
    for_stencil(a.S, cx, cy, cz, make_float3(q.x, q.y, q.z), false,
                [&](int cell, float qx, float qy, float qz, bool) {
                    const uint32_t beg = __ldg(a.cell_start + cell), end = __ldg(a.cell_start + cell + 1);
                    for (uint32_t p = beg; p < end; ++p) {
                        const float4 c = __ldg(a.pts + p);
                        const float3 d = cand_disp(a.S, a.bf, c, qx, qy, qz);
                        const float r2 = r2_f32(d.x, d.y, d.z);
                        if (r2 < a.band.hi) {
                            const int j = __float_as_int(c.w);
                            if (j == excl) continue;
                            if (r2 < a.band.lo) {
                                fn(j, d, r2, -1.0);
                            } else {
                                const double e = exact_r2_idx(a.bd, a.q_orig, i, a.p_orig, j);
                                ++nesc;
                                if (e < a.T) fn(j, d, r2, e);
                            }
                        }
                    }
                });
    return nesc;
}

}  // namespace fgb
