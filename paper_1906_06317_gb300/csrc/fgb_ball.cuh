// Ball-query candidate walk shared by the neighbor-list build, the fused Steinhardt
// forward pass and the batched kernel.
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
    int self;                   // query points are the points (the self pair has d = 0 exactly)
    unsigned long long *esc;    // FP64 re-decisions
    int *err;                   // internal consistency flag
};

template <int MODE>
__device__ __forceinline__ float3 cand_disp_m(const BoxF &bf, float4 c, float qx, float qy, float qz) {
    float3 d = make_float3(c.x - qx, c.y - qy, c.z - qz);
    if (MODE != 0) d = min_image_f32(bf, d);
    return d;
}

// Number of neighbors of one sorted query (exact), and the FP64 re-decisions it took.
// CHECKJ: test the excluded index on every certain hit (queries that are not the points
// themselves); otherwise the self pair, found once with d = 0, is subtracted at the end.
template <int MODE, bool CHECKJ>
__device__ __forceinline__ uint32_t ball_count_walk(const BallArgs &a, float4 q, uint32_t qc, int i, int &nesc) {
    int cx, cy, cz;
    cell_coords(qc, a.S.nc, cx, cy, cz);
    const int excl = a.exclude ? i : -1;
    const float lo = a.band.lo, hi = a.band.hi;
    uint32_t cnt = 0;
    for_stencil(a.S, cx, cy, cz, make_float3(q.x, q.y, q.z), false,
                [&](int cell, float qx, float qy, float qz, bool) {
                    const uint32_t beg = __ldg(a.cell_start + cell), end = __ldg(a.cell_start + cell + 1);
#pragma unroll 2
                    for (uint32_t p = beg; p < end; ++p) {
                        const float4 c = __ldg(a.pts + p);
                        const float3 d = cand_disp_m<MODE>(a.bf, c, qx, qy, qz);
                        const float r2 = r2_f32(d.x, d.y, d.z);
                        if (CHECKJ)
                            cnt += (r2 < lo && __float_as_int(c.w) != excl) ? 1u : 0u;
                        else
                            cnt += r2 < lo ? 1u : 0u;
                        if (r2 >= lo && r2 < hi) {
                            const int j = __float_as_int(c.w);
                            if (j != excl) {
                                ++nesc;
                                cnt += exact_r2_idx(a.bd, a.q_orig, i, a.p_orig, j) < a.T ? 1u : 0u;
                            }
                        }
                    }
                });
    if (!CHECKJ && a.exclude && lo > 0.f) --cnt;  // the self pair (r2 = 0 < lo) was counted
    return cnt;
}

// Visits every neighbor (exactly decided) of one sorted query: fn(j, d, r2f, e) with the
// FP32 displacement d, its FP32 r2 and the FP64 r2 when the pair was re-decided (else -1).
template <int MODE, class F>
__device__ __forceinline__ int ball_visit_m(const BallArgs &a, float4 q, uint32_t qc, int i, F &&fn) {
    int cx, cy, cz;
    cell_coords(qc, a.S.nc, cx, cy, cz);
    const int excl = a.exclude ? i : -1;
    const float lo = a.band.lo, hi = a.band.hi;
    int nesc = 0;
    for_stencil(a.S, cx, cy, cz, make_float3(q.x, q.y, q.z), false,
                [&](int cell, float qx, float qy, float qz, bool) {
                    const uint32_t beg = __ldg(a.cell_start + cell), end = __ldg(a.cell_start + cell + 1);
#pragma unroll 2
                    for (uint32_t p = beg; p < end; ++p) {
                        const float4 c = __ldg(a.pts + p);
                        const float3 d = cand_disp_m<MODE>(a.bf, c, qx, qy, qz);
                        const float r2 = r2_f32(d.x, d.y, d.z);
                        if (r2 < hi) {
                            const int j = __float_as_int(c.w);
                            if (j == excl) continue;
                            if (r2 < lo) {
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

template <class F>
__device__ __forceinline__ int ball_visit(const BallArgs &a, float4 q, uint32_t qc, int i, F &&fn) {
    if (a.S.mode == 0) return ball_visit_m<0>(a, q, qc, i, fn);
    return ball_visit_m<1>(a, q, qc, i, fn);
}

}  // namespace fgb
