// Device-side helpers shared by the kernels: the exact FP64 pair sequence, FP32
// minimum image, and the stencil description of a cell-list query.
#pragma once

#include "fgb_internal.cuh"

namespace fgb {

constexpr float kU32 = 5.9604644775390625e-8f;  // 2^-24, unit roundoff of float32

// n = rint(d / L).  The product with 1/L differs from the IEEE quotient by a few ulps,
// so when it sits clear of a half-integer both round to the same integer; otherwise the
// IEEE division is taken.  Either way n equals rint of the correctly rounded quotient.
__device__ __forceinline__ double rint_quot(double d, double L, double invL) {
    double q = __dmul_rn(d, invL);
    double n = rint(q);
    if (fabs(__dsub_rn(q, n)) > 0.49) n = rint(__ddiv_rn(d, L));
    return n;
}

// r^2 of the minimum-image displacement x_j - x_i by the defining FP64 sequence:
// reduce along a3, then a2, then a1; r2 = (dx*dx + dy*dy) + dz*dz; every operation
// rounded separately (no fused multiply-add).  A step with n = 0 is skipped, which
// leaves every value unchanged.
__device__ __forceinline__ double exact_r2(const BoxD &b, float xi0, float xi1, float xi2, float xj0, float xj1,
                                           float xj2) {
    double dx = __dsub_rn((double)xj0, (double)xi0);
    double dy = __dsub_rn((double)xj1, (double)xi1);
    double dz = __dsub_rn((double)xj2, (double)xi2);
    double nz = rint_quot(dz, b.L[2], b.invL[2]);
    if (nz != 0.0) {
        dx = __dsub_rn(dx, __dmul_rn(nz, b.a3x));
        dy = __dsub_rn(dy, __dmul_rn(nz, b.a3y));
        dz = __dsub_rn(dz, __dmul_rn(nz, b.L[2]));
    }
    double ny = rint_quot(dy, b.L[1], b.invL[1]);
    if (ny != 0.0) {
        dx = __dsub_rn(dx, __dmul_rn(ny, b.a2x));
        dy = __dsub_rn(dy, __dmul_rn(ny, b.L[1]));
    }
    double nx = rint_quot(dx, b.L[0], b.invL[0]);
    if (nx != 0.0) dx = __dsub_rn(dx, __dmul_rn(nx, b.L[0]));
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

__device__ __forceinline__ double exact_r2_idx(const BoxD &b, const float *xi_arr, int64_t i, const float *xj_arr,
                                               int64_t j) {
    return exact_r2(b, __ldg(xi_arr + 3 * i), __ldg(xi_arr + 3 * i + 1), __ldg(xi_arr + 3 * i + 2),
                    __ldg(xj_arr + 3 * j), __ldg(xj_arr + 3 * j + 1), __ldg(xj_arr + 3 * j + 2));
}

// FP32 minimum image with box vectors split hi+lo (accurate to a few ulps of |d|).
__device__ __forceinline__ float3 min_image_f32(const BoxF &b, float3 d) {
    float nz = rintf(d.z * b.invL[2]);
    d.x = fmaf(-nz, b.a3x_hi, d.x);
    d.x = fmaf(-nz, b.a3x_lo, d.x);
    d.y = fmaf(-nz, b.a3y_hi, d.y);
    d.y = fmaf(-nz, b.a3y_lo, d.y);
    d.z = fmaf(-nz, b.Lhi[2], d.z);
    d.z = fmaf(-nz, b.Llo[2], d.z);
    float ny = rintf(d.y * b.invL[1]);
    d.x = fmaf(-ny, b.a2x_hi, d.x);
    d.x = fmaf(-ny, b.a2x_lo, d.x);
    d.y = fmaf(-ny, b.Lhi[1], d.y);
    d.y = fmaf(-ny, b.Llo[1], d.y);
    float nx = rintf(d.x * b.invL[0]);
    d.x = fmaf(-nx, b.Lhi[0], d.x);
    d.x = fmaf(-nx, b.Llo[0], d.x);
    return d;
}

__device__ __forceinline__ float r2_f32(float dx, float dy, float dz) {
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// Pair decision bands: r2 < lo is certainly inside the edge, r2 >= hi certainly outside;
// anything between goes to exact_r2.
struct Band {
    float lo, hi;
};

// How a query enumerates candidate cells.
//  mode 0 (shift): every axis has 2s+1 <= nc, so each stencil offset o names a distinct
//    cell and the image of its points is fixed: d = local_j - (local_i - OFF[o]),
//    OFF[o] = M (o / nc) rounded once from FP64.
//  mode 1 (general): an axis with 2s+1 > nc is scanned whole once; the offset is built
//    per cell from the steps a_k / nc_k and each candidate is reduced by rint.
struct Stencil {
    int nc[3];
    int s[3];          // half-width of the stencil walked
    int ts[3];         // half-width the offset table was built for (>= s in mode 0)
    int full[3];       // axis scanned whole (mode 1)
    int mode;
    const float4 *off; // mode 0 offsets, index ((oz+s2)*(2 s1+1) + (oy+s1))*(2 s0+1) + (ox+s0)
    float3 step[3];    // a_k / nc_k (mode 1)
};

__device__ __forceinline__ void cell_coords(uint32_t c, const int *nc, int &cx, int &cy, int &cz) {
    cx = (int)(c % (uint32_t)nc[0]);
    uint32_t r = c / (uint32_t)nc[0];
    cy = (int)(r % (uint32_t)nc[1]);
    cz = (int)(r / (uint32_t)nc[1]);
}

__device__ __forceinline__ int wrap_cell(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Visits every candidate cell of a query in cell (cx, cy, cz) with local coordinate ql.
// fn(cell, qx, qy, qz) receives the query position shifted into the frame of that cell's
// points (mode 0) or the general offset frame (mode 1).  half != 0 keeps only offsets
// lexicographically after (0,0,0) plus the own cell (mode 0 only).
template <class F>
__device__ __forceinline__ void for_stencil(const Stencil &S, int cx, int cy, int cz, float3 ql, bool half, F &&fn) {
    if (S.mode == 0) {
        const int wx = 2 * S.ts[0] + 1, wy = 2 * S.ts[1] + 1;
        const int oz0 = half ? 0 : -S.s[2];
        for (int oz = oz0; oz <= S.s[2]; ++oz) {
            const int zz = wrap_cell(cz + oz, S.nc[2]);
            const int oy0 = (half && oz == 0) ? 0 : -S.s[1];
            for (int oy = oy0; oy <= S.s[1]; ++oy) {
                const int yy = wrap_cell(cy + oy, S.nc[1]);
                const int base = (zz * S.nc[1] + yy) * S.nc[0];
                const int ox0 = (half && oz == 0 && oy == 0) ? 0 : -S.s[0];
                const float4 *orow = S.off + ((oz + S.ts[2]) * wy + (oy + S.ts[1])) * wx + S.ts[0];
                for (int ox = ox0; ox <= S.s[0]; ++ox) {
                    const int xx = wrap_cell(cx + ox, S.nc[0]);
                    const float4 o = __ldg(orow + ox);
                    fn(base + xx, ql.x - o.x, ql.y - o.y, ql.z - o.z, oz == 0 && oy == 0 && ox == 0);
                }
            }
        }
    } else {
        int lo[3], hi[3], c[3] = {cx, cy, cz};
        for (int k = 0; k < 3; ++k) {
            lo[k] = S.full[k] ? -c[k] : -S.s[k];
            hi[k] = S.full[k] ? S.nc[k] - 1 - c[k] : S.s[k];
        }
        for (int oz = lo[2]; oz <= hi[2]; ++oz) {
            const int zz = wrap_cell(cz + oz, S.nc[2]);
            for (int oy = lo[1]; oy <= hi[1]; ++oy) {
                const int yy = wrap_cell(cy + oy, S.nc[1]);
                const int base = (zz * S.nc[1] + yy) * S.nc[0];
                for (int ox = lo[0]; ox <= hi[0]; ++ox) {
                    const int xx = wrap_cell(cx + ox, S.nc[0]);
                    const float fx = (float)ox, fy = (float)oy, fz = (float)oz;
                    const float offx = fmaf(fz, S.step[2].x, fmaf(fy, S.step[1].x, fx * S.step[0].x));
                    const float offy = fmaf(fz, S.step[2].y, fy * S.step[1].y);
                    const float offz = fz * S.step[2].z;
                    fn(base + xx, ql.x - offx, ql.y - offy, ql.z - offz, oz == 0 && oy == 0 && ox == 0);
                }
            }
        }
    }
}

// Displacement from the shifted query to a candidate (cell-local coordinates).
__device__ __forceinline__ float3 cand_disp(const Stencil &S, const BoxF &bf, float4 c, float qx, float qy,
                                            float qz) {
    float3 d = make_float3(c.x - qx, c.y - qy, c.z - qz);
    if (S.mode != 0) d = min_image_f32(bf, d);
    return d;
}

Stencil to_device(const fgb_nq *nq, const StencilPlan &p);

}  // namespace fgb
