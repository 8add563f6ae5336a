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

// The minimum-image displacement x_j - x_i itself, by the same FP64 sequence as exact_r2.
__device__ __forceinline__ double3 exact_disp(const BoxD &b, const float *xi, const float *xj) {
    double dx = __dsub_rn((double)__ldg(xj), (double)__ldg(xi));
    double dy = __dsub_rn((double)__ldg(xj + 1), (double)__ldg(xi + 1));
    double dz = __dsub_rn((double)__ldg(xj + 2), (double)__ldg(xi + 2));
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
    return make_double3(dx, dy, dz);
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

// Bond vector x_j - x_i under the minimum image in FP32.  When no image shift is needed
// the plain difference is already accurate (|d| is a bond length); otherwise the
// difference and the shifts are carried as hi + lo pairs so the large intermediate
// values lose nothing.
__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void ds_sub_shift(float &h, float &l, float n, float ahi, float alo) {
    float s, e;
    // n is a small integer: n * ahi is formed exactly through its error term
    const float p = __fmul_rn(n, ahi);
    const float pe = __fmaf_rn(n, ahi, -p);
    two_sum_f(h, -p, s, e);
    h = s;
    l = __fadd_rn(l, __fsub_rn(__fsub_rn(e, pe), __fmul_rn(n, alo)));
}

__device__ __forceinline__ float3 bond_f32v(const BoxF &b, float xi0, float xi1, float xi2, float xj0, float xj1,
                                            float xj2) {
    float3 d = make_float3(xj0 - xi0, xj1 - xi1, xj2 - xi2);
    const float nz = rintf(d.z * b.invL[2]);
    const float ny = rintf((d.y - nz * b.a3y) * b.invL[1]);
    const float nx = rintf((d.x - nz * b.a3x - ny * b.a2x) * b.invL[0]);
    if (nz == 0.f && ny == 0.f && nx == 0.f) return d;
    float hx, lx, hy, ly, hz, lz;
    two_sum_f(xj0, -xi0, hx, lx);
    two_sum_f(xj1, -xi1, hy, ly);
    two_sum_f(xj2, -xi2, hz, lz);
    ds_sub_shift(hx, lx, nz, b.a3x_hi, b.a3x_lo);
    ds_sub_shift(hy, ly, nz, b.a3y_hi, b.a3y_lo);
    ds_sub_shift(hz, lz, nz, b.Lhi[2], b.Llo[2]);
    ds_sub_shift(hx, lx, ny, b.a2x_hi, b.a2x_lo);
    ds_sub_shift(hy, ly, ny, b.Lhi[1], b.Llo[1]);
    ds_sub_shift(hx, lx, nx, b.Lhi[0], b.Llo[0]);
    return make_float3(hx + lx, hy + ly, hz + lz);
}

__device__ __forceinline__ float3 bond_f32(const BoxF &b, const float *x, int64_t i, int64_t j) {
    return bond_f32v(b, __ldg(x + 3 * i), __ldg(x + 3 * i + 1), __ldg(x + 3 * i + 2), __ldg(x + 3 * j),
                     __ldg(x + 3 * j + 1), __ldg(x + 3 * j + 2));
}

// 1/sqrt(x) by the hardware approximation (PTX rsqrt.approx, relative error below
// 2^-22), with subnormal inputs taken as zero: skips the subnormal rescaling that the
// non-ftz form adds.  Callers only pass r2 > 0 of pairs that matter or test the result.
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float r2_f32(float dx, float dy, float dz) {
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// Top-KT list by (r2, index), kept sorted in registers (kNN kernels).
template <int KT>
__device__ __forceinline__ void topk_insert(float (&br)[KT], int (&bj)[KT], float r2, int j) {
    float cr = r2;
    int cj = j;
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        const bool less = cr < br[q] || (cr == br[q] && cj < bj[q]);
        const float tr = less ? br[q] : cr;
        const int tj = less ? bj[q] : cj;
        br[q] = less ? cr : br[q];
        bj[q] = less ? cj : bj[q];
        cr = tr;
        cj = tj;
    }
}

// a[idx] for a runtime idx without dynamic register indexing (keeps the list in registers)
template <int KT, class T>
__device__ __forceinline__ T pick(const T (&v)[KT], int idx) {
    T out = v[0];
#pragma unroll
    for (int q = 1; q < KT; ++q)
        if (q == idx) out = v[q];
    return out;
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

// ------------------------------------------------------------------ RDF binning

// Bin of one pair for the RDF.  The fast test places x = (r - r_min)/Delta from the FP32
// r and accepts bin floor(x) when x sits further than e from both edges, with
//   e = g2h / r + 8u (bins + r_min/Delta + 2)  (x < bins + 1 wherever it matters),
// g2h = 0.55 G2 / Delta bounding the shift of x caused by an r2 error of at most G2
// (valid once r2 > 16 G2), the 8u term covering rsqrt, the product with 1/Delta and the
// FP64 edge positions.  Otherwise the FP32 bands around the exact edge thresholds decide,
// and pairs inside a band are left to the FP64 sequence.
struct BinParams {
    int bins;
    float rmin, invdelta, rmin_invdelta, g2h, r2_fast;  // r2_fast = 16 G2
    float eps;                                            // 8u (bins + r_min/Delta + 2)
    float rmax_hi, rmin_lo;                               // bands of the outer edges
    const float2 *band;                                   // (bins+1) bands [lo, hi)
};

// Bin of an in-range pair from the FP32 bands around the exact edge thresholds (the
// fast test of rdf_bin failed): >= 0 the bin, -2 decide in FP64.
__device__ __forceinline__ int rdf_bin_band(const BinParams &P, float r2) {
    const float r = r2 > 0.f ? r2 * rsqrtf(r2) : 0.f;
    int b = (int)((r - P.rmin) * P.invdelta);
    b = min(max(b, 0), P.bins - 1);
    float2 e0 = __ldg(P.band + b), e1 = __ldg(P.band + b + 1);
    if (r2 < e0.x && b > 0) {
        --b;
        e1 = e0;
        e0 = __ldg(P.band + b);
    } else if (r2 >= e1.y && b + 1 < P.bins) {
        ++b;
        e0 = e1;
        e1 = __ldg(P.band + b + 1);
    }
    if (r2 >= e0.y && r2 < e1.x) return b;
    return -2;
}

// >= 0: the bin; -1: certainly outside [r_min, r_max); -2: decide in FP64.
// The fast test needs neither 0 <= b nor b < bins: an x just outside [0, bins) lies
// within e of an edge and fails it.
__device__ __forceinline__ int rdf_bin(const BinParams &P, float r2) {
    if (r2 >= P.rmax_hi || r2 < P.rmin_lo) return -1;
    const float inv = rsqrtf(r2);
    const float x = fmaf(r2 * inv, P.invdelta, -P.rmin_invdelta);
    const float fb = floorf(x);
    const float e = fmaf(P.g2h, inv, P.eps);
    if (r2 > P.r2_fast && fabsf((x - fb) - 0.5f) < 0.5f - e) return (int)fb;
    return rdf_bin_band(P, r2);
}
Stencil to_device(const BoxHost &b, const GridHost &g, const StencilPlan &p, const float4 *table);

// ------------------------------------------------------------------ binning

struct GridDev {
    int nc[3];
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Sum of three hi/lo pairs, returned as hi + lo.
__device__ __forceinline__ float2 ds_sum3(float2 a, float2 b, float2 c) {
    float s1, e1, s2, e2;
    two_sum(a.x, b.x, s1, e1);
    two_sum(s1, c.x, s2, e2);
    float lo = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(__fadd_rn(a.y, b.y), c.y));
    float hi = __fadd_rn(s2, lo);
    lo = __fsub_rn(lo, __fsub_rn(hi, s2));
    return make_float2(hi, lo);
}

// Cell and cell-local coordinate of one point.  The fractional coordinate is formed in
// FP32 (it only selects a cell; the stencil margin absorbs its rounding).  The local
// coordinate x - M (n + c/nc - 1/2) is formed from hi/lo origin tables, so its error is a
// few ulps of the cell size rather than of the box size.  Points more than a few box
// lengths away, or outside the primary box, take an FP64 route.
__device__ __forceinline__ void bin_point(const BoxF &b, const BoxD &bd, const GridDev &g, const OriginTables &org,
                                          float x, float y, float z, uint32_t &key, float4 &loc) {
    float s[3];
    s[2] = __fmaf_rn(z, b.inv22, 0.5f);
    s[1] = __fmaf_rn(z, b.inv12, __fmaf_rn(y, b.inv11, 0.5f));
    s[0] = __fmaf_rn(z, b.inv02, __fmaf_rn(y, b.inv01, __fmaf_rn(x, b.inv00, 0.5f)));
    int c[3];
    bool inbox = true;
    float n[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        n[k] = floorf(s[k]);
        float f = __fsub_rn(s[k], n[k]);
        int ck = (int)(f * (float)g.nc[k]);
        c[k] = min(max(ck, 0), g.nc[k] - 1);
        inbox &= (n[k] == 0.0f);
    }
    if (inbox) {
        float2 ox = ds_sum3(__ldg(org.Tx + c[0]), __ldg(org.Txy + c[1]), __ldg(org.Txz + c[2]));
        float2 oy = ds_sum3(__ldg(org.Ty + c[1]), __ldg(org.Tyz + c[2]), make_float2(0.f, 0.f));
        float2 oz = __ldg(org.Tz + c[2]);
        loc.x = __fsub_rn(__fsub_rn(x, ox.x), ox.y);
        loc.y = __fsub_rn(__fsub_rn(y, oy.x), oy.y);
        loc.z = __fsub_rn(__fsub_rn(z, oz.x), oz.y);
    } else {
        // FP64 route: fractional coordinate, wrap count and cell again in double
        double xd = x, yd = y, zd = z;
        double sd[3];
        sd[2] = zd * bd.invL[2] + 0.5;
        sd[1] = (yd - (sd[2] - 0.5) * bd.a3y) * bd.invL[1] + 0.5;
        sd[0] = (xd - (sd[1] - 0.5) * bd.a2x - (sd[2] - 0.5) * bd.a3x) * bd.invL[0] + 0.5;
        double gk[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double nk = floor(sd[k]);
            double f = sd[k] - nk;
            int ck = (int)(f * g.nc[k]);
            c[k] = min(max(ck, 0), g.nc[k] - 1);
            gk[k] = nk + (double)c[k] / g.nc[k] - 0.5;
        }
        double Ox = gk[0] * bd.L[0] + gk[1] * bd.a2x + gk[2] * bd.a3x;
        double Oy = gk[1] * bd.L[1] + gk[2] * bd.a3y;
        double Oz = gk[2] * bd.L[2];
        loc.x = (float)(xd - Ox);
        loc.y = (float)(yd - Oy);
        loc.z = (float)(zd - Oz);
    }
    key = (uint32_t)((c[2] * g.nc[1] + c[1]) * g.nc[0] + c[0]);
}


}  // namespace fgb
