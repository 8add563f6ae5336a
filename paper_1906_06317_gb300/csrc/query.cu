// NeighborQuery.query (Section "Implementation": queries by cutoff distance or by
// number of neighbors; Section "General Utilities": NeighborList storage, sorted).
//
// Ball query: count pass -> exclusive scan into int64 segments -> write pass.  One thread
// per query point in cell order (threads of a warp share stencil cells, so candidate
// loads hit L1); each candidate is decided in FP32 against a band around r_max and the
// few inside the band are re-decided with the defining FP64 sequence.  The write pass
// keeps each query's hits sorted by point index in shared memory (insertion as they
// arrive) and the warp then stores whole segments with coalesced writes.
//
// kNN: one thread per query keeps the k+1 best (r2, j) in registers, widening the
// stencil until the k-th distance is inside the radius the stencil is known to cover.
// Queries whose ranking has a gap within the FP32 error band are redone by a second
// kernel that ranks the close candidates with FP64 distances.
#include <cmath>
#include <cstring>

#include "fgb_device.cuh"

namespace fgb {

// ------------------------------------------------------------------ host: stencil plan

static double vnorm(double x, double y, double z) { return std::sqrt(x * x + y * y + z * z); }

// Offset table of mode 0: entry o holds M (o / nc), rounded once from FP64.
__global__ void k_offset_table(double m00, double m01, double m02, double m11, double m12, double m22, int nx, int ny,
                               int nz, int tx, int ty, int tz, float4 *out) {
    const int wx = 2 * tx + 1, wy = 2 * ty + 1, wz = 2 * tz + 1;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= wx * wy * wz) return;
    const int ox = t % wx - tx, oy = (t / wx) % wy - ty, oz = t / (wx * wy) - tz;
    const double fx = (double)ox / nx, fy = (double)oy / ny, fz = (double)oz / nz;
    out[t] = make_float4((float)(m00 * fx + m01 * fy + m02 * fz), (float)(m11 * fy + m12 * fz), (float)(m22 * fz), 0.f);
}

int plan_stencil_host(const BoxHost &b, const GridHost &g, double R, int s_table_min, StencilPlan *p,
                      std::vector<float4> *table) {
    memset(p, 0, sizeof(*p));
    int smax = 0;
    for (int k = 0; k < 3; ++k) {
        int s = (int)std::ceil(R * (1.0 + 0.5 * kCellMargin) / g.wc[k]);
        if (s < 1) s = 1;
        p->s[k] = s;
        if (2 * s + 1 > g.nc[k]) {
            p->full[k] = 1;
            p->mode = 1;
        }
        smax = std::max(smax, s);
    }
    if (p->mode == 0 && smax > kMaxStencil) p->mode = 1;  // very wide stencils: no table
    p->Lsum = vnorm(b.M[0][0], 0, 0) + vnorm(b.M[0][1], b.M[1][1], 0) + vnorm(b.M[0][2], b.M[1][2], b.M[2][2]);
    const double u = std::ldexp(1.0, -24);
    if (p->mode == 0) {
        for (int k = 0; k < 3; ++k)
            p->ts[k] = std::max(p->s[k], std::min(std::min(s_table_min, kMaxStencil), (g.nc[k] - 1) / 2));
        double offmax = 0;
        for (int r = 0; r < (b.is2d ? 2 : 3); ++r) {  // 2D: pairs come from the z = 0 layer only
            double e = 0;
            for (int c = 0; c < 3; ++c) e += std::fabs(b.M[r][c]) * p->ts[c] / g.nc[c];
            offmax = std::max(offmax, e);
        }
        if (table) {
            table->clear();
            for (int oz = -p->ts[2]; oz <= p->ts[2]; ++oz)
                for (int oy = -p->ts[1]; oy <= p->ts[1]; ++oy)
                    for (int ox = -p->ts[0]; ox <= p->ts[0]; ++ox) {
                        const double fx = (double)ox / g.nc[0], fy = (double)oy / g.nc[1], fz = (double)oz / g.nc[2];
                        table->push_back(make_float4((float)(b.M[0][0] * fx + b.M[0][1] * fy + b.M[0][2] * fz),
                                                     (float)(b.M[1][1] * fy + b.M[1][2] * fz), (float)(b.M[2][2] * fz),
                                                     0.f));
                    }
        }
        // error of one displacement component:
        //   local_i, local_j: 2 roundings each of a value <= ext      -> 4 u ext
        //   offset rounded once from FP64 (|off| <= offmax)          -> u offmax
        //   q' = local_i - off (|q'| <= ext + offmax)                -> u (ext + offmax)
        //   d = local_j - q' (|d| <= R for pairs that matter)        -> u R
        // doubled for slack.
        p->eps_d = 2.0 * u * (5.0 * g.ext + 2.0 * offmax + R);
    } else {
        // general route: offsets formed in FP32 from a_k/nc_k (|off| <= Lsum), rint
        // reduction with split box vectors (|intermediate| <= 2 Lsum + R), local
        // coordinates as above; doubled for slack.
        p->eps_d = 2.0 * u * (5.0 * g.ext + 8.0 * p->Lsum + 4.0 * R);
    }
    return FGB_OK;
}

int plan_stencil(const fgb_nq *nq, double R, int s_table_min, cudaStream_t st, StencilPlan *p) {
    FGB_TRY(plan_stencil_host(nq->box, nq->grid, R, s_table_min, p, nullptr));
    if (p->mode == 0) {
        const BoxHost &b = nq->box;
        const GridHost &g = nq->grid;
        const int total = (2 * p->ts[0] + 1) * (2 * p->ts[1] + 1) * (2 * p->ts[2] + 1);
        FGB_TRY(dalloc_n(&p->table, total, st));
        {
            FGB_KSCOPE("k_offset_table", st);
            k_offset_table<<<(total + 127) / 128, 128, 0, st>>>(b.M[0][0], b.M[0][1], b.M[0][2], b.M[1][1], b.M[1][2],
                                                                b.M[2][2], g.nc[0], g.nc[1], g.nc[2], p->ts[0],
                                                                p->ts[1], p->ts[2], p->table);
        }
        FGB_LAUNCH_CHECK();
    }
    return FGB_OK;
}

int launch_offset_table(const BoxHost &b, const GridHost &g, const StencilPlan &p, float4 *table, cudaStream_t st) {
    const int total = (2 * p.ts[0] + 1) * (2 * p.ts[1] + 1) * (2 * p.ts[2] + 1);
    {
        FGB_KSCOPE("k_offset_table", st);
        k_offset_table<<<(total + 127) / 128, 128, 0, st>>>(b.M[0][0], b.M[0][1], b.M[0][2], b.M[1][1], b.M[1][2],
                                                            b.M[2][2], g.nc[0], g.nc[1], g.nc[2], p.ts[0], p.ts[1],
                                                            p.ts[2], table);
    }
    FGB_LAUNCH_CHECK();
    return FGB_OK;
}

double r2_error_bound_eps(double e, double Lsum, double R) {
    const double u = std::ldexp(1.0, -24);
    // r2 = fma(dz,dz, fma(dy,dy, dx*dx)): |sum 2 d_k e| + 3 e^2 from the displacement,
    // 3 u r2 from the three roundings, plus slack for the FP64 reference's own rounding.
    return 2.0 * std::sqrt(3.0) * R * e + 3.0 * e * e + 3.0 * u * (R + e) * (R + e) + 1e-12 * (R + Lsum) * (R + Lsum);
}

double r2_error_bound(const StencilPlan &p, double R) { return r2_error_bound_eps(p.eps_d, p.Lsum, R); }

void band_around(double T, double delta, float *lo, float *hi) {
    double l = T - delta, h = T + delta;
    float lf = (float)l, hf = (float)h;
    if ((double)lf > l) lf = std::nextafter(lf, -INFINITY);
    if ((double)hf < h) hf = std::nextafter(hf, INFINITY);
    *lo = lf;
    *hi = hf;
}

Stencil to_device(const fgb_nq *nq, const StencilPlan &p) { return to_device(nq->box, nq->grid, p, p.table); }

Stencil to_device(const BoxHost &b, const GridHost &g, const StencilPlan &p, const float4 *table) {
    Stencil S;
    memset(&S, 0, sizeof(S));
    for (int k = 0; k < 3; ++k) {
        S.nc[k] = g.nc[k];
        S.s[k] = p.s[k];
        S.ts[k] = p.ts[k];
        S.full[k] = p.full[k];
    }
    S.mode = p.mode;
    S.off = table;
    S.step[0] = make_float3((float)(b.M[0][0] / g.nc[0]), 0.f, 0.f);
    S.step[1] = make_float3((float)(b.M[0][1] / g.nc[1]), (float)(b.M[1][1] / g.nc[1]), 0.f);
    S.step[2] = make_float3((float)(b.M[0][2] / g.nc[2]), (float)(b.M[1][2] / g.nc[2]), (float)(b.M[2][2] / g.nc[2]));
    return S;
}

}  // namespace fgb
