// Solid-liquid order parameter (order module, Section "Analysis Modules": a solid-liquid
// order parameter for identifying generic ordered phases, after ten Wolde, Ruiz-Montero
// and Frenkel 1996):
//   s_ij = Re sum_{m=-l..l} Q_lm(i) conj(Q_lm(j)) / (|Q_l(i)| |Q_l(j)|)   (per bond),
// a bond is solid-like when s_ij > q_threshold, a particle is solid when it has at least
// solid_threshold solid-like bonds, and clusters join solid particles through solid-like
// bonds (cluster.cu).
//
// The bond decision turns a real number into an integer outcome.  It is screened in
// FP32 with a proven enclosure and settled in FP64 only where the enclosure is too wide:
//   * per particle, Q_lm in FP32 carried with a radius (midpoint-radius arithmetic: each
//     operation's radius adds the operands' radii times the other operand and the
//     operation's own rounding, 2^-23 |result|, every radius term rounded upward), from
//     the defining FP64 displacement (exact_disp) rounded to FP32 with its exact radius,
//     coefficients carried with their own rounding radius;
//   * per bond, the enclosure [s_lo, s_hi] of the score from the enclosures of the dot
//     product and the two norms (finished in FP64 with a relative slack);
//   * a bond whose enclosure lies more than 1e-12 above or below the threshold is
//     decided from it (the FP64 evaluation differs from the exact score by far less);
//     the others (and their end points' Q_lm) are evaluated in FP64 as before: Q_lm in
//     double from exact_disp and the harmonics by the same recurrence with double
//     coefficients.  Only a bond whose FP64 score lies within about 1e-12 of the
//     threshold could be decided differently by another FP64 evaluation.
// The scores reported per bond are the FP32 midpoints (FP64 for the bonds settled in
// FP64): float32 accuracy.
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "fgb_device.cuh"

namespace fgb {

constexpr int kSlLMax = 12;

struct LegendreConsts64 {
    double amm[kSlLMax + 1];
    double first[kSlLMax + 1];
    double alpha[kSlLMax + 1][kSlLMax + 1];
    double beta[kSlLMax + 1][kSlLMax + 1];
};

static __constant__ LegendreConsts64 c_leg64;

// Abar_lm = c_lm d^m P_l / dz^m with c_lm = (-1)^m sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!):
// Abar_mm, Abar_{m+1,m} = first z Abar_mm, then the three-term recurrence in l.
static int ensure_consts64() {
    static bool done = false;
    if (done) return FGB_OK;
    auto fact = [](int n) {
        double f = 1;
        for (int i = 2; i <= n; ++i) f *= i;
        return f;
    };
    auto c = [&](int l, int m) {
        return ((m & 1) ? -1.0 : 1.0) * std::sqrt((2 * l + 1) / (4.0 * M_PI) * fact(l - m) / fact(l + m));
    };
    LegendreConsts64 h;
    memset(&h, 0, sizeof(h));
    for (int m = 0; m <= kSlLMax; ++m) {
        double dfact = 1;  // (2m-1)!!
        for (int k = 2 * m - 1; k > 1; k -= 2) dfact *= k;
        h.amm[m] = c(m, m) * dfact;
        if (m + 1 <= kSlLMax) h.first[m] = (2 * m + 1) * c(m + 1, m) / c(m, m);
        for (int l = m + 2; l <= kSlLMax; ++l) {
            h.alpha[l][m] = (2.0 * l - 1) / (l - m) * c(l, m) / c(l - 1, m);
            h.beta[l][m] = (double)(l + m - 1) / (l - m) * c(l, m) / c(l - 2, m);
        }
    }
    FGB_CUDA(cudaMemcpyToSymbol(c_leg64, &h, sizeof(h)));
    done = true;
    return FGB_OK;
}

// Q_lm(i), m = 0..l, in FP64 over the bonds of row i (coincident points skipped).
__device__ __forceinline__ void sl_qlm64_row(const BoxD &bd, const float *__restrict__ x,
                                             const int64_t *__restrict__ seg, const int32_t *__restrict__ pj, int64_t i,
                                             int l, double2 *__restrict__ Q) {
    double sr[kSlLMax + 1], si[kSlLMax + 1];
    for (int m = 0; m <= l; ++m) sr[m] = si[m] = 0.0;
    const int64_t beg = seg[i], end = seg[i + 1];
    int nb = 0;
    for (int64_t e = beg; e < end; ++e) {
        const double3 d = exact_disp(bd, x + 3 * i, x + 3 * (int64_t)pj[e]);
        const double r2 = d.x * d.x + d.y * d.y + d.z * d.z;
        ++nb;
        if (!(r2 > 0.0)) continue;
        const double inv = 1.0 / sqrt(r2);
        const double ux = d.x * inv, uy = d.y * inv, uz = d.z * inv;
        double wr = 1.0, wi = 0.0;  // (ux + i uy)^m
        for (int m = 0; m <= l; ++m) {
            double p0 = c_leg64.amm[m], a = p0;
            if (l > m) {
                double p1 = c_leg64.first[m] * uz * p0;
                for (int ll = m + 2; ll <= l; ++ll) {
                    const double p2 = c_leg64.alpha[ll][m] * uz * p1 - c_leg64.beta[ll][m] * p0;
                    p0 = p1;
                    p1 = p2;
                }
                a = p1;
            }
            sr[m] += a * wr;
            si[m] += a * wi;
            const double nr = wr * ux - wi * uy, ni = wr * uy + wi * ux;
            wr = nr;
            wi = ni;
        }
    }
    const double invn = nb > 0 ? 1.0 / nb : 0.0;
    for (int m = 0; m <= l; ++m) Q[i * (l + 1) + m] = make_double2(sr[m] * invn, si[m] * invn);
}

__global__ void __launch_bounds__(128) k_sl_qlm64(BoxD bd, const float *__restrict__ x, const int64_t *__restrict__ seg,
                                                  const int32_t *__restrict__ pj, int64_t n, int l,
                                                  double2 *__restrict__ Q) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    sl_qlm64_row(bd, x, seg, pj, i, l, Q);
}

// s_ij of bond e (FP64), the solid-like flag, and it as FP32 for the caller.
__device__ __forceinline__ void sl_bond64(const int32_t *__restrict__ qi, const int32_t *__restrict__ pj, int64_t e,
                                          const double2 *__restrict__ Q, int l, double thr, int normalize,
                                          float *__restrict__ s_out, uint8_t *__restrict__ solid) {
    const double2 *a = Q + (int64_t)qi[e] * (l + 1), *b = Q + (int64_t)pj[e] * (l + 1);
    // the m < 0 terms equal the m > 0 ones: Q_{l,-m} conj(Q'_{l,-m}) = conj(Q_lm conj(Q'_lm))
    double dot = a[0].x * b[0].x + a[0].y * b[0].y, na = a[0].x * a[0].x + a[0].y * a[0].y,
           nb = b[0].x * b[0].x + b[0].y * b[0].y;
    for (int m = 1; m <= l; ++m) {
        dot += 2.0 * (a[m].x * b[m].x + a[m].y * b[m].y);
        na += 2.0 * (a[m].x * a[m].x + a[m].y * a[m].y);
        nb += 2.0 * (b[m].x * b[m].x + b[m].y * b[m].y);
    }
    double s = dot;
    if (normalize) s = (na > 0.0 && nb > 0.0) ? dot / sqrt(na * nb) : 0.0;
    if (s_out) s_out[e] = (float)s;
    solid[e] = s > thr ? 1 : 0;
}

__global__ void k_sl_bonds(const int32_t *__restrict__ qi, const int32_t *__restrict__ pj, int64_t mpairs,
                           const double2 *__restrict__ Q, int l, double thr, int normalize, float *__restrict__ s_out,
                           uint8_t *__restrict__ solid) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= mpairs) return;
    sl_bond64(qi, pj, e, Q, l, thr, normalize, s_out, solid);
}

__global__ void k_sl_connections(const int64_t *__restrict__ seg, const uint8_t *__restrict__ solid, int64_t n,
                                 int32_t *__restrict__ nconn) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = 0;
    for (int64_t e = seg[i]; e < seg[i + 1]; ++e) c += solid[e];
    nconn[i] = c;
}

// A bond joins a cluster when it is solid-like and both ends are solid particles.
__global__ void k_sl_mask(const int32_t *__restrict__ qi, const int32_t *__restrict__ pj, int64_t mpairs,
                          const int32_t *__restrict__ nconn, int sthr, uint8_t *__restrict__ solid) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= mpairs) return;
    if (solid[e] && !(nconn[qi[e]] >= sthr && nconn[pj[e]] >= sthr)) solid[e] = 0;
}

static int grid1d(int64_t n, int t) { return (int)((n + t - 1) / t); }

// ------------------------------------------------------------------ FP32 screen

// A value with a radius that bounds its distance to the exact one.
struct Mr {
    float v, r;
};

constexpr float kMrU = 1.1920928955078125e-7f;  // 2^-23 >= |fl(x) - x| / |fl(x)| for round to nearest
constexpr float kMrEta = 1e-44f;                // >= the absolute error of a subnormal result

__device__ __forceinline__ float mr_round(float v) { return __fmaf_ru(kMrU, fabsf(v), kMrEta); }

__device__ __forceinline__ Mr mr_add(Mr a, Mr b) {
    const float v = __fadd_rn(a.v, b.v);
    return {v, __fadd_ru(__fadd_ru(a.r, b.r), mr_round(v))};
}
__device__ __forceinline__ Mr mr_sub(Mr a, Mr b) {
    const float v = __fsub_rn(a.v, b.v);
    return {v, __fadd_ru(__fadd_ru(a.r, b.r), mr_round(v))};
}
__device__ __forceinline__ Mr mr_mul(Mr a, Mr b) {
    const float v = __fmul_rn(a.v, b.v);
    // |ab - a'b'| <= |a'| rb + |b'| ra + ra rb for |a - a'| <= ra, |b - b'| <= rb
    const float r = __fmaf_ru(fabsf(a.v), b.r, __fmaf_ru(fabsf(b.v), a.r, __fmaf_ru(a.r, b.r, mr_round(v))));
    return {v, r};
}

struct MrConsts {
    Mr amm[kSlLMax + 1];
    Mr first[kSlLMax + 1];
    Mr alpha[kSlLMax + 1][kSlLMax + 1];
    Mr beta[kSlLMax + 1][kSlLMax + 1];
};
static __constant__ MrConsts c_mr;

// FP32 coefficients with the radius of their rounding from the exact values (computed in
// long double on the host, plus a relative 1e-15 for that computation's own error).
static long double sl_fact(int n) {
    long double f = 1;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

static long double sl_clm(int l, int m) {
    return ((m & 1) ? -1.0L : 1.0L) * std::sqrt((2 * l + 1) / (4.0L * (long double)M_PI) * sl_fact(l - m) / sl_fact(l + m));
}

static Mr sl_mr(long double x) {
    const float v = (float)x;
    const long double d = std::fabs((long double)v - x) + 1e-15L * std::fabs(x);
    float r = (float)d;
    if ((long double)r < d) r = std::nextafter(r, INFINITY);
    return Mr{v, r};
}

static int ensure_mr_consts() {
    static bool done = false;
    if (done) return FGB_OK;
    MrConsts h;
    memset(&h, 0, sizeof(h));
    for (int m = 0; m <= kSlLMax; ++m) {
        long double dfact = 1;
        for (int k = 2 * m - 1; k > 1; k -= 2) dfact *= k;
        h.amm[m] = sl_mr(sl_clm(m, m) * dfact);
        if (m + 1 <= kSlLMax) h.first[m] = sl_mr((2 * m + 1) * sl_clm(m + 1, m) / sl_clm(m, m));
        for (int l = m + 2; l <= kSlLMax; ++l) {
            h.alpha[l][m] = sl_mr((2.0L * l - 1) / (l - m) * sl_clm(l, m) / sl_clm(l - 1, m));
            h.beta[l][m] = sl_mr((long double)(l + m - 1) / (l - m) * sl_clm(l, m) / sl_clm(l - 2, m));
        }
    }
    FGB_CUDA(cudaMemcpyToSymbol(c_mr, &h, sizeof(h)));
    done = true;
    return FGB_OK;
}

// Q_lm(i), m = 0..L, in FP32 with radii (real and imaginary parts).
template <int L>
__global__ void __launch_bounds__(128) k_sl_qlm_screen(BoxD bd, const float *__restrict__ x,
                                                       const int64_t *__restrict__ seg, const int32_t *__restrict__ pj,
                                                       int64_t n, float4 *__restrict__ Q) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Mr sr[L + 1], si[L + 1];
#pragma unroll
    for (int m = 0; m <= L; ++m) sr[m] = si[m] = Mr{0.f, 0.f};
    const int64_t beg = seg[i], end = seg[i + 1];
    int nb = 0;
    for (int64_t e = beg; e < end; ++e) {
        const double3 d64 = exact_disp(bd, x + 3 * i, x + 3 * (int64_t)pj[e]);
        ++nb;
        if (!(d64.x * d64.x + d64.y * d64.y + d64.z * d64.z > 0.0)) continue;  // as the FP64 path
        Mr d[3];
        const double dv[3] = {d64.x, d64.y, d64.z};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            d[k].v = (float)dv[k];
            d[k].r = __double2float_ru(fabs((double)d[k].v - dv[k]));
        }
        const Mr r2 = mr_add(mr_add(mr_mul(d[0], d[0]), mr_mul(d[1], d[1])), mr_mul(d[2], d[2]));
        // 1/|d|: rsqrtf is within 2 ulp; the exact r2 lies in [r2 - r, r2 + r], where the
        // derivative of t^-1/2 is at most (r2 - r)^-3/2 / 2 (bounded above by directed
        // rounding: numerator up, denominator down)
        Mr inv;
        inv.v = rsqrtf(r2.v);
        {
            const float lo = __fsub_rd(r2.v, r2.r);
            const float spread =
                lo > 0.f ? __fdiv_ru(__fmul_ru(0.5f, r2.r), __fmul_rd(lo, __fsqrt_rd(lo))) : INFINITY;
            inv.r = __fmaf_ru(2.384185791015625e-7f, fabsf(inv.v), spread);
        }
        const Mr ux = mr_mul(d[0], inv), uy = mr_mul(d[1], inv), uz = mr_mul(d[2], inv);
        Mr wr = Mr{1.f, 0.f}, wi = Mr{0.f, 0.f};
#pragma unroll
        for (int m = 0; m <= L; ++m) {
            Mr p0 = c_mr.amm[m], a = p0;
            if (m < L) {
                Mr p1 = mr_mul(mr_mul(c_mr.first[m], uz), p0);
#pragma unroll
                for (int ll = m + 2; ll <= L; ++ll) {
                    const Mr p2 = mr_sub(mr_mul(mr_mul(c_mr.alpha[ll][m], uz), p1), mr_mul(c_mr.beta[ll][m], p0));
                    p0 = p1;
                    p1 = p2;
                }
                a = p1;
            }
            sr[m] = mr_add(sr[m], mr_mul(a, wr));
            si[m] = mr_add(si[m], mr_mul(a, wi));
            const Mr nr = mr_sub(mr_mul(wr, ux), mr_mul(wi, uy));
            const Mr ni = mr_add(mr_mul(wr, uy), mr_mul(wi, ux));
            wr = nr;
            wi = ni;
        }
    }
    Mr invn = {0.f, 0.f};
    if (nb > 0) {
        invn.v = __fdiv_rn(1.f, (float)nb);
        invn.r = mr_round(invn.v);
    }
#pragma unroll
    for (int m = 0; m <= L; ++m) {
        const Mr a = mr_mul(sr[m], invn), b = mr_mul(si[m], invn);
        Q[i * (L + 1) + m] = make_float4(a.v, b.v, a.r, b.r);
    }
}

// Per bond: the score's FP32 midpoint and enclosure; decided bonds get their solid flag,
// the others are listed and their end points flagged for the FP64 pass.
__global__ void k_sl_screen(const int32_t *__restrict__ qi, const int32_t *__restrict__ pj, int64_t mpairs,
                            const float4 *__restrict__ Q, int l, double thr, int normalize, float *__restrict__ s_out,
                            uint8_t *__restrict__ solid, int *__restrict__ amb, int *__restrict__ namb,
                            uint8_t *__restrict__ need64) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= mpairs) return;
    const int i = qi[e], j = pj[e];
    const float4 *a = Q + (int64_t)i * (l + 1), *b = Q + (int64_t)j * (l + 1);
    Mr dot = {0.f, 0.f}, na = {0.f, 0.f}, nb = {0.f, 0.f};
    for (int m = 0; m <= l; ++m) {
        const float4 x = a[m], y = b[m];
        const Mr xr = {x.x, x.z}, xi = {x.y, x.w}, yr = {y.x, y.z}, yi = {y.y, y.w};
        // the m < 0 terms equal the m > 0 ones: weight 2 (exact) for m > 0
        const Mr f = {m ? 2.f : 1.f, 0.f};
        dot = mr_add(dot, mr_mul(f, mr_add(mr_mul(xr, yr), mr_mul(xi, yi))));
        na = mr_add(na, mr_mul(f, mr_add(mr_mul(xr, xr), mr_mul(xi, xi))));
        nb = mr_add(nb, mr_mul(f, mr_add(mr_mul(yr, yr), mr_mul(yi, yi))));
    }
    // enclosure of the score, every bound rounded outward (FP32 directed rounding)
    float lo, hi, mid;
    const float dlo = __fsub_rd(dot.v, dot.r), dhi = __fadd_ru(dot.v, dot.r);
    if (!normalize) {
        lo = dlo;
        hi = dhi;
        mid = dot.v;
    } else if ((na.v == 0.f && na.r == 0.f) || (nb.v == 0.f && nb.r == 0.f)) {
        lo = hi = 0.f;  // a particle without bonds: the score is 0 by definition
        mid = 0.f;
    } else {
        const float alo = __fsub_rd(na.v, na.r), ahi = __fadd_ru(na.v, na.r);
        const float blo = __fsub_rd(nb.v, nb.r), bhi = __fadd_ru(nb.v, nb.r);
        if (alo > 0.f && blo > 0.f) {
            // s = D / sqrt(A B) rises with D and falls with A B where D >= 0 (rises where
            // D < 0): the lower end takes the larger norms for D >= 0, the smaller ones else
            const float plo = __fsqrt_rd(__fmul_rd(alo, blo)), phi = __fsqrt_ru(__fmul_ru(ahi, bhi));
            lo = __fdiv_rd(dlo, dlo >= 0.f ? phi : plo);
            hi = __fdiv_ru(dhi, dhi >= 0.f ? plo : phi);
        } else {
            lo = -INFINITY;
            hi = INFINITY;
        }
        mid = dot.v / sqrtf(na.v * nb.v);
    }
    if (s_out) s_out[e] = mid;
    // the FP64 evaluation of the score differs from the exact one by far less than tau
    const double tau = 1e-12;
    if ((double)lo > thr + tau) {
        solid[e] = 1;
    } else if ((double)hi < thr - tau) {
        solid[e] = 0;
    } else {
        solid[e] = 0;
        const int k = atomicAdd(namb, 1);
        amb[k] = (int)e;  // the list has room for every bond
        need64[i] = 1;
        need64[j] = 1;
    }
}

// Q_lm in FP64 for the particles flagged by the screen.
__global__ void __launch_bounds__(128) k_sl_qlm64_flagged(BoxD bd, const float *__restrict__ x,
                                                          const int64_t *__restrict__ seg, const int32_t *__restrict__ pj,
                                                          int64_t n, int l, const uint8_t *__restrict__ need64,
                                                          double2 *__restrict__ Q) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !need64[i]) return;
    sl_qlm64_row(bd, x, seg, pj, i, l, Q);
}

// The listed bonds decided from FP64 Q_lm (grid-stride over the device count).
__global__ void k_sl_bonds_listed(const int32_t *__restrict__ qi, const int32_t *__restrict__ pj,
                                  const int *__restrict__ amb, const int *__restrict__ namb, const double2 *__restrict__ Q,
                                  int l, double thr, int normalize, float *__restrict__ s_out,
                                  uint8_t *__restrict__ solid) {
    const int m = *namb;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x)
        sl_bond64(qi, pj, amb[k], Q, l, thr, normalize, s_out, solid);
}

template <int L>
static void launch_qlm_screen(const BoxD &bd, const float *x, const fgb_nlist *nl, float4 *Q, cudaStream_t s) {
    const int64_t n = nl->n_query;
    FGB_KSCOPE("k_sl_qlm_screen", s);
    k_sl_qlm_screen<L><<<grid1d(n, 128), 128, 0, s>>>(bd, x, nl->segments, nl->pj, n, Q);
}

static void qlm_screen(int l, const BoxD &bd, const float *x, const fgb_nlist *nl, float4 *Q, cudaStream_t s) {
    switch (l) {
        case 0: launch_qlm_screen<0>(bd, x, nl, Q, s); break;
        case 1: launch_qlm_screen<1>(bd, x, nl, Q, s); break;
        case 2: launch_qlm_screen<2>(bd, x, nl, Q, s); break;
        case 3: launch_qlm_screen<3>(bd, x, nl, Q, s); break;
        case 4: launch_qlm_screen<4>(bd, x, nl, Q, s); break;
        case 5: launch_qlm_screen<5>(bd, x, nl, Q, s); break;
        case 6: launch_qlm_screen<6>(bd, x, nl, Q, s); break;
        case 7: launch_qlm_screen<7>(bd, x, nl, Q, s); break;
        case 8: launch_qlm_screen<8>(bd, x, nl, Q, s); break;
        case 9: launch_qlm_screen<9>(bd, x, nl, Q, s); break;
        case 10: launch_qlm_screen<10>(bd, x, nl, Q, s); break;
        case 11: launch_qlm_screen<11>(bd, x, nl, Q, s); break;
        default: launch_qlm_screen<12>(bd, x, nl, Q, s); break;
    }
}

// FGB_SL_SCREEN=0 decides every bond in FP64 (comparisons and tests of that path).
static bool sl_screen_enabled() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("FGB_SL_SCREEN");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

}  // namespace fgb

using namespace fgb;

extern "C" int fgb_solid_liquid(const fgb_box *box, const float *points, const fgb_nlist *nlist, int32_t l,
                                double q_threshold, int32_t solid_threshold, int32_t normalize_q, float *ql_ij,
                                int32_t *num_connections, void *stream, fgb_clusters **clusters_out) {
    clear_error();
    if (!box || !nlist || !clusters_out) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    FGB_TRY(nlist_ready(nlist));
    *clusters_out = nullptr;
    if (l < 0 || l > kSlLMax) return fail(FGB_ERR_INVALID_ARG, "l must be in [0, %d]", kSlLMax);
    if (nlist->n_query != nlist->n_points) return fail(FGB_ERR_INVALID_ARG, "needs a self neighbor list");
    const int64_t n = nlist->n_query, mp = nlist->n_pairs;
    if (n > 0 && (!points || !num_connections)) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    BoxHost b;
    FGB_TRY(make_box(box, &b));
    FGB_TRY(ensure_consts64());
    const bool screen = sl_screen_enabled() && mp > 0 && mp < ((int64_t)1 << 31);
    if (screen) FGB_TRY(ensure_mr_consts());
    cudaStream_t s = as_stream(stream);
    double2 *Q = nullptr;
    uint8_t *solid = nullptr;
    float4 *Q32 = nullptr;
    int *amb = nullptr;
    uint8_t *need64 = nullptr;
    int st = dalloc_n(&Q, (size_t)std::max<int64_t>(n, 1) * (l + 1), s);
    st = st ? st : dalloc_n(&solid, std::max<int64_t>(mp, 1), s);
    if (screen) {
        st = st ? st : dalloc_n(&Q32, (size_t)std::max<int64_t>(n, 1) * (l + 1), s);
        st = st ? st : dalloc_n(&amb, (size_t)mp + 1, s);  // [0]: count, then the listed bonds
        st = st ? st : dalloc_n(&need64, (size_t)std::max<int64_t>(n, 1), s);
    }
    if (st == FGB_OK && n > 0 && screen) {
        cudaMemsetAsync(amb, 0, sizeof(int), s);
        cudaMemsetAsync(need64, 0, (size_t)n, s);
        qlm_screen(l, b.d, points, nlist, Q32, s);
        {
            FGB_KSCOPE("k_sl_screen", s);
            k_sl_screen<<<grid1d(mp, 256), 256, 0, s>>>(nlist->qi, nlist->pj, mp, Q32, l, q_threshold,
                                                         normalize_q ? 1 : 0, ql_ij, solid, amb + 1, amb, need64);
        }
        {
            FGB_KSCOPE("k_sl_qlm64_flagged", s);
            k_sl_qlm64_flagged<<<grid1d(n, 128), 128, 0, s>>>(b.d, points, nlist->segments, nlist->pj, n, l, need64, Q);
        }
        {
            FGB_KSCOPE("k_sl_bonds_listed", s);
            k_sl_bonds_listed<<<num_sms() * 4, 256, 0, s>>>(nlist->qi, nlist->pj, amb + 1, amb, Q, l, q_threshold,
                                                            normalize_q ? 1 : 0, ql_ij, solid);
        }
    } else if (st == FGB_OK && n > 0) {
        {
            FGB_KSCOPE("k_sl_qlm64", s);
            k_sl_qlm64<<<grid1d(n, 128), 128, 0, s>>>(b.d, points, nlist->segments, nlist->pj, n, l, Q);
        }
        if (mp > 0) {
            FGB_KSCOPE("k_sl_bonds", s);
            k_sl_bonds<<<grid1d(mp, 256), 256, 0, s>>>(nlist->qi, nlist->pj, mp, Q, l, q_threshold, normalize_q ? 1 : 0,
                                                        ql_ij, solid);
        }
    }
    if (st == FGB_OK && n > 0) {
        {
            FGB_KSCOPE("k_sl_connections", s);
            k_sl_connections<<<grid1d(n, 256), 256, 0, s>>>(nlist->segments, solid, n, num_connections);
        }
        if (mp > 0) {
            FGB_KSCOPE("k_sl_mask", s);
            k_sl_mask<<<grid1d(mp, 256), 256, 0, s>>>(nlist->qi, nlist->pj, mp, num_connections, solid_threshold, solid);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = fail(FGB_ERR_CUDA, "solid-liquid launch failed: %s", cudaGetErrorString(e));
    }
    if (st == FGB_OK) st = fgb_cluster_compute(n, nlist, solid, stream, clusters_out);
    dfree(Q, s);
    dfree(solid, s);
    dfree(Q32, s);
    dfree(amb, s);
    dfree(need64, s);
    return st;
}
