// Solid-liquid order parameter (order module, Section "Analysis Modules": a solid-liquid
// order parameter for identifying generic ordered phases, after ten Wolde, Ruiz-Montero
// and Frenkel 1996):
//   s_ij = Re sum_{m=-l..l} Q_lm(i) conj(Q_lm(j)) / (|Q_l(i)| |Q_l(j)|)   (per bond),
// a bond is solid-like when s_ij > q_threshold, a particle is solid when it has at least
// solid_threshold solid-like bonds, and clusters join solid particles through solid-like
// bonds (cluster.cu).
//
// The bond decision turns a real number into an integer outcome, so it is taken in FP64
// on the device: Q_lm in double from the defining FP64 displacement (exact_disp) and the
// harmonics by the same recurrence as the FP32 kernels with double coefficients.  Only a
// bond whose FP64 score lies within about 1e-12 of the threshold could then be decided
// differently by another FP64 evaluation.
#include <cmath>
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
__global__ void __launch_bounds__(128) k_sl_qlm64(BoxD bd, const float *__restrict__ x, const int64_t *__restrict__ seg,
                                                  const int32_t *__restrict__ pj, int64_t n, int l,
                                                  double2 *__restrict__ Q) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
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

// s_ij per bond (FP64), the solid-like flag, and it as FP32 for the caller.
__global__ void k_sl_bonds(const int32_t *__restrict__ qi, const int32_t *__restrict__ pj, int64_t mpairs,
                           const double2 *__restrict__ Q, int l, double thr, int normalize, float *__restrict__ s_out,
                           uint8_t *__restrict__ solid) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= mpairs) return;
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

}  // namespace fgb

using namespace fgb;

extern "C" int fgb_solid_liquid(const fgb_box *box, const float *points, const fgb_nlist *nlist, int32_t l,
                                double q_threshold, int32_t solid_threshold, int32_t normalize_q, float *ql_ij,
                                int32_t *num_connections, void *stream, fgb_clusters **clusters_out) {
    clear_error();
    if (!box || !nlist || !clusters_out) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    *clusters_out = nullptr;
    if (l < 0 || l > kSlLMax) return fail(FGB_ERR_INVALID_ARG, "l must be in [0, %d]", kSlLMax);
    if (nlist->n_query != nlist->n_points) return fail(FGB_ERR_INVALID_ARG, "needs a self neighbor list");
    const int64_t n = nlist->n_query, mp = nlist->n_pairs;
    if (n > 0 && (!points || !num_connections)) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    BoxHost b;
    FGB_TRY(make_box(box, &b));
    FGB_TRY(ensure_consts64());
    cudaStream_t s = as_stream(stream);
    double2 *Q = nullptr;
    uint8_t *solid = nullptr;
    int st = dalloc_n(&Q, (size_t)std::max<int64_t>(n, 1) * (l + 1), s);
    st = st ? st : dalloc_n(&solid, std::max<int64_t>(mp, 1), s);
    if (st == FGB_OK && n > 0) {
        {
            FGB_KSCOPE("k_sl_qlm64", s);
            k_sl_qlm64<<<grid1d(n, 128), 128, 0, s>>>(b.d, points, nlist->segments, nlist->pj, n, l, Q);
        }
        if (mp > 0) {
            FGB_KSCOPE("k_sl_bonds", s);
            k_sl_bonds<<<grid1d(mp, 256), 256, 0, s>>>(nlist->qi, nlist->pj, mp, Q, l, q_threshold, normalize_q ? 1 : 0,
                                                        ql_ij, solid);
        }
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
    return st;
}
