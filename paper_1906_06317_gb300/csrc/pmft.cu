// Potential of mean force and torque in the plane, PMFT(x, y) (pmft module; Section
// "Potentials of Mean Force and Torque", the PMFT relation and Fig. 6): every bond (i, j)
// of a 2D system, the minimum-image d = x_j - q_i, is written in the frame of query
// particle i, whose orientation is the angle theta_i about z (the bond turned by
// -theta_i):
//   x' = cos(theta_i) d_x + sin(theta_i) d_y,   y' = cos(theta_i) d_y - sin(theta_i) d_x,
// and counted in bin (floor((x' + x_max) / dx), floor((y' + y_max) / dy)),
// dx = 2 x_max / bins_x, dy = 2 y_max / bins_y (an index equal to the bin count clamps
// to the last bin), when -x_max <= x' < x_max and -y_max <= y' < y_max.  The histogram
// accumulates over calls (reset = 0) like the RDF; pcf = counts / (norm * bin area) with
// norm = sum over frames of N_query N_points / A, and the PMFT is -log(pcf).
//
// Binning turns real numbers into integers, so every bond is decided in FP64 from the
// defining FP64 displacement (exact_disp) with (cos, sin) of the FP32 angle in FP64.
#include <cmath>
#include <cstring>
#include <vector>

#include "fgb_device.cuh"

struct fgb_pmft {
    double x_max, y_max;
    int bx, by;
    unsigned long long *hist;  // device, bx * by, x major
    double2 *trig;             // device, (cos, sin) of the query orientations
    int64_t trig_cap;
    double norm;               // sum over frames of N_query * N_points / area
    cudaStream_t stream;
};

namespace fgb {

struct PmftBins {
    double x_max, y_max, dx, dy;
    int bx, by;
};

__global__ void k_pmft_trig(const float *__restrict__ theta, int64_t n, double2 *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s, c;
    sincos((double)theta[i], &s, &c);
    out[i] = make_double2(c, s);
}

// Bin index of one bond in the frame (FP64, the defining sequence); -1 outside.
__device__ __forceinline__ int pmft_bin64(const PmftBins &B, double2 cs, double3 d) {
    const double xr = __dadd_rn(__dmul_rn(cs.x, d.x), __dmul_rn(cs.y, d.y));
    const double yr = __dsub_rn(__dmul_rn(cs.x, d.y), __dmul_rn(cs.y, d.x));
    if (!(xr >= -B.x_max && xr < B.x_max && yr >= -B.y_max && yr < B.y_max)) return -1;
    const int ix = min((int)floor(__ddiv_rn(__dadd_rn(xr, B.x_max), B.dx)), B.bx - 1);
    const int iy = min((int)floor(__ddiv_rn(__dadd_rn(yr, B.y_max), B.dy)), B.by - 1);
    return ix * B.by + iy;
}

// One thread per bond of a NeighborList (query_point_indices address qp and trig).
__global__ void k_pmft_list(BoxD bd, const float *__restrict__ p, const float *__restrict__ qp,
                            const double2 *__restrict__ trig, const int32_t *__restrict__ qi,
                            const int32_t *__restrict__ pj, int64_t m, PmftBins B,
                            unsigned long long *__restrict__ hist) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = __ldg(qi + e), j = __ldg(pj + e);
        const double3 d = exact_disp(bd, qp + 3 * (int64_t)i, p + 3 * (int64_t)j);
        const int b = pmft_bin64(B, __ldg(trig + i), d);
        if (b >= 0) atomicAdd(hist + b, 1ull);
    }
}

}  // namespace fgb

using namespace fgb;

extern "C" int fgb_pmftxy_create(double x_max, double y_max, int32_t bins_x, int32_t bins_y, fgb_pmft **out) {
    clear_error();
    if (!out) return fail(FGB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!(x_max > 0.0) || !(y_max > 0.0) || !std::isfinite(x_max) || !std::isfinite(y_max))
        return fail(FGB_ERR_INVALID_ARG, "x_max and y_max must be positive and finite");
    if (bins_x <= 0 || bins_y <= 0 || (int64_t)bins_x * bins_y > ((int64_t)1 << 26))
        return fail(FGB_ERR_INVALID_ARG, "bin counts must be positive, at most 2^26 bins in all");
    fgb_pmft *P = new fgb_pmft();
    P->x_max = x_max;
    P->y_max = y_max;
    P->bx = bins_x;
    P->by = bins_y;
    *out = P;
    return FGB_OK;
}

extern "C" void fgb_pmftxy_destroy(fgb_pmft *P) {
    if (!P) return;
    dfree(P->hist, P->stream);
    dfree(P->trig, P->stream);
    delete P;
}

extern "C" int fgb_pmftxy_compute(fgb_pmft *P, fgb_nq *nq, const float *query_points, const float *query_orientations,
                                  int64_t n_query, const fgb_nlist *nlist, int32_t reset, void *stream) {
    clear_error();
    if (!P || !nq) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    if (!nq->box.is2d) return fail(FGB_ERR_INVALID_ARG, "PMFT(x, y) needs a 2D box (Lz = 0)");
    if (n_query < 0 || (!query_points && n_query != nq->n))
        return fail(FGB_ERR_INVALID_ARG, "n_query must be the point count when query_points is NULL");
    if (n_query > 0 && !query_orientations) return fail(FGB_ERR_INVALID_ARG, "query_orientations is NULL");
    if (nlist && (nlist->n_query != n_query || nlist->n_points != nq->n))
        return fail(FGB_ERR_INVALID_ARG, "the neighbor list does not match the query and point counts");
    const double reach = std::sqrt(P->x_max * P->x_max + P->y_max * P->y_max);
    if (!(reach < 0.5 * nq->box.wmin * (1.0 - 1e-5)))
        return fail(FGB_ERR_BOX_TOO_SMALL, "sqrt(x_max^2 + y_max^2) = %g must be below half the smallest box width (%g)",
                    reach, 0.5 * nq->box.wmin);
    cudaStream_t s = as_stream(stream);
    const size_t nb = (size_t)P->bx * P->by;
    if (!P->hist) {
        FGB_TRY(dalloc_n(&P->hist, nb, s));
        P->stream = s;
        reset = 1;
    }
    if (reset) {
        FGB_CUDA(cudaMemsetAsync(P->hist, 0, sizeof(unsigned long long) * nb, s));
        P->norm = 0.0;
    }
    if (n_query > 0 && nq->n > 0) {
        if (P->trig_cap < n_query) {
            dfree(P->trig, P->stream);
            P->trig = nullptr;
            P->trig_cap = 0;
            FGB_TRY(dalloc_n(&P->trig, n_query, s));
            P->trig_cap = n_query;
        }
        {
            FGB_KSCOPE("k_pmft_trig", s);
            k_pmft_trig<<<(unsigned)((n_query + 255) / 256), 256, 0, s>>>(query_orientations, n_query, P->trig);
        }
        FGB_LAUNCH_CHECK();
        fgb_nlist *own = nullptr;
        if (!nlist) {
            fgb_query_args qa;
            qa.r_max = reach;
            qa.num_neighbors = 0;
            qa.exclude_ii = query_points ? 0 : 1;
            FGB_TRY(fgb_nq_query(nq, query_points, n_query, &qa, stream, &own));
            nlist = own;
        }
        PmftBins B;
        B.x_max = P->x_max;
        B.y_max = P->y_max;
        B.dx = 2.0 * P->x_max / P->bx;
        B.dy = 2.0 * P->y_max / P->by;
        B.bx = P->bx;
        B.by = P->by;
        int st = FGB_OK;
        if (nlist->n_pairs > 0) {
            const unsigned grid = (unsigned)std::min<int64_t>((nlist->n_pairs + 255) / 256, (int64_t)num_sms() * 16);
            FGB_KSCOPE("k_pmft_list", s);
            k_pmft_list<<<grid, 256, 0, s>>>(nq->box.d, nq->points, query_points ? query_points : nq->points, P->trig,
                                             nlist->qi, nlist->pj, nlist->n_pairs, B, P->hist);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) st = fail(FGB_ERR_CUDA, "pmft launch failed: %s", cudaGetErrorString(e));
        }
        if (own) fgb_nlist_destroy(own);
        if (st != FGB_OK) return st;
    }
    P->norm += (double)n_query * (double)nq->n / (nq->box.p[0] * nq->box.p[1]);
    return FGB_OK;
}

extern "C" int fgb_pmftxy_result(const fgb_pmft *P, uint64_t *counts, double *pcf, double *pmft, void *stream) {
    clear_error();
    if (!P) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    const size_t nb = (size_t)P->bx * P->by;
    std::vector<unsigned long long> h(nb, 0ull);
    if (P->hist) {
        cudaStream_t s = as_stream(stream);
        FGB_CUDA(cudaMemcpyAsync(h.data(), P->hist, sizeof(unsigned long long) * nb, cudaMemcpyDeviceToHost, s));
        FGB_CUDA(cudaStreamSynchronize(s));
    }
    const double area = (2.0 * P->x_max / P->bx) * (2.0 * P->y_max / P->by);
    for (size_t k = 0; k < nb; ++k) {
        const double g = P->norm > 0 ? (double)h[k] / (P->norm * area) : 0.0;
        if (counts) counts[k] = h[k];
        if (pcf) pcf[k] = g;
        if (pmft) pmft[k] = g > 0 ? -std::log(g) : INFINITY;
    }
    return FGB_OK;
}

extern "C" int fgb_pmftxy_counts_device(const fgb_pmft *P, const uint64_t **counts) {
    if (!P || !counts) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    *counts = reinterpret_cast<const uint64_t *>(P->hist);
    return FGB_OK;
}
