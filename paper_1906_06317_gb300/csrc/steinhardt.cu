// Steinhardt bond-orientational order q_l (order module, Section "Analysis Modules";
// definition of Steinhardt, Nelson and Ronchetti 1983) and the gradient of the global
// Q = (1/N) sum_i q_l(i) with respect to the positions, neighbor list held fixed.
//
// Spherical harmonics in FP32 without trigonometry: for a unit bond u = (x, y, z),
//   Y_lm(u) = Abar_lm(z) (x + i y)^m,   Abar_lm = c_lm d^m P_l / dz^m,
//   c_lm = (-1)^m sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),
// with Abar_lm built by the three-term recurrence in l at fixed m (normalisation folded
// into the coefficients) and (x + i y)^m by repeated complex products.  m < 0 follows
// from Y_{l,-m} = (-1)^m conj(Y_lm), so sum_m |Q_lm|^2 = |Q_l0|^2 + 2 sum_{m>0} |Q_lm|^2.
// The gradient uses the same basis: Y~_lm(u) = Abar_lm(z) (x + i y)^m is a homogeneous
// polynomial of degree l, so
//   d/dx Y~ = m Abar_lm w^(m-1),  d/dy Y~ = i m Abar_lm w^(m-1),
//   d/dz Y~ = (c_lm / c_l,m+1) Abar_l,m+1 w^m,
// projected on the sphere with (I - u u^T)/|d|, and the gradient at -u is (-1)^(l-1)
// times the gradient at u.
// Spherical-harmonic helpers: fgb_ylm.cuh.
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "fgb_ball.cuh"
#include "fgb_ylm.cuh"

namespace fgb {

// Forward pass over a NeighborList: one thread per query particle.
template <int L>
__global__ void __launch_bounds__(128) k_st_nlist(BoxF b, const float *__restrict__ x, const int64_t *__restrict__ seg,
                                                  const int32_t *__restrict__ pj, int64_t n, float *__restrict__ q,
                                                  float2 *__restrict__ Q, int32_t *__restrict__ nn) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float sr[L + 1], si[L + 1];
#pragma unroll
    for (int m = 0; m <= L; ++m) sr[m] = si[m] = 0.f;
    const int64_t beg = seg[i], end = seg[i + 1];
    for (int64_t e = beg; e < end; ++e) accumulate_bond<L>(bond_f32(b, x, i, pj[e]), sr, si);
    finish<L>(i, (int)(end - beg), sr, si, q, Q, nn);
}

// Forward pass fused with the cell-list ball query (no neighbor list is stored).
template <int L>
__global__ void __launch_bounds__(128) k_st_fused(BallArgs a, float *__restrict__ q, float2 *__restrict__ Q,
                                                  int32_t *__restrict__ nn) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.nq) return;
    const float4 p = a.qs[t];
    const int i = __float_as_int(p.w);
    float sr[L + 1], si[L + 1];
#pragma unroll
    for (int m = 0; m <= L; ++m) sr[m] = si[m] = 0.f;
    int n = 0;
    BondBuffer<L> bb;
    const int nesc = ball_visit(a, p, a.qcell[t], i, [&](int, float3 d, float, double) {
        ++n;
        bb.add(d, sr, si);
    });
    bb.flush(sr, si);
    if (nesc) atomicAdd(a.esc, (unsigned long long)nesc);
    finish<L>(i, n, sr, si, q, Q, nn);
}

// Gradient, symmetric neighbor list (j in nb(k) <=> k in nb(j)):
//   dQ/dx_k = (s/N) sum_{j in nb(k)} [ dq_j/dd_jk - dq_k/dd_kj ],  d_kj = x_j - x_k.
template <int L>
__global__ void __launch_bounds__(128) k_st_bwd_gather(BoxF b, const float *__restrict__ x, const int64_t *__restrict__ seg,
                                                       const int32_t *__restrict__ pj, int64_t n, const float *__restrict__ q,
                                                       const float2 *__restrict__ Q, const int32_t *__restrict__ nn,
                                                       float scale, float3 *__restrict__ grad) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float pref = 4.f * (float)M_PI / (2 * L + 1);
    const float qk = q[k];
    const int nk = nn[k];
    const float ck = (qk > 0.f && nk > 0) ? pref / (qk * (float)nk) : 0.f;
    const float sgn = (L & 1) ? 1.f : -1.f;  // (-1)^(L-1)
    float gx = 0.f, gy = 0.f, gz = 0.f;
    const int64_t beg = seg[k], end = seg[k + 1];
    for (int64_t e = beg; e < end; ++e) {
        const int j = pj[e];
        const float3 d = bond_f32(b, x, k, j);
        const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
        if (!(r2 > 0.f)) continue;
        const float inv = rsqrtf(r2);
        const float3 u = make_float3(d.x * inv, d.y * inv, d.z * inv);
        float A[L + 2], wr[L + 1], wi[L + 1];
        legendre_row<L>(u.z, A);
        powers<L>(u.x, u.y, wr, wi);
        const float qj = q[j];
        const int nj = nn[j];
        const float cj = (qj > 0.f && nj > 0) ? pref / (qj * (float)nj) : 0.f;
        const float3 own = project(contract_grad<L>(A, wr, wi, Q + k * (L + 1)), u, inv);
        const float3 nbr = project(contract_grad<L>(A, wr, wi, Q + (int64_t)j * (L + 1)), u, inv);
        gx += sgn * cj * nbr.x - ck * own.x;
        gy += sgn * cj * nbr.y - ck * own.y;
        gz += sgn * cj * nbr.z - ck * own.z;
    }
    grad[k] = make_float3(scale * gx, scale * gy, scale * gz);
}

// The same gradient with the next neighbour's data (its index, Q_lm, q and bond count)
// loaded before the current bond is computed, so the gathers of consecutive bonds
// overlap instead of each waiting on the last.
template <int L>
__global__ void __launch_bounds__(128) k_st_bwd_gather_pf(BoxF b, const float *__restrict__ x,
                                                          const int64_t *__restrict__ seg,
                                                          const int32_t *__restrict__ pj, int64_t n,
                                                          const float *__restrict__ q, const float2 *__restrict__ Q,
                                                          const int32_t *__restrict__ nn, float scale,
                                                          float3 *__restrict__ grad) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float pref = 4.f * (float)M_PI / (2 * L + 1);
    const float qk = q[k];
    const int nk = nn[k];
    const float ck = (qk > 0.f && nk > 0) ? pref / (qk * (float)nk) : 0.f;
    const float sgn = (L & 1) ? 1.f : -1.f;  // (-1)^(L-1)
    float2 Qk[L + 1];
#pragma unroll
    for (int m = 0; m <= L; ++m) Qk[m] = Q[k * (L + 1) + m];
    float gx = 0.f, gy = 0.f, gz = 0.f;
    const int64_t beg = seg[k], end = seg[k + 1];
    int j = beg < end ? pj[beg] : 0;
    float2 Qj[L + 1];
    float qj = 0.f;
    int nj = 0;
    if (beg < end) {
#pragma unroll
        for (int m = 0; m <= L; ++m) Qj[m] = Q[(int64_t)j * (L + 1) + m];
        qj = q[j];
        nj = nn[j];
    }
    for (int64_t e = beg; e < end; ++e) {
        const int jc = j;
        float2 Qc[L + 1];
#pragma unroll
        for (int m = 0; m <= L; ++m) Qc[m] = Qj[m];
        const float qc = qj;
        const int nc = nj;
        if (e + 1 < end) {  // the next neighbour's data, in flight during this bond
            j = pj[e + 1];
#pragma unroll
            for (int m = 0; m <= L; ++m) Qj[m] = Q[(int64_t)j * (L + 1) + m];
            qj = q[j];
            nj = nn[j];
        }
        const float3 d = bond_f32(b, x, k, jc);
        const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
        if (!(r2 > 0.f)) continue;
        const float inv = rsqrtf(r2);
        const float3 u = make_float3(d.x * inv, d.y * inv, d.z * inv);
        float A[L + 2], wr[L + 1], wi[L + 1];
        legendre_row<L>(u.z, A);
        powers<L>(u.x, u.y, wr, wi);
        const float cj = (qc > 0.f && nc > 0) ? pref / (qc * (float)nc) : 0.f;
        const float3 own = project(contract_grad<L>(A, wr, wi, Qk), u, inv);
        const float3 nbr = project(contract_grad<L>(A, wr, wi, Qc), u, inv);
        gx += sgn * cj * nbr.x - ck * own.x;
        gy += sgn * cj * nbr.y - ck * own.y;
        gz += sgn * cj * nbr.z - ck * own.z;
    }
    grad[k] = make_float3(scale * gx, scale * gy, scale * gz);
}

// Gradient, any neighbor list: one thread per pair, float atomics.
template <int L>
__global__ void __launch_bounds__(128) k_st_bwd_scatter(BoxF b, const float *__restrict__ x, const int32_t *__restrict__ qi,
                                                        const int32_t *__restrict__ pj, int64_t m, const float *__restrict__ q,
                                                        const float2 *__restrict__ Q, const int32_t *__restrict__ nn,
                                                        float scale, float *__restrict__ grad) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const int i = qi[e], j = pj[e];
    const float qv = q[i];
    const int ni = nn[i];
    if (!(qv > 0.f) || ni == 0) return;
    const float3 d = bond_f32(b, x, i, j);
    const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
    if (!(r2 > 0.f)) return;
    const float inv = rsqrtf(r2);
    const float3 u = make_float3(d.x * inv, d.y * inv, d.z * inv);
    float A[L + 2], wr[L + 1], wi[L + 1];
    legendre_row<L>(u.z, A);
    powers<L>(u.x, u.y, wr, wi);
    const float c = scale * 4.f * (float)M_PI / (2 * L + 1) / (qv * (float)ni);
    const float3 g = project(contract_grad<L>(A, wr, wi, Q + (int64_t)i * (L + 1)), u, inv);
    atomicAdd(grad + 3 * j + 0, c * g.x);
    atomicAdd(grad + 3 * j + 1, c * g.y);
    atomicAdd(grad + 3 * j + 2, c * g.z);
    atomicAdd(grad + 3 * i + 0, -c * g.x);
    atomicAdd(grad + 3 * i + 1, -c * g.y);
    atomicAdd(grad + 3 * i + 2, -c * g.z);
}

// FGB_ST_PREFETCH=0 takes the gradient kernel without the prefetch (comparisons).
static bool bwd_prefetch() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("FGB_ST_PREFETCH");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

template <int L>
struct StLaunch {
    static void nlist(const BoxF &b, const float *x, const fgb_nlist *nl, float *q, float2 *Q, int32_t *nn,
                      cudaStream_t s) {
        {
            FGB_KSCOPE("k_st_nlist", s);
            k_st_nlist<L><<<(unsigned)((nl->n_query + 127) / 128), 128, 0, s>>>(b, x, nl->segments, nl->pj, nl->n_query, q,
                                                                               Q, nn);
        }
    }
    static void fused(const BallArgs &a, float *q, float2 *Q, int32_t *nn, cudaStream_t s) {
        {
            FGB_KSCOPE("k_st_fused", s);
            k_st_fused<L><<<(unsigned)((a.nq + 127) / 128), 128, 0, s>>>(a, q, Q, nn);
        }
    }
    static void bwd(const BoxF &b, const float *x, const fgb_nlist *nl, const float *q, const float2 *Q,
                    const int32_t *nn, float scale, float *grad, cudaStream_t s) {
        if (nl->symmetric) {
            FGB_KSCOPE("k_st_bwd_gather", s);
            if (bwd_prefetch())
                k_st_bwd_gather_pf<L><<<(unsigned)((nl->n_query + 127) / 128), 128, 0, s>>>(
                    b, x, nl->segments, nl->pj, nl->n_query, q, Q, nn, scale, reinterpret_cast<float3 *>(grad));
            else
                k_st_bwd_gather<L><<<(unsigned)((nl->n_query + 127) / 128), 128, 0, s>>>(
                    b, x, nl->segments, nl->pj, nl->n_query, q, Q, nn, scale, reinterpret_cast<float3 *>(grad));
        } else {
            cudaMemsetAsync(grad, 0, sizeof(float) * 3 * nl->n_points, s);
            if (nl->n_pairs > 0)
                {
                    FGB_KSCOPE("k_st_bwd_scatter", s);
                    k_st_bwd_scatter<L><<<(unsigned)((nl->n_pairs + 127) / 128), 128, 0, s>>>(b, x, nl->qi, nl->pj, nl->n_pairs,
                                                                                            q, Q, nn, scale, grad);
                }
        }
    }
};

template <template <int> class F, class... Args>
static bool dispatch_l(int l, Args &&...args) {
    switch (l) {
#define FGB_L(V)                                \
    case V:                                     \
        F<V>::run(std::forward<Args>(args)...); \
        return true;
        FGB_L(0) FGB_L(1) FGB_L(2) FGB_L(3) FGB_L(4) FGB_L(5) FGB_L(6) FGB_L(7) FGB_L(8) FGB_L(9) FGB_L(10) FGB_L(11)
        FGB_L(12)
#undef FGB_L
    }
    return false;
}

template <int L>
struct RunNlist {
    static void run(const BoxF &b, const float *x, const fgb_nlist *nl, float *q, float2 *Q, int32_t *nn, cudaStream_t s) {
        StLaunch<L>::nlist(b, x, nl, q, Q, nn, s);
    }
};
template <int L>
struct RunFused {
    static void run(const BallArgs &a, float *q, float2 *Q, int32_t *nn, cudaStream_t s) { StLaunch<L>::fused(a, q, Q, nn, s); }
};
template <int L>
struct RunBwd {
    static void run(const BoxF &b, const float *x, const fgb_nlist *nl, const float *q, const float2 *Q,
                    const int32_t *nn, float scale, float *grad, cudaStream_t s) {
        StLaunch<L>::bwd(b, x, nl, q, Q, nn, scale, grad, s);
    }
};

}  // namespace fgb


using namespace fgb;

extern "C" int fgb_steinhardt_create(int32_t l, fgb_steinhardt **out) {
    clear_error();
    if (!out) return fail(FGB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (l < 0 || l > kLMax) return fail(FGB_ERR_INVALID_ARG, "l must be in [0, %d]", kLMax);
    FGB_TRY(ensure_consts());
    fgb_steinhardt *st = new fgb_steinhardt();
    memset(st, 0, sizeof(*st));
    st->l = l;
    *out = st;
    return FGB_OK;
}

extern "C" void fgb_steinhardt_destroy(fgb_steinhardt *st) {
    if (!st) return;
    dfree(st->Q, st->stream);
    dfree(st->nn, st->stream);
    dfree(st->Qtmp, st->stream);
    dfree(st->w3j, st->stream);
    delete st;
}

static int st_ensure(fgb_steinhardt *st, int64_t n, cudaStream_t s) {
    st->averaged = 0;
    if (st->n != n || !st->Q) {
        dfree(st->Q, s);
        dfree(st->nn, s);
        st->Q = nullptr;
        st->nn = nullptr;
        FGB_TRY(dalloc_n(&st->Q, (size_t)n * (st->l + 1), s));
        FGB_TRY(dalloc_n(&st->nn, n, s));
        st->n = n;
        st->stream = s;
    }
    return FGB_OK;
}

extern "C" int fgb_steinhardt_compute(fgb_steinhardt *st, fgb_nq *nq, const fgb_nlist *nlist,
                                      const fgb_query_args *qargs, float *q_out, void *stream) {
    clear_error();
    if (!st || !nq || (nq->n > 0 && !q_out)) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    FGB_TRY(nlist_ready(nlist));
    cudaStream_t s = as_stream(stream);
    FGB_TRY(st_ensure(st, nq->n, s));
    st->last_nlist = nlist;
    if (nq->n == 0) return FGB_OK;
    if (nlist) {
        if (nlist->n_query != nq->n) return fail(FGB_ERR_INVALID_ARG, "nlist must have one segment per point");
        dispatch_l<RunNlist>(st->l, nq->box.f, nq->points, nlist, q_out, st->Q, st->nn, s);
    } else {
        if (!qargs || !(qargs->r_max > 0.0))
            return fail(FGB_ERR_UNSUPPORTED, "without a NeighborList the neighbors must be a ball query (r_max > 0)");
        if (nq->kind != 0)
            return fail(FGB_ERR_UNSUPPORTED, "the fused query walks a cell list; pass a NeighborList from the tree query");
        const double R = qargs->r_max;
        if (!(R < 0.5 * nq->box.wmin * (1.0 - 1e-5)))
            return fail(FGB_ERR_BOX_TOO_SMALL, "r_max must be below half the smallest box width");
        StencilPlan plan;
        FGB_TRY(plan_stencil(nq, R, 0, s, &plan));
        BallArgs a;
        memset(&a, 0, sizeof(a));
        a.S = to_device(nq, plan);
        a.bf = nq->box.f;
        a.bd = nq->box.d;
        a.pts = nq->sorted;
        a.cell_start = nq->cell_start;
        a.qs = nq->sorted;
        a.qcell = nq->sorted_cell;
        a.nq = nq->n;
        a.p_orig = nq->points;
        a.q_orig = nq->points;
        a.T = sqrt_threshold(R);
        band_around(a.T, r2_error_bound(plan, R), &a.band.lo, &a.band.hi);
        a.exclude = qargs->exclude_ii ? 1 : 0;
        unsigned long long *esc = nullptr;
        int rc = dalloc_n(&esc, 2, s);
        if (rc == FGB_OK) {
            a.esc = esc;
            a.err = reinterpret_cast<int *>(esc + 1);
            dispatch_l<RunFused>(st->l, a, q_out, st->Q, st->nn, s);
        }
        dfree(esc, s);
        dfree(plan.table, s);
        FGB_TRY(rc);
    }
    FGB_LAUNCH_CHECK();
    return FGB_OK;
}

extern "C" int fgb_steinhardt_state(const fgb_steinhardt *st, const float **qlm, const int32_t **n_neighbors) {
    if (!st) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    if (qlm) *qlm = reinterpret_cast<const float *>(st->Q);
    if (n_neighbors) *n_neighbors = st->nn;
    return FGB_OK;
}

extern "C" int fgb_steinhardt_backward(fgb_steinhardt *st, fgb_nq *nq, const fgb_nlist *nlist, const float *q,
                                       float upstream, float *grad_out, void *stream) {
    clear_error();
    if (!st || !nq || !nlist || (nq->n > 0 && (!q || !grad_out))) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    FGB_TRY(nlist_ready(nlist));
    if (!st->Q || st->n != nq->n) return fail(FGB_ERR_INVALID_ARG, "call fgb_steinhardt_compute first");
    if (st->averaged) return fail(FGB_ERR_UNSUPPORTED, "the backward pass is for q_l, not the averaged q_l");
    if (nlist->n_query != nq->n || nlist->n_points != nq->n)
        return fail(FGB_ERR_INVALID_ARG, "backward needs a self neighbor list over the same points");
    cudaStream_t s = as_stream(stream);
    if (nq->n == 0) return FGB_OK;
    const float scale = (float)(upstream / (double)nq->n);
    dispatch_l<RunBwd>(st->l, nq->box.f, nq->points, nlist, q, st->Q, st->nn, scale, grad_out, s);
    FGB_LAUNCH_CHECK();
    return FGB_OK;
}
