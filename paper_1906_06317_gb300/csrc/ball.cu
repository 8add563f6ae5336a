// Ball query (r_max) and the NeighborList handle.  See query.cu for the overview.
#include <cmath>
#include <cstring>

#include "fgb_ball.cuh"

namespace fgb {

int knn_query(fgb_nq *nq, const QueryPoints &Q, const fgb_query_args *a, cudaStream_t s, fgb_nlist *nl);

__global__ void __launch_bounds__(128) k_ball_count(BallArgs a, uint32_t *__restrict__ counts) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.nq) return;
    const float4 q = a.qs[t];
    const int i = __float_as_int(q.w);
    uint32_t cnt = 0;
    const int nesc = ball_visit(a, q, a.qcell[t], i, [&](int, float3, float, double) { ++cnt; });
    counts[i] = cnt;
    if (nesc) atomicAdd(a.esc, (unsigned long long)nesc);
}

// Write pass.  SHARED: each thread appends its query's hits (j, distance bits) to a
// shared slab laid out [slot][thread], sorts them by j once the walk is done, and the warp
// then writes each query's segment with coalesced stores.  !SHARED (very large neighbor
// counts): insertion happens in the output arrays themselves.
template <bool SHARED>
__global__ void __launch_bounds__(128) k_ball_write(BallArgs a, const int64_t *__restrict__ seg,
                                                    const uint32_t *__restrict__ counts, int cap,
                                                    int32_t *__restrict__ qi_out, int32_t *__restrict__ pj_out,
                                                    float *__restrict__ d_out) {
    extern __shared__ uint2 slab[];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = t < a.nq;
    int i = -1;
    uint32_t n = 0, want = 0;
    int64_t off = 0;
    if (valid) {
        const float4 q = a.qs[t];
        i = __float_as_int(q.w);
        off = seg[i];
        want = counts[i];
        const uint32_t lim = SHARED ? (uint32_t)cap : want;
        ball_visit(a, q, a.qcell[t], i, [&](int j, float3, float r2, double e) {
            if (n >= lim) {
                atomicExch(a.err, 1);
                return;
            }
            const float dist = e < 0.0 ? sqrtf(r2) : (float)sqrt(e);
            if (SHARED) {
                slab[n * blockDim.x + threadIdx.x] = make_uint2((uint32_t)j, __float_as_uint(dist));
            } else {
                uint32_t pos = n;
                while (pos > 0) {
                    const int pj = pj_out[off + pos - 1];
                    if (pj < j) break;
                    pj_out[off + pos] = pj;
                    d_out[off + pos] = d_out[off + pos - 1];
                    --pos;
                }
                pj_out[off + pos] = j;
                d_out[off + pos] = dist;
            }
            ++n;
        });
        if (SHARED) {
            // hits arrive as one index-sorted run per stencil cell; a shell sort (gaps
            // 57, 23, 10, 4, 1) orders them by point index with few moves
            const int gaps[5] = {57, 23, 10, 4, 1};
            const int B = blockDim.x, me = threadIdx.x;
            for (int gi = 0; gi < 5; ++gi) {
                const int g = gaps[gi];
                for (int k = g; k < (int)n; ++k) {
                    const uint2 v = slab[k * B + me];
                    int m = k;
                    while (m >= g) {
                        const uint2 u = slab[(m - g) * B + me];
                        if ((int)u.x < (int)v.x) break;
                        slab[m * B + me] = u;
                        m -= g;
                    }
                    slab[m * B + me] = v;
                }
            }
        }
        if (n != want) atomicExch(a.err, 2);
    }
    if (SHARED) {
        const int lane = threadIdx.x & 31;
        const int wbase = threadIdx.x & ~31;
        for (int L = 0; L < 32; ++L) {
            const int iL = __shfl_sync(0xffffffffu, i, L);
            const uint32_t nL = __shfl_sync(0xffffffffu, n, L);
            const int64_t oL = __shfl_sync(0xffffffffu, off, L);
            for (uint32_t k = lane; k < nL; k += 32) {
                const uint2 e = slab[k * blockDim.x + wbase + L];
                qi_out[oL + k] = iL;
                pj_out[oL + k] = (int32_t)e.x;
                d_out[oL + k] = __uint_as_float(e.y);
            }
        }
    } else if (valid) {
        for (uint32_t k = 0; k < n; ++k) qi_out[off + k] = i;
    }
}

struct QueryStatus {
    int64_t total;
    unsigned long long esc;
    uint32_t maxcount;
    int err;
};

static int ball_query(fgb_nq *nq, const QueryPoints &Q, const fgb_query_args *args, cudaStream_t s, fgb_nlist *nl) {
    const double R = args->r_max;
    StencilPlan plan;
    FGB_TRY(plan_stencil(nq, R, 0, s, &plan));
    BallArgs a;
    memset(&a, 0, sizeof(a));
    a.S = to_device(nq, plan);
    a.bf = nq->box.f;
    a.bd = nq->box.d;
    a.pts = nq->sorted;
    a.cell_start = nq->cell_start;
    a.qs = Q.sorted;
    a.qcell = Q.cell;
    a.nq = Q.n;
    a.p_orig = nq->points;
    a.q_orig = Q.orig;
    a.T = sqrt_threshold(R);
    band_around(a.T, r2_error_bound(plan, R), &a.band.lo, &a.band.hi);
    a.exclude = args->exclude_ii ? 1 : 0;
    QueryStatus *dst = nullptr;
    int st = dalloc_n(&dst, 1, s);
    if (st) {
        dfree(plan.table, s);
        return st;
    }
    cudaMemsetAsync(dst, 0, sizeof(QueryStatus), s);
    a.esc = &dst->esc;
    a.err = &dst->err;
    const int64_t nqq = Q.n;
    nl->n_query = nqq;
    nl->n_points = nq->n;
    st = st ? st : dalloc_n(&nl->counts, nqq, s);
    st = st ? st : dalloc_n(&nl->segments, nqq + 1, s);
    uint32_t *counts = reinterpret_cast<uint32_t *>(nl->counts);
    if (st == FGB_OK && nqq > 0) {
        {
            FGB_KSCOPE("k_ball_count", s);
            k_ball_count<<<(unsigned)((nqq + 127) / 128), 128, 0, s>>>(a, counts);
        }
        st = scan_u32_i64(counts, nl->segments, nqq, &dst->maxcount, s);
    } else if (st == FGB_OK) {
        cudaMemsetAsync(nl->segments, 0, sizeof(int64_t), s);
    }
    QueryStatus hs;
    memset(&hs, 0, sizeof(hs));
    if (st == FGB_OK && nqq > 0) {
        cudaMemcpyAsync(&hs.total, nl->segments + nqq, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&hs.maxcount, &dst->maxcount, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = fail(FGB_ERR_CUDA, "ball query count pass failed: %s", cudaGetErrorString(e));
    }
    if (st == FGB_OK && hs.total >= ((int64_t)1 << 40))
        st = fail(FGB_ERR_CAPACITY, "neighbor list of %lld pairs is too large", (long long)hs.total);
    nl->n_pairs = hs.total;
    st = st ? st : dalloc_n(&nl->qi, hs.total, s);
    st = st ? st : dalloc_n(&nl->pj, hs.total, s);
    st = st ? st : dalloc_n(&nl->dist, hs.total, s);
    if (st == FGB_OK && nqq > 0 && hs.total > 0) {
        int cap = (int)((hs.maxcount + 3) & ~3u);
        int block = 128;
        while (block > 32 && (size_t)cap * block * sizeof(uint2) > 96 * 1024) block >>= 1;
        const size_t smem = (size_t)cap * block * sizeof(uint2);
        const unsigned grid = (unsigned)((nqq + block - 1) / block);
        if (smem <= 200 * 1024) {
            if (smem > 48 * 1024)
                cudaFuncSetAttribute(k_ball_write<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            {
                FGB_KSCOPE("k_ball_write", s);
                k_ball_write<true><<<grid, block, smem, s>>>(a, nl->segments, counts, cap, nl->qi, nl->pj, nl->dist);
            }
        } else {
            {
                FGB_KSCOPE("k_ball_write", s);
                k_ball_write<false><<<(unsigned)((nqq + 127) / 128), 128, 0, s>>>(a, nl->segments, counts, 0, nl->qi,
                                                                                 nl->pj, nl->dist);
            }
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = fail(FGB_ERR_CUDA, "ball query write launch failed: %s", cudaGetErrorString(e));
    }
    if (st == FGB_OK) {
        cudaMemcpyAsync(&hs.esc, &dst->esc, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&hs.err, &dst->err, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = fail(FGB_ERR_CUDA, "ball query write pass failed: %s", cudaGetErrorString(e));
        else if (hs.err) st = fail(FGB_ERR_CUDA, "ball query: count and write passes disagree (code %d)", hs.err);
    }
    nl->escalations = (int64_t)hs.esc;
    nl->symmetric = Q.self ? 1 : 0;
    nl->kind = 0;
    dfree(dst, s);
    dfree(plan.table, s);
    return st;
}

}  // namespace fgb

using namespace fgb;

extern "C" int fgb_nq_query(fgb_nq *nq, const float *query_points, int64_t n_query, const fgb_query_args *args,
                            void *stream, fgb_nlist **out) {
    clear_error();
    if (!nq || !args || !out) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    const bool ball = args->r_max > 0.0;
    const bool knn = args->num_neighbors > 0;
    if (ball == knn) return fail(FGB_ERR_INVALID_ARG, "set exactly one of r_max > 0 and num_neighbors > 0");
    if (ball && !std::isfinite(args->r_max)) return fail(FGB_ERR_INVALID_ARG, "r_max must be finite");
    if (ball && !(args->r_max < 0.5 * nq->box.wmin * (1.0 - 1e-5)))
        return fail(FGB_ERR_BOX_TOO_SMALL, "r_max=%g must be below half the smallest box width (%g)", args->r_max,
                    0.5 * nq->box.wmin);
    if (query_points && query_points != nq->points && n_query < 0)
        return fail(FGB_ERR_INVALID_ARG, "n_query must be >= 0");
    cudaStream_t s = as_stream(stream);
    QueryPoints Q;
    int st = prepare_queries(nq, query_points, n_query, s, &Q);
    fgb_nlist *nl = new fgb_nlist();
    memset(nl, 0, sizeof(*nl));
    nl->stream = s;
    if (st == FGB_OK) st = ball ? ball_query(nq, Q, args, s, nl) : knn_query(nq, Q, args, s, nl);
    release_queries(&Q, s);
    if (st != FGB_OK) {
        fgb_nlist_destroy(nl);
        return st;
    }
    *out = nl;
    return FGB_OK;
}

extern "C" int fgb_nlist_size(const fgb_nlist *nl, int64_t *n_pairs, int64_t *n_query) {
    if (!nl) return fail(FGB_ERR_INVALID_ARG, "nlist is NULL");
    if (n_pairs) *n_pairs = nl->n_pairs;
    if (n_query) *n_query = nl->n_query;
    return FGB_OK;
}

extern "C" int fgb_nlist_arrays(const fgb_nlist *nl, const int32_t **qi, const int32_t **pj, const float **dist,
                                const int64_t **segments, const int32_t **counts) {
    if (!nl) return fail(FGB_ERR_INVALID_ARG, "nlist is NULL");
    if (qi) *qi = nl->qi;
    if (pj) *pj = nl->pj;
    if (dist) *dist = nl->dist;
    if (segments) *segments = nl->segments;
    if (counts) *counts = nl->counts;
    return FGB_OK;
}

extern "C" int fgb_nlist_escalations(const fgb_nlist *nl, int64_t *n) {
    if (!nl || !n) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    *n = nl->escalations;
    return FGB_OK;
}

namespace fgb {
// counts[q] from a non-decreasing query index array (one thread per pair).
__global__ void k_count_from_qi(const int32_t *__restrict__ qi, int64_t m, int64_t nq, uint32_t *__restrict__ counts,
                                int *err) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const int32_t q = qi[e];
    if (q < 0 || q >= nq || (e > 0 && qi[e - 1] > q)) {
        atomicExch(err, 1);
        return;
    }
    atomicAdd(counts + q, 1u);
}
}  // namespace fgb

extern "C" int fgb_nlist_from_arrays(int64_t n_query, int64_t n_points, const int32_t *qi, const int32_t *pj,
                                     const float *dist, int64_t m, int32_t symmetric, void *stream, fgb_nlist **out) {
    clear_error();
    if (!out) return fail(FGB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_query < 0 || n_points < 0 || m < 0 || (m > 0 && (!qi || !pj)))
        return fail(FGB_ERR_INVALID_ARG, "invalid arrays");
    cudaStream_t s = as_stream(stream);
    fgb_nlist *nl = new fgb_nlist();
    memset(nl, 0, sizeof(*nl));
    nl->stream = s;
    nl->n_query = n_query;
    nl->n_points = n_points;
    nl->n_pairs = m;
    nl->symmetric = symmetric ? 1 : 0;
    nl->kind = 2;
    int *err = nullptr;
    int st = dalloc_n(&nl->qi, m, s);
    st = st ? st : dalloc_n(&nl->pj, m, s);
    st = st ? st : dalloc_n(&nl->dist, m, s);
    st = st ? st : dalloc_n(&nl->counts, n_query, s);
    st = st ? st : dalloc_n(&nl->segments, n_query + 1, s);
    st = st ? st : dalloc_n(&err, 1, s);
    if (st == FGB_OK) {
        cudaMemcpyAsync(nl->qi, qi, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(nl->pj, pj, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, s);
        if (dist)
            cudaMemcpyAsync(nl->dist, dist, sizeof(float) * m, cudaMemcpyDeviceToDevice, s);
        else
            cudaMemsetAsync(nl->dist, 0, sizeof(float) * (m > 0 ? m : 1), s);
        cudaMemsetAsync(nl->counts, 0, sizeof(int32_t) * (n_query > 0 ? n_query : 1), s);
        cudaMemsetAsync(err, 0, sizeof(int), s);
        if (m > 0)
            {
                FGB_KSCOPE("k_count_from_qi", s);
                k_count_from_qi<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(
                    nl->qi, m, n_query, reinterpret_cast<uint32_t *>(nl->counts), err);
            }
        st = scan_u32_i64(reinterpret_cast<uint32_t *>(nl->counts), nl->segments, n_query, nullptr, s);
        int herr = 0;
        cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (st == FGB_OK && e != cudaSuccess) st = fail(FGB_ERR_CUDA, "nlist_from_arrays: %s", cudaGetErrorString(e));
        if (st == FGB_OK && herr)
            st = fail(FGB_ERR_INVALID_ARG, "query_point_indices must be non-decreasing and in [0, n_query)");
    }
    dfree(err, s);
    if (st != FGB_OK) {
        fgb_nlist_destroy(nl);
        return st;
    }
    *out = nl;
    return FGB_OK;
}

extern "C" void fgb_nlist_destroy(fgb_nlist *nl) {
    if (!nl) return;
    dfree(nl->qi, nl->stream);
    dfree(nl->pj, nl->stream);
    dfree(nl->dist, nl->stream);
    dfree(nl->counts, nl->stream);
    dfree(nl->segments, nl->stream);
    delete nl;
}
