// One frame split across ranks by contiguous ranges of query cells (the paper's parallel
// wrappers split per-particle work across workers, Section "Implementation"; here each
// rank is one GPU holding every point and walking a range of the query cells).
//
// fgb_nq_count_cells: half-stencil counts of the pairs whose first point lies in the
// range (every unordered pair belongs to exactly one cell's half stencil, hence to one
// range); summing every rank's partial counts gives the exact neighbor counts.
// fgb_nq_shard_segments: row starts of the range's own queries (a scan of the summed
// counts masked to them) and of the whole list.  fgb_nq_write_cells: the rows of the
// range's queries, sorted by point index, at the given row starts.
// fgb_rdf_compute_cells: the RDF histogram of the pairs whose first point lies in the
// range; the ranks' histograms sum to the frame's.
//
// The collectives between these calls (sums of counts and histograms) are the caller's.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "fgb_internal.cuh"

namespace fgb {

namespace {

struct ShardStatus {
    unsigned long long esc;
    int err;
    uint32_t maxcount;
    int64_t local_total;
};

// Narrows the cell-tile kernels of nq to [lo, hi) for one call.
struct WalkScope {
    fgb_nq *nq;
    WalkScope(fgb_nq *q, int64_t lo, int64_t hi) : nq(q) {
        nq->walk_set = 1;
        nq->walk_lo = lo;
        nq->walk_hi = hi;
    }
    ~WalkScope() { nq->walk_set = 0; }
};

int check_shard(const fgb_nq *nq, double r_max, int64_t cell_lo, int64_t cell_hi, StencilPlan *plan) {
    if (!nq) return fail(FGB_ERR_INVALID_ARG, "nq is NULL");
    if (nq->kind != 0) return fail(FGB_ERR_UNSUPPORTED, "sharded calls walk a cell list");
    if (cell_lo < 0 || cell_hi < cell_lo || cell_hi > nq->grid.ncell)
        return fail(FGB_ERR_INVALID_ARG, "cell range [%lld, %lld) outside [0, %lld)", (long long)cell_lo,
                    (long long)cell_hi, (long long)nq->grid.ncell);
    if (!(r_max > 0.0) || !std::isfinite(r_max)) return fail(FGB_ERR_INVALID_ARG, "r_max must be > 0");
    if (!(r_max < 0.5 * nq->box.wmin * (1.0 - 1e-5)))
        return fail(FGB_ERR_BOX_TOO_SMALL, "r_max=%g must be below half the smallest box width (%g)", r_max,
                    0.5 * nq->box.wmin);
    FGB_TRY(plan_stencil_host(nq->box, nq->grid, r_max, 0, plan, nullptr));
    if (!tile_ok(*plan))
        return fail(FGB_ERR_UNSUPPORTED, "sharded calls need the cell-tile route (every axis at least 2s+1 cells)");
    return FGB_OK;
}

// masked[index] = counts[index] for the points in sorted positions
// [cell_start[lo], cell_start[hi]), else 0.
__global__ void k_shard_mask(const float4 *__restrict__ pts, const uint32_t *__restrict__ cell_start, int64_t n,
                             int64_t lo, int64_t hi, const uint32_t *__restrict__ counts,
                             uint32_t *__restrict__ masked) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t plo = __ldg(cell_start + lo), phi = __ldg(cell_start + hi);
    const int i = __float_as_int(__ldg(pts + p).w);
    masked[i] = (p >= plo && p < phi) ? __ldg(counts + i) : 0u;
}

}  // namespace

}  // namespace fgb

using namespace fgb;

extern "C" int fgb_nq_count_cells(fgb_nq *nq, double r_max, int32_t exclude_ii, int64_t cell_lo, int64_t cell_hi,
                                  uint32_t *counts, void *stream) {
    clear_error();
    StencilPlan plan;
    FGB_TRY(check_shard(nq, r_max, cell_lo, cell_hi, &plan));
    if (nq->n > 0 && !counts) return fail(FGB_ERR_INVALID_ARG, "counts is NULL");
    if (nq->n == 0) return FGB_OK;
    cudaStream_t s = as_stream(stream);
    FGB_TRY(plan_stencil(nq, r_max, 0, s, &plan));
    ShardStatus *dst = nullptr;
    int st = dalloc_n(&dst, 1, s);
    if (st == FGB_OK) {
        FGB_CUDA(cudaMemsetAsync(dst, 0, sizeof(ShardStatus), s));
        WalkScope walk(nq, cell_lo, cell_hi);
        st = nl_count(nq, plan, r_max, exclude_ii ? 1 : 0, &dst->esc, &dst->err, counts, s);
    }
    dfree(dst, s);
    dfree(plan.table, s);
    return st;
}

extern "C" int fgb_nq_shard_segments(const fgb_nq *nq, int64_t cell_lo, int64_t cell_hi, const uint32_t *counts,
                                     int64_t *local_segments, int64_t *global_segments, int64_t *n_local_pairs,
                                     uint32_t *max_count, void *stream) {
    clear_error();
    if (!nq || nq->kind != 0) return fail(FGB_ERR_INVALID_ARG, "nq must be a cell-list NeighborQuery");
    if (cell_lo < 0 || cell_hi < cell_lo || cell_hi > nq->grid.ncell)
        return fail(FGB_ERR_INVALID_ARG, "cell range outside the grid");
    if (!local_segments || (nq->n > 0 && !counts)) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = as_stream(stream);
    const int64_t n = nq->n;
    uint32_t *masked = nullptr;
    ShardStatus *dst = nullptr;
    int st = dalloc_n(&masked, (size_t)std::max<int64_t>(n, 1), s);
    st = st ? st : dalloc_n(&dst, 1, s);
    if (st == FGB_OK && n > 0) {
        {
            FGB_KSCOPE("k_shard_mask", s);
            k_shard_mask<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(nq->sorted, nq->cell_start, n, cell_lo, cell_hi,
                                                                    counts, masked);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = fail(FGB_ERR_CUDA, "shard mask launch failed: %s", cudaGetErrorString(e));
        st = st ? st : scan_u32_i64(masked, local_segments, n, &dst->maxcount, s);
        if (st == FGB_OK && global_segments) st = scan_u32_i64(counts, global_segments, n, nullptr, s);
    } else if (st == FGB_OK) {
        cudaMemsetAsync(local_segments, 0, sizeof(int64_t), s);
        if (global_segments) cudaMemsetAsync(global_segments, 0, sizeof(int64_t), s);
        cudaMemsetAsync(dst, 0, sizeof(ShardStatus), s);
    }
    ShardStatus hs;
    memset(&hs, 0, sizeof(hs));
    if (st == FGB_OK) {
        cudaMemcpyAsync(&hs.local_total, local_segments + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&hs.maxcount, &dst->maxcount, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = fail(FGB_ERR_CUDA, "shard segments failed: %s", cudaGetErrorString(e));
    }
    if (st == FGB_OK && n_local_pairs) *n_local_pairs = hs.local_total;
    if (st == FGB_OK && max_count) *max_count = hs.maxcount;
    dfree(masked, s);
    dfree(dst, s);
    return st;
}

extern "C" int fgb_nq_write_cells(fgb_nq *nq, double r_max, int32_t exclude_ii, int64_t cell_lo, int64_t cell_hi,
                                  const int64_t *segments, const uint32_t *counts, uint32_t max_count, int32_t *qi,
                                  int32_t *pj, float *dist, void *stream) {
    clear_error();
    StencilPlan plan;
    FGB_TRY(check_shard(nq, r_max, cell_lo, cell_hi, &plan));
    if (nq->n == 0 || cell_hi == cell_lo) return FGB_OK;
    if (!segments || !counts || !qi || !pj || !dist) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    if (max_count > 16384) return fail(FGB_ERR_UNSUPPORTED, "more than 16384 neighbors of one point");
    cudaStream_t s = as_stream(stream);
    FGB_TRY(plan_stencil(nq, r_max, 0, s, &plan));
    ShardStatus *dst = nullptr;
    int st = dalloc_n(&dst, 1, s);
    if (st == FGB_OK) {
        FGB_CUDA(cudaMemsetAsync(dst, 0, sizeof(ShardStatus), s));
        const int cap = (int)((max_count + 3) & ~3u);
        WalkScope walk(nq, cell_lo, cell_hi);
        st = nl_write(nq, plan, r_max, exclude_ii ? 1 : 0, &dst->err, segments, counts, std::max(cap, 4), nq->n, qi,
                      pj, dist, s);
    }
    ShardStatus hs;
    memset(&hs, 0, sizeof(hs));
    if (st == FGB_OK) {
        cudaMemcpyAsync(&hs.err, &dst->err, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = fail(FGB_ERR_CUDA, "sharded write failed: %s", cudaGetErrorString(e));
        else if (hs.err) st = fail(FGB_ERR_CUDA, "sharded write: rows disagree with the given counts (code %d)", hs.err);
    }
    dfree(dst, s);
    dfree(plan.table, s);
    return st;
}

extern "C" int fgb_rdf_compute_cells(fgb_rdf *r, fgb_nq *nq, int64_t cell_lo, int64_t cell_hi, int32_t reset,
                                     void *stream) {
    clear_error();
    if (!r) return fail(FGB_ERR_INVALID_ARG, "rdf is NULL");
    double r_max = 0.0, r_min = 0.0;
    int32_t bins = 0;
    FGB_TRY(fgb_rdf_params(r, &bins, &r_max, &r_min));
    StencilPlan plan;
    FGB_TRY(check_shard(nq, r_max, cell_lo, cell_hi, &plan));
    if (bins > 1024) return fail(FGB_ERR_UNSUPPORTED, "sharded RDF: at most 1024 bins");
    const int nfull = (2 * plan.s[0] + 1) * (2 * plan.s[1] + 1) * (2 * plan.s[2] + 1);
    if ((nfull + 1) / 2 > 128) return fail(FGB_ERR_UNSUPPORTED, "sharded RDF: stencil too wide");
    WalkScope walk(nq, cell_lo, cell_hi);
    return fgb_rdf_compute(r, nq, nullptr, 0, nullptr, reset, stream);
}
