// Ball query (r_max) and the NeighborList handle.  See query.cu for the overview.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "fgb_ball.cuh"

namespace fgb {

// FGB_THREAD_KERNELS=1 selects the thread-per-query kernels even where the cell-tile
// kernels apply (for comparisons).
bool force_thread_kernels() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("FGB_THREAD_KERNELS");
        v = (e && e[0] == '1') ? 1 : 0;
    }
    return v == 1;
}

// FGB_SPLIT_KERNELS=0 keeps few-query grids on the one-thread-per-query kernels (ball
// count and write, per-point RDF) instead of the ones that give a query 8 lanes or a
// warp (so that both stay covered by tests).
bool split_kernels_enabled() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("FGB_SPLIT_KERNELS");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

bool force_tile_kernels() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("FGB_TILE_KERNELS");
        v = (e && e[0] == '1') ? 1 : 0;
    }
    return v == 1;
}

int knn_query(fgb_nq *nq, const QueryPoints &Q, const fgb_query_args *a, cudaStream_t s, fgb_nlist *nl);

template <int MODE, bool CHECKJ>
__global__ void __launch_bounds__(128) k_ball_count(BallArgs a, uint32_t *__restrict__ counts) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.nq) return;
    const float4 q = a.qs[t];
    const int i = __float_as_int(q.w);
    int nesc = 0;
    counts[i] = ball_count_walk<MODE, CHECKJ>(a, q, a.qcell[t], i, nesc);
    if (nesc) atomicAdd(a.esc, (unsigned long long)nesc);
}

// Write pass.  Each thread walks its query again and appends the neighbor indices to a
// shared slab laid out [slot][thread] (4 bytes per hit keeps occupancy up).  The warp
// then takes its 32 queries one at a time: up to 64 hits are sorted by a bitonic network
// across the warp (two keys per lane); longer lists are ranked by counting the smaller
// indices in the slab column (broadcast reads).  The float32 distance is recomputed from
// the input coordinates and every segment is stored sorted by point index with
// coalesced stores.
template <int MODE>
__global__ void __launch_bounds__(128) k_ball_write(BallArgs a, const int64_t *__restrict__ seg,
                                                    const uint32_t *__restrict__ counts, int cap,
                                                    int32_t *__restrict__ qi_out, int32_t *__restrict__ pj_out,
                                                    float *__restrict__ d_out) {
    extern __shared__ uint32_t slab[];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int B = blockDim.x + 1;  // odd row stride: a column read by 32 lanes hits 32 banks
    int i = -1;
    uint32_t n = 0;
    int64_t off = 0;
    if (t < a.nq) {
        const float4 q = a.qs[t];
        i = __float_as_int(q.w);
        off = seg[i];
        const uint32_t want = counts[i];
        ball_visit_m<MODE>(a, q, a.qcell[t], i, [&](int j, float3, float, double) {
            if (n < (uint32_t)cap) slab[n * B + threadIdx.x] = (uint32_t)j;
            ++n;
        });
        if (n != want || n > (uint32_t)cap) atomicExch(a.err, n > (uint32_t)cap ? 1 : 2);
        n = min(n, (uint32_t)cap);
    }
    const int lane = threadIdx.x & 31;
    const uint32_t *wslab = slab + (threadIdx.x & ~31);
    for (int L = 0; L < 32; ++L) {
        const uint32_t nL = __shfl_sync(0xffffffffu, n, L);
        if (nL == 0) continue;
        const int iL = __shfl_sync(0xffffffffu, i, L);
        const int64_t oL = __shfl_sync(0xffffffffu, off, L);
        const uint32_t *col = wslab + L;
        const float xi0 = __ldg(a.q_orig + 3 * (int64_t)iL), xi1 = __ldg(a.q_orig + 3 * (int64_t)iL + 1),
                    xi2 = __ldg(a.q_orig + 3 * (int64_t)iL + 2);
        if (nL <= 64) {
            // bitonic sort of 64 keys, two per lane (elements 2 lane and 2 lane + 1)
            uint32_t v0 = 2 * lane < (int)nL ? col[(2 * lane) * B] : 0xffffffffu;
            uint32_t v1 = 2 * lane + 1 < (int)nL ? col[(2 * lane + 1) * B] : 0xffffffffu;
#pragma unroll
            for (int k = 2; k <= 64; k <<= 1) {
                const bool asc = ((2 * lane) & k) == 0;
#pragma unroll
                for (int jj = k >> 1; jj > 0; jj >>= 1) {
                    if (jj == 1) {
                        const uint32_t lo = min(v0, v1), hi = max(v0, v1);
                        v0 = asc ? lo : hi;
                        v1 = asc ? hi : lo;
                    } else {
                        const int lm = jj >> 1;
                        const uint32_t p0 = __shfl_xor_sync(0xffffffffu, v0, lm);
                        const uint32_t p1 = __shfl_xor_sync(0xffffffffu, v1, lm);
                        const bool takemin = ((lane & lm) == 0) == asc;
                        v0 = takemin ? min(v0, p0) : max(v0, p0);
                        v1 = takemin ? min(v1, p1) : max(v1, p1);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const uint32_t k = 2 * lane + r;
                const uint32_t j = r ? v1 : v0;
                if (k < nL) {
                    const float3 d = bond_f32v(a.bf, xi0, xi1, xi2, __ldg(a.p_orig + 3 * (int64_t)j),
                                               __ldg(a.p_orig + 3 * (int64_t)j + 1), __ldg(a.p_orig + 3 * (int64_t)j + 2));
                    __stcs(qi_out + oL + k, iL);
                    __stcs(pj_out + oL + k, (int32_t)j);
                    __stcs(d_out + oL + k, sqrtf(r2_f32(d.x, d.y, d.z)));
                }
            }
            continue;
        }
        for (uint32_t base = 0; base < nL; base += 32) {
            const uint32_t k = base + lane;
            const bool act = k < nL;
            const uint32_t j = act ? col[k * B] : 0u;
            uint32_t rank = 0;
            for (uint32_t m = 0; m < nL; ++m) rank += col[m * B] < j ? 1u : 0u;
            if (act) {
                const float3 d = bond_f32v(a.bf, xi0, xi1, xi2, __ldg(a.p_orig + 3 * (int64_t)j),
                                           __ldg(a.p_orig + 3 * (int64_t)j + 1), __ldg(a.p_orig + 3 * (int64_t)j + 2));
                // streaming stores: the list is not re-read here, keep L2 for the walks
                __stcs(qi_out + oL + rank, iL);
                __stcs(pj_out + oL + rank, (int32_t)j);
                __stcs(d_out + oL + rank, sqrtf(r2_f32(d.x, d.y, d.z)));
            }
        }
    }
}

// ------------------------------------------------------------------ split queries
//
// Few queries (a small grid): G consecutive lanes share one query, lane g taking the
// candidates beg + g, beg + g + G, ... of every stencil cell (coalesced across the
// group), so the GPU holds G times as many warps.  Pairs are decided exactly as in the
// single-lane walks.  G = 8 below 128 queries per SM, a whole warp below 32.

constexpr int kSplitG = 8;

template <int MODE, bool CHECKJ, int G, class F>
__device__ __forceinline__ void split_walk(const BallArgs &a, float4 q, uint32_t qc, int i, int g, F &&fn) {
    int cx, cy, cz;
    cell_coords(qc, a.S.nc, cx, cy, cz);
    const int excl = a.exclude ? i : -1;
    const float lo = a.band.lo, hi = a.band.hi;
    for_stencil(a.S, cx, cy, cz, make_float3(q.x, q.y, q.z), false,
                [&](int cell, float qx, float qy, float qz, bool) {
                    const uint32_t beg = __ldg(a.cell_start + cell), end = __ldg(a.cell_start + cell + 1);
                    for (uint32_t p = beg + (uint32_t)g; p < end; p += G) {
                        const float4 c = __ldg(a.pts + p);
                        const float3 d = cand_disp_m<MODE>(a.bf, c, qx, qy, qz);
                        const float r2 = r2_f32(d.x, d.y, d.z);
                        if (r2 < hi) {
                            const int j = __float_as_int(c.w);
                            if (j == excl) continue;
                            if (r2 < lo)
                                fn(j, 0);
                            else if (exact_r2_idx(a.bd, a.q_orig, i, a.p_orig, j) < a.T)
                                fn(j, 1);
                            else
                                fn(-1, 1);
                        }
                    }
                });
}

// Neighbor count of every query (G lanes per query).
template <int MODE, int G>
__global__ void __launch_bounds__(128) k_ball_count_split(BallArgs a, uint32_t *__restrict__ counts) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t qx = t / G;
    const int g = (int)(t % G);
    const bool act = qx < a.nq;
    uint32_t cnt = 0;
    int nesc = 0, i = -1;
    if (act) {
        const float4 q = a.qs[qx];
        i = __float_as_int(q.w);
        split_walk<MODE, true, G>(a, q, a.qcell[qx], i, g, [&](int j, int esc) {
            nesc += esc;
            cnt += j >= 0 ? 1u : 0u;
        });
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (act && g == 0) counts[i] = cnt;
    if (nesc) atomicAdd(a.esc, (unsigned long long)nesc);
}

// Rows of every query (G lanes per query), unsorted: each lane counts its share,
// takes its offset in the row from an exclusive scan over the group, and writes its
// neighbors there (bounded by the row's count); sort_segments sorts the rows.
template <int MODE, int G>
__global__ void __launch_bounds__(128) k_ball_write_split(BallArgs a, const int64_t *__restrict__ seg,
                                                          const uint32_t *__restrict__ counts,
                                                          int32_t *__restrict__ qi_out, int32_t *__restrict__ pj_out,
                                                          float *__restrict__ d_out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t qx = t / G;
    const int g = (int)(t % G);
    const bool act = qx < a.nq;
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t qc = 0, mine = 0;
    int i = -1;
    if (act) {
        q = a.qs[qx];
        qc = a.qcell[qx];
        i = __float_as_int(q.w);
        split_walk<MODE, true, G>(a, q, qc, i, g, [&](int j, int) { mine += j >= 0 ? 1u : 0u; });
    }
    uint32_t inc = mine;
#pragma unroll
    for (int d = 1; d < G; d <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, d);
        if (g >= d) inc += u;
    }
    if (!act) return;
    const int64_t off = seg[i];
    const uint32_t want = counts[i];
    if (g == G - 1 && inc != want) atomicExch(a.err, 2);
    const float xi0 = __ldg(a.q_orig + 3 * (int64_t)i), xi1 = __ldg(a.q_orig + 3 * (int64_t)i + 1),
                xi2 = __ldg(a.q_orig + 3 * (int64_t)i + 2);
    uint32_t n = inc - mine;
    split_walk<MODE, true, G>(a, q, qc, i, g, [&](int j, int) {
        if (j < 0) return;
        if (n < want) {
            const float3 d = bond_f32v(a.bf, xi0, xi1, xi2, __ldg(a.p_orig + 3 * (int64_t)j),
                                       __ldg(a.p_orig + 3 * (int64_t)j + 1), __ldg(a.p_orig + 3 * (int64_t)j + 2));
            qi_out[off + n] = i;
            pj_out[off + n] = j;
            d_out[off + n] = sqrtf(r2_f32(d.x, d.y, d.z));
        }
        ++n;
    });
}

// Write pass for long rows (thread per query): each query appends its neighbors to its
// segment in walk order (bounded by its count), and sort_segments then sorts every row
// by point index with a warp per row.
template <int MODE>
__global__ void __launch_bounds__(128) k_ball_write_rows(BallArgs a, const int64_t *__restrict__ seg,
                                                         const uint32_t *__restrict__ counts,
                                                         int32_t *__restrict__ qi_out, int32_t *__restrict__ pj_out,
                                                         float *__restrict__ d_out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.nq) return;
    const float4 q = a.qs[t];
    const int i = __float_as_int(q.w);
    const int64_t off = seg[i];
    const uint32_t want = counts[i];
    const float xi0 = __ldg(a.q_orig + 3 * (int64_t)i), xi1 = __ldg(a.q_orig + 3 * (int64_t)i + 1),
                xi2 = __ldg(a.q_orig + 3 * (int64_t)i + 2);
    uint32_t n = 0;
    ball_visit_m<MODE>(a, q, a.qcell[t], i, [&](int j, float3, float, double) {
        if (n < want) {
            const float3 d = bond_f32v(a.bf, xi0, xi1, xi2, __ldg(a.p_orig + 3 * (int64_t)j),
                                       __ldg(a.p_orig + 3 * (int64_t)j + 1), __ldg(a.p_orig + 3 * (int64_t)j + 2));
            qi_out[off + n] = i;
            pj_out[off + n] = j;
            d_out[off + n] = sqrtf(r2_f32(d.x, d.y, d.z));
        }
        ++n;
    });
    if (n != want) atomicExch(a.err, 2);
}

// Write pass for very large neighbor counts: insertion straight into the output arrays.
template <int MODE>
__global__ void __launch_bounds__(128) k_ball_write_global(BallArgs a, const int64_t *__restrict__ seg,
                                                           const uint32_t *__restrict__ counts,
                                                           int32_t *__restrict__ qi_out, int32_t *__restrict__ pj_out,
                                                           float *__restrict__ d_out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.nq) return;
    const float4 q = a.qs[t];
    const int i = __float_as_int(q.w);
    const int64_t off = seg[i];
    const uint32_t want = counts[i];
    uint32_t n = 0;
    ball_visit_m<MODE>(a, q, a.qcell[t], i, [&](int j, float3, float r2, double e) {
        if (n >= want) {
            atomicExch(a.err, 1);
            return;
        }
        const float dist = e < 0.0 ? sqrtf(r2) : (float)sqrt(e);
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
        ++n;
    });
    if (n != want) atomicExch(a.err, 2);
    for (uint32_t k = 0; k < n; ++k) qi_out[off + k] = i;
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
    a.self = Q.self ? 1 : 0;
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
    const bool checkj = !Q.self && a.exclude;
    const bool tile = Q.self && tile_ok(plan) && tile_worth(nq) && (nq->walk_set || !force_thread_kernels());
    // few queries: several lanes per query (the single-lane kernels would leave most SMs idle)
    const bool split = !tile && nqq < (int64_t)num_sms() * 128 && split_kernels_enabled();
    const int split_g = nqq < (int64_t)num_sms() * 32 ? 32 : kSplitG;
    if (st == FGB_OK && nqq > 0 && tile) {
        // 2D: the tile kernels walk only the points' layer; a point off the plane keeps a
        // count of zero instead of an unwritten one
        if (nq->box.is2d && cudaMemsetAsync(counts, 0, sizeof(uint32_t) * nqq, s) != cudaSuccess)
            st = fail(FGB_ERR_CUDA, "memset failed");
        if (nl_kernels_enabled())
            st = st ? st : nl_count(nq, plan, R, a.exclude, a.esc, a.err, counts, s);
        else
            st = st ? st : tile_count(nq, plan, R, a.exclude, a.esc, a.err, counts, s);
        st = st ? st : scan_u32_i64(counts, nl->segments, nqq, &dst->maxcount, s);
    } else if (st == FGB_OK && nqq > 0 && split) {
        {
            FGB_KSCOPE("k_ball_count_split", s);
            const unsigned g2 = (unsigned)((nqq * split_g + 127) / 128);
            if (split_g == 32)
                (a.S.mode == 0 ? k_ball_count_split<0, 32> : k_ball_count_split<1, 32>)<<<g2, 128, 0, s>>>(a, counts);
            else
                (a.S.mode == 0 ? k_ball_count_split<0, kSplitG>
                               : k_ball_count_split<1, kSplitG>)<<<g2, 128, 0, s>>>(a, counts);
        }
        st = scan_u32_i64(counts, nl->segments, nqq, &dst->maxcount, s);
    } else if (st == FGB_OK && nqq > 0) {
        const unsigned grid = (unsigned)((nqq + 127) / 128);
        {
            FGB_KSCOPE("k_ball_count", s);
            if (a.S.mode == 0 && !checkj)
                k_ball_count<0, false><<<grid, 128, 0, s>>>(a, counts);
            else if (a.S.mode == 0)
                k_ball_count<0, true><<<grid, 128, 0, s>>>(a, counts);
            else if (!checkj)
                k_ball_count<1, false><<<grid, 128, 0, s>>>(a, counts);
            else
                k_ball_count<1, true><<<grid, 128, 0, s>>>(a, counts);
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
        const int cap = (int)((hs.maxcount + 3) & ~3u);
        if (tile && nl_kernels_enabled()) {
            st = nl_write(nq, plan, R, a.exclude, a.err, nl->segments, counts, cap, nqq, nl->qi, nl->pj, nl->dist, s);
        } else if (tile && cap <= 128 && tile_write_smem(cap) <= 160 * 1024) {
            st = tile_write(nq, plan, R, a.exclude, a.err, nl->segments, counts, cap, nl->qi, nl->pj, nl->dist, s);
        } else if (tile && cap <= 16384) {
            // long rows: appended to the list by the cell tiles, then sorted per row
            st = tile_write_global(nq, plan, R, a.exclude, a.err, nl->segments, counts, nl->qi, nl->pj, nl->dist, s);
            st = st ? st
                    : sort_segments(nl->segments, nqq, cap, nq->n, nl->qi, nl->pj, nl->dist, s);
        } else if (cap <= 16384 && (split || cap > 64)) {
            // rows written unsorted, then sorted per row by a warp (a rank sort of each
            // row by one warp costs O(row^2) and held c1's 268-entry rows to 128 warps)
            if (split) {
                FGB_KSCOPE("k_ball_write_split", s);
                const unsigned g2 = (unsigned)((nqq * split_g + 127) / 128);
                auto kern = split_g == 32 ? (a.S.mode == 0 ? k_ball_write_split<0, 32> : k_ball_write_split<1, 32>)
                                          : (a.S.mode == 0 ? k_ball_write_split<0, kSplitG>
                                                           : k_ball_write_split<1, kSplitG>);
                kern<<<g2, 128, 0, s>>>(a, nl->segments, counts, nl->qi, nl->pj, nl->dist);
            } else {
                FGB_KSCOPE("k_ball_write_rows", s);
                const unsigned g2 = (unsigned)((nqq + 127) / 128);
                if (a.S.mode == 0)
                    k_ball_write_rows<0><<<g2, 128, 0, s>>>(a, nl->segments, counts, nl->qi, nl->pj, nl->dist);
                else
                    k_ball_write_rows<1><<<g2, 128, 0, s>>>(a, nl->segments, counts, nl->qi, nl->pj, nl->dist);
            }
            st = sort_segments(nl->segments, nqq, cap, nq->n, nl->qi, nl->pj, nl->dist, s);
        } else {
        int block = 128;
        while (block > 32 && (size_t)cap * (block + 1) * sizeof(uint32_t) > 100 * 1024) block >>= 1;
        const size_t smem = (size_t)cap * (block + 1) * sizeof(uint32_t);
        const unsigned grid = (unsigned)((nqq + block - 1) / block);
        if (smem <= 200 * 1024) {
            if (a.S.mode == 0) {
                if (smem > 48 * 1024)
                    cudaFuncSetAttribute(k_ball_write<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                FGB_KSCOPE("k_ball_write", s);
                k_ball_write<0><<<grid, block, smem, s>>>(a, nl->segments, counts, cap, nl->qi, nl->pj, nl->dist);
            } else {
                if (smem > 48 * 1024)
                    cudaFuncSetAttribute(k_ball_write<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                FGB_KSCOPE("k_ball_write", s);
                k_ball_write<1><<<grid, block, smem, s>>>(a, nl->segments, counts, cap, nl->qi, nl->pj, nl->dist);
            }
        } else {
            const unsigned g2 = (unsigned)((nqq + 127) / 128);
            FGB_KSCOPE("k_ball_write_global", s);
            if (a.S.mode == 0)
                k_ball_write_global<0><<<g2, 128, 0, s>>>(a, nl->segments, counts, nl->qi, nl->pj, nl->dist);
            else
                k_ball_write_global<1><<<g2, 128, 0, s>>>(a, nl->segments, counts, nl->qi, nl->pj, nl->dist);
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

// Pairs of a self ball query on uniformly spread points, n (n - 1) v / V (v the ball's
// volume, the disc's area in 2D), with a margin of 10 % plus 8 per point.
static int64_t capacity_estimate(const fgb_nq *nq, double R) {
    const double n = (double)nq->n;
    const double v = nq->box.is2d ? M_PI * R * R : 4.0 / 3.0 * M_PI * R * R * R;
    const double V = nq->box.is2d ? nq->box.p[0] * nq->box.p[1] : nq->box.p[0] * nq->box.p[1] * nq->box.p[2];
    const double est = n * std::max(n - 1.0, 0.0) * v / V;
    return (int64_t)std::min(1.1 * est + 8.0 * n + 1024.0, (double)((int64_t)1 << 40));
}

// The self ball query without host synchronisation: count, scan and write are queued on
// s into arrays of `capacity` pairs; the status words (list size, longest row, FP64
// decisions, error flag) are copied to a pinned slot and `done` recorded after them.
// nlist_ready completes it.  Only the cell-tile route of the NeighborList kernels has
// this form; the caller runs ball_query otherwise.
static int ball_query_async(fgb_nq *nq, const fgb_query_args *args, int64_t capacity, cudaStream_t s,
                            fgb_nlist *nl) {
    const double R = args->r_max;
    StencilPlan plan;
    FGB_TRY(plan_stencil(nq, R, 0, s, &plan));
    const int64_t n = nq->n;
    if (capacity <= 0) capacity = capacity_estimate(nq, R);
    nl->n_query = n;
    nl->n_points = n;
    nl->symmetric = 1;
    nl->kind = 0;
    nl->src = nq;
    nl->r_max = R;
    nl->exclude = args->exclude_ii ? 1 : 0;
    nl->capacity = capacity;
    QueryStatus *dst = nullptr;
    int st = dalloc_n(&dst, 1, s);
    st = st ? st : pinned_slot(&nl->hstatus);
    if (st == FGB_OK && cudaEventCreateWithFlags(&nl->done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        nl->done = nullptr;
        st = fail(FGB_ERR_CUDA, "event creation failed");
    }
    nl->dstatus = dst;
    st = st ? st : dalloc_n(&nl->counts, n, s);
    st = st ? st : dalloc_n(&nl->segments, n + 1, s);
    st = st ? st : dalloc_n(&nl->qi, capacity, s);
    st = st ? st : dalloc_n(&nl->pj, capacity, s);
    st = st ? st : dalloc_n(&nl->dist, capacity, s);
    uint32_t *counts = reinterpret_cast<uint32_t *>(nl->counts);
    if (st == FGB_OK && cudaMemsetAsync(dst, 0, sizeof(QueryStatus), s) != cudaSuccess)
        st = fail(FGB_ERR_CUDA, "memset failed");
    if (st == FGB_OK && nq->box.is2d && cudaMemsetAsync(counts, 0, sizeof(uint32_t) * n, s) != cudaSuccess)
        st = fail(FGB_ERR_CUDA, "memset failed");
    st = st ? st : nl_count(nq, plan, R, nl->exclude, &dst->esc, &dst->err, counts, s);
    st = st ? st : scan_u32_i64(counts, nl->segments, n, &dst->maxcount, s);
    st = st ? st
            : nl_write(nq, plan, R, nl->exclude, &dst->err, nl->segments, counts, 0, n, nl->qi, nl->pj, nl->dist, s,
                       capacity);
    if (st == FGB_OK) {
        QueryStatus *h = static_cast<QueryStatus *>(nl->hstatus);
        cudaMemcpyAsync(h, dst, sizeof(QueryStatus), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&h->total, nl->segments + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        cudaEventRecord(nl->done, s);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = fail(FGB_ERR_CUDA, "asynchronous ball query: %s", cudaGetErrorString(e));
    }
    dfree(plan.table, s);
    if (st == FGB_OK) nl->pending = 1;
    return st;
}

// The waiting half: a list that did not fit its capacity, or held a row the
// asynchronous fallback could not take, is written again by the synchronous route
// (counts and segments are final by then).
static int nlist_finish(fgb_nlist *nl) {
    cudaStream_t s = nl->stream;
    nl->pending = 0;
    if (cudaEventSynchronize(nl->done) != cudaSuccess) {
        const cudaError_t e = cudaGetLastError();
        return fail(FGB_ERR_CUDA, "asynchronous ball query failed: %s", cudaGetErrorString(e));
    }
    const QueryStatus h = *static_cast<const QueryStatus *>(nl->hstatus);
    pinned_release(nl->hstatus, nullptr);
    cudaEventDestroy(nl->done);
    nl->hstatus = nullptr;
    nl->done = nullptr;
    QueryStatus *dst = static_cast<QueryStatus *>(nl->dstatus);
    int st = FGB_OK;
    if (h.total >= ((int64_t)1 << 40))
        st = fail(FGB_ERR_CAPACITY, "neighbor list of %lld pairs is too large", (long long)h.total);
    const bool grow = h.total > nl->capacity;
    if (st == FGB_OK && (grow || h.err)) {
        fgb_nq *nq = nl->src;
        if (grow) {
            dfree(nl->qi, s);
            dfree(nl->pj, s);
            dfree(nl->dist, s);
            nl->qi = nl->pj = nullptr;
            nl->dist = nullptr;
            st = dalloc_n(&nl->qi, h.total, s);
            st = st ? st : dalloc_n(&nl->pj, h.total, s);
            st = st ? st : dalloc_n(&nl->dist, h.total, s);
            nl->capacity = h.total;
        }
        StencilPlan plan;
        plan.table = nullptr;
        st = st ? st : plan_stencil(nq, nl->r_max, 0, s, &plan);
        if (st == FGB_OK && cudaMemsetAsync(&dst->err, 0, sizeof(int), s) != cudaSuccess)
            st = fail(FGB_ERR_CUDA, "memset failed");
        const int cap = (int)((h.maxcount + 3) & ~3u);
        st = st ? st
                : nl_write(nq, plan, nl->r_max, nl->exclude, &dst->err, nl->segments,
                           reinterpret_cast<const uint32_t *>(nl->counts), std::max(cap, 4), nl->n_query, nl->qi,
                           nl->pj, nl->dist, s);
        int err = 0;
        if (st == FGB_OK) {
            cudaMemcpyAsync(&err, &dst->err, sizeof(int), cudaMemcpyDeviceToHost, s);
            const cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = fail(FGB_ERR_CUDA, "ball query rewrite failed: %s", cudaGetErrorString(e));
            else if (err) st = fail(FGB_ERR_CUDA, "ball query: count and write passes disagree (code %d)", err);
        }
        dfree(plan.table, s);
        nl->repaired = 1;
    }
    dfree(nl->dstatus, s);
    nl->dstatus = nullptr;
    nl->n_pairs = h.total;
    nl->escalations = (int64_t)h.esc;
    return st;
}

int nlist_ready(const fgb_nlist *nl) {
    if (!nl || !nl->pending) return FGB_OK;
    return nlist_finish(const_cast<fgb_nlist *>(nl));
}

}  // namespace fgb

using namespace fgb;

extern "C" int fgb_nq_query_async(fgb_nq *nq, const fgb_query_args *args, int64_t capacity, void *stream,
                                  fgb_nlist **out) {
    clear_error();
    if (!nq || !args || !out) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (!(args->r_max > 0.0) || args->num_neighbors > 0 || !std::isfinite(args->r_max))
        return fail(FGB_ERR_INVALID_ARG, "an asynchronous query is a ball query: r_max > 0, num_neighbors 0");
    if (capacity < 0) return fail(FGB_ERR_INVALID_ARG, "capacity must be >= 0");
    if (!(args->r_max < 0.5 * nq->box.wmin * (1.0 - 1e-5)))
        return fail(FGB_ERR_BOX_TOO_SMALL, "r_max=%g must be below half the smallest box width (%g)", args->r_max,
                    0.5 * nq->box.wmin);
    bool async = nq->kind == 0 && nq->n > 0 && !nq->walk_set && nl_kernels_enabled() && tile_worth(nq) &&
                 !force_thread_kernels();
    if (async) {
        StencilPlan plan;
        FGB_TRY(plan_stencil_host(nq->box, nq->grid, args->r_max, 0, &plan, nullptr));
        async = tile_ok(plan);
    }
    if (!async) return fgb_nq_query(nq, nullptr, 0, args, stream, out);
    cudaStream_t s = as_stream(stream);
    fgb_nlist *nl = new fgb_nlist();
    memset(nl, 0, sizeof(*nl));
    nl->stream = s;
    const int st = ball_query_async(nq, args, capacity, s, nl);
    if (st != FGB_OK) {
        if (nl->done) cudaEventSynchronize(nl->done);
        fgb_nlist_destroy(nl);
        return st;
    }
    *out = nl;
    return FGB_OK;
}

extern "C" int fgb_nlist_wait(fgb_nlist *nl, int32_t *rewritten) {
    clear_error();
    if (!nl) return fail(FGB_ERR_INVALID_ARG, "nlist is NULL");
    FGB_TRY(nlist_ready(nl));
    if (rewritten) *rewritten = nl->repaired;
    return FGB_OK;
}

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
    fgb_nlist *nl = new fgb_nlist();
    memset(nl, 0, sizeof(*nl));
    nl->stream = s;
    int st = FGB_OK;
    if (nq->kind == 2) {
        st = fail(FGB_ERR_UNSUPPORTED, "a NeighborQuery of points only answers no query; pass a NeighborList");
    } else if (nq->kind == 1) {
        st = ball ? aabb_ball_query(nq, query_points, n_query, args, s, nl)
                  : aabb_knn_query(nq, query_points, n_query, args, s, nl);
    } else {
        QueryPoints Q;
        st = prepare_queries(nq, query_points, n_query, s, &Q);
        if (st == FGB_OK) st = ball ? ball_query(nq, Q, args, s, nl) : knn_query(nq, Q, args, s, nl);
        release_queries(&Q, s);
    }
    if (st != FGB_OK) {
        fgb_nlist_destroy(nl);
        return st;
    }
    *out = nl;
    return FGB_OK;
}

extern "C" int fgb_nlist_size(const fgb_nlist *nl, int64_t *n_pairs, int64_t *n_query) {
    if (!nl) return fail(FGB_ERR_INVALID_ARG, "nlist is NULL");
    FGB_TRY(nlist_ready(nl));
    if (n_pairs) *n_pairs = nl->n_pairs;
    if (n_query) *n_query = nl->n_query;
    return FGB_OK;
}

extern "C" int fgb_nlist_arrays(const fgb_nlist *nl, const int32_t **qi, const int32_t **pj, const float **dist,
                                const int64_t **segments, const int32_t **counts) {
    if (!nl) return fail(FGB_ERR_INVALID_ARG, "nlist is NULL");
    FGB_TRY(nlist_ready(nl));
    if (qi) *qi = nl->qi;
    if (pj) *pj = nl->pj;
    if (dist) *dist = nl->dist;
    if (segments) *segments = nl->segments;
    if (counts) *counts = nl->counts;
    return FGB_OK;
}

extern "C" int fgb_nlist_escalations(const fgb_nlist *nl, int64_t *n) {
    if (!nl || !n) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    FGB_TRY(nlist_ready(nl));
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
    // a list still in flight: its status slot is reused once its copies have completed
    // (the arrays' frees are ordered on the stream behind the kernels)
    if (nl->hstatus) pinned_release(nl->hstatus, nl->done);
    else if (nl->done) cudaEventDestroy(nl->done);
    dfree(nl->dstatus, nl->stream);
    dfree(nl->qi, nl->stream);
    dfree(nl->pj, nl->stream);
    dfree(nl->dist, nl->stream);
    dfree(nl->counts, nl->stream);
    dfree(nl->segments, nl->stream);
    delete nl;
}
