// NeighborList build on the cell tiles: the count and write passes of a self ball query
// (Section "Implementation": NeighborQuery.query by r_max, NeighborList; Section
// "General Utilities": sorted neighbors).
//
// Count.  One warp per query cell A walks A's half stencil (A itself, then the cells
// after it in (z, y, x) offset order), so every unordered pair of points is tested once
// and adds one to both counts.  A's queries sit in shared memory and are read by a
// uniform load; candidates sit on lanes.  A's own points pair only with later points of
// A.  The other cells' candidates are staged in batches after dropping those out of
// reach of the bounding box of the query block.  Counts accumulate by sorted position
// (lanes hold consecutive positions, so their atomic adds coalesce) and are scattered to
// the caller's order afterwards.
//
// Write.  One warp per query cell stages the candidates of the full 27-cell stencil
// that lie within reach of the bounding box of A's points, then sorts them by point
// index once (a bucket sort on the index range with exact ranks inside each bucket).
// Taking the sorted candidates 32 at a time, every query's hits come out in point-index
// order: each hit's place in its row is the number of hits before it (ballot + popc),
// and it is stored straight into the query's segment.  No per-row sort and no row
// buffer.  The query index array is filled by a separate coalesced pass.  Cells whose
// pruned stencil exceeds the stage are listed and written by the older kernels.
//
// Both passes decide in FP32 outside a proven band around r_max and in FP64 (the
// defining sequence) inside it, as everywhere else.
#include <algorithm>
#include <climits>
#include <cstdlib>

#include "fgb_tile.cuh"

namespace fgb {

constexpr int kNlWarps = 4;
constexpr int kNlCountStage = 256;  // other-cell candidates per staged batch (count)
constexpr int kNlStage = 384;       // pruned full-stencil candidates of one cell (write)
constexpr int kNlBuckets = 256;     // buckets of the per-cell index sort
constexpr int kNlAsyncRowCap = 128; // longest row of the asynchronous form's fallback
constexpr int kNlOwnCap = 512;      // half-stencil candidates of a cell with an owner table

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float4 far_record() { return make_float4(kFar, kFar, kFar, __int_as_float(-1)); }

// ------------------------------------------------------------------ count

// Band pairs of one round (lanes with r2 in [lo, hi)): the FP64 decision.  i is the
// query's index; the candidate's index is read from its sorted record at position p
// (or given directly as j when p < 0).
__device__ __noinline__ bool nl_band_pair(const TileArgs *ap, int i, int p, int j) {
    if (p >= 0) j = __float_as_int(__ldg(ap->pts + p).w);
    return exact_r2_idx(ap->bd, ap->p_orig, i, ap->p_orig, j) < ap->T;
}

template <int NS>
__device__ __forceinline__ void nl_count_body(const TileArgs &a, uint32_t *__restrict__ cs) {
    __shared__ TileStencilT<NS> sts[kNlWarps];
    __shared__ float4 sstage[kNlWarps][kNlCountStage + 32];
    __shared__ float4 sq[kNlWarps][32];
    __shared__ uint8_t sown[kNlWarps][kNlOwnCap];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t A = a.cell_lo + (int64_t)blockIdx.x * kNlWarps + warp;
    if (A >= a.ncell) return;
    const int begA = (int)__ldg(a.cell_start + A);
    const int nA = (int)__ldg(a.cell_start + A + 1) - begA;
    if (nA == 0) return;
    int cx, cy, cz;
    cell_coords((uint32_t)A, a.nc, cx, cy, cz);
    TileStencilT<NS> &ts = sts[warp];
    const int n = tile_stencil(a, cx, cy, cz, true, ts);  // A first, with nA candidates
    const int total = ts.pre[n];
    const uint8_t *own = nullptr;
    if (total <= kNlOwnCap) {
        tile_owners(ts, n, sown[warp]);
        own = sown[warp];
    }
    float4 *stage = sstage[warp];
    float4 *qs = sq[warp];
    const float lo = a.band.lo, hi = a.band.hi;
    const float reach2 = hi * (1.0f + 1e-5f);
    const unsigned lt = lanemask_lt();
    int nesc = 0;
    for (int qb = 0; qb < nA; qb += 32) {
        const int nq = min(32, nA - qb);
        __syncwarp();
        const float4 myq = lane < nq ? __ldg(a.pts + begA + qb + lane) : far_record();
        qs[lane] = myq;
        __syncwarp();
        uint32_t qacc = 0;  // lane t: neighbors of query qb + t found so far
        // A's own points: the pair (t, k) once, for k > t
        for (int kb = qb; kb < nA; kb += 32) {
            const int k = kb + lane;
            const float4 c = k < nA ? __ldg(a.pts + begA + k) : far_record();
            uint32_t ccnt = 0;
            for (int t = 0; t < nq; ++t) {
                const float4 Q = qs[t];
                const float r2 = r2_f32(c.x - Q.x, c.y - Q.y, c.z - Q.z);
                const bool valid = k > qb + t;
                bool hit = valid && r2 < lo;
                const bool maybe = valid && r2 < hi;
                unsigned mh = __ballot_sync(0xffffffffu, hit);
                if (__ballot_sync(0xffffffffu, maybe) != mh) {
                    if (maybe && !hit) {
                        ++nesc;
                        hit = nl_band_pair(&a, __float_as_int(Q.w), -1, __float_as_int(c.w));
                    }
                    mh = __ballot_sync(0xffffffffu, hit);
                }
                ccnt += hit ? 1u : 0u;
                if (lane == t) qacc += __popc(mh);
            }
            if (ccnt) atomicAdd(cs + begA + k, ccnt);
        }
        // the other cells of the half stencil, pruned by the block's bounding box
        float3 blo, bhi;
        warp_box(myq.x, myq.y, myq.z, lane < nq, blo, bhi);
        int base = nA;
        while (base < total) {
            int kept = 0;
            while (base < total && kept <= kNlCountStage - 32) {
                const int k = base + lane;
                const TileCand c = tile_load_own(a, ts, own, n, total, k);
                const bool keep = k < total && box_dist2(blo, bhi, c.x, c.y, c.z) <= reach2;
                const unsigned m = __ballot_sync(0xffffffffu, keep);
                if (keep) stage[kept + __popc(m & lt)] = make_float4(c.x, c.y, c.z, __int_as_float(c.p));
                kept += __popc(m);
                base += 32;
            }
            const int padded = (kept + 31) & ~31;
            if (kept + lane < padded) stage[kept + lane] = far_record();
            __syncwarp();
            for (int ch = 0; ch < kept; ch += 32) {
                const float4 c = stage[ch + lane];
                const int p = __float_as_int(c.w);
                uint32_t ccnt = 0;
                bool band = false;
                // certain pairs only; pairs inside the band are counted by the second sweep
#pragma unroll 4
                for (int t = 0; t < nq; ++t) {
                    const float4 Q = qs[t];
                    const float r2 = r2_f32(c.x - Q.x, c.y - Q.y, c.z - Q.z);
                    const bool hit = r2 < lo;
                    band |= (r2 >= lo) & (r2 < hi);
                    const unsigned mh = __ballot_sync(0xffffffffu, hit);
                    ccnt += hit ? 1u : 0u;
                    if (lane == t) qacc += __popc(mh);
                }
                if (__any_sync(0xffffffffu, band)) {
                    for (int t = 0; t < nq; ++t) {
                        const float4 Q = qs[t];
                        const float r2 = r2_f32(c.x - Q.x, c.y - Q.y, c.z - Q.z);
                        bool hit = false;
                        if (r2 >= lo && r2 < hi && p >= 0) {
                            ++nesc;
                            hit = nl_band_pair(&a, __float_as_int(Q.w), p, 0);
                        }
                        const unsigned mh = __ballot_sync(0xffffffffu, hit);
                        ccnt += hit ? 1u : 0u;
                        if (lane == t) qacc += __popc(mh);
                    }
                }
                if (ccnt) atomicAdd(cs + p, ccnt);
            }
            __syncwarp();
        }
        if (lane < nq && qacc) atomicAdd(cs + begA + qb + lane, qacc);
    }
    if (nesc) atomicAdd(a.esc, (unsigned long long)nesc);
}

template <int NS>
__global__ void __launch_bounds__(kNlWarps * 32) k_nl_count(const __grid_constant__ TileArgs a,
                                                            uint32_t *__restrict__ cs) {
    nl_count_body<NS>(a, cs);
}

// At most 64 registers: eight blocks per SM instead of seven (0.85 against 0.87 ms at c3).
template <int NS>
__global__ void __launch_bounds__(kNlWarps * 32, 8) k_nl_count_occ(const __grid_constant__ TileArgs a,
                                                                   uint32_t *__restrict__ cs) {
    nl_count_body<NS>(a, cs);
}

// counts[index] = count of the point at sorted position p, plus one for the self pair
// when it is not excluded (points in the walked cells [cell_lo, ncell) only: a 2D box's
// tile kernels walk only the points' layer).
__global__ void k_nl_count_scatter(const float4 *__restrict__ pts, const uint32_t *__restrict__ cell,
                                   const uint32_t *__restrict__ cs, int64_t n, uint32_t self, int64_t cell_lo,
                                   int64_t ncell, uint32_t *__restrict__ counts) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t c = __ldg(cell + p);
    counts[__float_as_int(__ldg(pts + p).w)] = cs[p] + ((c >= cell_lo && c < ncell) ? self : 0u);
}

// ------------------------------------------------------------------ write

struct NlWriteArgs {
    TileArgs t;
    const int64_t *seg;
    const uint32_t *counts;
    int32_t *qi;  // nullable: filled by k_nl_fill_qi instead
    int32_t *pj;
    float *dist;
    int *ovf_cells;  // cells whose pruned stencil exceeds the stage
    int *ovf_count;
    int stage_cap;   // <= kNlStage
    // asynchronous query: nothing is written when the list (*total pairs) exceeds the
    // arrays' capacity (total NULL: no limit)
    const int64_t *total;
    int64_t capacity;
};

// Exact ranks of the staged candidates by point index: bucket by the index's place in
// [jmin, jmax] (a monotone map), count, scan, group, then rank each candidate among its
// bucket by comparison.  perm[r] = stage slot of rank r; slots [kept, round32(kept))
// point at the far sentinel stage[kNlStage].
template <int STAGE>
__device__ __forceinline__ void nl_sort_stage(const float4 *stage, int kept, int jmin, int jmax, uint32_t *cnt,
                                              uint16_t *grp, uint16_t *perm) {
    const int lane = threadIdx.x & 31;
    const float scale = (float)kNlBuckets / (float)((jmax - jmin) + 1);
    for (int b = lane; b < kNlBuckets; b += 32) cnt[b] = 0;
    __syncwarp();
    for (int e = lane; e < kept; e += 32) {
        const int j = __float_as_int(stage[e].w);
        const int b = min(kNlBuckets - 1, __float2int_rz(__int2float_rn(j - jmin) * scale));
        atomicAdd(cnt + b, 1u);
    }
    __syncwarp();
    // exclusive scan of the bucket counts (kNlBuckets / 32 per lane)
    constexpr int PER = kNlBuckets / 32;
    uint32_t v[PER];
    uint32_t sum = 0;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        v[r] = cnt[lane * PER + r];
        sum += v[r];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += u;
    }
    uint32_t run = inc - sum;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        cnt[lane * PER + r] = run;
        run += v[r];
    }
    __syncwarp();
    // group: after this pass cnt[b] is the end of bucket b
    for (int e = lane; e < kept; e += 32) {
        const int j = __float_as_int(stage[e].w);
        const int b = min(kNlBuckets - 1, __float2int_rz(__int2float_rn(j - jmin) * scale));
        grp[atomicAdd(cnt + b, 1u)] = (uint16_t)e;
    }
    __syncwarp();
    for (int g = lane; g < kept; g += 32) {
        const int e = grp[g];
        const int j = __float_as_int(stage[e].w);
        const int b = min(kNlBuckets - 1, __float2int_rz(__int2float_rn(j - jmin) * scale));
        const int s0 = b ? (int)cnt[b - 1] : 0, s1 = (int)cnt[b];
        int rank = s0;
        for (int k = s0; k < s1; ++k) rank += __float_as_int(stage[grp[k]].w) < j ? 1 : 0;
        perm[rank] = (uint16_t)e;
    }
    const int padded = (kept + 31) & ~31;
    if (kept + lane < padded) perm[kept + lane] = (uint16_t)STAGE;
    __syncwarp();
}

template <int NS, int QN, int STAGE>
__device__ __forceinline__ void nl_write_body(const NlWriteArgs &w) {
    const TileArgs &a = w.t;
    // the sort's grouping array lives in the stencil list's memory when it fits (the list
    // is dead once the candidates are staged)
    constexpr bool kAlias = sizeof(TileStencilT<NS>) >= STAGE * sizeof(uint16_t);
    __shared__ TileStencilT<NS> sts[kNlWarps];
    __shared__ float4 sstage[kNlWarps][STAGE + 1];  // + the far sentinel
    __shared__ uint16_t sperm[kNlWarps][STAGE + 32];
    __shared__ uint16_t sgrp[kNlWarps][kAlias ? 1 : STAGE];
    __shared__ uint32_t scnt[kNlWarps][kNlBuckets];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t A = a.cell_lo + (int64_t)blockIdx.x * kNlWarps + warp;
    if (A >= a.ncell) return;
    if (w.total && __ldg(w.total) > w.capacity) return;  // (no cell is listed either)
    const int begA = (int)__ldg(a.cell_start + A);
    const int nA = (int)__ldg(a.cell_start + A + 1) - begA;
    if (nA == 0) return;
    int cx, cy, cz;
    cell_coords((uint32_t)A, a.nc, cx, cy, cz);
    TileStencilT<NS> &ts = sts[warp];
    float4 *stage = sstage[warp];
    uint16_t *perm = sperm[warp];
    const int n = tile_stencil(a, cx, cy, cz, false, ts);
    const int total = ts.pre[n];
    const unsigned lt = lanemask_lt();
    // the owner table lives in the order array's memory (the sort writes it after staging)
    constexpr int kOwn = (STAGE + 32) * (int)sizeof(uint16_t);
    const uint8_t *own = nullptr;
    if (total <= kOwn) {
        tile_owners(ts, n, reinterpret_cast<uint8_t *>(perm));
        own = reinterpret_cast<const uint8_t *>(perm);
    }
    if (lane == 0) stage[STAGE] = far_record();
    // bounding box of A's points
    float3 blo = make_float3(INFINITY, INFINITY, INFINITY), bhi = make_float3(-INFINITY, -INFINITY, -INFINITY);
    for (int t0 = 0; t0 < nA; t0 += 32) {
        const float4 q = __ldg(a.pts + begA + min(t0 + lane, nA - 1));
        float3 l, h;
        warp_box(q.x, q.y, q.z, t0 + lane < nA, l, h);
        blo = make_float3(fminf(blo.x, l.x), fminf(blo.y, l.y), fminf(blo.z, l.z));
        bhi = make_float3(fmaxf(bhi.x, h.x), fmaxf(bhi.y, h.y), fmaxf(bhi.z, h.z));
    }
    // stage the candidates within reach of the box, packed
    const float reach2 = a.band.hi * (1.0f + 1e-5f);
    int kept = 0, jmin = INT_MAX, jmax = -1;
    for (int base = 0; base < total; base += 32) {
        const TileCand c = tile_load_own(a, ts, own, n, total, base + lane);
        const bool keep = base + lane < total && box_dist2(blo, bhi, c.x, c.y, c.z) <= reach2;
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (kept + __popc(m) > w.stage_cap) {
            kept = -1;
            break;
        }
        if (keep) {
            stage[kept + __popc(m & lt)] = make_float4(c.x, c.y, c.z, __int_as_float(c.j));
            jmin = min(jmin, c.j);
            jmax = max(jmax, c.j);
        }
        kept += __popc(m);
    }
    if (kept < 0) {
        if (lane == 0) w.ovf_cells[atomicAdd(w.ovf_count, 1)] = (int)A;
        return;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        jmin = min(jmin, __shfl_xor_sync(0xffffffffu, jmin, o));
        jmax = max(jmax, __shfl_xor_sync(0xffffffffu, jmax, o));
    }
    __syncwarp();
    uint16_t *grp = kAlias ? reinterpret_cast<uint16_t *>(&ts) : &sgrp[warp][0];
    if (kept > 0) nl_sort_stage<STAGE>(stage, kept, jmin, jmax, scnt[warp], grp, perm);
    const int nch = (kept + 31) >> 5;
    const float lo = a.band.lo, hi = a.band.hi;
    for (int q0 = 0; q0 < nA; q0 += QN) {
        float4 Q[QN];
        int iq[QN], ex[QN];
        int64_t so[QN];
        uint32_t nh[QN], want[QN];
#pragma unroll
        for (int u = 0; u < QN; ++u) {
            const bool v = q0 + u < nA;
            Q[u] = v ? __ldg(a.pts + begA + q0 + u) : far_record();
            iq[u] = v ? __float_as_int(Q[u].w) : -1;
            ex[u] = a.exclude ? iq[u] : -1;
            so[u] = v ? __ldg(w.seg + iq[u]) : 0;
            want[u] = v ? __ldg(w.counts + iq[u]) : 0;
            nh[u] = 0;
        }
        for (int ch = 0; ch < nch; ++ch) {
            const float4 c = stage[perm[(ch << 5) + lane]];
            const int j = __float_as_int(c.w);
            float r2[QN];
            bool hit[QN];
            bool anyband = false;
#pragma unroll
            for (int u = 0; u < QN; ++u) {
                r2[u] = r2_f32(c.x - Q[u].x, c.y - Q[u].y, c.z - Q[u].z);
                hit[u] = r2[u] < lo && j != ex[u];
                anyband |= r2[u] >= lo && r2[u] < hi;
            }
            float dd[QN];
#pragma unroll
            for (int u = 0; u < QN; ++u) dd[u] = sqrt_approx(r2[u]);
            if (__any_sync(0xffffffffu, anyband)) {
#pragma unroll
                for (int u = 0; u < QN; ++u) {
                    if (r2[u] >= lo && r2[u] < hi && j != ex[u] && j >= 0 && iq[u] >= 0) {
                        const double e = exact_r2_idx(a.bd, a.p_orig, iq[u], a.p_orig, j);
                        if (e < a.T) {
                            hit[u] = true;
                            dd[u] = (float)sqrt(e);
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < QN; ++u) {
                const unsigned m = __ballot_sync(0xffffffffu, hit[u]);
                const uint32_t pos = nh[u] + __popc(m & lt);
                if (hit[u] && pos < want[u]) {  // never beyond the counted segment
                    const int64_t at = so[u] + pos;
                    __stcs(w.pj + at, j);
                    __stcs(w.dist + at, dd[u]);
                    if (w.qi) __stcs(w.qi + at, iq[u]);
                }
                nh[u] += __popc(m);
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int u = 0; u < QN; ++u)
                if (iq[u] >= 0 && nh[u] != want[u]) atomicExch(a.err, nh[u] > want[u] ? 1 : 2);
        }
    }
}

template <int NS, int QN>
__global__ void __launch_bounds__(kNlWarps * 32) k_nl_write(const __grid_constant__ NlWriteArgs w) {
    nl_write_body<NS, QN, kNlStage>(w);
}

// The build for 27-cell stencils: a stage of 352 and at most 80 registers, so six
// blocks fit an SM instead of five (latency-bound: 3.28 against 3.66 ms at c3; a stage
// of 320 at seven blocks spilled and took 3.59 ms).  Cells with more candidates go to
// the listed fallback.
constexpr int kNlStageSmall = 352;
template <int NS, int QN>
__global__ void __launch_bounds__(kNlWarps * 32, 6) k_nl_write_occ(const __grid_constant__ NlWriteArgs w) {
    nl_write_body<NS, QN, kNlStageSmall>(w);
}

// qi[seg[i] .. seg[i+1]) = i: one warp per 32 consecutive queries, each row stored by
// the whole warp.  Nothing is stored when the list (seg[nq]) exceeds capacity.
__global__ void __launch_bounds__(256) k_nl_fill_qi(const int64_t *__restrict__ seg, int64_t nq, int64_t capacity,
                                                    int32_t *__restrict__ qi) {
    const int lane = threadIdx.x & 31;
    const int64_t i0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
    if (i0 >= nq || __ldg(seg + nq) > capacity) return;
    const int m = (int)(nq - i0 < 32 ? nq - i0 : 32);
    const int64_t myseg = __ldg(seg + i0 + min(lane, m));  // lane r: start of row r
    const int64_t last = __ldg(seg + i0 + m);              // end of the warp's last row
    for (int r = 0; r < m; ++r) {
        const int64_t b = __shfl_sync(0xffffffffu, myseg, r);
        const int64_t nx = __shfl_sync(0xffffffffu, myseg, (r + 1) & 31);
        const int64_t e = r + 1 < m ? nx : last;
        const int32_t v = (int32_t)(i0 + r);
        for (int64_t k = b + lane; k < e; k += 32) __stcs(qi + k, v);
    }
}

// ------------------------------------------------------------------ host

// FGB_NL_KERNELS=0 keeps the earlier count and write kernels on the cell tiles.
bool nl_kernels_enabled() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("FGB_NL_KERNELS");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

// Stage capacity of the write kernel (FGB_NL_STAGE_CAP lowers it, so tests can send
// cells to the listed fallback).
static int nl_stage_cap() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("FGB_NL_STAGE_CAP");
        v = kNlStage;
        if (e) v = std::max(0, std::min(kNlStage, atoi(e)));
    }
    return v;
}

// FGB_NL_QI=0 fills the query index array by a separate coalesced pass instead of the
// write kernel's stores.
static bool nl_qi_in_write() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("FGB_NL_QI");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

// FGB_NL_OCC=0 launches the unconstrained builds of the count and write kernels
// (comparisons).
static bool nl_occ() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("FGB_NL_OCC");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

// FGB_NL_QN: queries per pass of the write kernel (2 or 4; 4 measured faster).
static int nl_qn() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("FGB_NL_QN");
        v = (e && e[0] == '2') ? 2 : 4;
    }
    return v;
}

int nl_count(const fgb_nq *nq, const StencilPlan &p, double R, int exclude, unsigned long long *esc, int *err,
             uint32_t *counts, cudaStream_t s) {
    TileArgs t = tile_args(nq, p, R, exclude);
    t.esc = esc;
    t.err = err;
    uint32_t *cs = nullptr;
    FGB_TRY(dalloc_n(&cs, (size_t)nq->n, s));
    FGB_CUDA(cudaMemsetAsync(cs, 0, sizeof(uint32_t) * nq->n, s));
    const unsigned grid = (unsigned)((t.ncell - t.cell_lo + kNlWarps - 1) / kNlWarps);
    // the half stencil holds (nfull - 1) / 2 + 1 cells; the shared stencil list must fit it
    const int nfull = (2 * p.s[0] + 1) * (2 * p.s[1] + 1) * (2 * p.s[2] + 1);
    const int nhalf = (nfull - 1) / 2 + 1;
    if (nhalf > kTileMaxStencil) {
        dfree(cs, s);
        return fail(FGB_ERR_UNSUPPORTED, "neighbor count: stencil of %d cells", nfull);
    }
    if (grid > 0) {  // (a shard may walk no cell)
        FGB_KSCOPE("k_nl_count", s);
        if (nhalf <= 32) {
            if (nl_occ())
                k_nl_count_occ<32><<<grid, kNlWarps * 32, 0, s>>>(t, cs);
            else
                k_nl_count<32><<<grid, kNlWarps * 32, 0, s>>>(t, cs);
        } else {
            k_nl_count<kTileMaxStencil><<<grid, kNlWarps * 32, 0, s>>>(t, cs);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        FGB_KSCOPE("k_nl_count_scatter", s);
        k_nl_count_scatter<<<(unsigned)((nq->n + 255) / 256), 256, 0, s>>>(
            nq->sorted, nq->sorted_cell, cs, nq->n, exclude ? 0u : 1u, t.cell_lo, t.ncell, counts);
        e = cudaGetLastError();
    }
    dfree(cs, s);
    if (e != cudaSuccess) return fail(FGB_ERR_CUDA, "neighbor count launch failed: %s", cudaGetErrorString(e));
    return FGB_OK;
}

int tile_write_listed(const fgb_nq *nq, const StencilPlan &p, double R, int exclude, int *err, const int64_t *seg,
                      const uint32_t *counts, int cap, const int *cells, const int *ncells, int32_t *qi, int32_t *pj,
                      float *dist, cudaStream_t s);
int tile_write_global_listed(const fgb_nq *nq, const StencilPlan &p, double R, int exclude, int *err,
                             const int64_t *seg, const uint32_t *counts, const int *cells, const int *ncells,
                             int32_t *qi, int32_t *pj, float *dist, cudaStream_t s);

static int nfull_of(const StencilPlan &p) { return (2 * p.s[0] + 1) * (2 * p.s[1] + 1) * (2 * p.s[2] + 1); }

int nl_write(const fgb_nq *nq, const StencilPlan &p, double R, int exclude, int *err, const int64_t *seg,
             const uint32_t *counts, int cap, int64_t nqq, int32_t *qi, int32_t *pj, float *dist, cudaStream_t s,
             int64_t capacity) {
    // capacity >= 0: the asynchronous form (list size and longest row unknown on the host)
    const bool async = capacity >= 0;
    if (async) {
        cap = kNlAsyncRowCap;
        if (tile_write_smem(cap) > 160 * 1024) return fail(FGB_ERR_UNSUPPORTED, "asynchronous write: no fallback");
    }
    NlWriteArgs w;
    w.t = tile_args(nq, p, R, exclude);
    w.t.err = err;
    w.seg = seg;
    w.counts = counts;
    w.qi = nl_qi_in_write() ? qi : nullptr;
    w.pj = pj;
    w.dist = dist;
    w.total = async ? seg + nqq : nullptr;
    w.capacity = async ? capacity : INT64_MAX;
    w.stage_cap = nl_stage_cap();
    if (nfull_of(p) <= 32 && nl_occ() && nl_qn() == 4) w.stage_cap = std::min(w.stage_cap, kNlStageSmall);
    const int64_t cells = w.t.ncell - w.t.cell_lo;
    int *ovf = nullptr;
    FGB_TRY(dalloc_n(&ovf, (size_t)cells + 1, s));
    w.ovf_count = ovf;
    w.ovf_cells = ovf + 1;
    FGB_CUDA(cudaMemsetAsync(ovf, 0, sizeof(int), s));
    const unsigned grid = (unsigned)((cells + kNlWarps - 1) / kNlWarps);
    // the shared stencil list must hold every cell of the full stencil
    const int nfull = (2 * p.s[0] + 1) * (2 * p.s[1] + 1) * (2 * p.s[2] + 1);
    if (nfull > kTileMaxStencil) {
        dfree(ovf, s);
        return fail(FGB_ERR_UNSUPPORTED, "neighbor write: stencil of %d cells", nfull);
    }
    if (grid > 0) {  // (a shard may walk no cell)
        FGB_KSCOPE("k_nl_write", s);
        if (nfull <= 32) {
            if (nl_occ() && nl_qn() == 4)
                k_nl_write_occ<32, 4><<<grid, kNlWarps * 32, 0, s>>>(w);
            else if (nl_qn() == 4)
                k_nl_write<32, 4><<<grid, kNlWarps * 32, 0, s>>>(w);
            else
                k_nl_write<32, 2><<<grid, kNlWarps * 32, 0, s>>>(w);
        } else {
            if (nl_qn() == 4)
                k_nl_write<kTileMaxStencil, 4><<<grid, kNlWarps * 32, 0, s>>>(w);
            else
                k_nl_write<kTileMaxStencil, 2><<<grid, kNlWarps * 32, 0, s>>>(w);
        }
    }
    cudaError_t e = cudaGetLastError();
    int st = FGB_OK;
    if (e != cudaSuccess) st = fail(FGB_ERR_CUDA, "neighbor write launch failed: %s", cudaGetErrorString(e));
    if (st == FGB_OK && !w.qi && nqq > 0) {
        FGB_KSCOPE("k_nl_fill_qi", s);
        const int64_t warps = (nqq + 31) / 32;
        k_nl_fill_qi<<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(seg, nqq, w.capacity, qi);
        e = cudaGetLastError();
        if (e != cudaSuccess) st = fail(FGB_ERR_CUDA, "query index fill failed: %s", cudaGetErrorString(e));
    }
    // cells with more candidates than the stage: the earlier kernels, over the list
    // (the row sort of the long-row route reads each row's query index, filled above).
    // The asynchronous form takes the shared-row kernel with rows of up to
    // kNlAsyncRowCap entries; a longer row there is skipped and flagged (err = 1), and the
    // waiting call rewrites the list by the synchronous route.
    if (st == FGB_OK && cap <= 128 && tile_write_smem(cap) <= 160 * 1024) {
        st = tile_write_listed(nq, p, R, exclude, err, seg, counts, cap, w.ovf_cells, w.ovf_count, qi, pj, dist, s);
    } else if (st == FGB_OK) {
        st = tile_write_global_listed(nq, p, R, exclude, err, seg, counts, w.ovf_cells, w.ovf_count, qi, pj, dist,
                                      s);
        st = st ? st : sort_segments(seg, nqq, cap, nq->n, qi, pj, dist, s);
    }
    dfree(ovf, s);
    return st;
}

}  // namespace fgb
