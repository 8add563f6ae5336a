// Cell-tile kernels of the batched frames: the frames whose two stencils are on the shift
// route with at most kTileMaxStencil cells.  As in the single-frame tile kernels, one
// warp owns one query cell at a time; warps take work items (a frame and a range of its
// cells) from a counter and keep the frame's arguments in their own shared slot, so no
// warp waits on another.
//
// RDF: the candidates of the cell's half stencil stream through the lanes 32 at a time,
// shifted into the cell's frame, while the warp loops over the cell's queries (the own
// cell's points only against earlier queries, so each unordered pair is binned once with
// weight 2).  Counts go to the warp's shared histogram, added to the frame's row when
// the warp moves on to another frame.
//
// q_l: the candidates of the full ball stencil on lanes, the cell's queries looped, the
// exact ball test of the single-frame query (FP32 band, FP64 inside it).  Every bond
// found is queued in shared memory; 32 at a time, one lane per bond evaluates the
// harmonics and a segmented scan over the lanes sums them per query, in a fixed order,
// so the result does not depend on timing.
#include <algorithm>
#include <cstring>

#include "fgb_batch.cuh"
#include "fgb_ylm.cuh"

namespace fgb {

constexpr int kBtW = kBatchTileWarps;
constexpr int kBtOwnCap = 512;  // candidates of a stencil with an owner table
constexpr unsigned kFull = 0xffffffffu;

// Copies a frame's arguments into the warp's shared slot.
__device__ __forceinline__ void bt_load_frame(const FrameTile *g, FrameTile *s) {
    const int lane = threadIdx.x & 31;
    const int *src = reinterpret_cast<const int *>(g);
    int *dst = reinterpret_cast<int *>(s);
    __syncwarp();
    for (int k = lane; k < (int)(sizeof(FrameTile) / 4); k += 32) dst[k] = __ldg(src + k);
    __syncwarp();
}

// Next work item of the warp from counter ctl[slot]; false when none is left.
__device__ __forceinline__ bool bt_next(const BatchTileArgs &a, int slot, int4 &w) {
    int it = 0;
    if ((threadIdx.x & 31) == 0) it = atomicAdd(a.ctl + slot, 1);
    it = __shfl_sync(kFull, it, 0);
    if (it >= a.nitems) return false;
    w = __ldg(a.items + it);
    return true;
}

// ------------------------------------------------------------------ RDF

__device__ __forceinline__ int bt_exact_bin(const double *T, int bins, double e) {
    if (!(e >= T[0]) || !(e < T[bins])) return -1;
    int lo = 0, hi = bins;  // T[lo] <= e < T[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (T[mid] <= e)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Adds the warp's private counts (weight 2) to a frame's row and clears them.
__device__ __forceinline__ void bt_flush(uint32_t *h, int bins, unsigned long long *row) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    for (int b = lane; b < bins; b += 32) {
        const uint32_t v = h[b];
        if (v) {
            atomicAdd(row + b, 2ull * v);
            h[b] = 0;
        }
    }
    __syncwarp();
}

// A pair in [r_min, r_max) whose fast test failed: the band tables decide, else it is
// listed for the FP64 pass (or decided here when the list is full).
__device__ __noinline__ void bt_rdf_slow(const BatchTileArgs *ap, const FrameTile *fr, float r2, int i, int j,
                                         uint32_t *h) {
    const BatchTileArgs &a = *ap;
    const int b = rdf_bin_band(fr->P, r2);
    if (b >= 0) {
        atomicAdd(h + b, 1u);
        return;
    }
    const int slot = atomicAdd(a.ctl + 1, 1);
    if (slot < a.esc_cap) {
        a.esc[slot] = make_int4(fr->f, i, j, 2);
        return;
    }
    const int be = bt_exact_bin(a.T, a.bins, exact_r2_idx(fr->r.bd, a.pts, i, a.pts, j));
    if (be >= 0) atomicAdd(a.counts + (int64_t)fr->f * a.bins + be, 2ull);
}

// One candidate per lane against the queries [0, nq) of the pass, valid only for the
// queries lo <= tl < hi (lim = lo | hi << 8): the queries of the block cells whose half
// stencil holds the candidate's cell, and of its own cell only those before it (so each
// unordered pair is binned once, with weight 2).  The fast test is the single-frame one:
// bin floor(x) when x = (r - r_min)/Delta is further than the error bound from both
// edges.
__device__ __forceinline__ void bt_rdf_rounds(const BatchTileArgs &a, const FrameTile &fr, const float4 *qs, int nq,
                                              float cx, float cy, float cz, int cj, int lim, uint32_t *h) {
    const BinParams &P = fr.P;
    const float rhi = P.rmax_hi, rlo = P.rmin_lo;
    const float invd = P.invdelta, rmid = P.rmin_invdelta, g2h = P.g2h, eps = P.eps, r2f = P.r2_fast;
    const int llo = lim & 0xff, lhi = lim >> 8;
#pragma unroll 4
    for (int tl = 0; tl < nq; ++tl) {
        const float4 q = qs[tl];
        const float r2 = r2_f32(cx - q.x, cy - q.y, cz - q.z);
        if (r2 < rhi && r2 >= rlo && tl < lhi && tl >= llo) {
            const float inv = rsqrt_ftz(r2);
            const float x = fmaf(r2 * inv, invd, -rmid);
            const float fb = floorf(x);
            const float e = fmaf(g2h, inv, eps);
            if (r2 > r2f && fabsf((x - fb) - 0.5f) < 0.5f - e)
                atomicAdd(h + (int)fb, 1u);
            else
                bt_rdf_slow(&a, &fr, r2, __float_as_int(q.w), cj, h);
        }
    }
}

// Before a round could overflow a private 32-bit count, the warp flushes its histogram.
__device__ __forceinline__ void bt_guard(const BatchTileArgs &a, const FrameTile &fr, uint32_t *h, uint64_t &tests,
                                         int nq) {
    if (tests > 0xffffffffull - 32u * 32u) {
        bt_flush(h, a.bins, a.counts + (int64_t)fr.f * a.bins);
        tests = 0;
    }
    tests += 32u * (unsigned)nq;
}

// Query i of block cell b (sorted position p) in the frame of cell A: shifted by the
// table offset of (b, 0, 0), as the candidates are shifted by theirs.  qst[b] = start of
// block cell b's queries relative to the block's first point.
__device__ __forceinline__ float4 bt_block_query(const TileArgs &t, const int *qst, int len, int p, int rel) {
    float4 q = __ldg(t.pts + p);
    int b = 0;
    for (int c = 1; c < len; ++c) b += rel >= qst[c] ? 1 : 0;
    if (b > 0) {
        const int owx = 2 * t.ts[0] + 1, owy = 2 * t.ts[1] + 1;
        const float4 of = __ldg(t.off + (t.ts[2] * owy + t.ts[1]) * owx + (b + t.ts[0]));
        q.x += of.x;
        q.y += of.y;
        q.z += of.z;
    }
    return q;
}

// The queries of `len` x-adjacent cells A, A+1, ... of one row (contiguous in sorted
// order) against the union of their half stencils; each candidate keeps the range of
// query slots it pairs with.  The candidates are packed into full chunks of 32, dropping
// those out of reach of the pass's bounding box.
template <int NS>
__device__ __forceinline__ void bt_rdf_cell(const BatchTileArgs &a, const FrameTile &fr, int A, int len,
                                            TileStencilT<NS> &ts, uint8_t *ownbuf, int *qst, float4 *qs, float4 *buf,
                                            int *lim, uint32_t *h, uint64_t &tests) {
    const TileArgs &t = fr.r;
    const int lane = threadIdx.x & 31;
    const int begA = (int)__ldg(t.cell_start + A);
    const int nA = (int)__ldg(t.cell_start + A + len) - begA;
    if (nA == 0) return;
    int cx, cy, cz;
    cell_coords((uint32_t)A, t.nc, cx, cy, cz);
    __syncwarp();
    if (lane <= len) qst[lane] = (int)__ldg(t.cell_start + A + lane) - begA;
    const int n = tile_stencil(t, cx, cy, cz, true, ts, len);
    const int total = ts.pre[n];
    const uint8_t *own = nullptr;
    if (total <= kBtOwnCap) {
        tile_owners(ts, n, ownbuf);
        own = ownbuf;
    }
    const unsigned lt = lanemask_lt();
    // a candidate farther than this from the queries' bounding box reaches none of them
    const float reach2 = fr.P.rmax_hi * (1.0f + 1e-5f);
    for (int qb = 0; qb < nA; qb += 32) {
        const int nq = min(32, nA - qb);
        __syncwarp();
        if (lane < nq) qs[lane] = bt_block_query(t, qst, len, begA + qb + lane, qb + lane);
        __syncwarp();
        float3 blo, bhi;
        {
            const float4 q = qs[lane < nq ? lane : 0];
            warp_box(q.x, q.y, q.z, lane < nq, blo, bhi);
        }
        int cnt = 0;
        for (int base = 0; base < total; base += 32) {
            const int k = base + lane;
            const TileCand c = tile_load_own(t, ts, own, n, total, k);
            const bool keep = k < total && box_dist2(blo, bhi, c.x, c.y, c.z) <= reach2;
            const unsigned m = __ballot_sync(kFull, keep);
            if (keep) {
                const int rg = __float_as_int(ts.off[c.o].w);
                const int b0 = rg & 0xff, b1 = (rg >> 8) & 0xff;
                const int shi = (rg >> 16) ? c.p - begA : qst[b1 + 1];  // own cell: queries before it
                const int lo = min(max(qst[b0] - qb, 0), 32), hi = min(max(shi - qb, 0), 32);
                const int slot = cnt + __popc(m & lt);
                buf[slot] = make_float4(c.x, c.y, c.z, __int_as_float(c.j));
                lim[slot] = lo | (hi << 8);
            }
            cnt += __popc(m);
            if (cnt >= 32) {
                __syncwarp();
                bt_guard(a, fr, h, tests, nq);
                const float4 e = buf[lane];
                bt_rdf_rounds(a, fr, qs, nq, e.x, e.y, e.z, __float_as_int(e.w), lim[lane], h);
                const float4 rest = buf[32 + lane];
                const int rl = lim[32 + lane];
                __syncwarp();
                if (lane < cnt - 32) {
                    buf[lane] = rest;
                    lim[lane] = rl;
                }
                __syncwarp();
                cnt -= 32;
            }
        }
        if (cnt > 0) {
            __syncwarp();
            bt_guard(a, fr, h, tests, nq);
            const float4 e = lane < cnt ? buf[lane] : make_float4(kFar, kFar, kFar, __int_as_float(-1));
            bt_rdf_rounds(a, fr, qs, nq, e.x, e.y, e.z, __float_as_int(e.w), lane < cnt ? lim[lane] : 0, h);
        }
    }
}

template <int NS>
__global__ void __launch_bounds__(kBtW * 32, 7) k_batch_rtile(const __grid_constant__ BatchTileArgs a) {
    __shared__ FrameTile sfr[kBtW];
    __shared__ TileStencilT<NS> sts[kBtW];
    __shared__ float4 sq[kBtW][32];
    __shared__ float4 sbuf[kBtW][64];  // kept candidates
    __shared__ int slim[kBtW][64];     // their query limits
    __shared__ uint8_t sown[kBtW][kBtOwnCap];
    __shared__ int sqst[kBtW][8];      // query starts of the block's cells
    extern __shared__ uint32_t shist[];  // kBtW * bins
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *h = shist + warp * a.bins;
    for (int b = lane; b < a.bins; b += 32) h[b] = 0;
    FrameTile &fr = sfr[warp];
    int cur = -1;
    uint64_t tests = 0;  // pair tests since the last flush bound every private count
    int4 w;
    while (bt_next(a, 2, w)) {
        if (w.x != cur) {
            if (cur >= 0) bt_flush(h, a.bins, a.counts + (int64_t)fr.f * a.bins);
            tests = 0;
            bt_load_frame(a.ft + w.x, &fr);
            cur = w.x;
        }
        for (int c = w.y; c < w.z;) {
            // a block of up to qbr cells, within one x row and the work item
            const int len = min(min(fr.qbr, fr.r.nc[0] - c % fr.r.nc[0]), w.z - c);
            bt_rdf_cell<NS>(a, fr, c, len, sts[warp], sown[warp], sqst[warp], sq[warp], sbuf[warp], slim[warp], h,
                            tests);
            c += len;
        }
    }
    if (cur >= 0) bt_flush(h, a.bins, a.counts + (int64_t)fr.f * a.bins);
}

// ------------------------------------------------------------------ q_l

// Exact ball test of a pair inside the FP32 band.
__device__ __noinline__ bool bt_ball_exact(const BatchTileArgs *ap, const FrameTile *fr, int i, int j) {
    return exact_r2_idx(fr->b.bd, ap->pts, i, ap->pts, j) < fr->b.T;
}

// Harmonics of the first n queued bonds, one lane each, summed into the query rows
// acc[slot][2(L+1)].  The queue holds each round's hits (one query) together, so the
// bonds form runs of equal slot: a segmented inclusive scan over the lanes (the same
// tree for every component) leaves each run's sum on its last lane, which adds it to
// the row.
template <int L>
__device__ __forceinline__ void bt_drain(int n, const float4 *bond, float *acc) {
    constexpr int NC = 2 * (L + 1);
    const int lane = threadIdx.x & 31;
    __syncwarp();
    const bool have = lane < n;
    const float4 e = have ? bond[lane] : make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
    const int s = __float_as_int(e.w);
    float yr[L + 1], yi[L + 1];
    bond_harmonics<L>(make_float3(e.x, e.y, e.z), yr, yi);  // zero without a bond
    const int prev = __shfl_up_sync(kFull, s, 1), next = __shfl_down_sync(kFull, s, 1);
    const unsigned heads = __ballot_sync(kFull, lane == 0 || prev != s);
    const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));  // first lane of the run
    // steps beyond the longest run of bonds add nothing to a row: stop there (same sums,
    // same order; the lanes without a bond form a run of their own that no row takes)
    const int longest = (int)__reduce_max_sync(kFull, have ? (unsigned)(lane - start + 1) : 1u);
    for (int d = 1; d < longest; d <<= 1) {
        const bool take = lane - d >= start;
#pragma unroll
        for (int m = 0; m <= L; ++m) {
            const float ur = __shfl_up_sync(kFull, yr[m], d), ui = __shfl_up_sync(kFull, yi[m], d);
            if (take) {
                yr[m] += ur;
                yi[m] += ui;
            }
        }
    }
    // A slot can own several runs (hits of the same query from two staged chunks): each
    // pass adds, for every slot, the run of the lowest pending last lane, so a row takes
    // its runs one at a time and in lane order.
    unsigned pend = __ballot_sync(kFull, have && (lane == 31 || next != s));
    const unsigned lt = lanemask_lt();
    while (pend) {
        const bool mine = (pend >> lane) & 1u;
        const unsigned same = __match_any_sync(kFull, mine ? s : -1 - lane);
        const bool go = mine && (same & pend & lt) == 0;
        if (go) {
            float *row = acc + s * NC;
#pragma unroll
            for (int m = 0; m <= L; ++m) {
                row[m] += yr[m];
                row[L + 1 + m] += yi[m];
            }
        }
        pend &= ~__ballot_sync(kFull, go);
        __syncwarp();
    }
}

// The queries of `len` x-adjacent cells A, A+1, ... of one row (contiguous in sorted
// order) against the union of their ball stencils: a candidate outside a query's own
// stencil is farther than r_max from it (the stencil covers the ball), so testing it
// changes nothing.
template <int L, int NS>
__device__ __forceinline__ void bt_q_cell(const BatchTileArgs &a, const FrameTile &fr, int A, int len,
                                          TileStencilT<NS> &ts, uint8_t *ownbuf, float4 *qs, float4 *buf, float4 *bond,
                                          float *acc, int *snn, int &nesc) {
    constexpr int NC = 2 * (L + 1);
    const TileArgs &t = fr.b;
    const int lane = threadIdx.x & 31;
    const int begA = (int)__ldg(t.cell_start + A);
    const int nA = (int)__ldg(t.cell_start + A + len) - begA;
    if (nA == 0) return;
    int cx, cy, cz;
    cell_coords((uint32_t)A, t.nc, cx, cy, cz);
    __syncwarp();
    const int n = tile_stencil(t, cx, cy, cz, false, ts, len);
    const int total = ts.pre[n];
    const uint8_t *own = nullptr;
    if (total <= kBtOwnCap) {
        tile_owners(ts, n, ownbuf);
        own = ownbuf;
    }
    const float lo = t.band.lo, hi = t.band.hi;
    const float reach2 = hi * (1.0f + 1e-5f);
    const unsigned lt = lanemask_lt();
    for (int qb = 0; qb < nA; qb += 32) {
        const int nq = min(32, nA - qb);
        __syncwarp();
        if (lane < nq) {
            // a query of block cell b is local to that cell: shift it into cell A's frame
            // by the table offset of (b, 0, 0), as the candidates are shifted by theirs
            const int p = begA + qb + lane;
            float4 q = __ldg(t.pts + p);
            int b = 0;
            for (int c = 1; c < len; ++c) b += p >= (int)__ldg(t.cell_start + A + c) ? 1 : 0;
            if (b > 0) {
                const int owx = 2 * t.ts[0] + 1, owy = 2 * t.ts[1] + 1;
                const float4 of = __ldg(t.off + (t.ts[2] * owy + t.ts[1]) * owx + (b + t.ts[0]));
                q.x += of.x;
                q.y += of.y;
                q.z += of.z;
            }
            qs[lane] = q;
        }
        snn[lane] = 0;
        for (int k = lane; k < 32 * NC; k += 32) acc[k] = 0.f;
        __syncwarp();
        float3 blo, bhi;
        {
            const float4 q = qs[lane < nq ? lane : 0];
            warp_box(q.x, q.y, q.z, lane < nq, blo, bhi);
        }
        int kept = 0, qn = 0;
        for (int base = 0; base < total || kept > 0; base += 32) {
            if (base < total) {
                const TileCand c = tile_load_own(t, ts, own, n, total, base + lane);
                const bool keep = base + lane < total && box_dist2(blo, bhi, c.x, c.y, c.z) <= reach2;
                const unsigned m = __ballot_sync(kFull, keep);
                if (keep) buf[kept + __popc(m & lt)] = make_float4(c.x, c.y, c.z, __int_as_float(c.j));
                kept += __popc(m);
                if (kept < 32 && base + 32 < total) continue;
            }
            // a full chunk, or the last partial one (missing lanes far away)
            __syncwarp();
            const float4 e = lane < kept ? buf[lane] : make_float4(kFar, kFar, kFar, __int_as_float(-1));
            const int j = __float_as_int(e.w);
            for (int tl = 0; tl < nq; ++tl) {
                const float4 q = qs[tl];
                const float dx = e.x - q.x, dy = e.y - q.y, dz = e.z - q.z;
                const float r2 = r2_f32(dx, dy, dz);
                const int i = __float_as_int(q.w);
                bool hit = r2 < lo && j != i;
                if (r2 >= lo && r2 < hi && j != i && j >= 0) {
                    ++nesc;
                    hit = bt_ball_exact(&a, &fr, i, j);
                }
                const unsigned m = __ballot_sync(kFull, hit);
                if (m) {
                    if (hit) bond[qn + __popc(m & lt)] = make_float4(dx, dy, dz, __int_as_float(tl));
                    if (lane == 0) snn[tl] += __popc(m);
                    qn += __popc(m);
                    if (qn >= 32) {
                        bt_drain<L>(32, bond, acc);
                        const float4 r = bond[32 + lane];
                        __syncwarp();
                        if (lane < qn - 32) bond[lane] = r;
                        __syncwarp();
                        qn -= 32;
                    }
                }
            }
            const float4 rest = buf[32 + lane];
            __syncwarp();
            if (lane < kept - 32) buf[lane] = rest;
            __syncwarp();
            kept = max(kept - 32, 0);
            if (base >= total) break;
        }
        if (qn > 0) bt_drain<L>(qn, bond, acc);
        __syncwarp();
        if (lane < nq) {
            float sr[L + 1], si[L + 1];
            const float *row = acc + lane * NC;
#pragma unroll
            for (int m = 0; m <= L; ++m) {
                sr[m] = row[m];
                si[m] = row[L + 1 + m];
            }
            finish<L>(__float_as_int(qs[lane].w), snn[lane], sr, si, a.q, a.Q, a.nn);
        }
    }
}

template <int L, int NS>
__global__ void __launch_bounds__(kBtW * 32, 7) k_batch_qtile(const __grid_constant__ BatchTileArgs a) {
    __shared__ FrameTile sfr[kBtW];
    __shared__ TileStencilT<NS> sts[kBtW];
    __shared__ float4 sq[kBtW][32];
    __shared__ float4 sbuf[kBtW][64];   // kept candidates
    __shared__ float4 sbond[kBtW][64];  // queued bonds: displacement, query slot
    __shared__ int snn[kBtW][32];
    __shared__ float sacc[kBtW][32 * 2 * (L + 1)];  // per query: sums of Re, Im Y~_Lm
    __shared__ uint8_t sown[kBtW][kBtOwnCap];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    FrameTile &fr = sfr[warp];
    int cur = -1, nesc = 0;
    int4 w;
    while (bt_next(a, 3, w)) {
        if (w.x != cur) {
            bt_load_frame(a.ft + w.x, &fr);
            cur = w.x;
        }
        for (int c = w.y; c < w.z;) {
            // a block of up to qb cells, within one x row and the work item
            const int cx = c % fr.b.nc[0];
            const int len = min(min(fr.qb, fr.b.nc[0] - cx), w.z - c);
            bt_q_cell<L, NS>(a, fr, c, len, sts[warp], sown[warp], sq[warp], sbuf[warp], sbond[warp], sacc[warp],
                             snn[warp], nesc);
            c += len;
        }
    }
    nesc = __reduce_add_sync(kFull, nesc);
    if (lane == 0 && nesc) atomicAdd(a.qesc, (unsigned long long)nesc);
}

template <int L>
struct QTileKernel {
    template <int NS>
    static int occupancy(int *per_sm) {
        FGB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch_qtile<L, NS>, kBtW * 32, 0));
        return FGB_OK;
    }
    static int init(int *per_sm) {
        FGB_TRY(occupancy<32>(per_sm));
        FGB_TRY(occupancy<64>(per_sm + 1));
        return occupancy<kTileMaxStencil>(per_sm + 2);
    }
    static void launch(const BatchTileArgs &a, int ns, unsigned grid, cudaStream_t s) {
        FGB_KSCOPE("k_batch_qtile", s);
        if (ns <= 32)
            k_batch_qtile<L, 32><<<grid, kBtW * 32, 0, s>>>(a);
        else if (ns <= 64)
            k_batch_qtile<L, 64><<<grid, kBtW * 32, 0, s>>>(a);
        else
            k_batch_qtile<L, kTileMaxStencil><<<grid, kBtW * 32, 0, s>>>(a);
    }
};

template <class F>
static int dispatch_qtile(int l, F &&fn) {
    switch (l) {
#define FGB_QL(V) \
    case V:       \
        return fn(QTileKernel<V>());
        FGB_QL(0) FGB_QL(1) FGB_QL(2) FGB_QL(3) FGB_QL(4) FGB_QL(5) FGB_QL(6) FGB_QL(7) FGB_QL(8) FGB_QL(9) FGB_QL(10)
        FGB_QL(11) FGB_QL(12)
#undef FGB_QL
    }
    return fail(FGB_ERR_INVALID_ARG, "l = %d outside [0, 12]", l);
}

template <int NS>
static int rtile_init(size_t smem, int *per_sm) {
    FGB_CUDA(cudaFuncSetAttribute(k_batch_rtile<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FGB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch_rtile<NS>, kBtW * 32, smem));
    return FGB_OK;
}

int batch_tile_init(int bins, int l, BatchTileLaunch *out) {
    BatchTileLaunch g;
    memset(&g, 0, sizeof(g));
    g.smem_r = (size_t)kBtW * bins * sizeof(uint32_t);
    int per_sm[2] = {0, 0};
    FGB_TRY(rtile_init<64>(g.smem_r, &per_sm[0]));
    FGB_TRY(rtile_init<kTileMaxStencil>(g.smem_r, &per_sm[1]));
    for (int k = 0; k < 2; ++k) g.grid_r[k] = (unsigned)(num_sms() * std::max(per_sm[k], 1));
    g.warps = (int)g.grid_r[0] * kBtW;
    if (l >= 0) {
        FGB_TRY(ensure_consts());
        int q[3] = {0, 0, 0};
        FGB_TRY(dispatch_qtile(l, [&](auto k) { return k.init(q); }));
        for (int i = 0; i < 3; ++i) g.grid_q[i] = (unsigned)(num_sms() * std::max(q[i], 1));
    }
    *out = g;
    return FGB_OK;
}

int batch_tile_run(const BatchTileArgs &a, int l, const BatchTileLaunch &g, bool small_r, int q_ns, cudaStream_t s) {
    if (a.nitems <= 0) return FGB_OK;
    const unsigned want = (unsigned)((a.nitems + kBtW - 1) / kBtW);
    {
        FGB_KSCOPE("k_batch_rtile", s);
        const unsigned grid = std::min(g.grid_r[small_r ? 0 : 1], want);
        if (small_r)
            k_batch_rtile<64><<<grid, kBtW * 32, g.smem_r, s>>>(a);
        else
            k_batch_rtile<kTileMaxStencil><<<grid, kBtW * 32, g.smem_r, s>>>(a);
    }
    if (l >= 0)
        FGB_TRY(dispatch_qtile(l, [&](auto k) {
            k.launch(a, q_ns, std::min(g.grid_q[q_ns <= 32 ? 0 : q_ns <= 64 ? 1 : 2], want), s);
            return FGB_OK;
        }));
    FGB_LAUNCH_CHECK();
    return FGB_OK;
}

}  // namespace fgb
