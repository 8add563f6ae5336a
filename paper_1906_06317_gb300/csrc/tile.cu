// Ball-query and kNN cell-tile kernels: one warp per query cell.
//
// The warp lists the stencil cells of its cell A (offset, first point, running count),
// then stages their concatenated points 32 at a time in shared memory, already shifted
// into A's frame (cell-local coordinates + the cell's image offset).  The queries of A
// sit in registers, each spread over a group of lanes (QLayout); every round each lane
// tests its query against one staged candidate, so no lane waits on another lane's trip
// count.  Hits are counted, or appended to per-query rows that are sorted by index and
// stored.  This is the shift route only (every axis has at least 2s+1 cells and the
// stencil has at most kTileMaxStencil cells); other cases use the thread-per-query
// kernels.  The RDF's tile kernel (rdf.cu) puts candidates on lanes instead.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "fgb_tile.cuh"

namespace fgb {


// ------------------------------------------------------------------ ball-query count

// One staged chunk against the register-held queries: 32/G unrolled rounds, lane group g
// takes candidate r*G + g.  Pairs inside the FP32 band are only flagged here.
template <int G>
__device__ __forceinline__ uint32_t count_chunk(const float4 *sp, float4 Q, float lo, float hi, bool &band) {
    uint32_t cnt = 0;
#pragma unroll
    for (int r = 0; r < 32 / G; ++r) {
        const float4 c = sp[r * G];
        const float r2 = r2_f32(c.x - Q.x, c.y - Q.y, c.z - Q.z);
        cnt += r2 < lo ? 1u : 0u;
        band |= (r2 >= lo) & (r2 < hi);
    }
    return cnt;
}

// The same chunk again for the rare band pairs, decided by the FP64 sequence.
template <int G>
__device__ __forceinline__ uint32_t count_chunk_exact(const TileArgs &a, const float4 *sp, float4 Q, int i, int excl,
                                                      float lo, float hi, int &nesc) {
    uint32_t cnt = 0;
    for (int r = 0; r < 32 / G; ++r) {
        const float4 c = sp[r * G];
        const float r2 = r2_f32(c.x - Q.x, c.y - Q.y, c.z - Q.z);
        const int j = __float_as_int(c.w);
        if (r2 >= lo && r2 < hi && j != excl && j >= 0) {
            ++nesc;
            cnt += exact_r2_idx(a.bd, a.p_orig, i, a.p_orig, j) < a.T ? 1u : 0u;
        }
    }
    return cnt;
}

template <int NS>
__global__ void __launch_bounds__(kTileWarps * 32, 8) k_tile_count(TileArgs a, uint32_t *__restrict__ counts) {
    __shared__ TileStencilT<NS> sts[kTileWarps];
    __shared__ float4 sstage[kTileWarps][64];  // kept candidates, packed
    const int warp = threadIdx.x >> 5;
    const int64_t A = a.cell_lo + (int64_t)blockIdx.x * kTileWarps + warp;
    if (A >= a.ncell) return;
    const int begA = (int)__ldg(a.cell_start + A);
    const int nA = (int)__ldg(a.cell_start + A + 1) - begA;
    if (nA == 0) return;
    int cx, cy, cz;
    cell_coords((uint32_t)A, a.nc, cx, cy, cz);
    TileStencilT<NS> &ts = sts[warp];
    float4 *stage = sstage[warp];
    const int n = tile_stencil(a, cx, cy, cz, false, ts);
    const int total = ts.pre[n];
    const float lo = a.band.lo, hi = a.band.hi;
    const float reach2 = hi * (1.0f + 1e-5f);
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    int nesc = 0;
    for (int qb = 0; qb < nA; qb += 32) {
        const int nq = min(32, nA - qb);
        const QLayout L = qlayout(nq);
        const bool qact = L.myq < nq;
        const float4 Q = qact ? __ldg(a.pts + begA + qb + L.myq) : make_float4(kFar, kFar, kFar, __int_as_float(-1));
        const int i = __float_as_int(Q.w);
        const int excl = a.exclude ? i : -1;
        const float4 *sp = stage + L.g;
        uint32_t cnt = 0;
        // candidates out of reach of the pass's bounding box are dropped; the rest are
        // packed into full chunks (ballot + popc) before the rounds
        float3 blo, bhi;
        warp_box(Q.x, Q.y, Q.z, qact, blo, bhi);
        int kept = 0;
        for (int base = 0; base < total || kept > 0; base += 32) {
            if (base < total) {
                const TileCand c = tile_load(a, ts, n, total, base + lane);
                const bool keep = base + lane < total && box_dist2(blo, bhi, c.x, c.y, c.z) <= reach2;
                const unsigned m = __ballot_sync(0xffffffffu, keep);
                if (keep) stage[kept + __popc(m & lt)] = make_float4(c.x, c.y, c.z, __int_as_float(c.j));
                kept += __popc(m);
                if (kept < 32 && base + 32 < total) continue;
            }
            // a full chunk, or the last partial one padded with far entries
            if (kept < 32 && lane >= kept) stage[lane] = make_float4(kFar, kFar, kFar, __int_as_float(-1));
            __syncwarp();
            bool band = false;
#define FGB_CNT(GV) cnt += count_chunk<GV>(sp, Q, lo, hi, band)
            FGB_TILE_DISPATCH_G(L.G, FGB_CNT)
#undef FGB_CNT
            if (__any_sync(0xffffffffu, band)) {
#define FGB_CNTX(GV) cnt += count_chunk_exact<GV>(a, sp, Q, i, excl, lo, hi, nesc)
                FGB_TILE_DISPATCH_G(L.G, FGB_CNTX)
#undef FGB_CNTX
            }
            const float4 rest = stage[32 + lane];
            __syncwarp();
            if (lane < kept - 32) stage[lane] = rest;
            __syncwarp();
            kept = max(kept - 32, 0);
            if (base >= total) break;
        }
        for (int o = L.qpl; o < 32; o <<= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (L.g == 0 && qact) {
            if (a.exclude && lo > 0.f) --cnt;  // the query itself, found once at distance 0
            counts[i] = cnt;
        }
    }
    if (nesc) atomicAdd(a.esc, (unsigned long long)nesc);
}

// ------------------------------------------------------------------ ball-query write

// Each query's hits form a row of (index, distance) in shared memory; the row is sorted
// by index and stored as the query's segment.  Sort keys pack (index << 7 | slot) into
// 32 bits when indices fit 25 bits and rows 128 slots, so a bitonic network across the
// warp moves one word per key (2 or 4 keys per lane); otherwise hits are ranked by
// counting.

constexpr int kWriteStage = 512;  // candidates a cell's stencil may hold for the staged path
constexpr int kWriteQN = 2;       // queries per pass of the staged path

// Shared bytes one warp of the write kernel needs: the staged path's candidates and row,
// or the pass path's kTileQueries rows, whichever is larger.
inline __host__ __device__ size_t write_warp_bytes(int cap) {
    const size_t staged = (size_t)kWriteStage * 16 + (size_t)kWriteQN * cap * 8;
    const size_t passes = (size_t)kTileQueries * cap * 8;
    return ((staged > passes ? staged : passes) + 15) & ~(size_t)15;
}

template <int KPL>  // keys per lane (2 or 4): sorts 32 * KPL keys
__device__ __forceinline__ void bitonic_keys(uint32_t (&v)[KPL]) {
    const int lane = threadIdx.x & 31;
    constexpr int N = 32 * KPL;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            if (jj < KPL) {
                // partners inside the lane: elements e = KPL*lane + r
#pragma unroll
                for (int r = 0; r < KPL; ++r) {
                    const int p = r ^ jj;
                    if (p > r) {
                        const bool asc = (((KPL * lane + r) & k) == 0);
                        const uint32_t lo = min(v[r], v[p]), hi = max(v[r], v[p]);
                        v[r] = asc ? lo : hi;
                        v[p] = asc ? hi : lo;
                    }
                }
            } else {
                const int lm = jj / KPL;
                const bool lower = (lane & lm) == 0;
#pragma unroll
                for (int r = 0; r < KPL; ++r) {
                    const bool asc = (((KPL * lane + r) & k) == 0);
                    const uint32_t p = __shfl_xor_sync(0xffffffffu, v[r], lm);
                    v[r] = (lower == asc) ? min(v[r], p) : max(v[r], p);
                }
            }
        }
    }
}

// Two independent networks in one instruction stream (rows of two queries), so their
// shuffles and compare-exchanges overlap.
template <int KPL>
__device__ __forceinline__ void bitonic_keys2(uint32_t (&v)[KPL], uint32_t (&w)[KPL]) {
    const int lane = threadIdx.x & 31;
    constexpr int N = 32 * KPL;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            if (jj < KPL) {
#pragma unroll
                for (int r = 0; r < KPL; ++r) {
                    const int p = r ^ jj;
                    if (p > r) {
                        const bool asc = (((KPL * lane + r) & k) == 0);
                        const uint32_t lo = min(v[r], v[p]), hi = max(v[r], v[p]);
                        const uint32_t lo2 = min(w[r], w[p]), hi2 = max(w[r], w[p]);
                        v[r] = asc ? lo : hi;
                        v[p] = asc ? hi : lo;
                        w[r] = asc ? lo2 : hi2;
                        w[p] = asc ? hi2 : lo2;
                    }
                }
            } else {
                const int lm = jj / KPL;
                const bool lower = (lane & lm) == 0;
#pragma unroll
                for (int r = 0; r < KPL; ++r) {
                    const bool asc = (((KPL * lane + r) & k) == 0);
                    const uint32_t p = __shfl_xor_sync(0xffffffffu, v[r], lm);
                    const uint32_t p2 = __shfl_xor_sync(0xffffffffu, w[r], lm);
                    v[r] = (lower == asc) ? min(v[r], p) : max(v[r], p);
                    w[r] = (lower == asc) ? min(w[r], p2) : max(w[r], p2);
                }
            }
        }
    }
}

template <int KPL>
__device__ __forceinline__ void store_sorted_packed2(const uint2 *ra, uint32_t na, int ia, int64_t oa, const uint2 *rb,
                                                     uint32_t nb, int ib, int64_t ob, int32_t *__restrict__ qi_out,
                                                     int32_t *__restrict__ pj_out, float *__restrict__ d_out) {
    const int lane = threadIdx.x & 31;
    uint32_t v[KPL], w[KPL];
#pragma unroll
    for (int r = 0; r < KPL; ++r) {
        const uint32_t k = KPL * lane + r;
        v[r] = k < na ? (ra[k].x << 7) | k : 0xffffffffu;
        w[r] = k < nb ? (rb[k].x << 7) | k : 0xffffffffu;
    }
    bitonic_keys2<KPL>(v, w);
#pragma unroll
    for (int r = 0; r < KPL; ++r) {
        const uint32_t k = KPL * lane + r;
        if (k < na) {
            const uint2 e = ra[v[r] & 127u];
            __stcs(qi_out + oa + k, ia);
            __stcs(pj_out + oa + k, (int32_t)e.x);
            __stcs(d_out + oa + k, __uint_as_float(e.y));
        }
        if (k < nb) {
            const uint2 e = rb[w[r] & 127u];
            __stcs(qi_out + ob + k, ib);
            __stcs(pj_out + ob + k, (int32_t)e.x);
            __stcs(d_out + ob + k, __uint_as_float(e.y));
        }
    }
}

template <int KPL>
__device__ __forceinline__ void store_sorted_packed(const uint2 *row, uint32_t nL, int iL, int64_t oL,
                                                    int32_t *__restrict__ qi_out, int32_t *__restrict__ pj_out,
                                                    float *__restrict__ d_out) {
    const int lane = threadIdx.x & 31;
    uint32_t v[KPL];
#pragma unroll
    for (int r = 0; r < KPL; ++r) {
        const uint32_t k = KPL * lane + r;
        v[r] = k < nL ? (row[k].x << 7) | k : 0xffffffffu;
    }
    bitonic_keys<KPL>(v);
#pragma unroll
    for (int r = 0; r < KPL; ++r) {
        const uint32_t k = KPL * lane + r;
        if (k < nL) {
            const uint2 e = row[v[r] & 127u];
            __stcs(qi_out + oL + k, iL);
            __stcs(pj_out + oL + k, (int32_t)e.x);
            __stcs(d_out + oL + k, __uint_as_float(e.y));
        }
    }
}

__device__ __noinline__ void store_ranked(const uint2 *row, uint32_t nL, int iL, int64_t oL, int32_t *qi_out,
                                          int32_t *pj_out, float *d_out) {
    const int lane = threadIdx.x & 31;
    for (uint32_t b0 = 0; b0 < nL; b0 += 32) {
        const uint32_t k = b0 + lane;
        const bool act = k < nL;
        const uint2 e = act ? row[k] : make_uint2(0u, 0u);
        uint32_t rank = 0;
        for (uint32_t m = 0; m < nL; ++m) rank += row[m].x < e.x ? 1u : 0u;
        if (act) {
            __stcs(qi_out + oL + rank, iL);
            __stcs(pj_out + oL + rank, (int32_t)e.x);
            __stcs(d_out + oL + rank, __uint_as_float(e.y));
        }
    }
}

__device__ __forceinline__ void sort_store_row(const uint2 *row, uint32_t nL, int iL, int64_t oL, bool packable,
                                               int32_t *__restrict__ qi_out, int32_t *__restrict__ pj_out,
                                               float *__restrict__ d_out) {
    if (packable && nL <= 64)
        store_sorted_packed<2>(row, nL, iL, oL, qi_out, pj_out, d_out);
    else if (packable && nL <= 128)
        store_sorted_packed<4>(row, nL, iL, oL, qi_out, pj_out, d_out);
    else
        store_ranked(row, nL, iL, oL, qi_out, pj_out, d_out);
}

// Certain hits of one staged chunk; pairs inside the FP32 band are only flagged.
template <int G>
__device__ __forceinline__ void write_chunk(const float4 *sp, float4 Q, int excl, float lo, float hi, int *rowcnt,
                                            uint2 *myrow, int cap, bool &band) {
#pragma unroll 4
    for (int r = 0; r < 32 / G; ++r) {
        const float4 c = sp[r * G];
        const float r2 = r2_f32(c.x - Q.x, c.y - Q.y, c.z - Q.z);
        band |= (r2 >= lo) & (r2 < hi);
        if (r2 < lo) {
            const int j = __float_as_int(c.w);
            if (j != excl) {
                const int pos = atomicAdd(rowcnt, 1);
                if (pos < cap) myrow[pos] = make_uint2((uint32_t)j, __float_as_uint(r2 > 0.f ? r2 * rsqrt_ftz(r2) : 0.f));
            }
        }
    }
}

// The band pairs of one chunk, decided by the FP64 sequence.
__device__ __noinline__ void write_chunk_exact(const TileArgs &a, const float4 *sp, int G, float4 Q, int excl, float lo,
                                               float hi, int *rowcnt, uint2 *myrow, int cap) {
    const int i = __float_as_int(Q.w);
    for (int r = 0; r < 32 / G; ++r) {
        const float4 c = sp[r * G];
        const float r2 = r2_f32(c.x - Q.x, c.y - Q.y, c.z - Q.z);
        const int j = __float_as_int(c.w);
        if (r2 >= lo && r2 < hi && j != excl && j >= 0 && i >= 0) {
            const double e = exact_r2_idx(a.bd, a.p_orig, i, a.p_orig, j);
            if (e < a.T) {
                const int pos = atomicAdd(rowcnt, 1);
                if (pos < cap) myrow[pos] = make_uint2((uint32_t)j, __float_as_uint((float)sqrt(e)));
            }
        }
    }
}

// FP64 decision of a pair inside the band: its stored distance, or -1 when outside.
__device__ __noinline__ float write_band_pair(const TileArgs *ap, int i, int j) {
    const double e = exact_r2_idx(ap->bd, ap->p_orig, i, ap->p_orig, j);
    return e < ap->T ? (float)sqrt(e) : -1.f;
}

// Cells whose stencil holds at most kWriteStage candidates: the candidates within reach
// of the bounding box of A's points are staged once, packed and shifted into A's frame
// (a quarter of a 27-cell stencil of width r_max lies beyond that reach); then the
// queries of A are taken in pairs (two independent chains for the scheduler) with one
// candidate per lane.  Hits take consecutive row slots in candidate order (ballot +
// popc, no atomics); both rows are sorted by one interleaved network and stored before
// the next pair, so the warp needs kWriteQN = 2 rows.
template <class TS>
__device__ __forceinline__ void write_cell_staged(const TileArgs &a, const TS &ts, int n, int total, int begA,
                                                  int nA, float4 *stg, uint2 *row, const int64_t *__restrict__ seg,
                                                  const uint32_t *__restrict__ counts, int cap, bool packable,
                                                  int32_t *__restrict__ qi_out, int32_t *__restrict__ pj_out,
                                                  float *__restrict__ d_out) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    // bounding box of A's points (the queries)
    float3 blo = make_float3(INFINITY, INFINITY, INFINITY), bhi = make_float3(-INFINITY, -INFINITY, -INFINITY);
    for (int t0 = 0; t0 < nA; t0 += 32) {
        const float4 q = __ldg(a.pts + begA + min(t0 + lane, nA - 1));
        float3 l, h;
        warp_box(q.x, q.y, q.z, t0 + lane < nA, l, h);
        blo = make_float3(fminf(blo.x, l.x), fminf(blo.y, l.y), fminf(blo.z, l.z));
        bhi = make_float3(fmaxf(bhi.x, h.x), fmaxf(bhi.y, h.y), fmaxf(bhi.z, h.z));
    }
    // stage the candidates within reach of that box, packed (ballot + popc)
    const float reach2 = a.band.hi * (1.0f + 1e-5f);
    int kept = 0;
    for (int base = 0; base < total; base += 32) {
        const TileCand c = tile_load(a, ts, n, total, base + lane);
        const bool keep = base + lane < total && box_dist2(blo, bhi, c.x, c.y, c.z) <= reach2;
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) stg[kept + __popc(m & lt)] = make_float4(c.x, c.y, c.z, __int_as_float(c.j));
        kept += __popc(m);
    }
    for (int k = kept + lane; k < ((kept + 31) & ~31); k += 32) stg[k] = make_float4(kFar, kFar, kFar, __int_as_float(-1));
    __syncwarp();
    const int nch = (kept + 31) >> 5;
    const float lo = a.band.lo, hi = a.band.hi;
    uint2 *rowb = row + cap;
    for (int q = 0; q < nA; q += 2) {
        const bool two = q + 1 < nA;
        const float4 Qa = __ldg(a.pts + begA + q);
        const float4 Qb = two ? __ldg(a.pts + begA + q + 1) : make_float4(kFar, kFar, kFar, __int_as_float(-1));
        const int ia = __float_as_int(Qa.w), ib = __float_as_int(Qb.w);
        const int xa = a.exclude ? ia : -1, xb = a.exclude ? ib : -1;
        uint32_t na = 0, nb = 0;
        for (int ch = 0; ch < nch; ++ch) {
            const float4 c = stg[(ch << 5) + lane];
            const int j = __float_as_int(c.w);
            const float r2a = r2_f32(c.x - Qa.x, c.y - Qa.y, c.z - Qa.z);
            const float r2b = r2_f32(c.x - Qb.x, c.y - Qb.y, c.z - Qb.z);
            bool ha = r2a < lo && j != xa, hb = r2b < lo && j != xb;
            float da = r2a > 0.f ? r2a * rsqrt_ftz(r2a) : 0.f;
            float db = r2b > 0.f ? r2b * rsqrt_ftz(r2b) : 0.f;
            const bool ba = r2a >= lo && r2a < hi && j != xa && j >= 0;
            const bool bb = r2b >= lo && r2b < hi && j != xb && j >= 0 && ib >= 0;
            if (__any_sync(0xffffffffu, ba || bb)) {
                if (ba) {
                    const float d = write_band_pair(&a, ia, j);
                    if (d >= 0.f) {
                        ha = true;
                        da = d;
                    }
                }
                if (bb) {
                    const float d = write_band_pair(&a, ib, j);
                    if (d >= 0.f) {
                        hb = true;
                        db = d;
                    }
                }
            }
            const unsigned ma = __ballot_sync(0xffffffffu, ha), mb = __ballot_sync(0xffffffffu, hb);
            const uint32_t pa = na + __popc(ma & lt), pb = nb + __popc(mb & lt);
            if (ha && pa < (uint32_t)cap) row[pa] = make_uint2((uint32_t)j, __float_as_uint(da));
            if (hb && pb < (uint32_t)cap) rowb[pb] = make_uint2((uint32_t)j, __float_as_uint(db));
            na += __popc(ma);
            nb += __popc(mb);
        }
        __syncwarp();
        if (lane == 0 && (na > (uint32_t)cap || na != counts[ia])) atomicExch(a.err, na > (uint32_t)cap ? 1 : 2);
        if (lane == 0 && two && (nb > (uint32_t)cap || nb != counts[ib])) atomicExch(a.err, nb > (uint32_t)cap ? 1 : 2);
        const bool oka = na <= (uint32_t)cap, okb = two && nb <= (uint32_t)cap;
        if (packable && oka && okb && na <= 64 && nb <= 64) {
            store_sorted_packed2<2>(row, na, ia, seg[ia], rowb, nb, ib, seg[ib], qi_out, pj_out, d_out);
        } else if (packable && oka && okb && na <= 128 && nb <= 128) {
            store_sorted_packed2<4>(row, na, ia, seg[ia], rowb, nb, ib, seg[ib], qi_out, pj_out, d_out);
        } else {
            if (na != 0 && oka) sort_store_row(row, na, ia, seg[ia], packable, qi_out, pj_out, d_out);
            if (nb != 0 && okb) sort_store_row(rowb, nb, ib, seg[ib], packable, qi_out, pj_out, d_out);
        }
        __syncwarp();
    }
}

// Cells with larger stencils: blocks of kTileQueries queries on lane groups, the
// candidates staged 32 at a time, hits appended through per-row shared counters.
template <class TS>
__device__ __forceinline__ void write_cell_passes(const TileArgs &a, const TS &ts, int n, int total, int begA, int nA,
                                                  float4 *stage, int *rowlen, uint2 *slab,
                                                  const int64_t *__restrict__ seg, const uint32_t *__restrict__ counts,
                                                  int cap, bool packable, int32_t *__restrict__ qi_out,
                                                  int32_t *__restrict__ pj_out, float *__restrict__ d_out) {
    const int lane = threadIdx.x & 31;
    const float lo = a.band.lo, hi = a.band.hi;
    for (int qb = 0; qb < nA; qb += kTileQueries) {
        const int nq = min(kTileQueries, nA - qb);
        const QLayout L = qlayout(nq);
        const bool qact = L.myq < nq;
        const float4 Q = qact ? __ldg(a.pts + begA + qb + L.myq) : make_float4(kFar, kFar, kFar, __int_as_float(-1));
        const int excl = a.exclude ? __float_as_int(Q.w) : -1;
        if (lane < kTileQueries) rowlen[lane] = 0;
        __syncwarp();
        uint2 *myrow = slab + L.myq * cap;
        int *myrc = rowlen + L.myq;
        const float4 *sp = stage + L.g;
        for (int base = 0; base < total; base += 32) {
            tile_stage(a, ts, n, total, base, stage);
            bool band = false;
#define FGB_WR(GV) write_chunk<GV>(sp, Q, excl, lo, hi, myrc, myrow, cap, band)
            FGB_TILE_DISPATCH_G(L.G, FGB_WR)
#undef FGB_WR
            if (__any_sync(0xffffffffu, band)) write_chunk_exact(a, sp, L.G, Q, excl, lo, hi, myrc, myrow, cap);
            __syncwarp();
        }
        __syncwarp();
        for (int q = 0; q < nq; ++q) {
            const uint32_t nL = (uint32_t)rowlen[q];
            const int iL = __float_as_int(__ldg(a.pts + begA + qb + q).w);
            if (lane == 0 && (nL > (uint32_t)cap || nL != counts[iL])) atomicExch(a.err, nL > (uint32_t)cap ? 1 : 2);
            if (nL == 0 || nL > (uint32_t)cap) continue;
            sort_store_row(slab + q * cap, nL, iL, seg[iL], packable, qi_out, pj_out, d_out);
        }
        __syncwarp();
    }
}

// The write of one query cell A (one warp).
template <int NS>
__device__ __forceinline__ void tile_write_cell(const TileArgs &a, int64_t A, const int64_t *__restrict__ seg,
                                                const uint32_t *__restrict__ counts, int cap, int packable,
                                                int32_t *__restrict__ qi_out, int32_t *__restrict__ pj_out,
                                                float *__restrict__ d_out, unsigned char *tsm,
                                                TileStencilT<NS> &ts, float4 *stage1, int *rowlen) {
    const int warp = threadIdx.x >> 5;
    const int begA = (int)__ldg(a.cell_start + A);
    const int nA = (int)__ldg(a.cell_start + A + 1) - begA;
    if (nA == 0) return;
    int cx, cy, cz;
    cell_coords((uint32_t)A, a.nc, cx, cy, cz);
    const int n = tile_stencil(a, cx, cy, cz, false, ts);
    const int total = ts.pre[n];
    unsigned char *region = tsm + (size_t)warp * write_warp_bytes(cap);
    if (total <= kWriteStage)
        write_cell_staged(a, ts, n, total, begA, nA, reinterpret_cast<float4 *>(region),
                          reinterpret_cast<uint2 *>(region + kWriteStage * sizeof(float4)), seg, counts, cap,
                          packable != 0, qi_out, pj_out, d_out);
    else
        write_cell_passes(a, ts, n, total, begA, nA, stage1, rowlen, reinterpret_cast<uint2 *>(region), seg, counts,
                          cap, packable != 0, qi_out, pj_out, d_out);
}

template <int NS>
__global__ void __launch_bounds__(kTileWarps * 32, 5) k_tile_write(const __grid_constant__ TileArgs a,
                                                                   const int64_t *__restrict__ seg,
                                                                   const uint32_t *__restrict__ counts, int cap,
                                                                   int packable, int32_t *__restrict__ qi_out,
                                                                   int32_t *__restrict__ pj_out,
                                                                   float *__restrict__ d_out) {
    extern __shared__ __align__(16) unsigned char tsm[];  // kTileWarps * write_warp_bytes(cap)
    __shared__ TileStencilT<NS> sts[kTileWarps];
    __shared__ float4 sstage[kTileWarps][32];
    __shared__ int srow[kTileWarps][kTileQueries];
    const int warp = threadIdx.x >> 5;
    const int64_t A = a.cell_lo + (int64_t)blockIdx.x * kTileWarps + warp;
    if (A >= a.ncell) return;
    tile_write_cell<NS>(a, A, seg, counts, cap, packable, qi_out, pj_out, d_out, tsm, sts[warp], sstage[warp],
                        srow[warp]);
}

// The same over a device list of cells (warps stride through it).
template <int NS>
__global__ void __launch_bounds__(kTileWarps * 32, 5) k_tile_write_listed(const __grid_constant__ TileArgs a,
                                                                          const int *__restrict__ cells,
                                                                          const int *__restrict__ ncells,
                                                                          const int64_t *__restrict__ seg,
                                                                          const uint32_t *__restrict__ counts,
                                                                          int cap, int packable,
                                                                          int32_t *__restrict__ qi_out,
                                                                          int32_t *__restrict__ pj_out,
                                                                          float *__restrict__ d_out) {
    extern __shared__ __align__(16) unsigned char tsm[];
    __shared__ TileStencilT<NS> sts[kTileWarps];
    __shared__ float4 sstage[kTileWarps][32];
    __shared__ int srow[kTileWarps][kTileQueries];
    const int warp = threadIdx.x >> 5;
    const int m = *ncells;
    for (int k = blockIdx.x * kTileWarps + warp; k < m; k += gridDim.x * kTileWarps) {
        tile_write_cell<NS>(a, cells[k], seg, counts, cap, packable, qi_out, pj_out, d_out, tsm, sts[warp],
                            sstage[warp], srow[warp]);
        __syncwarp();
    }
}

// ---- dense cells: rows appended straight to the list, sorted afterwards ----
//
// When the longest row would not fit the write kernel's shared rows, hits go straight
// to the query's segment of the list: slots come from the row's shared counter (the row
// length is the count pass's, so every slot lies inside the segment), and
// sort_segments orders the rows by point index afterwards.

template <int G>
__device__ __forceinline__ void write_chunk_global(const float4 *sp, float4 Q, int i, int excl, float lo, float hi,
                                                   int *rowcnt, int64_t off, uint32_t want, int32_t *__restrict__ qi_out,
                                                   int32_t *__restrict__ pj_out, float *__restrict__ d_out,
                                                   bool &band) {
#pragma unroll 4
    for (int r = 0; r < 32 / G; ++r) {
        const float4 c = sp[r * G];
        const float r2 = r2_f32(c.x - Q.x, c.y - Q.y, c.z - Q.z);
        band |= (r2 >= lo) & (r2 < hi);
        if (r2 < lo) {
            const int j = __float_as_int(c.w);
            if (j != excl) {
                const uint32_t pos = (uint32_t)atomicAdd(rowcnt, 1);
                if (pos < want) {
                    qi_out[off + pos] = i;
                    pj_out[off + pos] = j;
                    d_out[off + pos] = r2 > 0.f ? r2 * rsqrt_ftz(r2) : 0.f;
                }
            }
        }
    }
}

// The band pairs of one chunk, decided by the FP64 sequence and appended.
__device__ __noinline__ void write_chunk_global_exact(const TileArgs &a, const float4 *sp, int G, float4 Q, int excl,
                                                      float lo, float hi, int *rowcnt, int64_t off, uint32_t want,
                                                      int32_t *qi_out, int32_t *pj_out, float *d_out) {
    const int i = __float_as_int(Q.w);
    for (int r = 0; r < 32 / G; ++r) {
        const float4 c = sp[r * G];
        const float r2 = r2_f32(c.x - Q.x, c.y - Q.y, c.z - Q.z);
        const int j = __float_as_int(c.w);
        if (r2 >= lo && r2 < hi && j != excl && j >= 0 && i >= 0) {
            const double e = exact_r2_idx(a.bd, a.p_orig, i, a.p_orig, j);
            if (e < a.T) {
                const uint32_t pos = (uint32_t)atomicAdd(rowcnt, 1);
                if (pos < want) {
                    qi_out[off + pos] = i;
                    pj_out[off + pos] = j;
                    d_out[off + pos] = (float)sqrt(e);
                }
            }
        }
    }
}

// Hits of one query cell A appended to their segments (one warp).
template <int NS>
__device__ __forceinline__ void tile_write_global_cell(const TileArgs &a, int64_t A, const int64_t *__restrict__ seg,
                                                       const uint32_t *__restrict__ counts,
                                                       int32_t *__restrict__ qi_out, int32_t *__restrict__ pj_out,
                                                       float *__restrict__ d_out, TileStencilT<NS> &ts, float4 *stage,
                                                       int *rowlen) {
    const int lane = threadIdx.x & 31;
    const int begA = (int)__ldg(a.cell_start + A);
    const int nA = (int)__ldg(a.cell_start + A + 1) - begA;
    if (nA == 0) return;
    int cx, cy, cz;
    cell_coords((uint32_t)A, a.nc, cx, cy, cz);
    const int n = tile_stencil(a, cx, cy, cz, false, ts);
    const int total = ts.pre[n];
    const float lo = a.band.lo, hi = a.band.hi;
    for (int qb = 0; qb < nA; qb += kTileQueries) {
        const int nq = min(kTileQueries, nA - qb);
        const QLayout L = qlayout(nq);
        const bool qact = L.myq < nq;
        const float4 Q = qact ? __ldg(a.pts + begA + qb + L.myq) : make_float4(kFar, kFar, kFar, __int_as_float(-1));
        const int i = __float_as_int(Q.w);
        const int excl = a.exclude ? i : -1;
        const int64_t off = qact ? seg[i] : 0;
        const uint32_t want = qact ? counts[i] : 0;
        if (lane < kTileQueries) rowlen[lane] = 0;
        __syncwarp();
        int *myrc = rowlen + L.myq;
        const float4 *sp = stage + L.g;
        for (int base = 0; base < total; base += 32) {
            tile_stage(a, ts, n, total, base, stage);
            bool band = false;
#define FGB_WG(GV) write_chunk_global<GV>(sp, Q, i, excl, lo, hi, myrc, off, want, qi_out, pj_out, d_out, band)
            FGB_TILE_DISPATCH_G(L.G, FGB_WG)
#undef FGB_WG
            if (__any_sync(0xffffffffu, band))
                write_chunk_global_exact(a, sp, L.G, Q, excl, lo, hi, myrc, off, want, qi_out, pj_out, d_out);
            __syncwarp();
        }
        if (L.g == 0 && qact && (uint32_t)*myrc != want) atomicExch(a.err, *myrc > (int)want ? 1 : 2);
        __syncwarp();
    }
}

template <int NS>
__global__ void __launch_bounds__(kTileWarps * 32) k_tile_write_global(const __grid_constant__ TileArgs a,
                                                                       const int64_t *__restrict__ seg,
                                                                       const uint32_t *__restrict__ counts,
                                                                       int32_t *__restrict__ qi_out,
                                                                       int32_t *__restrict__ pj_out,
                                                                       float *__restrict__ d_out) {
    __shared__ TileStencilT<NS> sts[kTileWarps];
    __shared__ float4 sstage[kTileWarps][32];
    __shared__ int srow[kTileWarps][kTileQueries];
    const int warp = threadIdx.x >> 5;
    const int64_t A = a.cell_lo + (int64_t)blockIdx.x * kTileWarps + warp;
    if (A >= a.ncell) return;
    tile_write_global_cell<NS>(a, A, seg, counts, qi_out, pj_out, d_out, sts[warp], sstage[warp], srow[warp]);
}

// The same over a device list of cells (warps stride through it).
template <int NS>
__global__ void __launch_bounds__(kTileWarps * 32) k_tile_write_global_listed(
    const __grid_constant__ TileArgs a, const int *__restrict__ cells, const int *__restrict__ ncells,
    const int64_t *__restrict__ seg, const uint32_t *__restrict__ counts, int32_t *__restrict__ qi_out,
    int32_t *__restrict__ pj_out, float *__restrict__ d_out) {
    __shared__ TileStencilT<NS> sts[kTileWarps];
    __shared__ float4 sstage[kTileWarps][32];
    __shared__ int srow[kTileWarps][kTileQueries];
    const int warp = threadIdx.x >> 5;
    const int m = *ncells;
    for (int k = blockIdx.x * kTileWarps + warp; k < m; k += gridDim.x * kTileWarps) {
        tile_write_global_cell<NS>(a, cells[k], seg, counts, qi_out, pj_out, d_out, sts[warp], sstage[warp],
                                   srow[warp]);
        __syncwarp();
    }
}

// Rows of up to 32 * KPL entries sorted on packed keys (index << SB | slot), for indices
// below 2^(32 - SB) and rows of at most 2^SB slots, then stored.
template <int KPL, int SB>
__device__ __forceinline__ void store_sorted_packed_sb(const uint2 *row, uint32_t nL, int iL, int64_t oL,
                                                       int32_t *__restrict__ qi_out, int32_t *__restrict__ pj_out,
                                                       float *__restrict__ d_out) {
    const int lane = threadIdx.x & 31;
    uint32_t v[KPL];
#pragma unroll
    for (int r = 0; r < KPL; ++r) {
        const uint32_t k = KPL * lane + r;
        v[r] = k < nL ? (row[k].x << SB) | k : 0xffffffffu;
    }
    bitonic_keys<KPL>(v);
#pragma unroll
    for (int r = 0; r < KPL; ++r) {
        const uint32_t k = KPL * lane + r;
        if (k < nL) {
            const uint2 e = row[v[r] & ((1u << SB) - 1u)];
            __stcs(qi_out + oL + k, iL);
            __stcs(pj_out + oL + k, (int32_t)e.x);
            __stcs(d_out + oL + k, __uint_as_float(e.y));
        }
    }
}

// A row of at most 32 (KPLA + KPLB) entries with point indices below 2^22 (one warp):
// keys (index << 10 | slot) in kb (padded with ~0 to that length) and distances in db
// by slot.  The first 32 KPLA keys and the next 32 KPLB are each sorted by the register
// network, the two sorted runs are merged (lane l produces its outputs from the
// merge-path split of its diagonal), and the merged row is stored coalesced.  Keys are
// distinct (indices are distinct within a row), so the merge needs no tie rule.
template <int KPLA, int KPLB>
__device__ __forceinline__ void sort_merge_store(uint32_t *kb, const float *db, uint32_t n, int iq, int64_t b,
                                                 int32_t *__restrict__ qi, int32_t *__restrict__ pj,
                                                 float *__restrict__ dist) {
    constexpr int LA = 32 * KPLA, LB = 32 * KPLB;  // lengths of the two runs
    constexpr int PER = KPLA + KPLB;               // outputs per lane
    const int lane = threadIdx.x & 31;
    {
        uint32_t v[KPLA];
#pragma unroll
        for (int r = 0; r < KPLA; ++r) v[r] = kb[KPLA * lane + r];
        bitonic_keys<KPLA>(v);
#pragma unroll
        for (int r = 0; r < KPLA; ++r) kb[KPLA * lane + r] = v[r];
    }
    {
        uint32_t v[KPLB];
#pragma unroll
        for (int r = 0; r < KPLB; ++r) v[r] = kb[LA + KPLB * lane + r];
        bitonic_keys<KPLB>(v);
#pragma unroll
        for (int r = 0; r < KPLB; ++r) kb[LA + KPLB * lane + r] = v[r];
    }
    __syncwarp();
    const uint32_t *A = kb, *B = kb + LA;
    const int d = PER * lane;
    int lo = max(0, d - LB), hi = min(d, LA);  // A elements among the first d outputs
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (A[mid] < B[d - mid - 1])
            lo = mid + 1;
        else
            hi = mid;
    }
    int ia = lo, ib = d - lo;
    uint32_t out[PER];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const uint32_t x = ia < LA ? A[ia] : 0xffffffffu, y = ib < LB ? B[ib] : 0xffffffffu;
        const bool ta = x < y;
        out[r] = ta ? x : y;
        ia += ta ? 1 : 0;
        ib += ta ? 0 : 1;
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < PER; ++r) kb[d + r] = out[r];
    __syncwarp();
    for (uint32_t k = lane; k < n; k += 32) {
        const uint32_t key = kb[k];
        __stcs(qi + b + k, iq);
        __stcs(pj + b + k, (int32_t)(key >> 10));
        __stcs(dist + b + k, db[key & 1023u]);
    }
}

// Rows of 257..MAXN entries (MAXN 512 or 1,024) by two sorted runs and a merge, in the
// warp's buffer of `width` entries (keys in its first half, distances in the second).
template <int MAXN>
__device__ __forceinline__ void sort_merge_row(uint2 *row, int width, uint32_t n, int64_t b, int32_t *__restrict__ qi,
                                               int32_t *__restrict__ pj, float *__restrict__ dist) {
    const int lane = threadIdx.x & 31;
    uint32_t *kb = reinterpret_cast<uint32_t *>(row);
    float *db = reinterpret_cast<float *>(kb + width);
    const uint32_t len = n <= 384 ? 384 : n <= 512 ? 512 : n <= 768 ? 768 : 1024;  // padded
    for (uint32_t k = lane; k < len; k += 32) {
        kb[k] = k < n ? ((uint32_t)pj[b + k] << 10) | k : 0xffffffffu;
        if (k < n) db[k] = dist[b + k];
    }
    const int iq = qi[b];
    __syncwarp();
    if (MAXN > 512 && n > 768)
        sort_merge_store<16, 16>(kb, db, n, iq, b, qi, pj, dist);
    else if (MAXN > 512 && n > 512)
        sort_merge_store<16, 8>(kb, db, n, iq, b, qi, pj, dist);
    else if (n > 384)
        sort_merge_store<8, 8>(kb, db, n, iq, b, qi, pj, dist);
    else
        sort_merge_store<8, 4>(kb, db, n, iq, b, qi, pj, dist);
}

// Sorts each segment [seg[q], seg[q+1]) of (qi, pj, dist) by point index in place: one
// warp per segment, staged as (index, distance) in shared memory, then the same network
// (or ranking) and stores as the write kernels.  WIDE (rows longer than 128): rows of up
// to 256 or 512 entries take a register network on packed keys when the point indices
// fit 23 bits; MERGE: rows of 257..MERGE entries (indices below 2^22) take two sorted
// runs and a merge (sort_merge_row) in the same buffer; other rows are sorted in shared memory by a bitonic
// network over the row padded to a power of two (width entries per warp), then stored
// coalesced.  packable: bit 0 indices below 2^25, bit 1 below 2^23, bit 2 below 2^22.
// Only the rows with nmin < length <= cap are sorted by one launch (nmin >= 1), so that
// rows of different length classes can take buffers of their own size.
template <bool WIDE, int MERGE>
__global__ void k_sort_segments(const int64_t *__restrict__ seg, int64_t nq, int nmin, int cap, int width,
                                int packable, int32_t *__restrict__ qi, int32_t *__restrict__ pj,
                                float *__restrict__ dist) {
    extern __shared__ uint2 srows[];  // (blockDim / 32) * (WIDE ? width : cap)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (q >= nq) return;
    const int64_t b = seg[q];
    const uint32_t n = (uint32_t)(seg[q + 1] - b);
    if (n <= (uint32_t)nmin || n > (uint32_t)cap) return;
    uint2 *row = srows + (size_t)warp * (WIDE ? width : cap);
    if (MERGE > 0 && WIDE && n > 256 && n <= (uint32_t)min(MERGE, width) && (packable & 4)) {
        sort_merge_row<MERGE>(row, width, n, b, qi, pj, dist);
        return;
    }
    for (uint32_t k = lane; k < n; k += 32) row[k] = make_uint2((uint32_t)pj[b + k], __float_as_uint(dist[b + k]));
    const int iq = qi[b];
    if (!WIDE || n <= 128) {
        __syncwarp();
        sort_store_row(row, n, iq, b, (packable & 1) != 0, qi, pj, dist);
        return;
    }
    if (n <= 256 && (packable & 2)) {
        __syncwarp();
        store_sorted_packed_sb<8, 8>(row, n, iq, b, qi, pj, dist);
        return;
    }
    if (n <= 512 && (packable & 2)) {
        __syncwarp();
        store_sorted_packed_sb<16, 9>(row, n, iq, b, qi, pj, dist);
        return;
    }

    uint32_t N = 256;
    while (N < n) N <<= 1;  // N <= width
    for (uint32_t k = n + lane; k < N; k += 32) row[k] = make_uint2(0xffffffffu, 0u);
    __syncwarp();
    for (uint32_t k = 2; k <= N; k <<= 1)
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t t = lane; t < N / 2; t += 32) {
                // the t-th compare-exchange pair of this step: e has bit j clear, l = e | j
                const uint32_t e = ((t & ~(j - 1)) << 1) | (t & (j - 1)), l = e | j;
                const uint2 x = row[e], y = row[l];
                const bool asc = (e & k) == 0;
                if ((x.x > y.x) == asc) {
                    row[e] = y;
                    row[l] = x;
                }
            }
            __syncwarp();
        }
    for (uint32_t k = lane; k < n; k += 32) {
        const uint2 e = row[k];
        __stcs(qi + b + k, iq);
        __stcs(pj + b + k, (int32_t)e.x);
        __stcs(dist + b + k, __uint_as_float(e.y));
    }
}

// One launch over the rows of length in (nmin, cap], each staged in a buffer of `width`
// entries (WIDE) or `cap` entries.
static int sort_segments_class(const int64_t *seg, int64_t nq, int nmin, int cap, int width, bool wide, int packable,
                               int32_t *qi, int32_t *pj, float *dist, cudaStream_t s) {
    const int stride = wide ? width : cap;
    int warps = 4;
    while (warps > 1 && (size_t)warps * stride * sizeof(uint2) > 96 * 1024) warps >>= 1;
    const size_t smem = (size_t)warps * stride * sizeof(uint2);
    if (smem > 200 * 1024) return fail(FGB_ERR_UNSUPPORTED, "more than %d neighbors of one point", 25600);
    const unsigned grid = (unsigned)((nq + warps - 1) / warps);
    // the merge of two sorted runs for the rows of 257..1,024 entries that the launch
    // holds (MERGE: the longest such row; the 1,024 build takes more registers)
    auto kern = !wide                                  ? k_sort_segments<false, 0>
                : (cap > 512 && nmin < 1024 && width >= 1024) ? k_sort_segments<true, 1024>
                : (cap > 256 && nmin < 512 && width >= 512)   ? k_sort_segments<true, 512>
                                                               : k_sort_segments<true, 0>;
    FGB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FGB_KSCOPE("k_sort_segments", s);
    kern<<<grid, 32 * warps, smem, s>>>(seg, nq, nmin, cap, width, packable, qi, pj, dist);
    FGB_LAUNCH_CHECK();
    return FGB_OK;
}

int sort_segments(const int64_t *seg, int64_t nq, int cap, int64_t npoints, int32_t *qi, int32_t *pj, float *dist,
                  cudaStream_t s) {
    if (nq == 0 || cap <= 1) return FGB_OK;
    const int packable = (npoints < ((int64_t)1 << 25) ? 1 : 0) | (npoints < ((int64_t)1 << 23) ? 2 : 0) |
                         (npoints < ((int64_t)1 << 22) ? 4 : 0);
    int width = 256;
    while (width < cap) width <<= 1;
    const bool wide = cap > 128 && (size_t)width * sizeof(uint2) <= 128 * 1024;
    if (!wide) return sort_segments_class(seg, nq, 1, cap, width, false, packable, qi, pj, dist, s);
    // long rows by length class (up to 512, up to 1,024, longer), each class with a row
    // buffer of its own size, so the common shorter rows keep more warps resident
    int lo = 1;
    for (const int hi : {512, 1024}) {
        if (lo >= cap) break;
        FGB_TRY(sort_segments_class(seg, nq, lo, std::min(cap, hi), std::min(width, hi), true, packable, qi, pj, dist,
                                    s));
        lo = hi;
    }
    if (cap > lo) FGB_TRY(sort_segments_class(seg, nq, lo, cap, width, true, packable, qi, pj, dist, s));
    return FGB_OK;
}

// ------------------------------------------------------------------ k nearest

// kNN by radius: every candidate within a collection radius rc <= r0 (the stencil's
// covered radius) is gathered as (r2 bits, index) into a 64-slot row per query, the row
// is sorted (bitonic network across the warp: one entry per lane up to 32, two up to
// 64), and the first m become the answer when the ranking is certain: every gap between
// neighbours among the first m+1 exceeds 2 delta and, if only m were found, the m-th
// sits more than 2 delta inside rc^2 (everything not gathered lies at rc or beyond, and
// inside r0 nothing is missed).  rc is set per query cell so that the stencil's mean
// density puts about m + 12 points inside it.  Other queries (fewer than m within rc,
// more than 64, or a near tie) are listed for the warp-per-query kernel.
struct KnnTile {
    float r0sq;      // the covered radius r0, squared (collection radii stay below it)
    float cnum;      // rc^dim = cnum / (candidates of the stencil): m + 12 expected inside
    int dim;         // 3, or 2 for a 2D box (cnum then gives rc^2)
    float delta;     // FP32 error bound on r2 at r0
    int k;
    int stride;      // output row length m
    int32_t *qi, *pj;
    float *dist;
    int32_t *counts;
    int *list;       // sorted positions of queries left to the thread kernel
    int *list_count;
};

// Sorts one gathered row (cnt <= 64 entries of (r2 bits, index) in shared memory) and
// writes its first m when the ranking is certain (the rule above); else lists the query
// (sorted position t) for the warp-per-query kernel.
__device__ __forceinline__ void knn_finish_row(const uint2 *row, int cnt, int m, float rcsq, const KnnTile &K, int iL,
                                               int t) {
    const int lane = threadIdx.x & 31;
    bool ok = cnt >= m && cnt <= 64;
    const float twod = 2.f * K.delta;
    if (ok && cnt <= 32) {
        // one 32-bit key per lane: the r2 bits with the low five replaced by the row slot
        // (r2 >= 0, so the bits order as the values).  Keys of distinct truncated r2
        // order as the true r2; equal truncated r2 is flagged as a tie below.
        uint32_t key = lane < cnt ? ((row[lane].x & ~31u) | (uint32_t)lane) : 0xffffffffu;
#pragma unroll
        for (int kk = 2; kk <= 32; kk <<= 1) {
            const bool asc = (lane & kk) == 0;
#pragma unroll
            for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                const uint32_t k0 = __shfl_xor_sync(0xffffffffu, key, jj);
                const bool takemin = ((lane & jj) == 0) == asc;
                if ((k0 < key) == takemin) key = k0;
            }
        }
        const uint2 e0 = lane < cnt ? row[key & 31u] : make_uint2(0xffffffffu, 0u);
        const float f0 = __uint_as_float(e0.x);
        const float fnext = __shfl_down_sync(0xffffffffu, f0, 1);
        const uint32_t knext = __shfl_down_sync(0xffffffffu, key, 1);
        bool amb = lane < m && lane + 1 < cnt && (fnext - f0 <= twod || (knext >> 5) == (key >> 5));
        const float fm = __shfl_sync(0xffffffffu, f0, m - 1);
        if (cnt == m && !(fm + twod < rcsq)) amb = true;
        ok = !__any_sync(0xffffffffu, amb);
        if (ok) {
            const int64_t row0 = (int64_t)iL * m;
            if (lane < m) {
                K.qi[row0 + lane] = iL;
                K.pj[row0 + lane] = (int32_t)e0.y;
                K.dist[row0 + lane] = sqrtf(f0);
            }
            if (lane == 0) K.counts[iL] = m;
        }
    } else if (ok) {
        uint2 e0 = 2 * lane < cnt ? row[2 * lane] : make_uint2(0xffffffffu, 0u);
        uint2 e1 = 2 * lane + 1 < cnt ? row[2 * lane + 1] : make_uint2(0xffffffffu, 0u);
#pragma unroll
        for (int kk = 2; kk <= 64; kk <<= 1) {
            const bool asc = ((2 * lane) & kk) == 0;
#pragma unroll
            for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                if (jj == 1) {
                    const bool sw = ((e0.x > e1.x) || (e0.x == e1.x && e0.y > e1.y)) == asc;
                    const uint2 t0 = sw ? e1 : e0, t1 = sw ? e0 : e1;
                    e0 = t0;
                    e1 = t1;
                } else {
                    const int lm = jj >> 1;
                    const uint32_t k0 = __shfl_xor_sync(0xffffffffu, e0.x, lm);
                    const uint32_t v0 = __shfl_xor_sync(0xffffffffu, e0.y, lm);
                    const uint32_t k1 = __shfl_xor_sync(0xffffffffu, e1.x, lm);
                    const uint32_t v1 = __shfl_xor_sync(0xffffffffu, e1.y, lm);
                    const bool takemin = ((lane & lm) == 0) == asc;
                    const bool l0 = k0 < e0.x || (k0 == e0.x && v0 < e0.y);
                    const bool l1 = k1 < e1.x || (k1 == e1.x && v1 < e1.y);
                    if (l0 == takemin) e0 = make_uint2(k0, v0);
                    if (l1 == takemin) e1 = make_uint2(k1, v1);
                }
            }
        }
        const float f0 = __uint_as_float(e0.x), f1 = __uint_as_float(e1.x);
        const float fnext = __shfl_down_sync(0xffffffffu, f0, 1);
        bool amb = false;
        if (2 * lane < m && 2 * lane + 1 < cnt) amb |= f1 - f0 <= twod;
        if (2 * lane + 1 < m && 2 * lane + 2 < cnt && lane < 31) amb |= fnext - f1 <= twod;
        const float fm = __shfl_sync(0xffffffffu, (m - 1) & 1 ? f1 : f0, (m - 1) >> 1);
        if (cnt == m && !(fm + twod < rcsq)) amb = true;
        ok = !__any_sync(0xffffffffu, amb);
        if (ok) {
            const int64_t row0 = (int64_t)iL * m;
            if (2 * lane < m) {
                K.qi[row0 + 2 * lane] = iL;
                K.pj[row0 + 2 * lane] = (int32_t)e0.y;
                K.dist[row0 + 2 * lane] = sqrtf(f0);
            }
            if (2 * lane + 1 < m) {
                K.qi[row0 + 2 * lane + 1] = iL;
                K.pj[row0 + 2 * lane + 1] = (int32_t)e1.y;
                K.dist[row0 + 2 * lane + 1] = sqrtf(f1);
            }
            if (lane == 0) K.counts[iL] = m;
        }
    }
    if (!ok && lane == 0) K.list[atomicAdd(K.list_count, 1)] = t;
}

// One warp per query cell: the cell's candidates within reach (rc) of the bounding box
// of its points are staged once (at most kKnnStage; a cell with more lists its queries),
// then each query in turn takes them 32 at a time, its hits packed into the row by
// ballot positions.
constexpr int kKnnStage = 224;
constexpr int kKnnOwnCap = 512;

template <int NS>
__global__ void __launch_bounds__(kTileWarps * 32, 9) k_tile_knn(TileArgs a, KnnTile K) {
    __shared__ TileStencilT<NS> sts[kTileWarps];
    __shared__ float4 sstage[kTileWarps][kKnnStage + 32];
    __shared__ uint2 srowbuf[kTileWarps][64];
    __shared__ uint8_t sown[kTileWarps][kKnnOwnCap];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t A = a.cell_lo + (int64_t)blockIdx.x * kTileWarps + warp;
    if (A >= a.ncell) return;
    const int begA = (int)__ldg(a.cell_start + A);
    const int nA = (int)__ldg(a.cell_start + A + 1) - begA;
    if (nA == 0) return;
    int cx, cy, cz;
    cell_coords((uint32_t)A, a.nc, cx, cy, cz);
    TileStencilT<NS> &ts = sts[warp];
    float4 *stage = sstage[warp];
    uint2 *row = srowbuf[warp];
    const int n = tile_stencil(a, cx, cy, cz, false, ts);
    const int total = ts.pre[n];
    const uint8_t *own = nullptr;
    if (total <= kKnnOwnCap) {
        tile_owners(ts, n, sown[warp]);
        own = sown[warp];
    }
    const int m = K.stride;
    float rcsq = K.r0sq;
    if (total > 0) {
        const float x = K.cnum / (float)total;
        const float r2 = K.dim == 3 ? cbrtf(x) * cbrtf(x) : x;
        rcsq = fminf(rcsq, r2);
    }
    float3 blo = make_float3(INFINITY, INFINITY, INFINITY), bhi = make_float3(-INFINITY, -INFINITY, -INFINITY);
    for (int t0 = 0; t0 < nA; t0 += 32) {
        const float4 q = __ldg(a.pts + begA + min(t0 + lane, nA - 1));
        float3 l, h;
        warp_box(q.x, q.y, q.z, t0 + lane < nA, l, h);
        blo = make_float3(fminf(blo.x, l.x), fminf(blo.y, l.y), fminf(blo.z, l.z));
        bhi = make_float3(fmaxf(bhi.x, h.x), fmaxf(bhi.y, h.y), fmaxf(bhi.z, h.z));
    }
    // a candidate farther than this from the box is at FP32 r2 >= rcsq from every query
    const float reach2 = rcsq * (1.0f + 1e-5f);
    const unsigned lt = lanemask_lt();
    int kept = total > 1024 ? -1 : 0;
    for (int base = 0; kept >= 0 && base < total; base += 32) {
        const TileCand c = tile_load_own(a, ts, own, n, total, base + lane);
        const bool keep = base + lane < total && box_dist2(blo, bhi, c.x, c.y, c.z) <= reach2;
        const unsigned mk = __ballot_sync(0xffffffffu, keep);
        if (kept + __popc(mk) > kKnnStage) {
            kept = -1;
            break;
        }
        if (keep) stage[kept + __popc(mk & lt)] = make_float4(c.x, c.y, c.z, __int_as_float(c.j));
        kept += __popc(mk);
    }
    if (kept < 0) {
        for (int q = lane; q < nA; q += 32) K.list[atomicAdd(K.list_count, 1)] = begA + q;
        return;
    }
    if (kept + lane < ((kept + 31) & ~31)) stage[kept + lane] = make_float4(kFar, kFar, kFar, __int_as_float(-1));
    __syncwarp();
    const int nch = (kept + 31) >> 5;
    float4 Qn = __ldg(a.pts + begA);  // the next query's record, loaded a query ahead
    for (int t = 0; t < nA; ++t) {
        const float4 Q = Qn;
        if (t + 1 < nA) Qn = __ldg(a.pts + begA + t + 1);
        const int iL = __float_as_int(Q.w);
        const int excl = a.exclude ? iL : -1;
        int cnt = 0;
        for (int ch = 0; ch < nch; ++ch) {
            const float4 c = stage[(ch << 5) + lane];
            const float r2 = r2_f32(c.x - Q.x, c.y - Q.y, c.z - Q.z);
            const int j = __float_as_int(c.w);
            const bool hit = r2 < rcsq && j != excl;
            const unsigned mh = __ballot_sync(0xffffffffu, hit);
            const int pos = cnt + __popc(mh & lt);
            if (hit && pos < 64) row[pos] = make_uint2(__float_as_uint(r2), (uint32_t)j);
            cnt += __popc(mh);
        }
        __syncwarp();
        knn_finish_row(row, cnt, m, rcsq, K, iL, begA + t);
        __syncwarp();
    }
}

// ------------------------------------------------------------------ host side

bool tile_ok(const StencilPlan &p) {
    if (p.mode != 0) return false;
    const int n = (2 * p.s[0] + 1) * (2 * p.s[1] + 1) * (2 * p.s[2] + 1);
    return n <= kTileMaxStencil;
}

bool tile_worth(const fgb_nq *nq) {
    const int64_t cells = nq->grid.ncell;
    // a sharded call walks cells, which only the cell-tile kernels do
    return nq->walk_set || force_tile_kernels() || (cells >= 4 * (int64_t)num_sms() && nq->n <= 64 * cells);
}

TileArgs tile_args(const fgb_nq *nq, const StencilPlan &p, double R, int exclude) {
    TileArgs t;
    memset(&t, 0, sizeof(t));
    for (int k = 0; k < 3; ++k) {
        t.nc[k] = nq->grid.nc[k];
        t.s[k] = p.s[k];
        t.ts[k] = p.ts[k];
    }
    t.off = p.table;
    t.pts = nq->sorted;
    t.cell_start = nq->cell_start;
    t.ncell = nq->grid.ncell;
    t.cell_lo = 0;
    if (nq->box.is2d) {
        // every point of a 2D box lies in the middle of the three z layers: its query cells
        // are that layer's (points elsewhere break the z = 0 rule and are not queried)
        const int64_t layer = (int64_t)nq->grid.nc[0] * nq->grid.nc[1];
        t.cell_lo = layer;
        t.ncell = 2 * layer;
    }
    if (nq->walk_set) {
        // a shard of the query cells (Section "Implementation": per-particle work split
        // across workers): walk only [walk_lo, walk_hi)
        t.cell_lo = std::max<int64_t>(t.cell_lo, nq->walk_lo);
        t.ncell = std::max<int64_t>(t.cell_lo, std::min<int64_t>(t.ncell, nq->walk_hi));
    }
    t.p_orig = nq->points;
    t.bf = nq->box.f;
    t.bd = nq->box.d;
    t.T = sqrt_threshold(R);
    band_around(t.T, r2_error_bound(p, R), &t.band.lo, &t.band.hi);
    t.exclude = exclude;
    return t;
}

int tile_count(const fgb_nq *nq, const StencilPlan &p, double R, int exclude, unsigned long long *esc, int *err,
               uint32_t *counts, cudaStream_t s) {
    TileArgs t = tile_args(nq, p, R, exclude);
    t.esc = esc;
    t.err = err;
    const unsigned grid = (unsigned)((t.ncell - t.cell_lo + kTileWarps - 1) / kTileWarps);
    if ((2 * p.s[0] + 1) * (2 * p.s[1] + 1) * (2 * p.s[2] + 1) <= 32) {
        FGB_KSCOPE("k_tile_count", s);
        k_tile_count<32><<<grid, kTileWarps * 32, 0, s>>>(t, counts);
    } else {
        FGB_KSCOPE("k_tile_count", s);
        k_tile_count<kTileMaxStencil><<<grid, kTileWarps * 32, 0, s>>>(t, counts);
    }
    FGB_LAUNCH_CHECK();
    return FGB_OK;
}

size_t tile_write_smem(int cap);

int tile_write(const fgb_nq *nq, const StencilPlan &p, double R, int exclude, int *err, const int64_t *seg,
               const uint32_t *counts, int cap, int32_t *qi, int32_t *pj, float *dist, cudaStream_t s) {
    TileArgs t = tile_args(nq, p, R, exclude);
    t.err = err;
    const size_t smem = tile_write_smem(cap);
    if (smem > 160 * 1024) return fail(FGB_ERR_UNSUPPORTED, "tile write: neighbor count too large");
    const unsigned grid = (unsigned)((t.ncell - t.cell_lo + kTileWarps - 1) / kTileWarps);
    const int packable = cap <= 128 && nq->n < ((int64_t)1 << 25);
    // the kernel also holds static shared memory: always raise the dynamic limit
    if ((2 * p.s[0] + 1) * (2 * p.s[1] + 1) * (2 * p.s[2] + 1) <= 32) {
        FGB_CUDA(cudaFuncSetAttribute(k_tile_write<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        FGB_KSCOPE("k_tile_write", s);
        k_tile_write<32><<<grid, kTileWarps * 32, smem, s>>>(t, seg, counts, cap, packable, qi, pj, dist);
    } else {
        FGB_CUDA(cudaFuncSetAttribute(k_tile_write<kTileMaxStencil>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        FGB_KSCOPE("k_tile_write", s);
        k_tile_write<kTileMaxStencil><<<grid, kTileWarps * 32, smem, s>>>(t, seg, counts, cap, packable, qi, pj, dist);
    }
    FGB_LAUNCH_CHECK();
    return FGB_OK;
}


int tile_knn(const fgb_nq *nq, const StencilPlan &p, int k, int m, int exclude, int32_t *qi, int32_t *pj, float *dist,
             int32_t *counts, int *list, int *list_count, cudaStream_t s) {
    TileArgs t = tile_args(nq, p, 1.0, exclude);
    double r0 = std::min(nq->grid.wc[0], std::min(nq->grid.wc[1], nq->grid.wc[2])) * p.s[0];
    for (int kk = 1; kk < 3; ++kk) r0 = std::min(r0, nq->grid.wc[kk] * p.s[kk]);
    r0 *= 0.99999;
    KnnTile K;
    K.r0sq = (float)(r0 * r0 * (1.0 - 1e-6));
    // the stencil's 27 cells (9 of them hold points in a 2D box) over the unit ball's
    // measure, times m + 12: rc^dim for the expected count m + 12 at the stencil's density
    const GridHost &g = nq->grid;
    const double area = nq->box.p[0] * nq->box.p[1] / ((double)g.nc[0] * g.nc[1]);
    const double extra = 12.0;  // under 1 % of uniform queries find fewer than m within rc
    if (nq->box.is2d) {
        K.dim = 2;
        K.cnum = (float)((m + extra) * 9.0 * area / M_PI);
    } else {
        K.dim = 3;
        K.cnum = (float)((m + extra) * 27.0 * area * nq->box.p[2] / g.nc[2] / (4.0 / 3.0 * M_PI));
    }
    K.delta = (float)r2_error_bound(p, r0);
    K.k = k;
    K.stride = m;
    K.qi = qi;
    K.pj = pj;
    K.dist = dist;
    K.counts = counts;
    K.list = list;
    K.list_count = list_count;
    const unsigned grid = (unsigned)((t.ncell - t.cell_lo + kTileWarps - 1) / kTileWarps);
    {
        FGB_KSCOPE("k_tile_knn", s);
        k_tile_knn<32><<<grid, kTileWarps * 32, 0, s>>>(t, K);
    }
    FGB_LAUNCH_CHECK();
    return FGB_OK;
}

size_t tile_write_smem(int cap) { return (size_t)kTileWarps * write_warp_bytes(cap); }

int tile_write_global(const fgb_nq *nq, const StencilPlan &p, double R, int exclude, int *err, const int64_t *seg,
                      const uint32_t *counts, int32_t *qi, int32_t *pj, float *dist, cudaStream_t s) {
    TileArgs t = tile_args(nq, p, R, exclude);
    t.err = err;
    const unsigned grid = (unsigned)((t.ncell - t.cell_lo + kTileWarps - 1) / kTileWarps);
    if ((2 * p.s[0] + 1) * (2 * p.s[1] + 1) * (2 * p.s[2] + 1) <= 32) {
        FGB_KSCOPE("k_tile_write_global", s);
        k_tile_write_global<32><<<grid, kTileWarps * 32, 0, s>>>(t, seg, counts, qi, pj, dist);
    } else {
        FGB_KSCOPE("k_tile_write_global", s);
        k_tile_write_global<kTileMaxStencil><<<grid, kTileWarps * 32, 0, s>>>(t, seg, counts, qi, pj, dist);
    }
    FGB_LAUNCH_CHECK();
    return FGB_OK;
}

// The write kernels over a device list of cells (the cells the staged-sort write
// kernel of nlist.cu could not take); the grid strides through the list.
int tile_write_listed(const fgb_nq *nq, const StencilPlan &p, double R, int exclude, int *err, const int64_t *seg,
                      const uint32_t *counts, int cap, const int *cells, const int *ncells, int32_t *qi, int32_t *pj,
                      float *dist, cudaStream_t s) {
    TileArgs t = tile_args(nq, p, R, exclude);
    t.err = err;
    const size_t smem = tile_write_smem(cap);
    if (smem > 160 * 1024) return fail(FGB_ERR_UNSUPPORTED, "tile write: neighbor count too large");
    const int packable = cap <= 128 && nq->n < ((int64_t)1 << 25);
    const unsigned grid = (unsigned)num_sms() * 4;
    if ((2 * p.s[0] + 1) * (2 * p.s[1] + 1) * (2 * p.s[2] + 1) <= 32) {
        FGB_CUDA(cudaFuncSetAttribute(k_tile_write_listed<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        FGB_KSCOPE("k_tile_write_listed", s);
        k_tile_write_listed<32><<<grid, kTileWarps * 32, smem, s>>>(t, cells, ncells, seg, counts, cap, packable, qi,
                                                                    pj, dist);
    } else {
        FGB_CUDA(cudaFuncSetAttribute(k_tile_write_listed<kTileMaxStencil>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        FGB_KSCOPE("k_tile_write_listed", s);
        k_tile_write_listed<kTileMaxStencil><<<grid, kTileWarps * 32, smem, s>>>(t, cells, ncells, seg, counts, cap,
                                                                                 packable, qi, pj, dist);
    }
    FGB_LAUNCH_CHECK();
    return FGB_OK;
}

int tile_write_global_listed(const fgb_nq *nq, const StencilPlan &p, double R, int exclude, int *err,
                             const int64_t *seg, const uint32_t *counts, const int *cells, const int *ncells,
                             int32_t *qi, int32_t *pj, float *dist, cudaStream_t s) {
    TileArgs t = tile_args(nq, p, R, exclude);
    t.err = err;
    const unsigned grid = (unsigned)num_sms() * 4;
    if ((2 * p.s[0] + 1) * (2 * p.s[1] + 1) * (2 * p.s[2] + 1) <= 32) {
        FGB_KSCOPE("k_tile_write_global_listed", s);
        k_tile_write_global_listed<32><<<grid, kTileWarps * 32, 0, s>>>(t, cells, ncells, seg, counts, qi, pj, dist);
    } else {
        FGB_KSCOPE("k_tile_write_global_listed", s);
        k_tile_write_global_listed<kTileMaxStencil><<<grid, kTileWarps * 32, 0, s>>>(t, cells, ncells, seg, counts,
                                                                                     qi, pj, dist);
    }
    FGB_LAUNCH_CHECK();
    return FGB_OK;
}

}  // namespace fgb
