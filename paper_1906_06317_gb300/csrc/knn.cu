// k-nearest-neighbor query (Section "Implementation": queries by number of neighbors;
// freud's num_neighbors).  Neighbors of a query are ordered by (r2, point index) with r2
// from the defining FP64 sequence; see query.cu for the overview.
#include <cmath>
#include <cstring>

#include "fgb_tile.cuh"

namespace fgb {

struct KnnArgs {
    int nc[3];
    int ts[3];             // offset-table half-width (mode 0 possible while s <= ts)
    const float4 *off;
    float3 step[3];
    float wc[3];           // perpendicular cell widths
    BoxF bf;
    BoxD bd;
    const float4 *pts;
    const uint32_t *cell_start;
    const float4 *qs;
    const uint32_t *qcell;
    int64_t nq;
    int64_t npts;
    const float *p_orig;
    const float *q_orig;
    int k;
    int exclude;
    int self;
    int stride;            // row stride of the output (m if uniform, else k)
    float ext, rowmax, Lsum;
    float half_wmin2;      // (w_min / 2)^2, slightly reduced
    int *flag_count;
    int4 *flags;           // (t, s, threshold bits, 0)
    int flag_cap;
    int *err;              // 1 = box too small, 2 = flag list overflow
    int32_t *qi_out, *pj_out;
    float *d_out;
    int32_t *counts;
    const int *list;        // when set: only these sorted positions, list_count of them
    const int *list_count;
};

// FP32 error bound on r2 at radius R for a walk with half-width s (mode 0) or the
// general route (mode 1); same terms as plan_stencil/r2_error_bound on the host.
__device__ __forceinline__ float knn_delta(const KnnArgs &a, int mode, int s, float R) {
    const float u = kU32;
    const float e = mode == 0 ? 2.f * u * (5.f * a.ext + 2.f * s * a.rowmax + R)
                              : 2.f * u * (5.f * a.ext + 8.f * a.Lsum + 4.f * R);
    const float d = 3.4641016f * R * e + 3.f * e * e + 3.f * u * (R + e) * (R + e) + 1e-12f * (R + a.Lsum) * (R + a.Lsum);
    return 1.5f * d;
}

__device__ __forceinline__ Stencil knn_stencil(const KnnArgs &a, int s, bool &all_full) {
    Stencil S;
    S.mode = 0;
    all_full = true;
    for (int k = 0; k < 3; ++k) {
        S.nc[k] = a.nc[k];
        S.s[k] = s;
        S.ts[k] = a.ts[k];
        S.full[k] = 2 * s + 1 > a.nc[k];
        if (S.full[k] || s > a.ts[k] || a.off == nullptr) S.mode = 1;
        all_full &= (bool)S.full[k];
        S.step[k] = a.step[k];
    }
    S.off = a.off;
    return S;
}

template <int KT>
__global__ void __launch_bounds__(128) k_knn(KnnArgs a) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a.list) {
        if (t >= *a.list_count) return;
        t = a.list[t];
    } else if (t >= a.nq) {
        return;
    }
    const float4 q = a.qs[t];
    const int i = __float_as_int(q.w);
    int cx, cy, cz;
    cell_coords(a.qcell[t], a.nc, cx, cy, cz);
    const int excl = a.exclude ? i : -1;
    const int avail = (int)min((int64_t)0x7fffffff, a.npts - ((a.exclude && i < a.npts) ? 1 : 0));
    const int m = min(a.k, avail);
    float br[KT];
    int bj[KT];
    int found = 0, s = 1, mode = 0;
    float delta = 0.f;
    for (;; ++s) {
        bool all_full;
        const Stencil S = knn_stencil(a, s, all_full);
        mode = S.mode;
#pragma unroll
        for (int q2 = 0; q2 < KT; ++q2) {
            br[q2] = INFINITY;
            bj[q2] = 0x7fffffff;
        }
        found = 0;
        for_stencil(S, cx, cy, cz, make_float3(q.x, q.y, q.z), false, [&](int cell, float qx, float qy, float qz, bool) {
            const uint32_t beg = __ldg(a.cell_start + cell), end = __ldg(a.cell_start + cell + 1);
            for (uint32_t p = beg; p < end; ++p) {
                const float4 c = __ldg(a.pts + p);
                const int j = __float_as_int(c.w);
                if (j == excl) continue;
                const float3 d = cand_disp(S, a.bf, c, qx, qy, qz);
                const float r2 = r2_f32(d.x, d.y, d.z);
                ++found;
                if (r2 < br[KT - 1] || (r2 == br[KT - 1] && j < bj[KT - 1])) topk_insert<KT>(br, bj, r2, j);
            }
        });
        if (all_full) {
            delta = knn_delta(a, mode, s, m > 0 ? sqrtf(pick<KT>(br, min(m, KT) - 1)) : 0.f);
            break;
        }
        float rcov = INFINITY;
        for (int k2 = 0; k2 < 3; ++k2)
            if (!S.full[k2]) rcov = fminf(rcov, s * a.wc[k2]);
        rcov *= 0.99999f;
        if (found >= m && m > 0) {
            const float rk2 = pick<KT>(br, m - 1);
            delta = knn_delta(a, mode, s, sqrtf(rk2) + 1e-3f);
            if (rk2 + delta < rcov * rcov) break;
        } else if (m == 0) {
            break;
        }
    }
    a.counts[i] = m;
    const float rm2 = m > 0 ? pick<KT>(br, m - 1) : 0.f;
    if (m > 0 && rm2 + delta >= a.half_wmin2) {
        atomicOr(a.err, 1);
        return;
    }
    // a ranking is certain when every neighboring gap among the first m+1 exceeds 2 delta
    bool ambiguous = false;
    const int last = min(found, KT) - 1;
#pragma unroll
    for (int q2 = 0; q2 + 1 < KT; ++q2)
        if (q2 < m && q2 + 1 <= last && br[q2 + 1] - br[q2] <= 2.f * delta) ambiguous = true;
    const int64_t row = (int64_t)i * a.stride;
    if (ambiguous) {
        const int slot = atomicAdd(a.flag_count, 1);
        if (slot < a.flag_cap) {
            const float thr = rm2 + 2.f * delta;
            a.flags[slot] = make_int4((int)t, s, __float_as_int(thr * 1.0000005f), 0);
        } else {
            atomicOr(a.err, 2);
        }
        return;
    }
#pragma unroll
    for (int q2 = 0; q2 < KT; ++q2)
        if (q2 < m) {
            a.qi_out[row + q2] = i;
            a.pj_out[row + q2] = bj[q2];
            a.d_out[row + q2] = sqrtf(br[q2]);
        }
}

// Listed queries (those the cell-tile kernel left: too many candidates for its rows,
// too few within its radius, or a near tie), a warp each: the same stencil walk,
// widening and ranking rule as k_knn, with each cell's candidates split across the
// lanes.  The best candidates so far are 64-bit keys (r2 bits << 32 | index: the (r2,
// index) order, r2 >= 0) in a per-warp shared buffer; a candidate enters when its key is
// below the KT-th best, and the buffer is sorted and cut back to KT entries whenever it
// holds 64 or more, so dense cells cost about one compare per candidate.
constexpr int kKnnWarps = 4;
constexpr int kKnnBuf = 128;

// Sorts buf[0, nb) (nb <= kKnnBuf, padded with ~0) and keeps the KT best; returns their
// number and sets thr to the KT-th key (all ones while fewer are kept).
template <int KT>
__device__ __forceinline__ int knn_trim(unsigned long long *buf, int nb, unsigned long long &thr) {
    const int lane = threadIdx.x & 31;
    for (int k = nb + lane; k < kKnnBuf; k += 32) buf[k] = ~0ull;
    __syncwarp();
    for (unsigned k = 2; k <= (unsigned)kKnnBuf; k <<= 1)
        for (unsigned j = k >> 1; j > 0; j >>= 1) {
            for (unsigned t = lane; t < kKnnBuf / 2; t += 32) {
                const unsigned e = ((t & ~(j - 1)) << 1) | (t & (j - 1)), l = e | j;
                const unsigned long long x = buf[e], y = buf[l];
                if ((x > y) == ((e & k) == 0)) {
                    buf[e] = y;
                    buf[l] = x;
                }
            }
            __syncwarp();
        }
    const int kept = min(nb, KT);
    thr = kept == KT ? buf[KT - 1] : ~0ull;
    return kept;
}

__device__ __forceinline__ float key_r2(unsigned long long key) { return __uint_as_float((uint32_t)(key >> 32)); }

template <int KT>
__global__ void __launch_bounds__(kKnnWarps * 32) k_knn_warp(KnnArgs a) {
    __shared__ unsigned long long sbuf[kKnnWarps][kKnnBuf];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned long long *buf = sbuf[warp];
    const unsigned lt = lanemask_lt();
    const int nlist = *a.list_count;
    for (int64_t w = (int64_t)blockIdx.x * kKnnWarps + warp; w < nlist; w += (int64_t)gridDim.x * kKnnWarps) {
        const int64_t t = a.list[w];
        const float4 q = a.qs[t];
        const int i = __float_as_int(q.w);
        int cx, cy, cz;
        cell_coords(a.qcell[t], a.nc, cx, cy, cz);
        const int excl = a.exclude ? i : -1;
        const int avail = (int)min((int64_t)0x7fffffff, a.npts - ((a.exclude && i < a.npts) ? 1 : 0));
        const int m = min(a.k, avail);
        int nb = 0, found = 0, s = 1, mode = 0;
        unsigned long long thr = ~0ull;
        float delta = 0.f;
        for (;; ++s) {
            bool all_full;
            const Stencil S = knn_stencil(a, s, all_full);
            mode = S.mode;
            nb = 0;
            found = 0;
            thr = ~0ull;
            // the query's own cell first (its points set a tight threshold at once), then
            // the rest of the stencil
            const int own = (cz * a.nc[1] + cy) * a.nc[0] + cx;
            for (int pass = 0; pass < 2; ++pass)
            for_stencil(S, cx, cy, cz, make_float3(q.x, q.y, q.z), false,
                        [&](int cell, float qx, float qy, float qz, bool) {
                            if ((cell == own) != (pass == 0)) return;
                            const uint32_t beg = __ldg(a.cell_start + cell), end = __ldg(a.cell_start + cell + 1);
                            for (uint32_t p0 = beg; p0 < end; p0 += 32) {
                                const uint32_t p = p0 + lane;
                                bool valid = false, take = false;
                                unsigned long long key = ~0ull;
                                if (p < end) {
                                    const float4 c = __ldg(a.pts + p);
                                    const int j = __float_as_int(c.w);
                                    if (j != excl) {
                                        const float3 d = cand_disp(S, a.bf, c, qx, qy, qz);
                                        const float r2 = r2_f32(d.x, d.y, d.z);
                                        key = ((unsigned long long)__float_as_uint(r2) << 32) | (uint32_t)j;
                                        valid = true;
                                        take = key < thr;
                                    }
                                }
                                found += __popc(__ballot_sync(0xffffffffu, valid));
                                const unsigned mk = __ballot_sync(0xffffffffu, take);
                                if (take) buf[nb + __popc(mk & lt)] = key;  // nb <= 63 here
                                nb += __popc(mk);
                                if (nb >= 64) {
                                    __syncwarp();
                                    nb = knn_trim<KT>(buf, nb, thr);
                                }
                            }
                        });
            __syncwarp();
            nb = knn_trim<KT>(buf, nb, thr);
            if (all_full) {
                delta = knn_delta(a, mode, s, m > 0 ? sqrtf(key_r2(buf[min(m, KT) - 1])) : 0.f);
                break;
            }
            float rcov = INFINITY;
            for (int k2 = 0; k2 < 3; ++k2)
                if (!S.full[k2]) rcov = fminf(rcov, s * a.wc[k2]);
            rcov *= 0.99999f;
            if (found >= m && m > 0) {
                const float rk2 = key_r2(buf[m - 1]);
                delta = knn_delta(a, mode, s, sqrtf(rk2) + 1e-3f);
                if (rk2 + delta < rcov * rcov) break;
            } else if (m == 0) {
                break;
            }
        }
        if (lane == 0) a.counts[i] = m;
        const float rm2 = m > 0 ? key_r2(buf[m - 1]) : 0.f;
        if (m > 0 && rm2 + delta >= a.half_wmin2) {
            if (lane == 0) atomicOr(a.err, 1);
            __syncwarp();
            continue;
        }
        // a ranking is certain when every neighbouring gap among the first m+1 exceeds 2 delta
        const int last = min(found, KT) - 1;
        const bool gap_small =
            lane < m && lane + 1 <= last && key_r2(buf[lane + 1]) - key_r2(buf[lane]) <= 2.f * delta;
        if (__any_sync(0xffffffffu, gap_small)) {
            if (lane == 0) {
                const int slot = atomicAdd(a.flag_count, 1);
                if (slot < a.flag_cap) {
                    const float thr2 = rm2 + 2.f * delta;
                    a.flags[slot] = make_int4((int)t, s, __float_as_int(thr2 * 1.0000005f), 0);
                } else {
                    atomicOr(a.err, 2);
                }
            }
            __syncwarp();
            continue;
        }
        const int64_t row = (int64_t)i * a.stride;
        if (lane < m) {
            const unsigned long long key = buf[lane];
            a.qi_out[row + lane] = i;
            a.pj_out[row + lane] = (int)(uint32_t)key;
            a.d_out[row + lane] = sqrtf(key_r2(key));
        }
        __syncwarp();
    }
}

// Exact ranking for flagged queries (near ties in FP32): candidates whose FP32 r2 is
// within the threshold get their FP64 r2 and are ranked by (r2, j) in double precision.
// A warp per flagged query: the lanes split the stencil's cells,
// list every candidate inside the threshold with its FP64 r2 in shared memory, and each
// listed candidate's rank by (r2, j) is counted against the others; ranks below m are
// written.  A query with more than kExactCap such candidates keeps the serial walk.
constexpr int kExactCap = 128;
constexpr int kExactWarps = 4;

template <int KT>
__device__ __noinline__ void knn_exact_serial(const KnnArgs &a, int64_t t, int s, float thr) {
    const float4 q = a.qs[t];
    const int i = __float_as_int(q.w);
    int cx, cy, cz;
    cell_coords(a.qcell[t], a.nc, cx, cy, cz);
    const int excl = a.exclude ? i : -1;
    const int m = a.counts[i];
    bool all_full;
    const Stencil S = knn_stencil(a, s, all_full);
    double br[KT];
    int bj[KT];
#pragma unroll
    for (int q2 = 0; q2 < KT; ++q2) {
        br[q2] = INFINITY;
        bj[q2] = 0x7fffffff;
    }
    for_stencil(S, cx, cy, cz, make_float3(q.x, q.y, q.z), false, [&](int cell, float qx, float qy, float qz, bool) {
        const uint32_t beg = __ldg(a.cell_start + cell), end = __ldg(a.cell_start + cell + 1);
        for (uint32_t p = beg; p < end; ++p) {
            const float4 c = __ldg(a.pts + p);
            const int j = __float_as_int(c.w);
            if (j == excl) continue;
            const float3 d = cand_disp(S, a.bf, c, qx, qy, qz);
            const float r2 = r2_f32(d.x, d.y, d.z);
            if (r2 > thr) continue;
            const double e = exact_r2_idx(a.bd, a.q_orig, i, a.p_orig, j);
            if (e < br[KT - 1] || (e == br[KT - 1] && j < bj[KT - 1])) {
                double cr = e;
                int cj = j;
#pragma unroll
                for (int q2 = 0; q2 < KT; ++q2) {
                    const bool less = cr < br[q2] || (cr == br[q2] && cj < bj[q2]);
                    const double tr = less ? br[q2] : cr;
                    const int tj = less ? bj[q2] : cj;
                    br[q2] = less ? cr : br[q2];
                    bj[q2] = less ? cj : bj[q2];
                    cr = tr;
                    cj = tj;
                }
            }
        }
    });
    const int64_t row = (int64_t)i * a.stride;
#pragma unroll
    for (int q2 = 0; q2 < KT; ++q2)
        if (q2 < m) {
            a.qi_out[row + q2] = i;
            a.pj_out[row + q2] = bj[q2];
            a.d_out[row + q2] = (float)sqrt(br[q2]);
        }
}

template <int KT>
__global__ void __launch_bounds__(kExactWarps * 32) k_knn_exact_warp(KnnArgs a) {
    __shared__ double se[kExactWarps][kExactCap];
    __shared__ int sj[kExactWarps][kExactCap];
    __shared__ int scnt[kExactWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nflag = min(*a.flag_count, a.flag_cap);
    for (int f = blockIdx.x * kExactWarps + warp; f < nflag; f += gridDim.x * kExactWarps) {
        const int4 fl = a.flags[f];
        const int64_t t = fl.x;
        const int s = fl.y;
        const float thr = __int_as_float(fl.z);
        const float4 q = a.qs[t];
        const int i = __float_as_int(q.w);
        int cx, cy, cz;
        cell_coords(a.qcell[t], a.nc, cx, cy, cz);
        const int excl = a.exclude ? i : -1;
        const int m = a.counts[i];
        bool all_full;
        const Stencil S = knn_stencil(a, s, all_full);
        // the stencil's offsets as a box [lo, hi] per axis (for_stencil's enumeration)
        int lo[3], hi[3];
        const int cc[3] = {cx, cy, cz};
        for (int k = 0; k < 3; ++k) {
            lo[k] = (S.mode != 0 && S.full[k]) ? -cc[k] : -S.s[k];
            hi[k] = (S.mode != 0 && S.full[k]) ? S.nc[k] - 1 - cc[k] : S.s[k];
        }
        const int wx = hi[0] - lo[0] + 1, wy = hi[1] - lo[1] + 1, wz = hi[2] - lo[2] + 1;
        if (lane == 0) scnt[warp] = 0;
        __syncwarp();
        for (int o = lane; o < wx * wy * wz; o += 32) {
            const int ox = o % wx + lo[0], oy = (o / wx) % wy + lo[1], oz = o / (wx * wy) + lo[2];
            const int xx = wrap_cell(cx + ox, S.nc[0]), yy = wrap_cell(cy + oy, S.nc[1]),
                      zz = wrap_cell(cz + oz, S.nc[2]);
            const int cell = (zz * S.nc[1] + yy) * S.nc[0] + xx;
            float qx, qy, qz;
            if (S.mode == 0) {
                const int twx = 2 * S.ts[0] + 1, twy = 2 * S.ts[1] + 1;
                const float4 of = __ldg(S.off + ((oz + S.ts[2]) * twy + (oy + S.ts[1])) * twx + (ox + S.ts[0]));
                qx = q.x - of.x;
                qy = q.y - of.y;
                qz = q.z - of.z;
            } else {
                const float fx = (float)ox, fy = (float)oy, fz = (float)oz;
                qx = q.x - fmaf(fz, S.step[2].x, fmaf(fy, S.step[1].x, fx * S.step[0].x));
                qy = q.y - fmaf(fz, S.step[2].y, fy * S.step[1].y);
                qz = q.z - fz * S.step[2].z;
            }
            const uint32_t beg = __ldg(a.cell_start + cell), end = __ldg(a.cell_start + cell + 1);
            for (uint32_t p = beg; p < end; ++p) {
                const float4 c = __ldg(a.pts + p);
                const int j = __float_as_int(c.w);
                if (j == excl) continue;
                const float3 d = cand_disp(S, a.bf, c, qx, qy, qz);
                if (r2_f32(d.x, d.y, d.z) > thr) continue;
                const int slot = atomicAdd(&scnt[warp], 1);
                if (slot < kExactCap) {
                    se[warp][slot] = exact_r2_idx(a.bd, a.q_orig, i, a.p_orig, j);
                    sj[warp][slot] = j;
                }
            }
        }
        __syncwarp();
        const int n = scnt[warp];
        if (n > kExactCap) {
            if (lane == 0) knn_exact_serial<KT>(a, t, s, thr);
        } else {
            const int64_t row = (int64_t)i * a.stride;
            for (int e = lane; e < n; e += 32) {
                const double me = se[warp][e];
                const int mj = sj[warp][e];
                int rank = 0;
                for (int k = 0; k < n; ++k) {
                    const double oe = se[warp][k];
                    rank += (oe < me || (oe == me && sj[warp][k] < mj)) ? 1 : 0;
                }
                if (rank < m) {
                    a.qi_out[row + rank] = i;
                    a.pj_out[row + rank] = mj;
                    a.d_out[row + rank] = (float)sqrt(me);
                }
            }
        }
        __syncwarp();
    }
}

// Packs rows of stride k into the final arrays (only when row lengths differ).
__global__ void k_knn_compact(const int64_t *__restrict__ seg, const int32_t *__restrict__ counts, int64_t nq, int k,
                              const int32_t *__restrict__ tqi, const int32_t *__restrict__ tpj,
                              const float *__restrict__ td, int32_t *qi, int32_t *pj, float *d) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    for (int a = 0; a < counts[i]; ++a) {
        qi[seg[i] + a] = tqi[i * k + a];
        pj[seg[i] + a] = tpj[i * k + a];
        d[seg[i] + a] = td[i * k + a];
    }
}

__global__ void k_knn_segments(int64_t nq, int m, int64_t *seg) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= nq) seg[i] = i * (int64_t)m;
}

template <int KT>
static void launch_knn(const KnnArgs &a, cudaStream_t s) {
    if (a.list) {
        // the queries the cell-tile kernel left, a warp each (the list length is on the
        // device: a grid of warps walks it)
        FGB_KSCOPE("k_knn_warp", s);
        k_knn_warp<KT><<<(unsigned)num_sms() * 8, kKnnWarps * 32, 0, s>>>(a);
    } else {
        FGB_KSCOPE("k_knn", s);
        k_knn<KT><<<(unsigned)((a.nq + 127) / 128), 128, 0, s>>>(a);
    }
    {
        FGB_KSCOPE("k_knn_exact", s);
        k_knn_exact_warp<KT><<<num_sms() * 4, kExactWarps * 32, 0, s>>>(a);
    }
}

int knn_query(fgb_nq *nq, const QueryPoints &Q, const fgb_query_args *args, cudaStream_t s, fgb_nlist *nl) {
    const int k = args->num_neighbors;
    if (k > 32) return fail(FGB_ERR_UNSUPPORTED, "num_neighbors > 32 is not supported");
    const int64_t nqq = Q.n, np = nq->n;
    const bool excl = args->exclude_ii != 0;
    // every query has the same row length unless exclusion removes a point for some
    // queries only (separate query points with at most k points)
    int64_t avail_min = np - ((excl && (Q.self || nqq > 0)) ? 1 : 0);
    const bool uniform = Q.self || !excl || np > k;
    const int m_uniform = (int)std::min<int64_t>(k, std::max<int64_t>(0, Q.self ? avail_min : (excl ? np - 1 : np)));
    StencilPlan plan;
    FGB_TRY(plan_stencil(nq, nq->grid.wc[0] * 0.5, kMaxStencil, s, &plan));
    KnnArgs a;
    memset(&a, 0, sizeof(a));
    const GridHost &g = nq->grid;
    const BoxHost &b = nq->box;
    for (int q = 0; q < 3; ++q) {
        a.nc[q] = g.nc[q];
        a.ts[q] = plan.mode == 0 ? plan.ts[q] : 0;
        a.wc[q] = (float)g.wc[q];
    }
    a.off = plan.mode == 0 ? plan.table : nullptr;
    a.step[0] = make_float3((float)(b.M[0][0] / g.nc[0]), 0.f, 0.f);
    a.step[1] = make_float3((float)(b.M[0][1] / g.nc[1]), (float)(b.M[1][1] / g.nc[1]), 0.f);
    a.step[2] = make_float3((float)(b.M[0][2] / g.nc[2]), (float)(b.M[1][2] / g.nc[2]), (float)(b.M[2][2] / g.nc[2]));
    a.bf = b.f;
    a.bd = b.d;
    a.pts = nq->sorted;
    a.cell_start = nq->cell_start;
    a.qs = Q.sorted;
    a.qcell = Q.cell;
    a.nq = nqq;
    a.npts = np;
    a.p_orig = nq->points;
    a.q_orig = Q.orig;
    a.k = k;
    a.exclude = excl ? 1 : 0;
    a.self = Q.self ? 1 : 0;
    a.stride = uniform ? m_uniform : k;
    double rowmax = 0;
    for (int r = 0; r < 3; ++r) {
        double e = 0;
        for (int c = 0; c < 3; ++c) e += std::fabs(b.M[r][c]) / g.nc[c];
        rowmax = std::max(rowmax, e);
    }
    a.ext = (float)g.ext;
    a.rowmax = (float)rowmax;
    a.Lsum = (float)plan.Lsum;
    a.half_wmin2 = (float)(0.25 * b.wmin * b.wmin * (1.0 - 1e-4));
    a.flag_cap = (int)std::min<int64_t>(std::max<int64_t>(nqq, 1), 1 << 24);
    int *ctl = nullptr;  // [0] flag count, [1] error bits, [2] list length, [4..] list
    nl->n_query = nqq;
    nl->n_points = np;
    const int64_t rows = uniform ? nqq * (int64_t)m_uniform : nqq * (int64_t)k;
    int32_t *tqi = nullptr, *tpj = nullptr;
    float *td = nullptr;
    int st = dalloc_n(&ctl, 5 + nqq, s);
    st = st ? st : dalloc_n(&a.flags, a.flag_cap, s);
    st = st ? st : dalloc_n(&nl->counts, nqq, s);
    st = st ? st : dalloc_n(&nl->segments, nqq + 1, s);
    st = st ? st : dalloc_n(&tqi, rows, s);
    st = st ? st : dalloc_n(&tpj, rows, s);
    st = st ? st : dalloc_n(&td, rows, s);
    if (st == FGB_OK) {
        cudaMemsetAsync(ctl, 0, 5 * sizeof(int), s);
        a.flag_count = ctl;
        a.err = ctl + 1;
        a.qi_out = tqi;
        a.pj_out = tpj;
        a.d_out = td;
        a.counts = nl->counts;
        // self queries on the shift route: radius kernel over cell tiles first, the
        // thread-per-query kernel only for the queries it leaves
        const bool tile = Q.self && plan.mode == 0 && plan.s[0] == 1 && plan.s[1] == 1 && plan.s[2] == 1 &&
                          m_uniform >= 1 && m_uniform <= 62 && tile_worth(nq) && !force_thread_kernels();
        if (tile && nqq > 0) {
            // 2D: only the points' layer is walked; a point off the plane keeps a zero count
            if (nq->box.is2d && cudaMemsetAsync(nl->counts, 0, sizeof(int32_t) * nqq, s) != cudaSuccess)
                st = fail(FGB_ERR_CUDA, "memset failed");
            st = st ? st : tile_knn(nq, plan, k, m_uniform, a.exclude, tqi, tpj, td, nl->counts, ctl + 4, ctl + 2, s);
            a.list = ctl + 4;
            a.list_count = ctl + 2;
        }
        if (nqq > 0) {
            const int KT = k + 1;
            if (KT <= 5) launch_knn<5>(a, s);
            else if (KT <= 9) launch_knn<9>(a, s);
            else if (KT <= 13) launch_knn<13>(a, s);
            else if (KT <= 17) launch_knn<17>(a, s);
            else if (KT <= 25) launch_knn<25>(a, s);
            else launch_knn<33>(a, s);
        }
        if (uniform) {
            {
                FGB_KSCOPE("k_knn_segments", s);
                k_knn_segments<<<(unsigned)((nqq + 256) / 256), 256, 0, s>>>(nqq, m_uniform, nl->segments);
            }
        } else {
            st = scan_u32_i64(reinterpret_cast<uint32_t *>(nl->counts), nl->segments, nqq, nullptr, s);
        }
        int hctl[2] = {0, 0};
        int64_t total = rows;
        cudaMemcpyAsync(hctl, ctl, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
        if (!uniform) cudaMemcpyAsync(&total, nl->segments + nqq, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (st == FGB_OK && e != cudaSuccess) st = fail(FGB_ERR_CUDA, "kNN query failed: %s", cudaGetErrorString(e));
        if (st == FGB_OK && (hctl[1] & 1))
            st = fail(FGB_ERR_BOX_TOO_SMALL, "a k-th nearest neighbor lies at or beyond half the smallest box width");
        if (st == FGB_OK && (hctl[1] & 2)) st = fail(FGB_ERR_CAPACITY, "kNN re-ranking list overflowed");
        nl->escalations = hctl[0];
        nl->n_pairs = total;
        if (st == FGB_OK && uniform) {
            nl->qi = tqi;
            nl->pj = tpj;
            nl->dist = td;
            tqi = tpj = nullptr;
            td = nullptr;
        } else if (st == FGB_OK) {
            st = st ? st : dalloc_n(&nl->qi, total, s);
            st = st ? st : dalloc_n(&nl->pj, total, s);
            st = st ? st : dalloc_n(&nl->dist, total, s);
            if (st == FGB_OK && nqq > 0)
                {
                    FGB_KSCOPE("k_knn_compact", s);
                    k_knn_compact<<<(unsigned)((nqq + 127) / 128), 128, 0, s>>>(nl->segments, nl->counts, nqq, k, tqi, tpj,
                                                                               td, nl->qi, nl->pj, nl->dist);
                }
        }
    }
    dfree(tqi, s);
    dfree(tpj, s);
    dfree(td, s);
    dfree(ctl, s);
    dfree(a.flags, s);
    dfree(plan.table, s);
    nl->symmetric = 0;
    nl->kind = 1;
    (void)avail_min;
    return st;
}

}  // namespace fgb
