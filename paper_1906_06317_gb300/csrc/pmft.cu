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
// The definition is FP64: the defining minimum-image displacement (exact_disp), cos and
// sin of the float32 angle in FP64, then the rotation and the bin index above, each
// operation rounded once.  Both routes (the fused cell-tile kernel and the list kernel)
// decide a bond in FP32 only when a proven error bound keeps it clear of every bin edge,
// and bin the rest by that FP64 sequence.
#include <cmath>
#include <cstring>
#include <vector>

#include "fgb_tile.cuh"

struct fgb_pmft {
    double x_max, y_max;
    int bx, by;
    unsigned long long *hist;  // device, bx * by, x major
    float2 *trig32;            // device, FP32 (cos, sin): by query (list route) or sorted position
    int64_t trig32_cap;
    int2 *esc;                 // bonds (query, point) left to the FP64 pass
    int esc_cap;
    unsigned *ctl;             // device [0] escalated bonds, [1] work counter
    int64_t last_esc;
    double norm;               // sum over frames of N_query * N_points / area
    cudaStream_t stream;
};

namespace fgb {

struct PmftBins {
    double x_max, y_max, dx, dy;
    int bx, by;
};

// FP32 (cos, sin) of the query orientations by query index (list route).
__global__ void k_pmft_trig(const float *__restrict__ theta, int64_t n, float2 *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s, c;
    sincosf(theta[i], &s, &c);
    out[i] = make_float2(c, s);
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

// FP32 (cos, sin) of every orientation by sorted position of the cell list (the fused
// kernel reads them next to the records).  sincosf is within 2 ulp of the exact values.
__global__ void k_pmft_trig_sorted(const float4 *__restrict__ sorted, const float *__restrict__ theta, int64_t n,
                                   float2 *__restrict__ out32) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int i = __float_as_int(__ldg(&sorted[p].w));
    float s, c;
    sincosf(__ldg(theta + i), &s, &c);
    out32[p] = make_float2(c, s);
}

// Bin of a bond at (tx, ty) in bin units (t = (x' + x_max) / dx in FP32) given decision
// margins (mx, my) in bins: >= 0 decided inside, -1 decided outside, -2 open.  An axis
// is decided when the fraction of t keeps the margin from both edges; a decided axis
// outside the range settles the bond.
__device__ __forceinline__ int pmft_decide(float tx, float ty, float mx, float my, int bx, int by) {
    const float fx = floorf(tx), fy = floorf(ty);
    const float rx = tx - fx, ry = ty - fy;
    const bool okx = rx > mx && rx < 1.f - mx, oky = ry > my && ry < 1.f - my;
    const bool inx = fx >= 0.f && fx < (float)bx, iny = fy >= 0.f && fy < (float)by;
    if ((okx && !inx) || (oky && !iny)) return -1;
    if (okx && oky) return (int)fx * by + (int)fy;
    return -2;
}

// FP64 (cos, sin) of one orientation, as the definition takes them.
__device__ __forceinline__ double2 trig64(const float *theta, int i) {
    double s, c;
    sincos((double)__ldg(theta + i), &s, &c);
    return make_double2(c, s);
}

struct PmftListArgs {
    BoxD bd;
    const float *p, *qp, *theta;
    const float2 *cs;          // FP32 (cos, sin) by query index
    const int32_t *qi, *pj;
    int64_t m;
    PmftBins B;
    float inv_dx, inv_dy, off_x, off_y;
    float kx, ky, cx, cy;      // margin in bins: k * max(|d_x|, |d_y|) + c
    float wx, wy, wz;          // 0.499 of the box lengths: plain differences below them
    unsigned long long *hist;
};

// One thread per bond of a NeighborList (query_point_indices address qp and cs).  The
// displacement is the defining FP64 one; rotation and binning run in FP32 and a bond
// within the margin of an edge is binned again by the FP64 sequence.  SHARED: the block
// counts into a shared histogram (bins <= kPmftListMaxBins) over its own contiguous
// range of at most 2^30 bonds, so no 32-bit count can overflow.
constexpr int kPmftListMaxBins = 16384;

template <bool SHARED>
__global__ void __launch_bounds__(256) k_pmft_list(const __grid_constant__ PmftListArgs a, int64_t per_block) {
    extern __shared__ uint32_t lh[];
    const int bins = a.B.bx * a.B.by;
    if (SHARED) {
        for (int b = threadIdx.x; b < bins; b += blockDim.x) lh[b] = 0;
        __syncthreads();
    }
    const int64_t e0 = (int64_t)blockIdx.x * per_block, e1 = min(a.m, e0 + per_block);
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int i = __ldg(a.qi + e), j = __ldg(a.pj + e);
        const float *xi = a.qp + 3 * (int64_t)i, *xj = a.p + 3 * (int64_t)j;
        // Below 0.499 of a box length on every axis, the defining sequence shifts by no
        // box vector and its displacement is the plain difference, which the FP32
        // difference matches within half an ulp.  Other bonds take the FP64 sequence.
        float dx = __ldg(xj) - __ldg(xi), dy = __ldg(xj + 1) - __ldg(xi + 1);
        const float dz = __ldg(xj + 2) - __ldg(xi + 2);
        double3 d;
        const bool plain = fabsf(dx) < a.wx && fabsf(dy) < a.wy && fabsf(dz) < a.wz;
        if (!plain) {
            d = exact_disp(a.bd, xi, xj);
            dx = (float)d.x;
            dy = (float)d.y;
        }
        const float dm = fmaxf(fabsf(dx), fabsf(dy));
        const float2 cs = __ldg(a.cs + i);
        const float xq = fmaf(cs.x, dx, cs.y * dy), yq = fmaf(cs.x, dy, -(cs.y * dx));
        int b = pmft_decide(fmaf(xq, a.inv_dx, a.off_x), fmaf(yq, a.inv_dy, a.off_y), fmaf(a.kx, dm, a.cx),
                            fmaf(a.ky, dm, a.cy), a.B.bx, a.B.by);
        if (b == -2) {
            if (plain) d = exact_disp(a.bd, xi, xj);
            b = pmft_bin64(a.B, trig64(a.theta, i), d);
        }
        if (b >= 0) {
            if (SHARED)
                atomicAdd(lh + b, 1u);
            else
                atomicAdd(a.hist + b, 1ull);
        }
    }
    if (SHARED) {
        __syncthreads();
        for (int b = threadIdx.x; b < bins; b += blockDim.x) {
            const uint32_t v = lh[b];
            if (v) atomicAdd(a.hist + b, (unsigned long long)v);
        }
    }
}

// ------------------------------------------------------------------ fused cell tiles
//
// Self bonds on the cell list's shift route, in the scheme of the RDF tile kernel:
// persistent warps take query cells A from a work counter (2D grids: only the layer
// holding the points), the half stencil's candidates stream through the lanes while the
// warp loops over A's queries, and every unordered pair within reach is binned twice:
// q -> c in q's frame and c -> q (the negated bond) in c's frame.  The block's warps
// share one shared histogram of 32-bit counts.

constexpr int kPmftTileWarps = 8;
constexpr int kPmftTileQ = 32;
constexpr int kPmftTileMaxBins = 16384;

struct PmftTileArgs {
    TileArgs t;
    PmftBins B;
    const float2 *cs32;        // sorted position -> (cos, sin) FP32
    const float *theta;        // original index -> orientation angle
    float reach2;              // FP32 bound: a bond beyond it lands in no bin
    float inv_dx, inv_dy, off_x, off_y;
    float mx, my;              // decision margins, in bins
    int bins;
    int cell_lo, cell_hi;      // query cells walked
    unsigned long long *hist;
    int2 *esc;
    int esc_cap;
    unsigned *ctl;             // [0] escalated, [1] work
};

// A bond the fast test left open: listed for the FP64 pass, or decided here in FP64 when
// the list is full.
__device__ __noinline__ void pmft_tile_slow(const PmftTileArgs *ap, int i, int j) {
    const PmftTileArgs &a = *ap;
    const unsigned slot = atomicAdd(a.ctl, 1u);
    if (slot < (unsigned)a.esc_cap) {
        a.esc[slot] = make_int2(i, j);
    } else {
        const double3 d = exact_disp(a.t.bd, a.t.p_orig + 3 * (int64_t)i, a.t.p_orig + 3 * (int64_t)j);
        const int b = pmft_bin64(a.B, trig64(a.theta, i), d);
        if (b >= 0) atomicAdd(a.hist + b, 1ull);
    }
}

// Bin of a bond at (tx, ty) in bin units with the kernel's margins.
__device__ __forceinline__ int pmft_fast_bin(const PmftTileArgs &a, float tx, float ty) {
    return pmft_decide(tx, ty, a.mx, a.my, a.B.bx, a.B.by);
}

// Rotates and bins one queued pair (both directions).  The pair tests of the rounds
// leave most lanes out of reach, so pairs within reach are first packed into a per-warp
// queue and binned 32 at a time with every lane busy.
__device__ __forceinline__ void pmft_bin_pair(const PmftTileArgs &a, const float4 *qs, const float2 *qcs, float4 e,
                                              int2 ix, uint32_t *h) {
    const float dx = e.x, dy = e.y;
    const float2 cq = qcs[ix.x];
    // q -> c in q's frame
    const float xq = fmaf(cq.x, dx, cq.y * dy), yq = fmaf(cq.x, dy, -(cq.y * dx));
    const int b1 = pmft_fast_bin(a, fmaf(xq, a.inv_dx, a.off_x), fmaf(yq, a.inv_dy, a.off_y));
    if (b1 >= 0)
        atomicAdd(h + b1, 1u);
    else if (b1 == -2)
        pmft_tile_slow(&a, __float_as_int(qs[ix.x].w), ix.y);
    // c -> q: the bond -d in c's frame
    const float xc = -fmaf(e.z, dx, e.w * dy), yc = -fmaf(e.z, dy, -(e.w * dx));
    const int b2 = pmft_fast_bin(a, fmaf(xc, a.inv_dx, a.off_x), fmaf(yc, a.inv_dy, a.off_y));
    if (b2 >= 0)
        atomicAdd(h + b2, 1u);
    else if (b2 == -2)
        pmft_tile_slow(&a, ix.y, __float_as_int(qs[ix.x].w));
}

// Per-warp queue of pairs within reach: (dx, dy, cos c, sin c) and (query slot, c's
// index); qn entries pending (warp-uniform), at most 31 between rounds.
struct PmftQueue {
    float4 *d;
    int2 *x;
    int qn;
};

__device__ __forceinline__ void pmft_queue_drain(const PmftTileArgs &a, const float4 *qs, const float2 *qcs,
                                                 PmftQueue &Q, uint32_t *h) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    if (lane < Q.qn) pmft_bin_pair(a, qs, qcs, Q.d[lane], Q.x[lane], h);
    __syncwarp();
    Q.qn = 0;
}

// One staged candidate (x, y, index j, its (cos, sin)) against the queries [0, nq) of
// the pass.  CENTER: the candidate may be one of A's own points, valid only against
// queries before it (tl < lim).  Pairs within reach join the queue.
template <bool CENTER>
__device__ __forceinline__ void pmft_tile_rounds(const PmftTileArgs &a, const float4 *qs, const float2 *qcs, int nq,
                                                 float cx, float cy, int cj, float2 ccs, int lim, PmftQueue &Q,
                                                 uint32_t *h) {
    const float r2hi = a.reach2;
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
#pragma unroll 2
    for (int tl = 0; tl < nq; ++tl) {
        const float4 q = qs[tl];
        const float dx = cx - q.x, dy = cy - q.y;
        const float r2 = fmaf(dx, dx, dy * dy);
        bool in = r2 < r2hi;
        if (CENTER) in = in && tl < lim;
        const unsigned m = __ballot_sync(0xffffffffu, in);
        if (in) {
            const int slot = Q.qn + __popc(m & lt);  // <= 31 + 31
            Q.d[slot] = make_float4(dx, dy, ccs.x, ccs.y);
            Q.x[slot] = make_int2(tl, cj);
        }
        Q.qn += __popc(m);
        if (Q.qn >= 32) {
            __syncwarp();
            pmft_bin_pair(a, qs, qcs, Q.d[lane], Q.x[lane], h);
            const float4 rd = Q.d[32 + lane];
            const int2 rx = Q.x[32 + lane];
            __syncwarp();
            if (lane < Q.qn - 32) {
                Q.d[lane] = rd;
                Q.x[lane] = rx;
            }
            __syncwarp();
            Q.qn -= 32;
        }
    }
}

// Adds the shared counts to the global histogram and clears them.  atomicExch takes each
// count whole while other warps keep adding, so no block barrier is needed.
__device__ __forceinline__ void pmft_tile_flush(uint32_t *h, int bins, unsigned long long *hist) {
    const int lane = threadIdx.x & 31;
    for (int b = lane; b < bins; b += 32) {
        const uint32_t v = atomicExch(h + b, 0u);
        if (v) atomicAdd(hist + b, (unsigned long long)v);
    }
}

template <int NS>
__global__ void __launch_bounds__(kPmftTileWarps * 32, 3) k_pmft_tile(const __grid_constant__ PmftTileArgs a) {
    __shared__ TileStencilT<NS> sts[kPmftTileWarps];
    __shared__ float4 sq[kPmftTileWarps][kPmftTileQ];
    __shared__ float2 sqcs[kPmftTileWarps][kPmftTileQ];
    __shared__ float4 sbuf[kPmftTileWarps][64];  // kept candidates: x, y, sorted position, index
    __shared__ float4 sqd[kPmftTileWarps][64];   // queued pairs
    __shared__ int2 sqx[kPmftTileWarps][64];
    extern __shared__ uint32_t shist[];          // bins, shared by the block's warps
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int b = threadIdx.x; b < a.bins; b += blockDim.x) shist[b] = 0;
    __syncthreads();
    TileStencilT<NS> &ts = sts[warp];
    float4 *qs = sq[warp];
    float2 *qcs = sqcs[warp];
    float4 *buf = sbuf[warp];
    PmftQueue Q;
    Q.d = sqd[warp];
    Q.x = sqx[warp];
    Q.qn = 0;
    const unsigned lt = lanemask_lt();
    // a candidate farther than this from the queries' bounding box reaches none of them
    const float reach2 = a.reach2 * (1.0f + 1e-5f);
    // this warp's additions since its last flush bound every shared count's share from
    // it; flushing at 2^28 keeps the sum over the block's warps below 2^32.  A chunk of
    // 32 candidates against nq <= 32 queries adds at most 64 nq; after a flush the at
    // most 31 queued pairs (62 additions) are still to come.
    uint32_t adds = 0;
    const uint32_t kFlushAt = 1u << 28;
    auto charge = [&](int nq) {
        if (adds > kFlushAt - 64u * kPmftTileQ) {
            pmft_tile_flush(shist, a.bins, a.hist);
            adds = 64u;
        }
        adds += 64u * (uint32_t)nq;
    };
    for (;;) {
        unsigned w = 0;
        if (lane == 0) w = atomicAdd(a.ctl + 1, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        const int64_t A = (int64_t)a.cell_lo + w;
        if (A >= a.cell_hi) break;
        const int begA = (int)__ldg(a.t.cell_start + A);
        const int nA = (int)__ldg(a.t.cell_start + A + 1) - begA;
        if (nA == 0) continue;
        int cx, cy, cz;
        cell_coords((uint32_t)A, a.t.nc, cx, cy, cz);
        __syncwarp();
        const int n = tile_stencil(a.t, cx, cy, cz, true, ts);
        const int total = ts.pre[n];
        for (int qb = 0; qb < nA; qb += kPmftTileQ) {
            const int nq = min(kPmftTileQ, nA - qb);
            __syncwarp();
            if (lane < nq) {
                qs[lane] = __ldg(a.t.pts + begA + qb + lane);
                qcs[lane] = __ldg(a.cs32 + begA + qb + lane);
            }
            __syncwarp();
            float3 blo, bhi;
            {
                const float4 q = qs[lane < nq ? lane : 0];
                warp_box(q.x, q.y, q.z, lane < nq, blo, bhi);
            }
            // A's own points first (they pair only with earlier queries)
            for (int base = 0; base < nA; base += 32) {
                const int k = base + lane;
                const TileCand c = tile_load(a.t, ts, n, nA, k);
                const float2 ccs = k < nA ? __ldg(a.cs32 + c.p) : make_float2(0.f, 0.f);
                charge(nq);
                pmft_tile_rounds<true>(a, qs, qcs, nq, c.x, c.y, c.j, ccs, k < nA ? k - qb : 0, Q, shist);
            }
            // the other cells: candidates out of reach of the whole pass are dropped, the
            // rest are packed into full chunks (ballot + popc) before the query rounds
            int cnt = 0;
            for (int base = nA; base < total; base += 32) {
                const int k = base + lane;
                const TileCand c = tile_load(a.t, ts, n, total, k);
                const bool keep = k < total && box_dist2(blo, bhi, c.x, c.y, c.z) <= reach2;
                const unsigned m = __ballot_sync(0xffffffffu, keep);
                if (keep) buf[cnt + __popc(m & lt)] = make_float4(c.x, c.y, __int_as_float(c.p), __int_as_float(c.j));
                cnt += __popc(m);
                if (cnt >= 32) {
                    __syncwarp();
                    const float4 e = buf[lane];
                    const float2 ecs = __ldg(a.cs32 + __float_as_int(e.z));
                    charge(nq);
                    pmft_tile_rounds<false>(a, qs, qcs, nq, e.x, e.y, __float_as_int(e.w), ecs, 0, Q, shist);
                    const float4 rest = buf[32 + lane];
                    __syncwarp();
                    if (lane < cnt - 32) buf[lane] = rest;
                    __syncwarp();
                    cnt -= 32;
                }
            }
            if (cnt > 0) {
                __syncwarp();
                const bool v = lane < cnt;
                const float4 e = v ? buf[lane] : make_float4(kFar, kFar, 0.f, __int_as_float(-1));
                const float2 ecs = v ? __ldg(a.cs32 + __float_as_int(e.z)) : make_float2(0.f, 0.f);
                charge(nq);
                pmft_tile_rounds<false>(a, qs, qcs, nq, e.x, e.y, __float_as_int(e.w), ecs, 0, Q, shist);
            }
            // the queue refers to this pass's staged queries: empty it before they change
            pmft_queue_drain(a, qs, qcs, Q, shist);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < a.bins; b += blockDim.x) {
        const uint32_t v = shist[b];
        if (v) atomicAdd(a.hist + b, (unsigned long long)v);
    }
}

// The bonds the fused kernel left open, decided by the FP64 sequence.
__global__ void k_pmft_escalated(const __grid_constant__ PmftTileArgs a) {
    const int m = min((int)min(*a.ctl, (unsigned)a.esc_cap), a.esc_cap);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x) {
        const int2 ij = a.esc[e];
        const double3 d = exact_disp(a.t.bd, a.t.p_orig + 3 * (int64_t)ij.x, a.t.p_orig + 3 * (int64_t)ij.y);
        const int b = pmft_bin64(a.B, trig64(a.theta, ij.x), d);
        if (b >= 0) atomicAdd(a.hist + b, 1ull);
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
    dfree(P->trig32, P->stream);
    dfree(P->esc, P->stream);
    dfree(P->ctl, P->stream);
    delete P;
}

// Queries and bonds farther than this reach no bin (the corner bond at exactly
// sqrt(x_max^2 + y_max^2) included, whatever the rounding of its rotation).
static double pmft_query_radius(const fgb_pmft *P) {
    return std::sqrt(P->x_max * P->x_max + P->y_max * P->y_max) * (1.0 + 1e-6);
}

static int pmft_launch_tile(fgb_pmft *P, fgb_nq *nq, const StencilPlan &plan, double R, const PmftBins &B, int nhalf,
                            const float *theta, cudaStream_t s) {
    PmftTileArgs a;
    memset(&a, 0, sizeof(a));
    a.t = tile_args(nq, plan, R, 1);
    a.B = B;
    a.cs32 = P->trig32;
    a.theta = theta;
    const double delta = r2_error_bound(plan, R);
    float lo, hi;
    band_around(R * R, delta, &lo, &hi);
    a.reach2 = std::nextafter(hi * (1.0f + 1e-6f), INFINITY);
    a.inv_dx = (float)(1.0 / B.dx);
    a.inv_dy = (float)(1.0 / B.dy);
    a.off_x = 0.5f * (float)B.bx;  // x_max / dx, exact
    a.off_y = 0.5f * (float)B.by;
    // Error of x' = cos d_x + sin d_y in FP32 against the FP64 definition, for |d| <= R:
    // sincosf (2 ulp, taken as 4u each), the displacement (eps_d per component, times
    // |cos| + |sin| <= sqrt 2), the product and the fused add (u |d| each): at most
    // 8 u R + 1.5 eps_d, doubled, plus the FP64 sequence's own rounding.  In bin units
    // the index t = x' / dx + bins / 2 adds the rounding of 1/dx and of the fused add.
    const double u = std::ldexp(1.0, -24);
    const double E = 2.0 * (8.0 * u * R + 1.5 * plan.eps_d) + 1e-12 * (R + plan.Lsum);
    a.mx = (float)(2.0 * (E / B.dx + u * B.bx * (R / B.x_max + 1.0)) + 1e-7);
    a.my = (float)(2.0 * (E / B.dy + u * B.by * (R / B.y_max + 1.0)) + 1e-7);
    a.bins = B.bx * B.by;
    const int64_t layer = (int64_t)nq->grid.nc[0] * nq->grid.nc[1];
    a.cell_lo = nq->box.is2d ? (int)layer : 0;  // 2D: the points sit in the middle layer
    a.cell_hi = nq->box.is2d ? (int)(2 * layer) : (int)nq->grid.ncell;
    a.hist = P->hist;
    a.esc = P->esc;
    a.esc_cap = P->esc_cap;
    a.ctl = P->ctl;
    FGB_CUDA(cudaMemsetAsync(P->ctl, 0, 2 * sizeof(unsigned), s));
    const size_t smem = (size_t)a.bins * sizeof(uint32_t);
    auto go = [&](auto kern) -> int {
        // static + dynamic shared memory above 48 KB needs the opt-in
        FGB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        FGB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPmftTileWarps * 32, smem));
        const int64_t want = ((int64_t)a.cell_hi - a.cell_lo + kPmftTileWarps - 1) / kPmftTileWarps;
        const unsigned grid =
            (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * std::max(per_sm, 1)));
        {
            FGB_KSCOPE("k_pmft_tile", s);
            kern<<<grid, kPmftTileWarps * 32, smem, s>>>(a);
        }
        FGB_LAUNCH_CHECK();
        {
            FGB_KSCOPE("k_pmft_escalated", s);
            k_pmft_escalated<<<num_sms() * 2, 256, 0, s>>>(a);
        }
        FGB_LAUNCH_CHECK();
        return FGB_OK;
    };
    if (nhalf <= 32) return go(k_pmft_tile<32>);
    if (nhalf <= 64) return go(k_pmft_tile<64>);
    return go(k_pmft_tile<kTileMaxStencil>);
}

static int pmft_ensure(fgb_pmft *P, int64_t n, bool sorted, cudaStream_t s) {
    if (P->trig32_cap < n) {
        dfree(P->trig32, P->stream);
        P->trig32 = nullptr;
        P->trig32_cap = 0;
        FGB_TRY(dalloc_n(&P->trig32, n, s));
        P->trig32_cap = n;
    }
    if (sorted) {
        const int64_t want = std::min<int64_t>(std::max<int64_t>(n / 8, 1 << 16), 1 << 26);
        if (P->esc_cap < want) {
            dfree(P->esc, P->stream);
            P->esc = nullptr;
            P->esc_cap = 0;
            FGB_TRY(dalloc_n(&P->esc, want, s));
            P->esc_cap = (int)want;
        }
        if (!P->ctl) FGB_TRY(dalloc_n(&P->ctl, 2, s));
    }
    return FGB_OK;
}

extern "C" int fgb_pmftxy_compute(fgb_pmft *P, fgb_nq *nq, const float *query_points, const float *query_orientations,
                                  int64_t n_query, const fgb_nlist *nlist, int32_t reset, void *stream) {
    clear_error();
    if (!P || !nq) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    FGB_TRY(nlist_ready(nlist));
    if (!nq->box.is2d) return fail(FGB_ERR_INVALID_ARG, "PMFT(x, y) needs a 2D box (Lz = 0)");
    if (n_query < 0 || (!query_points && n_query != nq->n))
        return fail(FGB_ERR_INVALID_ARG, "n_query must be the point count when query_points is NULL");
    if (n_query > 0 && !query_orientations) return fail(FGB_ERR_INVALID_ARG, "query_orientations is NULL");
    if (nlist && (nlist->n_query != n_query || nlist->n_points != nq->n))
        return fail(FGB_ERR_INVALID_ARG, "the neighbor list does not match the query and point counts");
    const double R = pmft_query_radius(P);
    if (!(R < 0.5 * nq->box.wmin * (1.0 - 1e-5)))
        return fail(FGB_ERR_BOX_TOO_SMALL, "sqrt(x_max^2 + y_max^2) = %g must be below half the smallest box width (%g)",
                    R, 0.5 * nq->box.wmin);
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
    P->last_esc = -1;
    PmftBins B;
    B.x_max = P->x_max;
    B.y_max = P->y_max;
    B.dx = 2.0 * P->x_max / P->bx;
    B.dy = 2.0 * P->y_max / P->by;
    B.bx = P->bx;
    B.by = P->by;
    if (n_query > 0 && nq->n > 0) {
        // fused route: self bonds on the cell list's shift route, histogram in shared memory
        bool fused = false;
        StencilPlan plan;
        memset(&plan, 0, sizeof(plan));
        if (!nlist && !query_points && nq->kind == 0 && nb <= (size_t)kPmftTileMaxBins && tile_worth(nq) &&
            !force_thread_kernels()) {
            FGB_TRY(plan_stencil(nq, R, 0, s, &plan));
            const int nfull = (2 * plan.s[0] + 1) * (2 * plan.s[1] + 1) * (2 * plan.s[2] + 1);
            const int nhalf = (nfull + 1) / 2;
            fused = plan.mode == 0 && nhalf <= kTileMaxStencil;
            int st = fused ? pmft_ensure(P, nq->n, true, s) : FGB_OK;
            if (st == FGB_OK && fused) {
                {
                    FGB_KSCOPE("k_pmft_trig_sorted", s);
                    k_pmft_trig_sorted<<<(unsigned)((nq->n + 255) / 256), 256, 0, s>>>(nq->sorted, query_orientations,
                                                                                       nq->n, P->trig32);
                }
                st = cudaGetLastError() == cudaSuccess ? FGB_OK : fail(FGB_ERR_CUDA, "pmft trig launch failed");
                if (st == FGB_OK) st = pmft_launch_tile(P, nq, plan, R, B, nhalf, query_orientations, s);
            }
            dfree(plan.table, s);
            if (st != FGB_OK) return st;
        }
        if (!fused) {
            FGB_TRY(pmft_ensure(P, n_query, false, s));
            {
                FGB_KSCOPE("k_pmft_trig", s);
                k_pmft_trig<<<(unsigned)((n_query + 255) / 256), 256, 0, s>>>(query_orientations, n_query, P->trig32);
            }
            FGB_LAUNCH_CHECK();
            fgb_nlist *own = nullptr;
            if (!nlist) {
                fgb_query_args qa;
                qa.r_max = R;
                qa.num_neighbors = 0;
                qa.exclude_ii = query_points ? 0 : 1;
                FGB_TRY(fgb_nq_query(nq, query_points, n_query, &qa, stream, &own));
                nlist = own;
            }
            int st = FGB_OK;
            if (nlist->n_pairs > 0) {
                PmftListArgs a;
                memset(&a, 0, sizeof(a));
                a.bd = nq->box.d;
                a.p = nq->points;
                a.qp = query_points ? query_points : nq->points;
                a.theta = query_orientations;
                a.cs = P->trig32;
                a.qi = nlist->qi;
                a.pj = nlist->pj;
                a.m = nlist->n_pairs;
                a.B = B;
                a.inv_dx = (float)(1.0 / B.dx);
                a.inv_dy = (float)(1.0 / B.dy);
                a.off_x = 0.5f * (float)B.bx;
                a.off_y = 0.5f * (float)B.by;
                // Error of x' in FP32 against the FP64 definition, dm = max(|d_x|, |d_y|):
                // sincosf (4u each) 8u dm, the displacement (the FP64 one rounded to FP32, or
                // the FP32 difference of the coordinates, within u |d| either way) sqrt(2) u dm,
                // the product and the fused add (1 + sqrt 2) u dm: at most 12.5 u dm.  The
                // index t = x' / dx + bins / 2 adds u bins (1.42 dm / x_max + 1).  Doubled,
                // plus the FP64 sequence's own rounding.
                const double u = std::ldexp(1.0, -24);
                a.kx = (float)(25.0 * u / B.dx + 2.84 * u * B.bx / B.x_max + 1e-12 / B.dx);
                a.ky = (float)(25.0 * u / B.dy + 2.84 * u * B.by / B.y_max + 1e-12 / B.dy);
                a.cx = (float)(2.0 * u * B.bx + 1e-12 / B.dx + 1e-7);
                a.cy = (float)(2.0 * u * B.by + 1e-12 / B.dy + 1e-7);
                a.wx = (float)(0.499 * nq->box.p[0]);
                a.wy = (float)(0.499 * nq->box.p[1]);
                a.wz = (float)(0.499 * nq->box.p[2]);
                a.hist = P->hist;
                const int bins = B.bx * B.by;
                const bool shared = bins <= kPmftListMaxBins;
                const size_t smem = shared ? (size_t)bins * sizeof(uint32_t) : 0;
                int per_sm = 8;
                if (shared) {
                    if (cudaFuncSetAttribute(k_pmft_list<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                            cudaSuccess ||
                        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pmft_list<true>, 256, smem) != cudaSuccess)
                        st = fail(FGB_ERR_CUDA, "pmft list kernel setup failed");
                }
                // enough blocks to fill the GPU, each over at most 2^30 bonds
                const int64_t m = nlist->n_pairs;
                int64_t grid = std::min<int64_t>((m + 255) / 256, (int64_t)num_sms() * std::max(per_sm, 1));
                grid = std::max<int64_t>(grid, (m + ((int64_t)1 << 30) - 1) >> 30);
                const int64_t per_block = (m + grid - 1) / grid;
                if (st == FGB_OK) {
                    FGB_KSCOPE("k_pmft_list", s);
                    if (shared)
                        k_pmft_list<true><<<(unsigned)grid, 256, smem, s>>>(a, per_block);
                    else
                        k_pmft_list<false><<<(unsigned)grid, 256, 0, s>>>(a, per_block);
                    cudaError_t e = cudaGetLastError();
                    if (e != cudaSuccess) st = fail(FGB_ERR_CUDA, "pmft launch failed: %s", cudaGetErrorString(e));
                }
            }
            if (own) fgb_nlist_destroy(own);
            if (st != FGB_OK) return st;
        } else {
            P->last_esc = -2;  // read from the device on request
        }
    }
    P->norm += (double)n_query * (double)nq->n / (nq->box.p[0] * nq->box.p[1]);
    return FGB_OK;
}

extern "C" int fgb_pmftxy_escalations(fgb_pmft *P, int64_t *n, void *stream) {
    clear_error();
    if (!P || !n) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    *n = 0;
    if (P->last_esc == -2 && P->ctl) {
        unsigned v = 0;
        cudaStream_t s = as_stream(stream);
        FGB_CUDA(cudaMemcpyAsync(&v, P->ctl, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        FGB_CUDA(cudaStreamSynchronize(s));
        *n = v;
    }
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
