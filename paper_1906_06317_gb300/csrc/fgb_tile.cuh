// Cell-tile building blocks shared by the ball-query, kNN and RDF tile kernels: the
// per-warp stencil list of a query cell, the candidate stream over it and the lane
// layouts that put queries or candidates on lanes.
#pragma once

#include "fgb_ball.cuh"

namespace fgb {

constexpr int kTileMaxStencil = 128;
constexpr int kTileWarps = 4;     // warps per block
constexpr int kTileQueries = 8;   // queries per pass of the write kernel

struct TileArgs {
    int nc[3];
    int s[3];
    int ts[3];
    const float4 *off;        // offset table of half-width ts
    const float4 *pts;        // sorted records
    const uint32_t *cell_start;
    int64_t ncell;            // query cells walked: [cell_lo, ncell)
    int64_t cell_lo;          // (2D grids: the layer that holds the points)
    const float *p_orig;
    BoxF bf;
    BoxD bd;
    Band band;
    double T;
    int exclude;
    int half;                 // half stencil (self pairs visited once)
    unsigned long long *esc;
    int *err;
};

template <int NS>
struct TileStencilT {
    int beg[NS];
    int pre[NS + 1];
    float4 off[NS];
};
using TileStencil = TileStencilT<kTileMaxStencil>;

// Builds the (half) stencil list of cell A in `ts` (one warp), returns the number of
// stencil cells; pre[n] holds the total number of candidates.  span > 1: the union of
// the (half) stencils of the span cells A, A+1, ... along x (offsets in x from -s to
// s + span - 1; the offset table must reach that far).  For a half stencil, off[].w of
// each listed cell holds (as int bits) the block cells b whose half stencil holds it,
// blo | bhi << 8, plus 1 << 16 when it is block cell bhi itself (then only points after
// the query in sorted order pair with it).
template <class TS>
__device__ __forceinline__ int tile_stencil(const TileArgs &a, int cx, int cy, int cz, bool half, TS &ts,
                                            int span = 1) {
    const int lane = threadIdx.x & 31;
    const int wx = 2 * a.s[0] + span, wy = 2 * a.s[1] + 1, wz = 2 * a.s[2] + 1;
    const int nfull = wx * wy * wz;
    const int owx = 2 * a.ts[0] + 1, owy = 2 * a.ts[1] + 1;
    // o -> (o mod wx, o / wx mod wy, o / (wx wy)) by float reciprocals: o < 2^8 and
    // w < 2^8, so (o + 1/2) / w lies at least 1/(2w) > 2^-9 from an integer while the
    // rounded product is within 2^-14 of it, and truncates to the exact quotient
    const float iwx = 1.0f / (float)wx, iwxy = 1.0f / (float)(wx * wy);
    int n = 0;
    // offsets in (oz, oy, ox) order; the half stencil keeps (0,0,0) and what follows it
    const int first = half ? (a.s[2] * wy + a.s[1]) * wx + a.s[0] : 0;
    for (int b = first; b < nfull; b += 32) {
        const int o = b + lane;
        int cnt = 0, beg = 0;
        float4 of = make_float4(0.f, 0.f, 0.f, 0.f);
        if (o < nfull) {
            const int qz = __float2int_rz(((float)o + 0.5f) * iwxy);
            const int rxy = o - qz * (wx * wy);
            const int qy = __float2int_rz(((float)rxy + 0.5f) * iwx);
            const int ox = rxy - qy * wx - a.s[0], oy = qy - a.s[1], oz = qz - a.s[2];
            const int xx = wrap_cell(cx + ox, a.nc[0]), yy = wrap_cell(cy + oy, a.nc[1]),
                      zz = wrap_cell(cz + oz, a.nc[2]);
            const int cell = (zz * a.nc[1] + yy) * a.nc[0] + xx;
            beg = (int)__ldg(a.cell_start + cell);
            cnt = (int)__ldg(a.cell_start + cell + 1) - beg;
            of = __ldg(a.off + ((oz + a.ts[2]) * owy + (oy + a.ts[1])) * owx + (ox + a.ts[0]));
            if (half) {
                const bool row = oz == 0 && oy == 0;  // the query cells' own row: ox >= 0
                const int blo = max(0, ox - a.s[0]), bhi = min(span - 1, row ? ox : ox + a.s[0]);
                of.w = __int_as_float(blo | (bhi << 8) | ((row && ox < span) ? (1 << 16) : 0));
            }
        }
        // inclusive scan of counts across the warp
        int inc = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += u;
        }
        const int base = n ? ts.pre[n] : 0;
        if (o < nfull) {
            const int idx = n + lane;
            ts.beg[idx] = beg;
            ts.pre[idx] = base + inc - cnt;
            ts.off[idx] = of;
        }
        const int tot = __shfl_sync(0xffffffffu, inc, 31);
        const int m = min(32, nfull - b);
        __syncwarp();
        if (lane == 0) ts.pre[n + m] = base + tot;
        __syncwarp();
        n += m;
    }
    return n;
}

// Stencil cell holding candidate k (largest o with pre[o] <= k; empty cells are skipped
// because the next non-empty cell shares their prefix).
template <class TS>
__device__ __forceinline__ int tile_find(const TS &ts, int n, int k) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (ts.pre[mid] <= k)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Candidate k of the current chunk: shifted position, index, sorted position, stencil slot.
struct TileCand {
    float x, y, z;
    int j;
    int p;
    int o;
};

template <class TS>
__device__ __forceinline__ TileCand tile_load(const TileArgs &a, const TS &ts, int n, int total, int k) {
    TileCand c;
    if (k < total) {
        const int o = tile_find(ts, n, k);
        const int p = ts.beg[o] + (k - ts.pre[o]);
        const float4 r = __ldg(a.pts + p);
        const float4 of = ts.off[o];
        c.x = r.x + of.x;
        c.y = r.y + of.y;
        c.z = r.z + of.z;
        c.j = __float_as_int(r.w);
        c.p = p;
        c.o = o;
    } else {
        c.x = c.y = c.z = 1e30f;
        c.j = -1;
        c.p = 0x7fffffff;
        c.o = -1;
    }
    return c;
}

// Owner table of a stencil list: own[k] = the stencil cell that holds candidate k, one
// byte each (at most kTileMaxStencil cells), for k < pre[n].  Built once per query cell,
// it turns each candidate's lookup into a table read instead of a binary search over the
// prefix sums.
template <class TS>
__device__ __forceinline__ void tile_owners(const TS &ts, int n, uint8_t *own) {
    const int lane = threadIdx.x & 31;
    for (int o = lane; o < n; o += 32) {
        const int b = ts.pre[o], e = ts.pre[o + 1];
        for (int k = b; k < e; ++k) own[k] = (uint8_t)o;
    }
    __syncwarp();
}

// tile_load with the owner table (own == nullptr: the binary search).
template <class TS>
__device__ __forceinline__ TileCand tile_load_own(const TileArgs &a, const TS &ts, const uint8_t *own, int n, int total,
                                                  int k) {
    if (!own) return tile_load(a, ts, n, total, k);
    TileCand c;
    if (k < total) {
        const int o = own[k];
        const int p = ts.beg[o] + (k - ts.pre[o]);
        const float4 r = __ldg(a.pts + p);
        const float4 of = ts.off[o];
        c.x = r.x + of.x;
        c.y = r.y + of.y;
        c.z = r.z + of.z;
        c.j = __float_as_int(r.w);
        c.p = p;
        c.o = o;
    } else {
        c.x = c.y = c.z = 1e30f;
        c.j = -1;
        c.p = 0x7fffffff;
        c.o = -1;
    }
    return c;
}

// Lanes hold queries, candidates are broadcast: a query block of nq <= 32 queries of the
// cell is spread over qpl = next power of two >= nq lanes, and the warp's 32/qpl lane
// groups take different candidates of the staged chunk in each round.
struct QLayout {
    int qpl, G, myq, g;
};

__device__ __forceinline__ QLayout qlayout(int nq) {
    QLayout L;
    L.qpl = 1;
    while (L.qpl < nq) L.qpl <<= 1;
    L.G = 32 / L.qpl;
    const int lane = threadIdx.x & 31;
    L.myq = lane & (L.qpl - 1);
    L.g = lane / L.qpl;
    return L;
}

constexpr float kFar = 1e30f;

// Stages candidates [base, base + 32) of the stencil list, shifted into the query cell's
// frame, as float4 (x, y, z, index bits); missing ones are placed far away.
template <class TS>
__device__ __forceinline__ void tile_stage(const TileArgs &a, const TS &ts, int n, int total, int base, float4 *stage) {
    const int lane = threadIdx.x & 31;
    const TileCand c = tile_load(a, ts, n, total, base + lane);
    stage[lane] = make_float4(c.x, c.y, c.z, __int_as_float(c.j));
    __syncwarp();
}

// Dispatches a body templated on the number of lane groups G = 32 / qpl (uniform per warp).
#define FGB_TILE_DISPATCH_G(G_, CALL) \
    switch (G_) {                     \
        case 32: CALL(32); break;     \
        case 16: CALL(16); break;     \
        case 8: CALL(8); break;       \
        case 4: CALL(4); break;       \
        case 2: CALL(2); break;       \
        default: CALL(1); break;      \
    }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Bounding box of one point per lane (lanes with valid == false take no part), reduced
// over the warp: every lane gets the box.
__device__ __forceinline__ void warp_box(float x, float y, float z, bool valid, float3 &lo, float3 &hi) {
    lo = valid ? make_float3(x, y, z) : make_float3(INFINITY, INFINITY, INFINITY);
    hi = valid ? make_float3(x, y, z) : make_float3(-INFINITY, -INFINITY, -INFINITY);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo.x = fminf(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, o));
        lo.y = fminf(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, o));
        lo.z = fminf(lo.z, __shfl_xor_sync(0xffffffffu, lo.z, o));
        hi.x = fmaxf(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, o));
        hi.y = fmaxf(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, o));
        hi.z = fmaxf(hi.z, __shfl_xor_sync(0xffffffffu, hi.z, o));
    }
}

// Squared distance from a point to a box (0 inside), in FP32.  Used to drop candidates
// that no query of a box can reach: for pairs that matter it is within a few ulps of the
// exact distance, so a slack factor of 1 + 1e-5 on the reach keeps every one of them.
__device__ __forceinline__ float box_dist2(float3 lo, float3 hi, float x, float y, float z) {
    const float dx = fmaxf(fmaxf(lo.x - x, x - hi.x), 0.f);
    const float dy = fmaxf(fmaxf(lo.y - y, y - hi.y), 0.f);
    const float dz = fmaxf(fmaxf(lo.z - z, z - hi.z), 0.f);
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// Kernel arguments for a self query of radius R on plan p (host).
TileArgs tile_args(const fgb_nq *nq, const StencilPlan &p, double R, int exclude);

}  // namespace fgb
