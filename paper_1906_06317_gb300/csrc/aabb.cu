// Bounding-volume-hierarchy neighbor query: the paper's AABBQuery (Section "General
// Utilities": the NeighborQuery family has a cell-list and a tree subclass, the tree
// adapted from HOOMD-blue; Fig. 3 benchmarks it), built GPU-first as a linear BVH.
//
// Build: every point is wrapped into the box, its fractional coordinates give a 30-bit
// Morton code, and the existing radix sort orders (code, index).  The internal nodes of
// the binary radix tree over the sorted codes are found independently per node (Karras,
// "Maximizing parallelism in the construction of BVHs, octrees, and k-d trees", HPG
// 2012: direction from the neighbouring common-prefix lengths, range end by exponential
// and binary search, split by binary search; equal codes are told apart by their sorted
// position).  Boxes are then refit bottom-up: one thread per leaf climbs while it is the
// second child to arrive at a node (atomic arrival counters; the first arrival stops, so
// nothing waits on another thread).
//
// Query: one thread per query (Morton order for self queries), one stack traversal per
// periodic image of the query that can reach the box, the same exact pair decision as
// the cell list (FP32 inside a proven band, the defining FP64 sequence inside it).  The
// count, scan and write passes give rows in traversal order; a warp per row then sorts
// it by point index, so the list equals the cell list's bit for bit.
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "fgb_tile.cuh"

namespace fgb {

// Internal node: child >= 0 names an internal node, child < 0 the leaf ~child (a
// position in Morton order).  lo/hi bound the wrapped coordinates of its points.
struct BvhNode {
    float lo[3];
    int left;
    float hi[3];
    int right;
};

constexpr int kBvhStack = 64;  // tree depth is at most 30 code bits + 31 position bits

// The point ranges stored after the n - 1 nodes of a tree over n >= 2 points.
__host__ __device__ inline int2 *bvh_ranges(BvhNode *nodes, int64_t n) {
    return reinterpret_cast<int2 *>(nodes + (n - 1));
}

// Bits of a 10-bit integer spread to every third position.
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Fractional coordinates s = M^-1 x + 1/2 (FP32).
__device__ __forceinline__ float3 frac_of(const BoxF &b, float x, float y, float z) {
    return make_float3(fmaf(b.inv00, x, fmaf(b.inv01, y, b.inv02 * z)) + 0.5f, fmaf(b.inv11, y, b.inv12 * z) + 0.5f,
                       b.inv22 * z + 0.5f);
}

// Wraps a point into the box: x - M floor(s).  Points already inside are unchanged
// (floor(s) = 0 makes every subtraction exact); others move by whole box vectors with
// one FP32 rounding per operation.  Also returns the wrapped fractional coordinates and
// flags: 1 the point moved, 2 a coordinate is beyond the supported range (|s - 1/2| > 2,
// where the error bound of this route no longer holds).
__device__ __forceinline__ float3 wrap_point(const BoxF &b, float x, float y, float z, float3 &f, int &flags) {
    const float3 s = frac_of(b, x, y, z);
    const float n0 = floorf(s.x), n1 = floorf(s.y), n2 = floorf(s.z);
    flags = (n0 != 0.f || n1 != 0.f || n2 != 0.f) ? 1 : 0;
    if (!(fabsf(s.x - 0.5f) <= 2.f && fabsf(s.y - 0.5f) <= 2.f && fabsf(s.z - 0.5f) <= 2.f)) flags |= 2;
    const float xw = x - n0 * b.L[0] - n1 * b.a2x - n2 * b.a3x;
    const float yw = y - n1 * b.L[1] - n2 * b.a3y;
    const float zw = z - n2 * b.L[2];
    f = make_float3(s.x - n0, s.y - n1, s.z - n2);
    return make_float3(xw, yw, zw);
}

__device__ __forceinline__ uint32_t morton30(float3 f) {
    const uint32_t qx = (uint32_t)min(1023, max(0, (int)(f.x * 1024.f)));
    const uint32_t qy = (uint32_t)min(1023, max(0, (int)(f.y * 1024.f)));
    const uint32_t qz = (uint32_t)min(1023, max(0, (int)(f.z * 1024.f)));
    return (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
}

__global__ void k_bvh_keys(BoxF b, const float *__restrict__ pts, int64_t n, uint32_t *__restrict__ keys,
                           uint32_t *__restrict__ vals, float4 *__restrict__ rec, int *flags_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float3 f;
    int fl;
    const float3 w = wrap_point(b, pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], f, fl);
    if (fl) atomicOr(flags_out, fl);
    keys[i] = morton30(f);
    vals[i] = (uint32_t)i;
    rec[i] = make_float4(w.x, w.y, w.z, __int_as_float((int)i));
}

// Common-prefix length of sorted keys i and j (positions break ties); -1 outside [0, n).
__device__ __forceinline__ int bvh_delta(const uint32_t *__restrict__ k, int n, int i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    const uint32_t a = __ldg(k + i), c = __ldg(k + j);
    if (a != c) return __clz(a ^ c);
    return 32 + __clz((uint32_t)i ^ (uint32_t)j);
}

// Internal node i of the radix tree over n >= 2 sorted keys; range[i] = the sorted
// positions (first, last) of its points.
__global__ void k_bvh_nodes(const uint32_t *__restrict__ keys, int n, BvhNode *__restrict__ nodes,
                            int2 *__restrict__ range, int *__restrict__ parent_int, int *__restrict__ parent_leaf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int d = bvh_delta(keys, n, i, i + 1) > bvh_delta(keys, n, i, i - 1) ? 1 : -1;
    const int dmin = bvh_delta(keys, n, i, i - d);
    int64_t lmax = 2;
    while (bvh_delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (bvh_delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
    const int j = (int)(i + l * d);
    const int dnode = bvh_delta(keys, n, i, j);
    int64_t s = 0;
    for (int64_t div = 2;; div <<= 1) {
        const int64_t t = (l + div - 1) / div;
        if (bvh_delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
        if (t <= 1) break;
    }
    const int g = (int)(i + s * d + min(d, 0));
    const int lo = min(i, j), hi = max(i, j);
    const int left = lo == g ? ~g : g;
    const int right = hi == g + 1 ? ~(g + 1) : g + 1;
    nodes[i].left = left;
    nodes[i].right = right;
    range[i] = make_int2(lo, hi);
    if (left < 0)
        parent_leaf[~left] = i;
    else
        parent_int[left] = i;
    if (right < 0)
        parent_leaf[~right] = i;
    else
        parent_int[right] = i;
}

__device__ __forceinline__ void child_box(const BvhNode *nodes, const float4 *pts, int c, float3 &lo, float3 &hi) {
    if (c < 0) {
        const float4 p = __ldcg(pts + ~c);
        lo = hi = make_float3(p.x, p.y, p.z);
    } else {
        const BvhNode *q = nodes + c;
        lo = make_float3(__ldcg(q->lo), __ldcg(q->lo + 1), __ldcg(q->lo + 2));
        hi = make_float3(__ldcg(q->hi), __ldcg(q->hi + 1), __ldcg(q->hi + 2));
    }
}

// Bottom-up boxes: a thread climbs from its leaf while it is the second arrival at each
// node; the fence orders its box stores before the arrival it signals.
__global__ void k_bvh_refit(const float4 *__restrict__ pts, int n, BvhNode *nodes, const int *__restrict__ parent_int,
                            const int *__restrict__ parent_leaf, int *flags) {
    const int leaf = blockIdx.x * blockDim.x + threadIdx.x;
    if (leaf >= n) return;
    int p = parent_leaf[leaf];
    for (int depth = 0; depth < 2 * kBvhStack; ++depth) {
        __threadfence();
        if (atomicAdd(flags + p, 1) == 0) return;
        float3 l0, h0, l1, h1;
        child_box(nodes, pts, __ldcg(&nodes[p].left), l0, h0);
        child_box(nodes, pts, __ldcg(&nodes[p].right), l1, h1);
        nodes[p].lo[0] = fminf(l0.x, l1.x);
        nodes[p].lo[1] = fminf(l0.y, l1.y);
        nodes[p].lo[2] = fminf(l0.z, l1.z);
        nodes[p].hi[0] = fmaxf(h0.x, h1.x);
        nodes[p].hi[1] = fmaxf(h0.y, h1.y);
        nodes[p].hi[2] = fmaxf(h0.z, h1.z);
        if (p == 0) return;
        p = parent_int[p];
    }
}

// ------------------------------------------------------------------ ball query

struct BvhArgs {
    BoxF bf;
    BoxD bd;
    float w[3];                 // perpendicular widths
    const BvhNode *nodes;       // n - 1 internal nodes (root 0) when n >= 2
    const int2 *range;          // their point ranges (first, last sorted position)
    const float4 *pts;          // wrapped points in Morton order, index bits in w
    int n;
    const float *p_orig;        // (n, 3) caller's points
    const float *q_orig;        // (nq, 3) caller's query points
    int64_t nq;
    int self;                   // queries are the points: thread t takes pts[t]
    int exclude;
    float reach2;               // node boxes farther than this (squared) are skipped
    float reach;                // images whose box distance exceeds this are skipped
    float group_ext;            // group kernels: a group wider than this is halved
    Band band;                  // FP32 band when neither point of a pair was moved by wrapping
    Band band_wide;             // band when one was (the points' flag or the query's own)
    int pts_moved;              // some point was moved by wrapping
    double T;
    unsigned long long *esc;
    int *err;
};

// Whether child c (node box or leaf point) lies within the traversal reach of (qx,qy,qz).
__device__ __forceinline__ bool bvh_near(const BvhArgs &a, int c, float qx, float qy, float qz) {
    float dx, dy, dz;
    if (c < 0) {
        const float4 p = __ldg(a.pts + ~c);
        dx = p.x - qx;
        dy = p.y - qy;
        dz = p.z - qz;
    } else {
        const BvhNode *cn = a.nodes + c;
        dx = fmaxf(fmaxf(__ldg(cn->lo) - qx, qx - __ldg(cn->hi)), 0.f);
        dy = fmaxf(fmaxf(__ldg(cn->lo + 1) - qy, qy - __ldg(cn->hi + 1)), 0.f);
        dz = fmaxf(fmaxf(__ldg(cn->lo + 2) - qz, qz - __ldg(cn->hi + 2)), 0.f);
    }
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= a.reach2;
}

// Visits every neighbor of one query (exactly decided): fn(j, dist).  Returns the number
// of FP64 decisions.
template <class F>
__device__ __forceinline__ int bvh_visit(const BvhArgs &a, int i, float3 qw, float3 qf, bool qmoved, F &&fn) {
    const bool wide = qmoved || a.pts_moved;
    const float lo = wide ? a.band_wide.lo : a.band.lo, hi = wide ? a.band_wide.hi : a.band.hi;
    const int excl = a.exclude ? i : -1;
    int nesc = 0;
    if (a.n == 0) return 0;
    int stack[kBvhStack];
    for (int sz = -1; sz <= 1; ++sz)
        for (int sy = -1; sy <= 1; ++sy)
            for (int sx = -1; sx <= 1; ++sx) {
                // distance from this image of the query to the box is at least the largest
                // of its distances to the three slabs
                const float gx = qf.x + sx, gy = qf.y + sy, gz = qf.z + sz;
                const float ex = fmaxf(fmaxf(-gx, gx - 1.f), 0.f) * a.w[0];
                const float ey = fmaxf(fmaxf(-gy, gy - 1.f), 0.f) * a.w[1];
                const float ez = fmaxf(fmaxf(-gz, gz - 1.f), 0.f) * a.w[2];
                if (fmaxf(ex, fmaxf(ey, ez)) > a.reach) continue;
                const float qx = qw.x + (float)sx * a.bf.L[0] + (float)sy * a.bf.a2x + (float)sz * a.bf.a3x;
                const float qy = qw.y + (float)sy * a.bf.L[1] + (float)sz * a.bf.a3y;
                const float qz = qw.z + (float)sz * a.bf.L[2];
                int sp = 0;
                int node = a.n >= 2 ? 0 : ~0;
                // a tree over n points has 2n - 1 nodes: a longer walk means a broken tree
                for (int64_t visits = 0;; ++visits) {
                    if (visits > 2 * (int64_t)a.n) {
                        atomicExch(a.err, 4);
                        break;
                    }
                    if (node < 0) {
                        const float4 c = __ldg(a.pts + ~node);
                        const float r2 = r2_f32(c.x - qx, c.y - qy, c.z - qz);
                        const int j = __float_as_int(c.w);
                        if (r2 < hi && j != excl) {
                            if (r2 < lo) {
                                fn(j, r2 > 0.f ? r2 * rsqrt_ftz(r2) : 0.f);
                            } else {
                                ++nesc;
                                const double e = exact_r2_idx(a.bd, a.q_orig, i, a.p_orig, j);
                                if (e < a.T) fn(j, (float)sqrt(e));
                            }
                        }
                    } else {
                        const BvhNode *nd = a.nodes + node;
                        const int c0 = __ldg(&nd->left), c1 = __ldg(&nd->right);
                        const bool t0 = bvh_near(a, c0, qx, qy, qz), t1 = bvh_near(a, c1, qx, qy, qz);
                        if (t0 && t1) {
                            if (sp < kBvhStack)
                                stack[sp++] = c1;
                            else
                                atomicExch(a.err, 3);  // deeper than any radix tree over 2^31 keys
                        }
                        if (t0 || t1) {
                            node = t0 ? c0 : c1;
                            continue;
                        }
                    }
                    if (sp == 0) break;
                    node = stack[--sp];
                }
            }
    return nesc;
}

// Query t: its index and wrapped position (self queries read the sorted record), and
// whether wrapping moved it (flags as in wrap_point).
__device__ __forceinline__ int bvh_query_point(const BvhArgs &a, int64_t t, float3 &qw, float3 &qf, int &flags) {
    if (a.self) {
        const float4 r = __ldg(a.pts + t);
        qw = make_float3(r.x, r.y, r.z);
        qf = frac_of(a.bf, r.x, r.y, r.z);
        flags = 0;
        return __float_as_int(r.w);
    }
    qw = wrap_point(a.bf, __ldg(a.q_orig + 3 * t), __ldg(a.q_orig + 3 * t + 1), __ldg(a.q_orig + 3 * t + 2), qf,
                    flags);
    return (int)t;
}

__global__ void __launch_bounds__(128) k_bvh_count(BvhArgs a, uint32_t *__restrict__ counts) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.nq) return;
    float3 qw, qf;
    int fl;
    const int i = bvh_query_point(a, t, qw, qf, fl);
    if (fl & 2) {
        atomicExch(a.err, 5);
        counts[i] = 0;
        return;
    }
    uint32_t cnt = 0;
    const int nesc = bvh_visit(a, i, qw, qf, fl != 0, [&](int, float) { ++cnt; });
    counts[i] = cnt;
    if (nesc) atomicAdd(a.esc, (unsigned long long)nesc);
}

// Rows in traversal order; sort_segments orders them by point index afterwards.
__global__ void __launch_bounds__(128) k_bvh_write(BvhArgs a, const int64_t *__restrict__ seg,
                                                   const uint32_t *__restrict__ counts, int32_t *__restrict__ qi_out,
                                                   int32_t *__restrict__ pj_out, float *__restrict__ d_out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.nq) return;
    float3 qw, qf;
    int fl;
    const int i = bvh_query_point(a, t, qw, qf, fl);
    if (fl & 2) return;
    const int64_t off = seg[i];
    const uint32_t want = counts[i];
    uint32_t k = 0;
    bvh_visit(a, i, qw, qf, fl != 0, [&](int j, float d) {
        if (k < want) {
            qi_out[off + k] = i;
            pj_out[off + k] = j;
            d_out[off + k] = d;
        }
        ++k;
    });
    if (k != want) atomicExch(a.err, 2);
}

// Squared distance between child c's box (a point for a leaf) and the box [blo, bhi]
// of a group's queries: every query is at least this far from every point of the child.
__device__ __forceinline__ float bvh_gap2(const BvhArgs &a, int c, float3 blo, float3 bhi) {
    float3 l, h;
    if (c < 0) {
        const float4 p = __ldg(a.pts + ~c);
        l = h = make_float3(p.x, p.y, p.z);
    } else {
        const BvhNode *cn = a.nodes + c;
        l = make_float3(__ldg(cn->lo), __ldg(cn->lo + 1), __ldg(cn->lo + 2));
        h = make_float3(__ldg(cn->hi), __ldg(cn->hi + 1), __ldg(cn->hi + 2));
    }
    const float dx = fmaxf(fmaxf(l.x - bhi.x, blo.x - h.x), 0.f);
    const float dy = fmaxf(fmaxf(l.y - bhi.y, blo.y - h.y), 0.f);
    const float dz = fmaxf(fmaxf(l.z - bhi.z, blo.z - h.z), 0.f);
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// One chunk of staged candidates (c on the lanes, valid when c.w >= 0) against the
// queries of lanes [l0, l1) in qs (w < 0: no query in this image), four queries per step
// so that their tests overlap.  Lane t keeps query t's count (cnt) and, when writing,
// its row start (off) and length (want); a hit's place in the row is the count so far
// plus the hits of lower lanes.
template <bool WRITE>
__device__ __forceinline__ void bvh_chunk(const BvhArgs &a, const float4 *qs, int l0, int l1, float4 c, float lo,
                                          float hi, unsigned lt, uint32_t &cnt, int64_t off, uint32_t want, int &nesc,
                                          int32_t *__restrict__ qi_out, int32_t *__restrict__ pj_out,
                                          float *__restrict__ d_out) {
    const int lane = threadIdx.x & 31;
    const int j = __float_as_int(c.w);
    for (int t0 = l0; t0 < l1; t0 += 4) {
        bool hit[4];
        float dist[4], r2[4];
        bool band = false;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float4 Q = qs[min(t0 + u, 31)];
            const int qi = __float_as_int(Q.w);
            const bool valid = t0 + u < l1 && j >= 0 && qi >= 0 && j != (a.exclude ? qi : -1);
            r2[u] = r2_f32(c.x - Q.x, c.y - Q.y, c.z - Q.z);
            hit[u] = valid && r2[u] < lo;
            band |= valid && r2[u] >= lo && r2[u] < hi;
            dist[u] = r2[u] > 0.f ? r2[u] * rsqrt_ftz(r2[u]) : 0.f;
        }
        if (__any_sync(0xffffffffu, band)) {  // pairs inside the FP32 band: the FP64 decision
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int qi = __float_as_int(qs[min(t0 + u, 31)].w);
                const bool valid = t0 + u < l1 && j >= 0 && qi >= 0 && j != (a.exclude ? qi : -1);
                if (valid && r2[u] >= lo && r2[u] < hi) {
                    ++nesc;
                    const double e = exact_r2_idx(a.bd, a.q_orig, qi, a.p_orig, j);
                    hit[u] = e < a.T;
                    dist[u] = (float)sqrt(e);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = t0 + u;
            const unsigned m = __ballot_sync(0xffffffffu, hit[u]);
            if (m == 0) continue;
            if (WRITE) {
                const uint32_t base = __shfl_sync(0xffffffffu, cnt, t);
                const int64_t row = __shfl_sync(0xffffffffu, off, t);
                const uint32_t rw = __shfl_sync(0xffffffffu, want, t);
                const uint32_t pos = base + __popc(m & lt);
                if (hit[u] && pos < rw) {
                    qi_out[row + pos] = __float_as_int(qs[t].w);
                    pj_out[row + pos] = j;
                    d_out[row + pos] = dist[u];
                }
            }
            if (lane == t) cnt += __popc(m);
        }
    }
}

// Self queries, a warp per group of 32 consecutive points in Morton order: the group's
// queries are walked down the tree together, a node kept when its box lies within reach
// of the bounding box of the group's queries (in the current periodic image), and a node
// of at most 32 points (its range of sorted positions) is taken as a bucket: its points
// staged into chunks of 32, each chunk against the group's queries in turn, one ballot
// per query.  A group whose box is wider than twice the radius (the Morton curve jumps
// between distant regions) is halved until it is not.  The pair decisions and images are those of bvh_visit, so the count
// and write passes give the same rows as the thread-per-query kernels (in another order
// before the row sort).
constexpr int kBvhWarps = 4;
constexpr int kBvhGroupSoft = 1024;                        // batched expansion below this
constexpr int kBvhGroupStack = kBvhGroupSoft + kBvhStack;  // + one entry per tree level

template <bool WRITE>
__global__ void __launch_bounds__(kBvhWarps * 32) k_bvh_group(BvhArgs a, uint32_t *__restrict__ counts,
                                                              const int64_t *__restrict__ seg,
                                                              int32_t *__restrict__ qi_out,
                                                              int32_t *__restrict__ pj_out, float *__restrict__ d_out) {
    __shared__ float4 sq[kBvhWarps][32];  // the group's queries in the current image (w: index, -1 none)
    __shared__ int sstk[kBvhWarps][kBvhGroupStack];
    __shared__ float4 sstg[kBvhWarps][64];  // bucket points staged into chunks of 32
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t g0 = ((int64_t)blockIdx.x * kBvhWarps + warp) * 32;
    if (g0 >= a.n) return;
    const int nq = (int)min((int64_t)32, (int64_t)a.n - g0);
    const bool qv = lane < nq;
    const float4 r = qv ? __ldg(a.pts + g0 + lane) : make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
    const int i = qv ? __float_as_int(r.w) : -1;
    const float3 qf = frac_of(a.bf, r.x, r.y, r.z);
    const float lo = a.pts_moved ? a.band_wide.lo : a.band.lo, hi = a.pts_moved ? a.band_wide.hi : a.band.hi;
    float4 *qs = sq[warp];
    int *stk = sstk[warp];
    float4 *stg = sstg[warp];
    int nst = 0;       // staged points
    uint32_t cnt = 0;  // lane t: hits of query t so far
    const int64_t off = WRITE && qv ? seg[i] : 0;
    const uint32_t want = WRITE && qv ? counts[i] : 0;
    const unsigned lt = lanemask_lt();
    int nesc = 0;
    // subgroups (lane ranges l0 | l1 << 8), depth first
    int pend[8];
    int np = 0;
    pend[np++] = nq << 8;
    while (np > 0) {
        const int rg = pend[--np];
        const int l0 = rg & 0xff, l1 = rg >> 8;
        const bool in = lane >= l0 && lane < l1;
        {
            float3 blo, bhi;
            warp_box(r.x, r.y, r.z, in, blo, bhi);
            const float ext = fmaxf(bhi.x - blo.x, fmaxf(bhi.y - blo.y, bhi.z - blo.z));
            if (ext > a.group_ext && l1 - l0 > 1) {
                const int mid = (l0 + l1) >> 1;
                pend[np++] = mid | (l1 << 8);
                pend[np++] = l0 | (mid << 8);
                continue;
            }
        }
        for (int im = 0; im < 27; ++im) {
            const int sx = im % 3 - 1, sy = (im / 3) % 3 - 1, sz = im / 9 - 1;
            // as in bvh_visit: this image of the query is at least its largest slab
            // distance away from the box
            const float gx = qf.x + sx, gy = qf.y + sy, gz = qf.z + sz;
            const float ex = fmaxf(fmaxf(-gx, gx - 1.f), 0.f) * a.w[0];
            const float ey = fmaxf(fmaxf(-gy, gy - 1.f), 0.f) * a.w[1];
            const float ez = fmaxf(fmaxf(-gz, gz - 1.f), 0.f) * a.w[2];
            const bool on = in && !(fmaxf(ex, fmaxf(ey, ez)) > a.reach);
            if (!__any_sync(0xffffffffu, on)) continue;
            const float qx = r.x + (float)sx * a.bf.L[0] + (float)sy * a.bf.a2x + (float)sz * a.bf.a3x;
            const float qy = r.y + (float)sy * a.bf.L[1] + (float)sz * a.bf.a3y;
            const float qz = r.z + (float)sz * a.bf.L[2];
            __syncwarp();
            qs[lane] = on ? make_float4(qx, qy, qz, __int_as_float(i)) : make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
            float3 blo, bhi;
            warp_box(qx, qy, qz, on, blo, bhi);
            // Depth first in batches: the top nodes of the warp's stack (up to 32, one
            // per lane) are expanded at once, their children within reach of the box
            // pushed back, nodes of at most 32 points kept as buckets.  Above the soft
            // capacity one node is expanded at a time, which adds at most one entry per
            // tree level, so the stack stays within kBvhGroupStack.
            if (lane == 0) stk[0] = a.n >= 2 ? 0 : ~0;
            int sp = 1;
            __syncwarp();
            for (int64_t steps = 0; sp > 0; ++steps) {
                if (steps > 2 * (int64_t)a.n + 2 || sp + 2 > kBvhGroupStack) {
                    if (lane == 0) atomicExch(a.err, steps > 2 * (int64_t)a.n + 2 ? 4 : 3);
                    break;
                }
                const int k = sp + 32 <= kBvhGroupSoft ? min(32, sp) : 1;
                const int node = lane < k ? stk[sp - k + lane] : 0;
                sp -= k;
                __syncwarp();
                bool bucket = false, t0 = false, t1 = false;
                int bfirst = 0, bcount = 0, c0 = 0, c1 = 0;
                if (lane < k) {
                    if (node < 0) {
                        bucket = true;
                        bfirst = ~node;
                        bcount = 1;
                    } else {
                        const int2 rn = __ldg(a.range + node);
                        bucket = rn.y - rn.x < 32;
                        bfirst = rn.x;
                        bcount = rn.y - rn.x + 1;
                    }
                    if (!bucket) {
                        const BvhNode *nd = a.nodes + node;
                        c0 = __ldg(&nd->left);
                        c1 = __ldg(&nd->right);
                        t0 = bvh_gap2(a, c0, blo, bhi) <= a.reach2;
                        t1 = bvh_gap2(a, c1, blo, bhi) <= a.reach2;
                    }
                }
                const unsigned m0 = __ballot_sync(0xffffffffu, t0), m1 = __ballot_sync(0xffffffffu, t1);
                if (t0) stk[sp + __popc(m0 & lt)] = c0;
                if (t1) stk[sp + __popc(m0) + __popc(m1 & lt)] = c1;
                sp += __popc(m0) + __popc(m1);
                __syncwarp();
                for (unsigned mb = __ballot_sync(0xffffffffu, bucket); mb; mb &= mb - 1) {
                    const int src = __ffs(mb) - 1;
                    const int bf = __shfl_sync(0xffffffffu, bfirst, src), bc = __shfl_sync(0xffffffffu, bcount, src);
                    // the bucket's points join the stage; each full chunk of 32 is tested
                    if (lane < bc) stg[nst + lane] = __ldg(a.pts + bf + lane);
                    nst += bc;
                    if (nst >= 32) {
                        __syncwarp();
                        bvh_chunk<WRITE>(a, qs, l0, l1, stg[lane], lo, hi, lt, cnt, off, want, nesc, qi_out, pj_out,
                                         d_out);
                        const float4 rest = stg[32 + lane];
                        __syncwarp();
                        if (lane < nst - 32) stg[lane] = rest;
                        nst -= 32;
                        __syncwarp();
                    }
                }
            }
            if (nst > 0) {  // the image's last, partial chunk
                __syncwarp();
                const float4 c = lane < nst ? stg[lane] : make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
                bvh_chunk<WRITE>(a, qs, l0, l1, c, lo, hi, lt, cnt, off, want, nesc, qi_out, pj_out, d_out);
                nst = 0;
                __syncwarp();
            }
        }
    }
    if (qv) {
        if (WRITE) {
            if (cnt != want) atomicExch(a.err, 2);
        } else {
            counts[i] = cnt;
        }
    }
    nesc = __reduce_add_sync(0xffffffffu, nesc);
    if (!WRITE && lane == 0 && nesc) atomicAdd(a.esc, (unsigned long long)nesc);
}

// ------------------------------------------------------------------ k nearest

// The same ranking rule as the cell-list kNN: the k+1 nearest by FP32 (r2, index) are
// kept; the ranking is accepted when every neighbouring gap among them exceeds 2 delta
// (delta = this route's FP32 error bound on r2 at the k-th distance, with 1.5x slack),
// otherwise every candidate within the k-th FP32 r2 + 2 delta is ranked by its FP64 r2.
struct BvhKnn {
    BvhArgs b;
    int k, m;                   // requested, per-row count (uniform)
    float Lsum;
    float half_wmin2;           // (w_min/2)^2, slightly reduced: a farther k-th neighbor is an error
    int *flag_count;
    int2 *flags;                // (query position t, threshold bits)
    int flag_cap;
    int32_t *qi_out, *pj_out;
    float *d_out;
};

__device__ __forceinline__ float bvh_knn_delta(const BvhKnn &a, float R, bool moved) {
    const float u = kU32;
    const float e = 2.f * u * ((moved ? 59.5f : 5.5f) * a.Lsum + R);
    const float d = 3.4641016f * R * e + 3.f * e * e + 3.f * u * (R + e) * (R + e) + 1e-12f * (R + a.Lsum) * (R + a.Lsum);
    return 1.5f * d;
}

// Best-first walk over every reachable image: fn(j, r2) for each leaf whose node boxes
// stayed within bound() (re-read after each leaf, so the bound may shrink).
template <class B, class F>
__device__ __forceinline__ void bvh_walk(const BvhArgs &a, float3 qw, float3 qf, B &&bound, F &&fn) {
    if (a.n == 0) return;
    int stack[kBvhStack];
    // the query's own image first: its neighbors set a tight bound at once, so most of
    // the other 26 images are skipped by their lower bound
    for (int t = 0; t < 27; ++t) {
        const int code = t == 0 ? 13 : (t <= 13 ? t - 1 : t);
        const int sx = code % 3 - 1, sy = (code / 3) % 3 - 1, sz = code / 9 - 1;
        const float gx = qf.x + sx, gy = qf.y + sy, gz = qf.z + sz;
        const float ex = fmaxf(fmaxf(-gx, gx - 1.f), 0.f) * a.w[0];
        const float ey = fmaxf(fmaxf(-gy, gy - 1.f), 0.f) * a.w[1];
        const float ez = fmaxf(fmaxf(-gz, gz - 1.f), 0.f) * a.w[2];
        const float lb = fmaxf(ex, fmaxf(ey, ez)) * (1.f - 1e-5f);
        if (lb * lb > bound()) continue;
        const float qx = qw.x + (float)sx * a.bf.L[0] + (float)sy * a.bf.a2x + (float)sz * a.bf.a3x;
        const float qy = qw.y + (float)sy * a.bf.L[1] + (float)sz * a.bf.a3y;
        const float qz = qw.z + (float)sz * a.bf.L[2];
        int sp = 0;
        int node = a.n >= 2 ? 0 : ~0;
        for (int64_t visits = 0;; ++visits) {
            if (visits > 2 * (int64_t)a.n) {
                atomicExch(a.err, 4);
                break;
            }
            if (node < 0) {
                const float4 c = __ldg(a.pts + ~node);
                fn(__float_as_int(c.w), r2_f32(c.x - qx, c.y - qy, c.z - qz));
            } else {
                const BvhNode *nd = a.nodes + node;
                const int c0 = __ldg(&nd->left), c1 = __ldg(&nd->right);
                float d0, d1;
                {
                    float dx, dy, dz;
                    if (c0 < 0) {
                        const float4 p = __ldg(a.pts + ~c0);
                        dx = p.x - qx, dy = p.y - qy, dz = p.z - qz;
                    } else {
                        const BvhNode *cn = a.nodes + c0;
                        dx = fmaxf(fmaxf(__ldg(cn->lo) - qx, qx - __ldg(cn->hi)), 0.f);
                        dy = fmaxf(fmaxf(__ldg(cn->lo + 1) - qy, qy - __ldg(cn->hi + 1)), 0.f);
                        dz = fmaxf(fmaxf(__ldg(cn->lo + 2) - qz, qz - __ldg(cn->hi + 2)), 0.f);
                    }
                    d0 = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * (1.f - 1e-5f);
                    if (c1 < 0) {
                        const float4 p = __ldg(a.pts + ~c1);
                        dx = p.x - qx, dy = p.y - qy, dz = p.z - qz;
                    } else {
                        const BvhNode *cn = a.nodes + c1;
                        dx = fmaxf(fmaxf(__ldg(cn->lo) - qx, qx - __ldg(cn->hi)), 0.f);
                        dy = fmaxf(fmaxf(__ldg(cn->lo + 1) - qy, qy - __ldg(cn->hi + 1)), 0.f);
                        dz = fmaxf(fmaxf(__ldg(cn->lo + 2) - qz, qz - __ldg(cn->hi + 2)), 0.f);
                    }
                    d1 = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * (1.f - 1e-5f);
                }
                const float lim = bound();
                const bool t0 = d0 <= lim, t1 = d1 <= lim;
                if (t0 && t1) {
                    const bool first0 = d0 <= d1;
                    if (sp < kBvhStack)
                        stack[sp++] = first0 ? c1 : c0;
                    else
                        atomicExch(a.err, 3);
                    node = first0 ? c0 : c1;
                    continue;
                }
                if (t0 || t1) {
                    node = t0 ? c0 : c1;
                    continue;
                }
            }
            // pop, skipping entries the shrinking bound has ruled out is left to the
            // child test of the next node (its box is re-tested when expanded)
            if (sp == 0) break;
            node = stack[--sp];
        }
    }
}
template <int KT>
__global__ void __launch_bounds__(128) k_bvh_knn(BvhKnn a) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.b.nq) return;
    float3 qw, qf;
    int fl;
    const int i = bvh_query_point(a.b, t, qw, qf, fl);
    if (fl & 2) {
        atomicExch(a.b.err, 5);
        return;
    }
    const int excl = a.b.exclude ? i : -1;
    const int m = a.m;
    float br[KT];
    int bj[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        br[q] = INFINITY;
        bj[q] = 0x7fffffff;
    }
    // bound: the (m+1)-th best so far (ties kept by the 1e-5 shrink of the box distances),
    // refreshed when a candidate enters the list
    float bnd = INFINITY;
    auto bound = [&]() { return bnd; };
    bvh_walk(a.b, qw, qf, bound, [&](int j, float r2) {
        if (j == excl) return;
        if (r2 < br[KT - 1] || (r2 == br[KT - 1] && j < bj[KT - 1])) {
            topk_insert<KT>(br, bj, r2, j);
            bnd = pick<KT>(br, min(m, KT - 1)) * (1.f + 1e-5f);
        }
    });
    if (m == 0) return;
    const bool moved = fl != 0 || a.b.pts_moved;
    const float rm2 = pick<KT>(br, m - 1);
    const float delta = bvh_knn_delta(a, sqrtf(rm2) + 1e-3f, moved);
    if (rm2 + delta >= a.half_wmin2) {
        atomicOr(a.b.err, 1);
        return;
    }
    bool ambiguous = false;
#pragma unroll
    for (int q = 0; q + 1 < KT; ++q)
        if (q < m && br[q + 1] - br[q] <= 2.f * delta) ambiguous = true;
    const int64_t row = (int64_t)i * m;
    if (ambiguous) {
        const int slot = atomicAdd(a.flag_count, 1);
        if (slot < a.flag_cap)
            a.flags[slot] = make_int2((int)t, __float_as_int((rm2 + 2.f * delta) * 1.0000005f));
        else
            atomicOr(a.b.err, 2);
        return;
    }
#pragma unroll
    for (int q = 0; q < KT; ++q)
        if (q < m) {
            a.qi_out[row + q] = i;
            a.pj_out[row + q] = bj[q];
            a.d_out[row + q] = sqrtf(br[q]);
        }
}

// Flagged queries: every candidate within the threshold ranked by its FP64 r2.
template <int KT>
__global__ void __launch_bounds__(64) k_bvh_knn_exact(BvhKnn a) {
    const int nflag = min(*a.flag_count, a.flag_cap);
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nflag; f += gridDim.x * blockDim.x) {
        const int2 flg = a.flags[f];
        float3 qw, qf;
        int fl;
        const int i = bvh_query_point(a.b, flg.x, qw, qf, fl);
        const float thr = __int_as_float(flg.y);
        const int excl = a.b.exclude ? i : -1;
        double br[KT];
        int bj[KT];
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            br[q] = INFINITY;
            bj[q] = 0x7fffffff;
        }
        bvh_walk(a.b, qw, qf, [&]() { return thr * (1.f + 1e-5f); }, [&](int j, float r2) {
            if (j == excl || r2 > thr) return;
            const double e = exact_r2_idx(a.b.bd, a.b.q_orig, i, a.b.p_orig, j);
            if (e < br[KT - 1] || (e == br[KT - 1] && j < bj[KT - 1])) {
                double cr = e;
                int cj = j;
#pragma unroll
                for (int q = 0; q < KT; ++q) {
                    const bool less = cr < br[q] || (cr == br[q] && cj < bj[q]);
                    const double tr = less ? br[q] : cr;
                    const int tj = less ? bj[q] : cj;
                    br[q] = less ? cr : br[q];
                    bj[q] = less ? cj : bj[q];
                    cr = tr;
                    cj = tj;
                }
            }
        });
        const int64_t row = (int64_t)i * a.m;
#pragma unroll
        for (int q = 0; q < KT; ++q)
            if (q < a.m) {
                a.qi_out[row + q] = i;
                a.pj_out[row + q] = bj[q];
                a.d_out[row + q] = (float)sqrt(br[q]);
            }
    }
}

// ------------------------------------------------------------------ host

static int grid1d(int64_t n, int t) { return (int)((n + t - 1) / t); }

// Blocks of kBvhWarps warps, one per 32 queries.
static unsigned group_grid(int64_t nq) { return (unsigned)(((nq + 31) / 32 + kBvhWarps - 1) / kBvhWarps); }

// FGB_BVH_GROUP=0 keeps self queries on the thread-per-query kernels (comparisons, and
// tests of those kernels).
static bool group_kernels() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("FGB_BVH_GROUP");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

int aabb_build(fgb_nq *nq, cudaStream_t s) {
    const int64_t n = nq->n;
    nq->kind = 1;
    if (n == 0) return FGB_OK;
    uint32_t *keys = nullptr, *vals = nullptr;
    float4 *rec = nullptr;
    void *ws = nullptr;
    int *parent_int = nullptr, *parent_leaf = nullptr, *flags = nullptr, *pflags = nullptr;
    BvhNode *nodes = nullptr;
    int st = dalloc_n(&pflags, 1, s);
    if (st == FGB_OK) st = cudaMemsetAsync(pflags, 0, sizeof(int), s) == cudaSuccess ? FGB_OK : fail(FGB_ERR_CUDA, "memset");
    st = st ? st : dalloc_n(&nq->sorted, n, s);
    st = st ? st : dalloc_n(&nq->sorted_cell, n, s);
    st = st ? st : dalloc_n(&keys, n, s);
    st = st ? st : dalloc_n(&vals, n, s);
    st = st ? st : dalloc_n(&rec, n, s);
    st = st ? st : dalloc(&ws, sort_ws_bytes(n), s);
    if (st == FGB_OK) {
        {
            FGB_KSCOPE("k_bvh_keys", s);
            k_bvh_keys<<<grid1d(n, 256), 256, 0, s>>>(nq->box.f, nq->points, n, keys, vals, rec, pflags);
        }
        st = radix_sort_cells(keys, vals, n, (int64_t)1 << 30, rec, nq->sorted, nq->sorted_cell, ws, s);
    }
    if (st == FGB_OK && n >= 2) {
        // the n - 1 nodes, then their n - 1 point ranges (int2), in one block
        static_assert(sizeof(BvhNode) % sizeof(int2) == 0, "ranges follow the nodes");
        st = dalloc(reinterpret_cast<void **>(&nodes), (size_t)(n - 1) * (sizeof(BvhNode) + sizeof(int2)), s);
        st = st ? st : dalloc_n(&parent_int, n - 1, s);
        st = st ? st : dalloc_n(&parent_leaf, n, s);
        st = st ? st : dalloc_n(&flags, n - 1, s);
        if (st == FGB_OK) {
            FGB_CUDA(cudaMemsetAsync(flags, 0, sizeof(int) * (n - 1), s));
            {
                FGB_KSCOPE("k_bvh_nodes", s);
                k_bvh_nodes<<<grid1d(n - 1, 256), 256, 0, s>>>(nq->sorted_cell, (int)n, nodes,
                                                               bvh_ranges(nodes, n), parent_int, parent_leaf);
            }
            {
                FGB_KSCOPE("k_bvh_refit", s);
                k_bvh_refit<<<grid1d(n, 256), 256, 0, s>>>(nq->sorted, (int)n, nodes, parent_int, parent_leaf, flags);
            }
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) st = fail(FGB_ERR_CUDA, "tree build launch failed: %s", cudaGetErrorString(e));
        }
    }
    int hflags = 0;
    if (st == FGB_OK) {
        cudaMemcpyAsync(&hflags, pflags, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = fail(FGB_ERR_CUDA, "tree build failed: %s", cudaGetErrorString(e));
    }
    if (st == FGB_OK && (hflags & 2))
        st = fail(FGB_ERR_INVALID_ARG, "tree query: points must lie within two box lengths of the box centre");
    nq->bvh_moved = (hflags & 1) ? 1 : 0;
    dfree(pflags, s);
    dfree(keys, s);
    dfree(vals, s);
    dfree(rec, s);
    dfree(ws, s);
    dfree(parent_int, s);
    dfree(parent_leaf, s);
    dfree(flags, s);
    if (st == FGB_OK)
        nq->bvh = nodes;
    else
        dfree(nodes, s);
    return st;
}

void aabb_free(fgb_nq *nq) {
    dfree(static_cast<BvhNode *>(nq->bvh), nq->stream);
    nq->bvh = nullptr;
}

int aabb_ball_query(fgb_nq *nq, const float *query_points, int64_t n_query, const fgb_query_args *args,
                    cudaStream_t s, fgb_nlist *nl) {
    const double R = args->r_max;
    const BoxHost &b = nq->box;
    const bool self = query_points == nullptr || query_points == nq->points;
    const int64_t nqq = self ? nq->n : n_query;
    BvhArgs a;
    memset(&a, 0, sizeof(a));
    a.bf = b.f;
    a.bd = b.d;
    for (int k = 0; k < 3; ++k) a.w[k] = (float)b.w[k];
    a.nodes = static_cast<const BvhNode *>(nq->bvh);
    a.range = nq->n >= 2 ? bvh_ranges(static_cast<BvhNode *>(nq->bvh), nq->n) : nullptr;
    a.pts = nq->sorted;
    a.n = (int)nq->n;
    a.p_orig = nq->points;
    a.q_orig = self ? nq->points : query_points;
    a.nq = nqq;
    a.self = self ? 1 : 0;
    a.exclude = args->exclude_ii ? 1 : 0;
    // Error of one displacement component, Lsum = sum of the box vector lengths.
    // Points that wrapping left in place (|x| <= Lsum / 2) keep their coordinates exactly:
    //   image shift of the query: FP32 box vectors (u Lsum) and 3 sums <= 1.5 Lsum
    //                                                                  -> 5.5 u Lsum
    //   d = p - q (|d| <= R for pairs that matter)                     -> u R
    // A point moved by wrapping (|s - 1/2| <= 2, so |x| <= 2 Lsum, |floor(s)| <= 3):
    //   3 products n a_k (<= 3 Lsum) and 3 differences (<= 5 Lsum), FP32 box vectors
    //   (3 u Lsum)                                              -> 27 u Lsum per point
    // Both doubled for slack.
    double Lsum = 0.0;
    for (int c = 0; c < 3; ++c) Lsum += std::sqrt(b.M[0][c] * b.M[0][c] + b.M[1][c] * b.M[1][c] + b.M[2][c] * b.M[2][c]);
    const double u = std::ldexp(1.0, -24);
    const double eps_in = 2.0 * u * (5.5 * Lsum + R);
    const double eps_moved = 2.0 * u * ((5.5 + 2.0 * 27.0) * Lsum + R);
    a.T = sqrt_threshold(R);
    band_around(a.T, r2_error_bound_eps(eps_in, Lsum, R), &a.band.lo, &a.band.hi);
    band_around(a.T, r2_error_bound_eps(eps_moved, Lsum, R), &a.band_wide.lo, &a.band_wide.hi);
    a.pts_moved = nq->bvh_moved;
    a.reach2 = a.band_wide.hi * (1.0f + 1e-5f) + 1e-30f;
    a.reach = (float)(R * (1.0 + 1e-4) + 1e-5 * Lsum);
    a.group_ext = (float)(2.0 * R);
    struct Status {
        unsigned long long esc;
        int err;
        uint32_t maxcount;
    };
    Status *dst = nullptr;
    FGB_TRY(dalloc_n(&dst, 1, s));
    FGB_CUDA(cudaMemsetAsync(dst, 0, sizeof(Status), s));
    a.esc = &dst->esc;
    a.err = &dst->err;
    nl->n_query = nqq;
    nl->n_points = nq->n;
    int st = dalloc_n(&nl->counts, nqq, s);
    st = st ? st : dalloc_n(&nl->segments, nqq + 1, s);
    uint32_t *counts = reinterpret_cast<uint32_t *>(nl->counts);
    Status hs;
    memset(&hs, 0, sizeof(hs));
    int64_t total = 0;
    if (st == FGB_OK && nqq > 0) {
        if (self && group_kernels()) {
            FGB_KSCOPE("k_bvh_group_count", s);
            k_bvh_group<false><<<group_grid(nqq), kBvhWarps * 32, 0, s>>>(a, counts, nullptr, nullptr, nullptr, nullptr);
        } else {
            FGB_KSCOPE("k_bvh_count", s);
            k_bvh_count<<<grid1d(nqq, 128), 128, 0, s>>>(a, counts);
        }
        st = scan_u32_i64(counts, nl->segments, nqq, &dst->maxcount, s);
        if (st == FGB_OK) {
            cudaMemcpyAsync(&total, nl->segments + nqq, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(&hs, dst, sizeof(Status), cudaMemcpyDeviceToHost, s);
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = fail(FGB_ERR_CUDA, "tree query count pass failed: %s", cudaGetErrorString(e));
        }
    } else if (st == FGB_OK) {
        FGB_CUDA(cudaMemsetAsync(nl->segments, 0, sizeof(int64_t), s));
    }
    if (st == FGB_OK && hs.err == 5)
        st = fail(FGB_ERR_INVALID_ARG, "tree query: query points must lie within two box lengths of the box centre");
    else if (st == FGB_OK && hs.err)
        st = fail(FGB_ERR_CUDA, "tree query: traversal failed (code %d)", hs.err);
    if (st == FGB_OK && total >= ((int64_t)1 << 40))
        st = fail(FGB_ERR_CAPACITY, "neighbor list of %lld pairs is too large", (long long)total);
    nl->n_pairs = total;
    st = st ? st : dalloc_n(&nl->qi, total, s);
    st = st ? st : dalloc_n(&nl->pj, total, s);
    st = st ? st : dalloc_n(&nl->dist, total, s);
    if (st == FGB_OK && total > 0) {
        if (self && group_kernels()) {
            FGB_KSCOPE("k_bvh_group_write", s);
            k_bvh_group<true><<<group_grid(nqq), kBvhWarps * 32, 0, s>>>(a, counts, nl->segments, nl->qi, nl->pj,
                                                                         nl->dist);
        } else {
            FGB_KSCOPE("k_bvh_write", s);
            k_bvh_write<<<grid1d(nqq, 128), 128, 0, s>>>(a, nl->segments, counts, nl->qi, nl->pj, nl->dist);
        }
        const int cap = (int)((hs.maxcount + 3) & ~3u);
        st = sort_segments(nl->segments, nqq, cap, nq->n, nl->qi, nl->pj, nl->dist, s);
    }
    if (st == FGB_OK) {
        cudaMemcpyAsync(&hs, dst, sizeof(Status), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = fail(FGB_ERR_CUDA, "tree query write pass failed: %s", cudaGetErrorString(e));
        else if (hs.err) st = fail(FGB_ERR_CUDA, "tree query: count and write passes disagree (code %d)", hs.err);
    }
    nl->escalations = (int64_t)hs.esc;
    nl->symmetric = self && a.exclude ? 1 : 0;
    nl->kind = 0;
    dfree(dst, s);
    return st;
}

__global__ void k_bvh_knn_rows(int64_t nq, int m, int64_t *__restrict__ seg, int32_t *__restrict__ counts) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= nq) seg[i] = i * (int64_t)m;
    if (i < nq) counts[i] = m;
}

template <int KT>
static void launch_bvh_knn(const BvhKnn &a, cudaStream_t s) {
    {
        FGB_KSCOPE("k_bvh_knn", s);
        k_bvh_knn<KT><<<grid1d(a.b.nq, 128), 128, 0, s>>>(a);
    }
    {
        FGB_KSCOPE("k_bvh_knn_exact", s);
        k_bvh_knn_exact<KT><<<num_sms() * 2, 64, 0, s>>>(a);
    }
}

int aabb_knn_query(fgb_nq *nq, const float *query_points, int64_t n_query, const fgb_query_args *args,
                   cudaStream_t s, fgb_nlist *nl) {
    const int k = args->num_neighbors;
    if (k > 32) return fail(FGB_ERR_UNSUPPORTED, "num_neighbors > 32 is not supported");
    const bool self = query_points == nullptr || query_points == nq->points;
    const bool excl = args->exclude_ii != 0;
    const int64_t np = nq->n, nqq = self ? np : n_query;
    if (!self && excl && np <= k)
        return fail(FGB_ERR_UNSUPPORTED, "tree kNN with exclude_ii needs more than k points (uniform rows)");
    const int m = (int)std::min<int64_t>(k, std::max<int64_t>(0, self && excl ? np - 1 : np));
    const BoxHost &b = nq->box;
    BvhKnn a;
    memset(&a, 0, sizeof(a));
    a.b.bf = b.f;
    a.b.bd = b.d;
    for (int q = 0; q < 3; ++q) a.b.w[q] = (float)b.w[q];
    a.b.nodes = static_cast<const BvhNode *>(nq->bvh);
    a.b.pts = nq->sorted;
    a.b.n = (int)np;
    a.b.p_orig = nq->points;
    a.b.q_orig = self ? nq->points : query_points;
    a.b.nq = nqq;
    a.b.self = self ? 1 : 0;
    a.b.exclude = excl ? 1 : 0;
    a.b.pts_moved = nq->bvh_moved;
    double Lsum = 0.0;
    for (int c = 0; c < 3; ++c) Lsum += std::sqrt(b.M[0][c] * b.M[0][c] + b.M[1][c] * b.M[1][c] + b.M[2][c] * b.M[2][c]);
    a.Lsum = (float)Lsum;
    const double hw = 0.5 * b.wmin * (1.0 - 1e-4);
    a.half_wmin2 = (float)(hw * hw);
    a.k = k;
    a.m = m;
    struct Status {
        int err;
        int flags;
    };
    Status *dst = nullptr;
    FGB_TRY(dalloc_n(&dst, 1, s));
    FGB_CUDA(cudaMemsetAsync(dst, 0, sizeof(Status), s));
    a.b.err = &dst->err;
    a.flag_count = &dst->flags;
    a.flag_cap = (int)std::max<int64_t>(1, nqq);
    nl->n_query = nqq;
    nl->n_points = np;
    nl->n_pairs = nqq * m;
    int st = dalloc_n(&nl->counts, nqq, s);
    st = st ? st : dalloc_n(&nl->segments, nqq + 1, s);
    st = st ? st : dalloc_n(&nl->qi, nl->n_pairs, s);
    st = st ? st : dalloc_n(&nl->pj, nl->n_pairs, s);
    st = st ? st : dalloc_n(&nl->dist, nl->n_pairs, s);
    st = st ? st : dalloc_n(&a.flags, a.flag_cap, s);
    if (st == FGB_OK) {
        {
            FGB_KSCOPE("k_bvh_knn_rows", s);
            k_bvh_knn_rows<<<grid1d(nqq + 1, 256), 256, 0, s>>>(nqq, m, nl->segments, nl->counts);
        }
        a.qi_out = nl->qi;
        a.pj_out = nl->pj;
        a.d_out = nl->dist;
        if (nqq > 0 && m > 0) {
            if (m + 1 <= 2)
                launch_bvh_knn<2>(a, s);
            else if (m + 1 <= 4)
                launch_bvh_knn<4>(a, s);
            else if (m + 1 <= 8)
                launch_bvh_knn<8>(a, s);
            else if (m + 1 <= 16)
                launch_bvh_knn<16>(a, s);
            else if (m + 1 <= 32)
                launch_bvh_knn<32>(a, s);
            else
                launch_bvh_knn<64>(a, s);
        }
        Status hs;
        cudaMemcpyAsync(&hs, dst, sizeof(Status), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess)
            st = fail(FGB_ERR_CUDA, "tree kNN failed: %s", cudaGetErrorString(e));
        else if (hs.err & 1)
            st = fail(FGB_ERR_BOX_TOO_SMALL, "a k-th neighbor lies at half the smallest box width or beyond");
        else if (hs.err == 5)
            st = fail(FGB_ERR_INVALID_ARG, "tree query: query points must lie within two box lengths of the box centre");
        else if (hs.err)
            st = fail(FGB_ERR_CUDA, "tree kNN: traversal failed (code %d)", hs.err);
    }
    dfree(a.flags, s);
    dfree(dst, s);
    nl->kind = 1;
    nl->symmetric = 0;
    return st;
}

}  // namespace fgb

using namespace fgb;

extern "C" int fgb_aabb_create(const fgb_box *box, const float *points, int64_t n, void *stream, fgb_nq **out) {
    clear_error();
    if (!out) return fail(FGB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 0 || (n > 0 && !points)) return fail(FGB_ERR_INVALID_ARG, "points/n invalid");
    if (n >= (int64_t)1 << 31) return fail(FGB_ERR_CAPACITY, "at most 2^31-1 points");
    cudaStream_t s = as_stream(stream);
    fgb_nq *nq = new fgb_nq();
    memset(nq, 0, sizeof(*nq));
    nq->points = points;
    nq->n = n;
    nq->stream = s;
    nq->kind = 1;
    int st = make_box(box, &nq->box);
    st = st ? st : aabb_build(nq, s);
    if (st != FGB_OK) {
        fgb_nq_destroy(nq);
        return st;
    }
    *out = nq;
    return FGB_OK;
}
