// Clusters of points joined by neighbor bonds and their properties (cluster module,
// Section "Analysis Modules": membership defined by neighbor bonds, then per-cluster
// properties such as gyration tensors).
//
// Connected components by a lock-free union-find on the device: every bond hooks the
// larger of its two current roots under the smaller with an atomic compare-and-swap
// (parents only ever decrease, so the forest stays acyclic and a component's root is its
// smallest index); a failed swap means another bond moved that root, and the bond simply
// looks its roots up again.  A sampling pass first joins every point with the other ends
// of its first two bonds, which in a neighbor graph already links most points into their
// final components; the full pass then skips every bond whose ends had the same root
// after sampling (such a bond joins nothing new), so crystals and dense clusters cost
// two loads per bond (sampling after Sutton, Ben-Nun and Barak, "Optimizing Parallel
// Graph Connectivity Computation via Subgraph Sampling", IPDPS 2018).  Clusters are then numbered by decreasing size, ties by
// their smallest member, through one stable radix sort of (n - size) over the roots.
//
// Properties: each member is unwrapped to the image nearest the cluster's smallest
// member (minimum image of x_j - x_root), the centre is that member plus the mean
// unwrapped offset, wrapped back into the box, and the gyration tensor is the mean outer
// product of the offsets from the centre; sums in FP64 atomics.
#include <cmath>
#include <cstring>

#include "fgb_device.cuh"

namespace fgb {

constexpr int kUnionRetries = 1 << 20;  // a bond retries only while other bonds move its roots

// Root of x (-1 if the walk did not end, which a forest whose parents only decrease
// rules out); halves the path on the way.
__device__ __forceinline__ int cc_find(int *parent, int x) {
    for (int it = 0; it < kUnionRetries; ++it) {
        const int p = __ldcg(parent + x);
        if (p == x) return x;
        const int g = __ldcg(parent + p);
        if (g != p) atomicMin(parent + x, g);
        x = g;
    }
    return -1;
}

__global__ void k_cc_init(int *parent, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) parent[i] = (int)i;
}

// Joins the components of a and b.
__device__ __forceinline__ void cc_link(int *parent, int a, int b, int *err) {
    for (int it = 0; it < kUnionRetries; ++it) {
        a = cc_find(parent, a);
        b = cc_find(parent, b);
        if (a < 0 || b < 0) break;
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(parent + a, a, b) == a) return;
    }
    atomicExch(err, 1);
}

// Sampling pass: the first two unmasked bonds of every segment [seg[i], seg[i+1]) join
// their two ends (for a query-ordered list, point i and two of its neighbors; each link
// is a bond of the list whatever its order, so the result never depends on it).
__global__ void k_cc_sample(const int64_t *__restrict__ seg, int64_t nq, const int32_t *__restrict__ qi,
                            const int32_t *__restrict__ pj, const uint8_t *__restrict__ mask, int *parent, int *err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    int taken = 0;
    for (int64_t e = seg[i]; e < seg[i + 1] && taken < 2; ++e) {
        if (mask && !mask[e]) continue;
        cc_link(parent, qi[e], pj[e], err);
        ++taken;
    }
}

// Every point's root after sampling (also written as its parent, one of its ancestors).
__global__ void k_cc_snapshot(int *parent, int64_t n, int *comp, int *err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = cc_find(parent, (int)i);
    if (r < 0) {
        atomicExch(err, 1);
        comp[i] = -1 - (int)i;  // matches no other point: its bonds take the full pass
        return;
    }
    comp[i] = r;
    parent[i] = r;
}

// One thread per bond (i, j); mask[e] == 0 skips the bond, and so does a bond whose ends
// had the same root after sampling (comp).
__global__ void k_cc_union(const int32_t *__restrict__ qi, const int32_t *__restrict__ pj,
                           const uint8_t *__restrict__ mask, int64_t m, const int *__restrict__ comp, int *parent,
                           int *err) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m || (mask && !mask[e])) return;
    const int a = qi[e], b = pj[e];
    if (__ldg(comp + a) == __ldg(comp + b)) return;
    cc_link(parent, a, b, err);
}

// Final roots and component sizes; the lanes of a warp with the same root add to its
// size once (one atomic per distinct root: a spanning cluster would otherwise put every
// point's addition on one address).
__global__ void k_cc_roots(int *parent, int64_t n, int *root, uint32_t *size, int *err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int r = -1;
    if (i < n) {
        r = cc_find(parent, (int)i);
        if (r < 0) {
            atomicExch(err, 1);
            r = (int)i;
        }
        root[i] = r;
    }
    const unsigned live = __ballot_sync(0xffffffffu, i < n);
    if (i >= n) return;
    const unsigned same = __match_any_sync(live, r);
    const int lane = threadIdx.x & 31;
    if (lane == __ffs(same) - 1) atomicAdd(size + r, (uint32_t)__popc(same));
}

__global__ void k_cc_is_root(const int *__restrict__ root, int64_t n, uint32_t *flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = root[i] == (int)i ? 1u : 0u;
}

// Sort records over the roots in increasing index order: key n - size, value the slot
// in the compacted root list, payload (root index, size).
__global__ void k_cc_keys(const int *__restrict__ root, const uint32_t *__restrict__ size, int64_t n,
                          const int64_t *__restrict__ slot_of, uint32_t *keys, uint32_t *vals, float4 *payload) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || root[i] != (int)i) return;
    const int64_t s = slot_of[i];
    keys[s] = (uint32_t)(n - size[i]);
    vals[s] = (uint32_t)s;
    payload[s] = make_float4(__int_as_float((int)i), __int_as_float((int)size[i]), 0.f, 0.f);
}

// Cluster id of every root from its sorted position.
__global__ void k_cc_ids(const float4 *__restrict__ sorted, int64_t nc, int *id_of_root, int32_t *sizes,
                         int32_t *roots_out) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const float4 v = sorted[c];
    id_of_root[__float_as_int(v.x)] = (int)c;
    sizes[c] = __float_as_int(v.y);
    roots_out[c] = __float_as_int(v.x);
}

__global__ void k_cc_label(const int *__restrict__ root, const int *__restrict__ id_of_root, int64_t n,
                           int32_t *cluster_idx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cluster_idx[i] = id_of_root[root[i]];
}

// ------------------------------------------------------------------ properties

// Adds v to *dst for every lane of the warp (live: the lanes holding a point; cluster c).
// A warp whose points all belong to one cluster (the usual case for large clusters, whose
// points sit together in index order more often than not) adds its sum once; otherwise
// every lane adds its own value.
__device__ __forceinline__ void warp_add(double *dst, double v, bool uniform) {
    if (uniform) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(dst, v);
    } else {
        atomicAdd(dst, v);
    }
}

__global__ void k_cl_offsets(BoxF b, const float *__restrict__ x, int64_t n, const int32_t *__restrict__ cid,
                             const int32_t *__restrict__ roots, double *sums) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < n;
    const int c = live ? cid[i] : -1;
    const int c0 = __shfl_sync(0xffffffffu, c, 0);
    const bool uniform = __all_sync(0xffffffffu, live && c == c0);
    if (!uniform && !live) return;
    const float3 d = live ? bond_f32(b, x, roots[c], i) : make_float3(0.f, 0.f, 0.f);
    warp_add(sums + 3 * c + 0, (double)d.x, uniform);
    warp_add(sums + 3 * c + 1, (double)d.y, uniform);
    warp_add(sums + 3 * c + 2, (double)d.z, uniform);
}

__global__ void k_cl_gyration(BoxF b, const float *__restrict__ x, int64_t n, const int32_t *__restrict__ cid,
                              const int32_t *__restrict__ roots, const int32_t *__restrict__ sizes,
                              const double *__restrict__ sums, double *g) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < n;
    const int c = live ? cid[i] : -1;
    const int c0 = __shfl_sync(0xffffffffu, c, 0);
    const bool uniform = __all_sync(0xffffffffu, live && c == c0);
    if (!uniform && !live) return;
    const float3 d = bond_f32(b, x, roots[c], i);
    const double inv = 1.0 / sizes[c];
    const double ex = d.x - sums[3 * c] * inv, ey = d.y - sums[3 * c + 1] * inv, ez = d.z - sums[3 * c + 2] * inv;
    double *gc = g + 6 * c;
    warp_add(gc + 0, ex * ex, uniform);
    warp_add(gc + 1, ex * ey, uniform);
    warp_add(gc + 2, ex * ez, uniform);
    warp_add(gc + 3, ey * ey, uniform);
    warp_add(gc + 4, ey * ez, uniform);
    warp_add(gc + 5, ez * ez, uniform);
}

// centre = x_root + mean offset, wrapped into the box; gyration = mean outer product
__global__ void k_cl_finish(BoxF b, const float *__restrict__ x, int64_t nc, const int32_t *__restrict__ roots,
                            const int32_t *__restrict__ sizes, const double *__restrict__ sums,
                            const double *__restrict__ g, float *centers, float *gyr) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const double inv = 1.0 / sizes[c];
    const int r = roots[c];
    float3 p = make_float3((float)(x[3 * r] + sums[3 * c] * inv), (float)(x[3 * r + 1] + sums[3 * c + 1] * inv),
                           (float)(x[3 * r + 2] + sums[3 * c + 2] * inv));
    const float s0 = fmaf(b.inv00, p.x, fmaf(b.inv01, p.y, b.inv02 * p.z)) + 0.5f;
    const float s1 = fmaf(b.inv11, p.y, b.inv12 * p.z) + 0.5f;
    const float s2 = b.inv22 * p.z + 0.5f;
    const float n0 = floorf(s0), n1 = floorf(s1), n2 = floorf(s2);
    p.x -= n0 * b.L[0] + n1 * b.a2x + n2 * b.a3x;
    p.y -= n1 * b.L[1] + n2 * b.a3y;
    p.z -= n2 * b.L[2];
    centers[3 * c] = p.x;
    centers[3 * c + 1] = p.y;
    centers[3 * c + 2] = p.z;
    const double *gc = g + 6 * c;
    float *o = gyr + 9 * c;
    o[0] = (float)(gc[0] * inv), o[1] = (float)(gc[1] * inv), o[2] = (float)(gc[2] * inv);
    o[3] = o[1], o[4] = (float)(gc[3] * inv), o[5] = (float)(gc[4] * inv);
    o[6] = o[2], o[7] = o[5], o[8] = (float)(gc[5] * inv);
}

static int grid1d(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace fgb

struct fgb_clusters {
    int64_t n, nc;
    int32_t *cluster_idx;   // (n)
    int32_t *sizes;         // (nc), non-increasing
    int32_t *roots;         // (nc) smallest member of each cluster
    cudaStream_t stream;
};

using namespace fgb;

extern "C" int fgb_cluster_compute(int64_t n, const fgb_nlist *nlist, const uint8_t *bond_mask, void *stream,
                                   fgb_clusters **out) {
    clear_error();
    if (!out || !nlist) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    FGB_TRY(nlist_ready(nlist));
    *out = nullptr;
    if (n < 0 || n >= ((int64_t)1 << 31) - 1) return fail(FGB_ERR_INVALID_ARG, "n out of range");
    if (nlist->n_query > n || nlist->n_points > n)
        return fail(FGB_ERR_INVALID_ARG, "the neighbor list indexes more than n points");
    cudaStream_t s = as_stream(stream);
    fgb_clusters *C = new fgb_clusters();
    memset(C, 0, sizeof(*C));
    C->n = n;
    C->stream = s;
    int *parent = nullptr, *root = nullptr, *err = nullptr, *id_of_root = nullptr;
    uint32_t *size = nullptr, *flag = nullptr, *keys = nullptr, *vals = nullptr, *okeys = nullptr;
    int64_t *slot = nullptr;
    float4 *payload = nullptr, *sorted = nullptr;
    void *ws = nullptr;
    int st = dalloc_n(&C->cluster_idx, n, s);
    st = st ? st : dalloc_n(&parent, n, s);
    st = st ? st : dalloc_n(&root, n, s);
    st = st ? st : dalloc_n(&size, n, s);
    st = st ? st : dalloc_n(&flag, n, s);
    st = st ? st : dalloc_n(&slot, n + 1, s);
    st = st ? st : dalloc_n(&err, 1, s);
    int64_t nc = 0;
    int herr = 0;
    if (st == FGB_OK && n > 0) {
        cudaMemsetAsync(size, 0, sizeof(uint32_t) * n, s);
        cudaMemsetAsync(err, 0, sizeof(int), s);
        {
            FGB_KSCOPE("k_cc_init", s);
            k_cc_init<<<grid1d(n, 256), 256, 0, s>>>(parent, n);
        }
        if (nlist->n_pairs > 0) {
            {
                FGB_KSCOPE("k_cc_sample", s);
                k_cc_sample<<<grid1d(nlist->n_query, 256), 256, 0, s>>>(nlist->segments, nlist->n_query, nlist->qi,
                                                                         nlist->pj, bond_mask, parent, err);
            }
            {
                FGB_KSCOPE("k_cc_snapshot", s);
                k_cc_snapshot<<<grid1d(n, 256), 256, 0, s>>>(parent, n, root, err);
            }
            FGB_KSCOPE("k_cc_union", s);
            k_cc_union<<<grid1d(nlist->n_pairs, 256), 256, 0, s>>>(nlist->qi, nlist->pj, bond_mask, nlist->n_pairs,
                                                                    root, parent, err);
        }
        {
            FGB_KSCOPE("k_cc_roots", s);
            k_cc_roots<<<grid1d(n, 256), 256, 0, s>>>(parent, n, root, size, err);
        }
        {
            FGB_KSCOPE("k_cc_is_root", s);
            k_cc_is_root<<<grid1d(n, 256), 256, 0, s>>>(root, n, flag);
        }
        st = scan_u32_i64(flag, slot, n, nullptr, s);
        if (st == FGB_OK) {
            cudaMemcpyAsync(&nc, slot + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = fail(FGB_ERR_CUDA, "clustering failed: %s", cudaGetErrorString(e));
            else if (herr) st = fail(FGB_ERR_CUDA, "clustering: union-find did not settle");
        }
        st = st ? st : dalloc_n(&keys, nc, s);
        st = st ? st : dalloc_n(&vals, nc, s);
        st = st ? st : dalloc_n(&okeys, nc, s);
        st = st ? st : dalloc_n(&payload, nc, s);
        st = st ? st : dalloc_n(&sorted, nc, s);
        st = st ? st : dalloc(&ws, sort_ws_bytes(nc), s);
        st = st ? st : dalloc_n(&id_of_root, n, s);
        st = st ? st : dalloc_n(&C->sizes, nc, s);
        st = st ? st : dalloc_n(&C->roots, nc, s);
        if (st == FGB_OK) {
            {
                FGB_KSCOPE("k_cc_keys", s);
                k_cc_keys<<<grid1d(n, 256), 256, 0, s>>>(root, size, n, slot, keys, vals, payload);
            }
            st = radix_sort_cells(keys, vals, nc, n + 1, payload, sorted, okeys, ws, s);
        }
        if (st == FGB_OK) {
            {
                FGB_KSCOPE("k_cc_ids", s);
                k_cc_ids<<<grid1d(nc, 256), 256, 0, s>>>(sorted, nc, id_of_root, C->sizes, C->roots);
            }
            {
                FGB_KSCOPE("k_cc_label", s);
                k_cc_label<<<grid1d(n, 256), 256, 0, s>>>(root, id_of_root, n, C->cluster_idx);
            }
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) st = fail(FGB_ERR_CUDA, "cluster labelling failed: %s", cudaGetErrorString(e));
        }
    }
    C->nc = nc;
    dfree(parent, s);
    dfree(root, s);
    dfree(size, s);
    dfree(flag, s);
    dfree(slot, s);
    dfree(err, s);
    dfree(keys, s);
    dfree(vals, s);
    dfree(okeys, s);
    dfree(payload, s);
    dfree(sorted, s);
    dfree(ws, s);
    dfree(id_of_root, s);
    if (st != FGB_OK) {
        fgb_cluster_destroy(C);
        return st;
    }
    *out = C;
    return FGB_OK;
}

extern "C" void fgb_cluster_destroy(fgb_clusters *C) {
    if (!C) return;
    dfree(C->cluster_idx, C->stream);
    dfree(C->sizes, C->stream);
    dfree(C->roots, C->stream);
    delete C;
}

extern "C" int fgb_cluster_result(const fgb_clusters *C, int64_t *num_clusters, const int32_t **cluster_idx,
                                  const int32_t **sizes) {
    if (!C) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    if (num_clusters) *num_clusters = C->nc;
    if (cluster_idx) *cluster_idx = C->cluster_idx;
    if (sizes) *sizes = C->sizes;
    return FGB_OK;
}

extern "C" int fgb_cluster_properties(const fgb_clusters *C, const fgb_box *box, const float *points,
                                      float *centers, float *gyration, void *stream) {
    clear_error();
    if (!C || !box || (C->n > 0 && (!points || !centers || !gyration))) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    BoxHost b;
    FGB_TRY(make_box(box, &b));
    if (C->nc == 0) return FGB_OK;
    cudaStream_t s = as_stream(stream);
    double *sums = nullptr, *g = nullptr;
    int st = dalloc_n(&sums, 3 * C->nc, s);
    st = st ? st : dalloc_n(&g, 6 * C->nc, s);
    if (st == FGB_OK) {
        cudaMemsetAsync(sums, 0, sizeof(double) * 3 * C->nc, s);
        cudaMemsetAsync(g, 0, sizeof(double) * 6 * C->nc, s);
        {
            FGB_KSCOPE("k_cl_offsets", s);
            k_cl_offsets<<<grid1d(C->n, 256), 256, 0, s>>>(b.f, points, C->n, C->cluster_idx, C->roots, sums);
        }
        {
            FGB_KSCOPE("k_cl_gyration", s);
            k_cl_gyration<<<grid1d(C->n, 256), 256, 0, s>>>(b.f, points, C->n, C->cluster_idx, C->roots, C->sizes,
                                                             sums, g);
        }
        {
            FGB_KSCOPE("k_cl_finish", s);
            k_cl_finish<<<grid1d(C->nc, 256), 256, 0, s>>>(b.f, points, C->nc, C->roots, C->sizes, sums, g, centers,
                                                           gyration);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = fail(FGB_ERR_CUDA, "cluster properties failed: %s", cudaGetErrorString(e));
    }
    dfree(sums, s);
    dfree(g, s);
    return st;
}
