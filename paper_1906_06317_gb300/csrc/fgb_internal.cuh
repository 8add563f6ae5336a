// Internal declarations shared by the libfgb translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <vector>

#include "fgb.h"

namespace fgb {

// ------------------------------------------------------------------ errors

int fail(int code, const char *fmt, ...);
void clear_error();

#define FGB_CUDA(expr)                                                                                   \
    do {                                                                                                 \
        cudaError_t fgb_e_ = (expr);                                                                     \
        if (fgb_e_ != cudaSuccess)                                                                       \
            return ::fgb::fail(FGB_ERR_CUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(fgb_e_), \
                               __FILE__, __LINE__);                                                      \
    } while (0)

#define FGB_LAUNCH_CHECK() FGB_CUDA(cudaGetLastError())

#define FGB_TRY(expr)              \
    do {                           \
        int fgb_s_ = (expr);       \
        if (fgb_s_ != FGB_OK)      \
            return fgb_s_;         \
    } while (0)

// Stream-ordered device allocation (a memory pool of the library's own, capi.cu).
int dalloc(void **p, size_t bytes, cudaStream_t s);
void dfree(void *p, cudaStream_t s);
int trim_memory();
int set_memory_cache(size_t bytes);
// A pinned host slot of 64 bytes for status words copied back by asynchronous calls;
// pinned_release hands it back, to be reused once `after` (nullable, then owned) has
// completed.
int pinned_slot(void **p);
void pinned_release(void *p, cudaEvent_t after);
template <class T>
int dalloc_n(T **p, size_t n, cudaStream_t s) {
    return dalloc(reinterpret_cast<void **>(p), n * sizeof(T), s);
}

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }
int num_sms();

// Every kernel launch goes through a KernelScope: it counts the launch and, when timing
// is enabled, brackets it with CUDA events on the launching stream.
void note_launch(const char *name, cudaStream_t s, bool begin);
struct KernelScope {
    const char *name;
    cudaStream_t s;
    KernelScope(const char *n, cudaStream_t st) : name(n), s(st) { note_launch(name, s, true); }
    ~KernelScope() { note_launch(name, s, false); }
};
#define FGB_KSCOPE_CAT2(a, b) a##b
#define FGB_KSCOPE_CAT(a, b) FGB_KSCOPE_CAT2(a, b)
#define FGB_KSCOPE(name, s) ::fgb::KernelScope FGB_KSCOPE_CAT(fgb_kscope_, __LINE__)(name, s)

// ------------------------------------------------------------------ box

// FP32 view of the box for the fast paths.  Box vectors a1 = (Lx,0,0),
// a2 = (a2x, Ly, 0), a3 = (a3x, a3y, Lz).  *_hi + *_lo splits carry the FP64 value to
// about 48 bits so a reduction by a whole box vector loses no accuracy.
struct BoxF {
    float L[3];
    float a2x, a3x, a3y;
    float inv00, inv01, inv02, inv11, inv12, inv22;  // upper-triangular M^-1
    float invL[3];
    float Lhi[3], Llo[3];
    float a2x_hi, a2x_lo, a3x_hi, a3x_lo, a3y_hi, a3y_lo;
};

// FP64 view for the exact decision sequence (identical operations to the definition).
struct BoxD {
    double L[3];
    double invL[3];
    double a2x, a3x, a3y;
};

struct BoxHost {
    double p[6];  // Lx Ly Lz xy xz yz
    double M[3][3];
    double Minv[3][3];
    double w[3];  // perpendicular widths
    double wmin;
    // 2D box (Lz = 0 on input, xz = yz = 0, every z coordinate 0): p[2] then holds an
    // internal thickness of twice the in-plane width, so no z image is ever within a
    // legal r_max, and the grid gets three z layers with the points in the middle one.
    int is2d;
    BoxF f;
    BoxD d;
};

int make_box(const fgb_box *in, BoxHost *out);

// Smallest double t with sqrt(t) >= R (IEEE sqrt, round to nearest): r >= R <=> r2 >= T(R).
double sqrt_threshold(double R);

// ------------------------------------------------------------------ cell grid

constexpr double kCellMargin = 1.0 / 256.0;  // relative slack between cell width and r_cell
constexpr int kMaxStencil = 8;               // largest stencil half-width

struct GridHost {
    int nc[3];
    int64_t ncell;
    double wc[3];        // perpendicular cell widths w_k / nc_k
    double ext;          // bound on |component| of a cell-local coordinate
    double origin_extent;
};

// Device tables of cell-corner origins along each axis, FP64 split in hi/lo floats:
// O_x = Tx[cx] + Txy[cy] + Txz[cz], O_y = Ty[cy] + Tyz[cz], O_z = Tz[cz].
struct OriginTables {
    const float2 *Tx, *Txy, *Txz, *Ty, *Tyz, *Tz;
};

}  // namespace fgb

// ------------------------------------------------------------------ handles

struct fgb_nq {
    fgb::BoxHost box;
    fgb::GridHost grid;
    const float *points;  // caller's (n,3)
    int64_t n;
    double r_cell;
    float4 *sorted;        // (n) cell-local xyz + index bits
    uint32_t *sorted_cell; // (n)
    uint32_t *cell_start;  // (ncell+1)
    float2 *origin_buf;    // all origin tables, packed
    fgb::OriginTables org;
    cudaStream_t stream;
    int kind;              // 0: cell list, 1: bounding-volume hierarchy (sorted = points in Morton order),
                           // 2: box and points only (consumers of a given NeighborList)
    void *bvh;             // kind 1: n-1 internal nodes (aabb.cu)
    int bvh_moved;         // kind 1: wrapping moved some point
    // query cells the cell-tile kernels walk: all cells unless a sharded call (shard.cu)
    // narrows them to [walk_lo, walk_hi) for its duration
    int walk_set;
    int64_t walk_lo, walk_hi;
};

// Steinhardt state (steinhardt.cu, order.cu): per-particle Q_lm, m = 0..l, and the
// neighbor counts of the last compute.
struct fgb_steinhardt {
    int l;
    int64_t n;
    float2 *Q;                  // (n, l+1): (1/n_i) sum_j Y_lm, or its neighbor average
    int32_t *nn;
    const fgb_nlist *last_nlist;
    cudaStream_t stream;
    int averaged;               // Q holds the neighbor-averaged Qbar_lm
    float2 *Qtmp;               // (n, l+1) scratch of the averaging
    float *w3j;                 // (2l+1)^2 Wigner 3j table (l l l; m1 m2 -m1-m2)
};

struct fgb_nlist {
    int64_t n_query, n_points, n_pairs;
    int32_t *qi, *pj, *counts;
    float *dist;
    int64_t *segments;
    int64_t escalations;
    int symmetric;
    int kind;  // 0 ball, 1 knn, 2 user arrays
    cudaStream_t stream;
    // asynchronous ball query (fgb_nq_query_async) in flight until fgb_nlist_wait: the
    // arrays hold `capacity` pairs; status words come back to `hstatus` (pinned) and
    // `done` follows their copy
    int pending, repaired;
    fgb_nq *src;
    double r_max;
    int exclude;
    int64_t capacity;
    void *dstatus, *hstatus;
    cudaEvent_t done;
};

namespace fgb {
// Completes an asynchronous list (waits, checks, rewrites it when it did not fit); every
// call that reads a list goes through it.  No-op for a complete list.
int nlist_ready(const fgb_nlist *nl);
}  // namespace fgb

namespace fgb {

// Sorted view of query points for a query launch (either the NeighborQuery's own
// sorted arrays or a separately binned copy of the query points).
struct QueryPoints {
    const float4 *sorted;
    const uint32_t *cell;
    const float *orig;  // (nq, 3) original coordinates
    int64_t n;
    bool self;
    // owned buffers (non-null when a separate copy was binned)
    float4 *own_sorted;
    uint32_t *own_cell;
};

int bin_points(const BoxHost &box, const GridHost &grid, const OriginTables &org, const float *pts, int64_t n,
               float4 *sorted, uint32_t *sorted_cell, uint32_t *cell_start, cudaStream_t s);
int grid_for(const BoxHost &box, double r_cell, int64_t n, GridHost *g);
int prepare_queries(fgb_nq *nq, const float *qpts, int64_t n_query, cudaStream_t s, QueryPoints *out);
void release_queries(QueryPoints *q, cudaStream_t s);

// Stencil set-up for a query radius R over nq's cell grid (query.cu): walked
// half-widths, the FP32 offset table (device, caller frees `table`) and the FP32 error
// bound on r^2 for pairs up to distance R.
struct StencilPlan {
    int s[3];       // half-width walked per axis (axes not scanned whole)
    int ts[3];      // half-width of the offset table (mode 0)
    int full[3];    // axis scanned whole once
    int mode;       // 0: fixed per-cell image offsets, 1: rint reduction per candidate
    float4 *table;  // owned (mode 0)
    double eps_d;   // bound on the FP32 error of one displacement component
    double Lsum;
};
int plan_stencil(const fgb_nq *nq, double R, int s_table_min, cudaStream_t st, StencilPlan *p);
// Same plan without device work; the mode-0 offset table is returned on the host.
int plan_stencil_host(const BoxHost &b, const GridHost &g, double R, int s_table_min, StencilPlan *p,
                      std::vector<float4> *table);
double r2_error_bound(const StencilPlan &p, double R);
// The same bound from a per-component displacement error eps_d (box vector length sum Lsum).
double r2_error_bound_eps(double eps_d, double Lsum, double R);
// FP32 band [lo, hi) around the exact threshold T, widened by `delta` and rounded outward.
void band_around(double T, double delta, float *lo, float *hi);

// Bounding-volume-hierarchy neighbor query (aabb.cu).
int aabb_build(fgb_nq *nq, cudaStream_t s);
void aabb_free(fgb_nq *nq);
int aabb_ball_query(fgb_nq *nq, const float *query_points, int64_t n_query, const fgb_query_args *args,
                    cudaStream_t s, fgb_nlist *nl);
int aabb_knn_query(fgb_nq *nq, const float *query_points, int64_t n_query, const fgb_query_args *args,
                   cudaStream_t s, fgb_nlist *nl);
// Sorts every segment of a list by point index in place (warp per segment, rows of at
// most cap entries staged in shared memory); tile.cu.
int sort_segments(const int64_t *seg, int64_t nq, int cap, int64_t npoints, int32_t *qi, int32_t *pj, float *dist,
                  cudaStream_t s);
// Ball-query write for rows too long for the write kernel's shared rows: hits appended to
// each query's segment in the list, unsorted (tile.cu; follow with sort_segments).
int tile_write_global(const fgb_nq *nq, const StencilPlan &p, double R, int exclude, int *err, const int64_t *seg,
                      const uint32_t *counts, int32_t *qi, int32_t *pj, float *dist, cudaStream_t s);

// Cell-tile kernels (tile.cu): one warp per query cell, self queries on the shift route.
bool tile_ok(const StencilPlan &p);
// Whether the grid gives the warp-per-cell kernels enough warps and short enough rows:
// at least 4 cells per SM and at most 64 points per cell on average (a small box with a
// few crowded cells runs faster one thread per query).
bool tile_worth(const fgb_nq *nq);
bool force_thread_kernels();
bool split_kernels_enabled();
// FGB_TILE_KERNELS=1: the cell-tile kernels wherever they apply, however small the grid.
bool force_tile_kernels();
int tile_count(const fgb_nq *nq, const StencilPlan &p, double R, int exclude, unsigned long long *esc, int *err,
               uint32_t *counts, cudaStream_t s);
size_t tile_write_smem(int cap);
// kNN by radius over cell tiles (self queries, 27-cell stencil, m <= 63); queries it
// cannot settle are appended (sorted positions) to `list`.
int tile_knn(const fgb_nq *nq, const StencilPlan &p, int k, int m, int exclude, int32_t *qi, int32_t *pj, float *dist,
             int32_t *counts, int *list, int *list_count, cudaStream_t s);
int tile_write(const fgb_nq *nq, const StencilPlan &p, double R, int exclude, int *err, const int64_t *seg,
               const uint32_t *counts, int cap, int32_t *qi, int32_t *pj, float *dist, cudaStream_t s);

// NeighborList count and write of a self ball query on the cell tiles (nlist.cu): the
// count tests each unordered pair once over half stencils; the write sorts each cell's
// pruned stencil by point index once and stores every hit in place.  FGB_NL_KERNELS=0
// keeps tile_count / tile_write instead.
bool nl_kernels_enabled();
int nl_count(const fgb_nq *nq, const StencilPlan &p, double R, int exclude, unsigned long long *esc, int *err,
             uint32_t *counts, cudaStream_t s);
// capacity >= 0: the asynchronous form: cap (the longest row) is not known and the arrays
// hold capacity pairs; nothing is written if seg[nqq] > capacity, and a row the stage
// fallback cannot hold sets *err = 1 (the caller rewrites the list synchronously).
int nl_write(const fgb_nq *nq, const StencilPlan &p, double R, int exclude, int *err, const int64_t *seg,
             const uint32_t *counts, int cap, int64_t nqq, int32_t *qi, int32_t *pj, float *dist, cudaStream_t s,
             int64_t capacity = -1);

// RDF bin parameters for an error bound G2 on r^2 (rdf.cu).
struct BinParams;
BinParams bin_params(int bins, double rmin, double rmax, double G2, const float2 *band, const std::vector<double> &T);

// Exclusive scan helpers (scan.cu).  out has n+1 entries (out[n] = total).
int scan_u32_i64(const uint32_t *in, int64_t *out, int64_t n, uint32_t *max_out, cudaStream_t s);
int scan_u32_u32(const uint32_t *in, uint32_t *out, int64_t n, cudaStream_t s);
size_t scan_ws_bytes(int64_t n);
int scan_u32_u32_ws(const uint32_t *in, uint32_t *out, int64_t n, void *ws, cudaStream_t s);

// Stable radix sort of (cell key, point index) with caller workspace of sort_ws_bytes(n)
// bytes; the final pass writes payload[index] records and keys in sorted order.
size_t sort_ws_bytes(int64_t n);
int radix_sort_cells(uint32_t *keys, uint32_t *vals, int64_t n, int64_t ncell, const float4 *payload, float4 *out_sorted,
                     uint32_t *out_keys, void *ws, cudaStream_t s);
int launch_cell_start(const uint32_t *skeys, int64_t n, int64_t ncell, uint32_t *start, cudaStream_t s);
// Cell-list build into caller buffers (origin tables, sorted records, keys, starts,
// radix workspace); launches only, no allocation.
int bin_points_into(const BoxHost &box, const GridHost &grid, const float *pts, int64_t n, float2 *origin_buf,
                    OriginTables *org, float4 *sorted, uint32_t *sorted_cell, uint32_t *cell_start, uint32_t *keys,
                    uint32_t *vals, float4 *local, void *sort_ws, cudaStream_t s);
// Mode-0 offset table of a plan into a caller buffer.
int launch_offset_table(const BoxHost &b, const GridHost &g, const StencilPlan &p, float4 *table, cudaStream_t st);

}  // namespace fgb
