// Box set-up and the cell-list build (Section "General Utilities": the cell-list
// NeighborQuery): box wrap + fractional transform, cell index per point, stable LSD
// radix sort of (cell, index), cell start offsets.
#include <cmath>
#include <cstring>

#include "fgb_device.cuh"

namespace fgb {

// ------------------------------------------------------------------ host: box

static void split(double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

int make_box(const fgb_box *in, BoxHost *b) {
    if (!in) return fail(FGB_ERR_INVALID_ARG, "box is NULL");
    double p[6] = {in->Lx, in->Ly, in->Lz, in->xy, in->xz, in->yz};
    for (int k = 0; k < 6; ++k)
        if (!std::isfinite(p[k])) return fail(FGB_ERR_INVALID_ARG, "box parameter %d is not finite", k);
    b->is2d = p[2] == 0.0;
    if (b->is2d) {
        // freud's 2D box: Lz = 0.  The plane's widths are Lx Ly / |a2| (across a1's
        // faces) and Ly; the internal thickness is twice the smaller one.
        if (p[4] != 0.0 || p[5] != 0.0) return fail(FGB_ERR_INVALID_ARG, "a 2D box (Lz = 0) must have xz = yz = 0");
        if (!(p[0] > 0 && p[1] > 0)) return fail(FGB_ERR_INVALID_ARG, "box lengths must be positive");
        const double w0 = p[0] * p[1] / std::sqrt(p[3] * p[1] * p[3] * p[1] + p[1] * p[1]);
        p[2] = 2.0 * std::fmin(w0, p[1]);
    } else if (!(p[0] > 0 && p[1] > 0 && p[2] > 0)) {
        return fail(FGB_ERR_INVALID_ARG, "box lengths must be positive (Lz = 0 for a 2D box)");
    }
    memcpy(b->p, p, sizeof(p));
    const double a2x = p[3] * p[1], a3x = p[4] * p[2], a3y = p[5] * p[2];
    double M[3][3] = {{p[0], a2x, a3x}, {0.0, p[1], a3y}, {0.0, 0.0, p[2]}};
    memcpy(b->M, M, sizeof(M));
    // inverse of the upper-triangular matrix
    double Mi[3][3] = {{0}};
    Mi[0][0] = 1.0 / p[0];
    Mi[1][1] = 1.0 / p[1];
    Mi[2][2] = 1.0 / p[2];
    Mi[0][1] = -a2x / (p[0] * p[1]);
    Mi[1][2] = -a3y / (p[1] * p[2]);
    Mi[0][2] = (a2x * a3y - a3x * p[1]) / (p[0] * p[1] * p[2]);
    memcpy(b->Minv, Mi, sizeof(Mi));
    // perpendicular widths: 1 / |row k of M^-1|
    for (int k = 0; k < 3; ++k) {
        double s = 0;
        for (int j = 0; j < 3; ++j) s += Mi[k][j] * Mi[k][j];
        b->w[k] = 1.0 / std::sqrt(s);
    }
    b->wmin = b->is2d ? std::fmin(b->w[0], b->w[1]) : std::fmin(b->w[0], std::fmin(b->w[1], b->w[2]));
    BoxF &f = b->f;
    for (int k = 0; k < 3; ++k) {
        f.L[k] = (float)p[k];
        f.invL[k] = (float)(1.0 / p[k]);
        split(p[k], f.Lhi[k], f.Llo[k]);
    }
    f.a2x = (float)a2x;
    f.a3x = (float)a3x;
    f.a3y = (float)a3y;
    split(a2x, f.a2x_hi, f.a2x_lo);
    split(a3x, f.a3x_hi, f.a3x_lo);
    split(a3y, f.a3y_hi, f.a3y_lo);
    f.inv00 = (float)Mi[0][0];
    f.inv01 = (float)Mi[0][1];
    f.inv02 = (float)Mi[0][2];
    f.inv11 = (float)Mi[1][1];
    f.inv12 = (float)Mi[1][2];
    f.inv22 = (float)Mi[2][2];
    BoxD &d = b->d;
    for (int k = 0; k < 3; ++k) {
        d.L[k] = p[k];
        d.invL[k] = 1.0 / p[k];
    }
    d.a2x = a2x;
    d.a3x = a3x;
    d.a3y = a3y;
    return FGB_OK;
}

double sqrt_threshold(double R) {
    if (!(R > 0.0)) return 0.0;
    double t = R * R;
    while (std::sqrt(t) < R) t = std::nextafter(t, INFINITY);
    for (;;) {
        double p = std::nextafter(t, 0.0);
        if (p >= 0.0 && std::sqrt(p) >= R && p < t)
            t = p;
        else
            break;
    }
    return t;
}

int grid_for(const BoxHost &box, double r_cell, int64_t n, GridHost *g) {
    if (!(r_cell > 0.0) || !std::isfinite(r_cell)) return fail(FGB_ERR_INVALID_ARG, "r_cell must be positive");
    // total cell count stays below ~4 cells per point (and 2^26) so empty space is cheap
    const double cap_total = std::fmax(64.0, std::fmin(67108864.0, 4.0 * (double)n + 64.0));
    double rc = r_cell;
    for (int it = 0; it < 200; ++it) {
        double tot = 1;
        for (int k = 0; k < 3; ++k) {
            double q = std::floor(box.w[k] / (rc * (1.0 + kCellMargin)));
            int nk = q > 1024.0 ? 1024 : (int)q;
            if (nk < 1) nk = 1;
            if (k == 2 && box.is2d) nk = 3;  // z layers below, at and above the plane
            g->nc[k] = nk;
            tot *= nk;
        }
        if (tot <= cap_total) break;
        rc *= 1.05;
    }
    g->ncell = (int64_t)g->nc[0] * g->nc[1] * g->nc[2];
    for (int k = 0; k < 3; ++k) g->wc[k] = box.w[k] / g->nc[k];
    // Largest cell-local component.  In a 2D box every point has z = 0 and lies in the
    // middle layer with the same local z, so candidates of the same layer give dz = 0
    // exactly and the z row adds no error.
    double ext = 0;
    for (int r = 0; r < (box.is2d ? 2 : 3); ++r) {
        double e = 0;
        for (int c = 0; c < 3; ++c) e += std::fabs(box.M[r][c]) * (1.0 / g->nc[c] + 1e-5);
        ext = std::fmax(ext, e);
    }
    g->ext = ext;
    return FGB_OK;
}

// ------------------------------------------------------------------ device: binning

__global__ void k_bin(BoxF b, BoxD bd, GridDev g, OriginTables org, const float *__restrict__ pts, int64_t n,
                      uint32_t *__restrict__ keys, uint32_t *__restrict__ vals, float4 *__restrict__ local) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
    uint32_t key;
    float4 loc;
    bin_point(b, bd, g, org, x, y, z, key, loc);
    loc.w = __int_as_float((int)i);
    keys[i] = key;
    vals[i] = (uint32_t)i;
    local[i] = loc;
}

// ------------------------------------------------------------------ radix sort

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // each warp owns 512 consecutive items

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t *__restrict__ keys, int64_t n, int shift,
                                                             int nblocks, uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[kRadix];
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) h[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int k = 0; k < kSortItems; ++k) {
        int64_t i = base + k * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) hist[(int64_t)d * nblocks + blockIdx.x] = h[d];
}

// Stable scatter of one tile.  Warp w ranks its 512 items in 16 rounds of 32 with
// match_any; per-warp digit counts are then scanned across warps.  When `payload` is
// given the final pass moves float4 records (looked up by the carried index).
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint32_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t n, int shift, int nblocks,
    const uint32_t *__restrict__ offs, uint32_t *__restrict__ okeys, uint32_t *__restrict__ ovals,
    const float4 *__restrict__ payload, float4 *__restrict__ opayload) {
    __shared__ uint32_t wcount[kSortThreads / 32][kRadix];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = lane; d < kRadix; d += 32) wcount[w][d] = 0;
    __syncwarp();
    const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)w * (kSortItems * 32);
    uint32_t rank[kSortItems];
    uint32_t digit[kSortItems];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int64_t i = base + r * 32 + lane;
        bool valid = i < n;
        uint32_t d = valid ? ((keys[i] >> shift) & (kRadix - 1)) : (uint32_t)kRadix;  // kRadix = none
        digit[r] = d;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t pre = valid ? wcount[w][d] : 0u;
        __syncwarp();
        if (valid && (peers & lt) == 0) wcount[w][d] = pre + __popc(peers);
        rank[r] = pre + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();
    // exclusive scan over warps per digit, plus the tile's global offset
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
        uint32_t run = offs[(int64_t)d * nblocks + blockIdx.x];
        for (int ww = 0; ww < kSortThreads / 32; ++ww) {
            uint32_t c = wcount[ww][d];
            wcount[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int64_t i = base + r * 32 + lane;
        if (i < n) {
            uint32_t pos = wcount[w][digit[r]] + rank[r];
            okeys[pos] = keys[i];
            uint32_t v = vals[i];
            if (opayload)
                opayload[pos] = payload[v];
            else
                ovals[pos] = v;
        }
    }
}

__global__ void k_cell_start(const uint32_t *__restrict__ skeys, int64_t n, int64_t ncell, uint32_t *__restrict__ start) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t cur = skeys[p];
    int64_t prev = p == 0 ? -1 : (int64_t)skeys[p - 1];
    for (int64_t c = prev + 1; c <= cur; ++c) start[c] = (uint32_t)p;
    if (p == n - 1)
        for (int64_t c = cur + 1; c <= ncell; ++c) start[c] = (uint32_t)n;
}

__global__ void k_fill_u32(uint32_t *p, int64_t n, uint32_t v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

static int grid1d(int64_t n, int t) { return (int)((n + t - 1) / t); }

size_t sort_ws_bytes(int64_t n) {
    const int64_t nblocks = (n + kSortTile - 1) / kSortTile;
    const int64_t hist = nblocks * kRadix;
    return 2 * sizeof(uint32_t) * (size_t)n + sizeof(uint32_t) * (size_t)(2 * hist + 1) + scan_ws_bytes(hist) + 1024;
}

int radix_sort_cells(uint32_t *keys, uint32_t *vals, int64_t n, int64_t ncell, const float4 *payload, float4 *out_sorted,
                     uint32_t *out_keys, void *ws, cudaStream_t s) {
    const int64_t nblocks = (n + kSortTile - 1) / kSortTile;
    const int64_t nh = nblocks * kRadix;
    char *w = static_cast<char *>(ws);
    uint32_t *kB = reinterpret_cast<uint32_t *>(w);
    uint32_t *vB = kB + n;
    uint32_t *hist = vB + n;
    uint32_t *offs = hist + nh;
    void *scan_ws = reinterpret_cast<void *>((reinterpret_cast<uintptr_t>(offs + nh + 1) + 255) & ~uintptr_t(255));
    int bits = 0;
    while (bits < 32 && ((uint64_t)1 << bits) < (uint64_t)ncell) ++bits;
    const int passes = (bits + kRadixBits - 1) / kRadixBits;
    uint32_t *ck = keys, *cv = vals, *nk = kB, *nv = vB;
    if (passes == 0) {
        FGB_CUDA(cudaMemcpyAsync(out_sorted, payload, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s));
        FGB_CUDA(cudaMemcpyAsync(out_keys, keys, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = pass * kRadixBits;
        const bool last = pass == passes - 1;
        {
            FGB_KSCOPE("k_radix_hist", s);
            k_radix_hist<<<(unsigned)nblocks, kSortThreads, 0, s>>>(ck, n, shift, (int)nblocks, hist);
        }
        FGB_TRY(scan_u32_u32_ws(hist, offs, nh, scan_ws, s));
        {
            FGB_KSCOPE("k_radix_scatter", s);
            k_radix_scatter<<<(unsigned)nblocks, kSortThreads, 0, s>>>(ck, cv, n, shift, (int)nblocks, offs,
                                                                       last ? out_keys : nk, nv, last ? payload : nullptr,
                                                                       last ? out_sorted : nullptr);
        }
        std::swap(ck, nk);
        std::swap(cv, nv);
    }
    FGB_LAUNCH_CHECK();
    return FGB_OK;
}

int launch_cell_start(const uint32_t *skeys, int64_t n, int64_t ncell, uint32_t *start, cudaStream_t s) {
    if (n == 0) {
        FGB_KSCOPE("k_fill_u32", s);
        k_fill_u32<<<grid1d(ncell + 1, 256), 256, 0, s>>>(start, ncell + 1, 0u);
    } else {
        FGB_KSCOPE("k_cell_start", s);
        k_cell_start<<<grid1d(n, 256), 256, 0, s>>>(skeys, n, ncell, start);
    }
    FGB_LAUNCH_CHECK();
    return FGB_OK;
}

int bin_points(const BoxHost &box, const GridHost &grid, const OriginTables &org, const float *pts, int64_t n,
               float4 *sorted, uint32_t *sorted_cell, uint32_t *cell_start, cudaStream_t s) {
    if (n == 0) return launch_cell_start(nullptr, 0, grid.ncell, cell_start, s);
    GridDev g = {{grid.nc[0], grid.nc[1], grid.nc[2]}};
    uint32_t *keys = nullptr, *vals = nullptr;
    float4 *local = nullptr;
    void *ws = nullptr;
    int st = dalloc_n(&keys, n, s);
    st = st ? st : dalloc_n(&vals, n, s);
    st = st ? st : dalloc_n(&local, n, s);
    st = st ? st : dalloc(&ws, sort_ws_bytes(n), s);
    if (st == FGB_OK) {
        {
            FGB_KSCOPE("k_bin", s);
            k_bin<<<grid1d(n, 256), 256, 0, s>>>(box.f, box.d, g, org, pts, n, keys, vals, local);
        }
        st = radix_sort_cells(keys, vals, n, grid.ncell, local, sorted, sorted_cell, ws, s);
        st = st ? st : launch_cell_start(sorted_cell, n, grid.ncell, cell_start, s);
    }
    dfree(keys, s);
    dfree(vals, s);
    dfree(local, s);
    dfree(ws, s);
    return st;
}

// Origin tables (see OriginTables): FP64 values split hi/lo, built on the device so the
// build needs no host synchronisation.
__global__ void k_origin_tables(double m00, double m01, double m11, double m02, double m12, double m22, int nx, int ny,
                                int nz, float2 *buf) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int total = nx + 2 * ny + 3 * nz;
    if (t >= total) return;
    double v;
    if (t < nx) {
        v = m00 * ((double)t / nx - 0.5);
    } else if (t < nx + ny) {
        int c = t - nx;
        v = m01 * ((double)c / ny - 0.5);
    } else if (t < nx + 2 * ny) {
        int c = t - nx - ny;
        v = m11 * ((double)c / ny - 0.5);
    } else {
        int r = t - nx - 2 * ny;
        int which = r / nz, c = r % nz;
        double m = which == 0 ? m02 : (which == 1 ? m12 : m22);
        v = m * ((double)c / nz - 0.5);
    }
    float hi = (float)v;
    buf[t] = make_float2(hi, (float)(v - (double)hi));
}

static int build_origin_tables(const BoxHost &box, const GridHost &g, float2 **buf, OriginTables *org, cudaStream_t s) {
    const int nx = g.nc[0], ny = g.nc[1], nz = g.nc[2];
    const int total = nx + 2 * ny + 3 * nz;
    FGB_TRY(dalloc_n(buf, total, s));
    {
        FGB_KSCOPE("k_origin_tables", s);
        k_origin_tables<<<(total + 255) / 256, 256, 0, s>>>(box.M[0][0], box.M[0][1], box.M[1][1], box.M[0][2], box.M[1][2],
                                                            box.M[2][2], nx, ny, nz, *buf);
    }
    FGB_LAUNCH_CHECK();
    org->Tx = *buf;
    org->Txy = *buf + nx;
    org->Ty = *buf + nx + ny;
    org->Txz = *buf + nx + 2 * ny;
    org->Tyz = *buf + nx + 2 * ny + nz;
    org->Tz = *buf + nx + 2 * ny + 2 * nz;
    return FGB_OK;
}

int bin_points_into(const BoxHost &box, const GridHost &grid, const float *pts, int64_t n, float2 *origin_buf,
                    OriginTables *org, float4 *sorted, uint32_t *sorted_cell, uint32_t *cell_start, uint32_t *keys,
                    uint32_t *vals, float4 *local, void *sort_ws, cudaStream_t s) {
    const int nx = grid.nc[0], ny = grid.nc[1], nz = grid.nc[2];
    const int total = nx + 2 * ny + 3 * nz;
    {
        FGB_KSCOPE("k_origin_tables", s);
        k_origin_tables<<<(total + 255) / 256, 256, 0, s>>>(box.M[0][0], box.M[0][1], box.M[1][1], box.M[0][2],
                                                            box.M[1][2], box.M[2][2], nx, ny, nz, origin_buf);
    }
    org->Tx = origin_buf;
    org->Txy = origin_buf + nx;
    org->Ty = origin_buf + nx + ny;
    org->Txz = origin_buf + nx + 2 * ny;
    org->Tyz = origin_buf + nx + 2 * ny + nz;
    org->Tz = origin_buf + nx + 2 * ny + 2 * nz;
    if (n == 0) return launch_cell_start(nullptr, 0, grid.ncell, cell_start, s);
    GridDev g = {{nx, ny, nz}};
    {
        FGB_KSCOPE("k_bin", s);
        k_bin<<<grid1d(n, 256), 256, 0, s>>>(box.f, box.d, g, *org, pts, n, keys, vals, local);
    }
    FGB_TRY(radix_sort_cells(keys, vals, n, grid.ncell, local, sorted, sorted_cell, sort_ws, s));
    return launch_cell_start(sorted_cell, n, grid.ncell, cell_start, s);
}

int prepare_queries(fgb_nq *nq, const float *qpts, int64_t n_query, cudaStream_t s, QueryPoints *q) {
    memset(q, 0, sizeof(*q));
    if (qpts == nullptr || qpts == nq->points) {
        q->sorted = nq->sorted;
        q->cell = nq->sorted_cell;
        q->orig = nq->points;
        q->n = nq->n;
        q->self = true;
        return FGB_OK;
    }
    if (n_query < 0) return fail(FGB_ERR_INVALID_ARG, "n_query must be >= 0");
    q->orig = qpts;
    q->n = n_query;
    q->self = false;
    uint32_t *start = nullptr;
    FGB_TRY(dalloc_n(&q->own_sorted, n_query, s));
    FGB_TRY(dalloc_n(&q->own_cell, n_query, s));
    FGB_TRY(dalloc_n(&start, nq->grid.ncell + 1, s));
    int st = bin_points(nq->box, nq->grid, nq->org, qpts, n_query, q->own_sorted, q->own_cell, start, s);
    dfree(start, s);
    q->sorted = q->own_sorted;
    q->cell = q->own_cell;
    return st;
}

void release_queries(QueryPoints *q, cudaStream_t s) {
    dfree(q->own_sorted, s);
    dfree(q->own_cell, s);
    q->own_sorted = nullptr;
    q->own_cell = nullptr;
}

}  // namespace fgb

using namespace fgb;

extern "C" int fgb_nq_create(const fgb_box *box, const float *points, int64_t n, double r_cell, void *stream,
                             fgb_nq **out) {
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
    nq->r_cell = r_cell;
    nq->stream = s;
    int st = make_box(box, &nq->box);
    st = st ? st : grid_for(nq->box, r_cell, n, &nq->grid);
    st = st ? st : build_origin_tables(nq->box, nq->grid, &nq->origin_buf, &nq->org, s);
    st = st ? st : dalloc_n(&nq->sorted, n, s);
    st = st ? st : dalloc_n(&nq->sorted_cell, n, s);
    st = st ? st : dalloc_n(&nq->cell_start, nq->grid.ncell + 1, s);
    st = st ? st : bin_points(nq->box, nq->grid, nq->org, points, n, nq->sorted, nq->sorted_cell, nq->cell_start, s);
    if (st != FGB_OK) {
        fgb_nq_destroy(nq);
        return st;
    }
    *out = nq;
    return FGB_OK;
}

extern "C" int fgb_nq_create_points(const fgb_box *box, const float *points, int64_t n, fgb_nq **out) {
    clear_error();
    if (!out) return fail(FGB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 0 || (n > 0 && !points)) return fail(FGB_ERR_INVALID_ARG, "points/n invalid");
    if (n >= (int64_t)1 << 31) return fail(FGB_ERR_CAPACITY, "at most 2^31-1 points");
    fgb_nq *nq = new fgb_nq();
    memset(nq, 0, sizeof(*nq));
    nq->points = points;
    nq->n = n;
    nq->kind = 2;
    const int st = make_box(box, &nq->box);
    if (st != FGB_OK) {
        delete nq;
        return st;
    }
    *out = nq;
    return FGB_OK;
}

extern "C" void fgb_nq_destroy(fgb_nq *nq) {
    if (!nq) return;
    dfree(nq->sorted, nq->stream);
    dfree(nq->sorted_cell, nq->stream);
    dfree(nq->cell_start, nq->stream);
    dfree(nq->origin_buf, nq->stream);
    if (nq->kind == 1) aabb_free(nq);
    delete nq;
}

extern "C" int fgb_nq_dims(const fgb_nq *nq, int32_t ncell[3], int64_t *n_points) {
    if (!nq) return fail(FGB_ERR_INVALID_ARG, "nq is NULL");
    if (ncell)
        for (int k = 0; k < 3; ++k) ncell[k] = nq->grid.nc[k];
    if (n_points) *n_points = nq->n;
    return FGB_OK;
}

extern "C" int fgb_nq_cells(const fgb_nq *nq, const float **sorted, const uint32_t **sorted_cell,
                            const uint32_t **cell_start) {
    if (!nq) return fail(FGB_ERR_INVALID_ARG, "nq is NULL");
    if (nq->kind != 0) return fail(FGB_ERR_UNSUPPORTED, "not a cell-list NeighborQuery");
    if (sorted) *sorted = reinterpret_cast<const float *>(nq->sorted);
    if (sorted_cell) *sorted_cell = nq->sorted_cell;
    if (cell_start) *cell_start = nq->cell_start;
    return FGB_OK;
}
