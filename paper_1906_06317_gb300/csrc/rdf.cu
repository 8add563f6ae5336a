// Radial distribution function (density module; reset=False accumulation of the
// Compute-class protocol in Section "Implementation").
//
// Fused query + histogram: pairs are never stored (the paper's lazy neighbor iterators,
// Section "General Utilities").  One thread per query point in cell order; for a self
// query each unordered pair is visited once (half stencil, same-cell pairs by sorted
// position) and counted twice.  Counts go to privatised shared-memory histograms
// (one copy per group of warps) merged into a global uint64 accumulator at block end
// (the thread-local histograms with lazy reduction of Section "Implementation").
// Pairs whose FP32 r2 lies inside the error band of a bin edge are appended to a list
// and binned by a second kernel with the defining FP64 sequence.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "fgb_tile.cuh"

struct fgb_rdf {
    int bins;
    double r_max, r_min;
    unsigned long long *hist;  // device, bins
    double *T;                 // device, exact r2 thresholds of the bins+1 edges
    std::vector<double> T_host;
    double norm;               // sum over frames of N_query * N_points / V (area in 2D)
    int dim;                   // 2 or 3 once a frame is accumulated, 0 before
    float2 *band;              // device, FP32 bands around the edges
    double band_delta;
    int2 *esc;
    int esc_cap;
    int *esc_count;            // device [0] count
    int64_t last_esc;
    cudaStream_t stream;
};

namespace fgb {

struct RdfArgs {
    Stencil S;
    BoxF bf;
    BoxD bd;
    const float4 *pts;
    const uint32_t *cell_start;
    const float4 *qs;
    const uint32_t *qcell;
    int64_t nq;
    const float *p_orig;
    const float *q_orig;
    int exclude;
    int half;
    int bins;
    int copies;
    BinParams P;
    const double *T;
    unsigned long long *hist;
    int2 *esc;
    int esc_cap;
    int *esc_count;
    unsigned weight;
};

BinParams bin_params(int bins, double rmin, double rmax, double G2, const float2 *band, const std::vector<double> &T) {
    BinParams P;
    P.bins = bins;
    const double invd = bins / (rmax - rmin);
    P.rmin = (float)rmin;
    P.invdelta = (float)invd;
    P.rmin_invdelta = (float)(rmin * invd);
    P.g2h = (float)(0.55 * G2 * invd);
    P.r2_fast = (float)(16.0 * G2);
    P.eps = (float)(8.0 * std::ldexp(1.0, -24) * (bins + rmin * invd + 2.0));
    float lo, hi;
    band_around(T[bins], G2, &lo, &hi);
    P.rmax_hi = hi;
    band_around(T[0], G2, &lo, &hi);
    P.rmin_lo = lo;
    P.band = band;
    return P;
}

__device__ __forceinline__ int exact_bin(const double *T, int bins, double e) {
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

// The same bin from a guess: the FP32 bin of sqrt(e), then stepped until
// T[b] <= e < T[b+1] holds in FP64 (T is increasing, so the result is the unique bin of
// the binary search; the guess is off by at most one in practice).
__device__ __forceinline__ int exact_bin_near(const double *T, int bins, double e, float rmin, float invdelta) {
    if (!(e >= T[0]) || !(e < T[bins])) return -1;
    int b = (int)((sqrtf((float)e) - rmin) * invdelta);
    b = min(max(b, 0), bins - 1);
    while (b > 0 && e < T[b]) --b;
    while (b + 1 < bins && e >= T[b + 1]) ++b;
    return b;
}

// HALF: self query with the half stencil; the pair (t, t) is never visited, so no index
// test is needed.  Otherwise a self query skips j == i explicitly.  LANES consecutive
// threads share a query (few queries: a small grid), thread g of the group taking the
// candidates beg + g, beg + g + LANES, ... of every stencil cell, so each candidate is
// still tested once.
template <bool SHARED, int MODE, bool HALF, int LANES>
__global__ void __launch_bounds__(256) k_rdf(RdfArgs a) {
    extern __shared__ uint32_t sh[];  // copies * bins
    if (SHARED) {
        for (int b = threadIdx.x; b < a.bins * a.copies; b += blockDim.x) sh[b] = 0;
        __syncthreads();
    }
    const int64_t tt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t t = tt / LANES;
    const uint32_t g = (uint32_t)(tt % LANES);
    uint32_t *my = sh + ((threadIdx.x >> 5) % a.copies) * a.bins;
    if (t < a.nq) {
        const float4 q = a.qs[t];
        const int i = __float_as_int(q.w);
        int cx, cy, cz;
        cell_coords(a.qcell[t], a.S.nc, cx, cy, cz);
        const int excl = a.exclude ? i : -1;
        for_stencil(a.S, cx, cy, cz, make_float3(q.x, q.y, q.z), HALF,
                    [&](int cell, float qx, float qy, float qz, bool center) {
                        uint32_t beg = __ldg(a.cell_start + cell);
                        const uint32_t end = __ldg(a.cell_start + cell + 1);
                        if (HALF && center) beg = max(beg, (uint32_t)t + 1u);
#pragma unroll 2
                        for (uint32_t p = beg + g; p < end; p += LANES) {
                            const float4 c = __ldg(a.pts + p);
                            const float3 d = cand_disp_m<MODE>(a.bf, c, qx, qy, qz);
                            const float r2 = r2_f32(d.x, d.y, d.z);
                            const int b = rdf_bin(a.P, r2);
                            if (b == -1) continue;
                            const int j = __float_as_int(c.w);
                            if (!HALF && j == excl) continue;
                            if (b >= 0) {
                                if (SHARED)
                                    atomicAdd(my + b, 1u);
                                else
                                    atomicAdd(a.hist + b, (unsigned long long)a.weight);
                            } else {
                                const int slot = atomicAdd(a.esc_count, 1);
                                if (slot < a.esc_cap) {
                                    a.esc[slot] = make_int2(i, j);
                                } else {
                                    const int be = exact_bin(a.T, a.bins, exact_r2_idx(a.bd, a.q_orig, i, a.p_orig, j));
                                    if (be >= 0) atomicAdd(a.hist + be, (unsigned long long)a.weight);
                                }
                            }
                        }
                    });
    }
    if (SHARED) {
        __syncthreads();
        for (int b = threadIdx.x; b < a.bins; b += blockDim.x) {
            uint32_t v = 0;
            for (int c = 0; c < a.copies; ++c) v += sh[c * a.bins + b];
            if (v) atomicAdd(a.hist + b, (unsigned long long)v * a.weight);
        }
    }
}

template <bool SHARED, int LANES>
static void launch_rdf_lanes(const RdfArgs &a, size_t smem, cudaStream_t s) {
    const unsigned grid = (unsigned)((a.nq * LANES + 255) / 256);
    if (a.half)
        k_rdf<SHARED, 0, true, LANES><<<grid, 256, smem, s>>>(a);
    else if (a.S.mode == 0)
        k_rdf<SHARED, 0, false, LANES><<<grid, 256, smem, s>>>(a);
    else
        k_rdf<SHARED, 1, false, LANES><<<grid, 256, smem, s>>>(a);
}

// Fewer than 128 queries per SM: 8 threads per query, fewer than 32: a warp per query
// (FGB_SPLIT_KERNELS=0: one thread).
template <bool SHARED>
static void launch_rdf(const RdfArgs &a, size_t smem, cudaStream_t s) {
    FGB_KSCOPE("k_rdf", s);
    if (a.nq < (int64_t)num_sms() * 32 && split_kernels_enabled())
        launch_rdf_lanes<SHARED, 32>(a, smem, s);
    else if (a.nq < (int64_t)num_sms() * 128 && split_kernels_enabled())
        launch_rdf_lanes<SHARED, 8>(a, smem, s);
    else
        launch_rdf_lanes<SHARED, 1>(a, smem, s);
}

// Band around each exact edge threshold, rounded outward.
__global__ void k_band(const double *__restrict__ T, int n, double delta, float2 *__restrict__ out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n) out[b] = make_float2(__double2float_rd(__dsub_rd(T[b], delta)), __double2float_ru(__dadd_ru(T[b], delta)));
}

// FP64 decisions of the listed band pairs.  SHARED: counted in a shared histogram per
// block and added to the global counts once per block and bin (the pairs crowd a few
// hundred bins, where one global atomic per pair contends).
constexpr int kEscSharedBins = 8192;

template <bool SHARED>
__global__ void k_rdf_escalated(RdfArgs a) {
    extern __shared__ uint32_t eh[];  // SHARED: bins
    if (SHARED) {
        for (int b = threadIdx.x; b < a.bins; b += blockDim.x) eh[b] = 0;
        __syncthreads();
    }
    const int n = min(*a.esc_count, a.esc_cap);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int2 p = a.esc[e];
        const int b =
            exact_bin_near(a.T, a.bins, exact_r2_idx(a.bd, a.q_orig, p.x, a.p_orig, p.y), a.P.rmin, a.P.invdelta);
        if (b >= 0) {
            if (SHARED)
                atomicAdd(eh + b, 1u);
            else
                atomicAdd(a.hist + b, (unsigned long long)a.weight);
        }
    }
    if (SHARED) {
        __syncthreads();
        for (int b = threadIdx.x; b < a.bins; b += blockDim.x)
            if (eh[b]) atomicAdd(a.hist + b, (unsigned long long)eh[b] * a.weight);
    }
}

static void launch_rdf_escalated(const RdfArgs &a, cudaStream_t s) {
    FGB_KSCOPE("k_rdf_escalated", s);
    if (a.bins <= kEscSharedBins)
        k_rdf_escalated<true><<<num_sms() * 2, 256, (size_t)a.bins * sizeof(uint32_t), s>>>(a);
    else
        k_rdf_escalated<false><<<num_sms() * 4, 256, 0, s>>>(a);
}

// ------------------------------------------------------------------ cell-tile RDF
//
// Self queries on the shift route: one warp per query cell A, taken from a work counter
// by persistent blocks.  The candidates of A's half stencil (A itself first, then the
// cells after it in (z, y, x) offset order) stream through the lanes 32 at a time,
// shifted into A's frame, while the warp loops over A's queries, read by a uniform
// shared-memory load.  Every lane tests one pair per round and no lane waits on another
// lane's trip count.  A's own points pair only with earlier queries of A, so each
// unordered pair is binned once (weight 2).  Each warp counts into its own shared
// histogram; the warps of a block merge theirs into the global counts at the end.

constexpr int kRdfTileWarps = 4;
constexpr int kRdfTileQ = 32;          // queries staged per pass
constexpr int kRdfOwnCap = 1024;       // candidates of a stencil with an owner table
constexpr int kRdfTileMaxBins = 1024;  // private histogram of every warp

struct RdfTileArgs {
    TileArgs t;
    BinParams P;
    const double *T;
    int bins;
    unsigned long long *hist;
    int2 *esc;
    int esc_cap;
    int *esc_count;
    unsigned weight;
    unsigned *work;
};

// A pair in [r_min, r_max) whose fast test failed: the band tables decide, else the pair
// is listed for the FP64 pass (or decided here when the list is full).
__device__ __noinline__ void rdf_tile_slow(const RdfTileArgs *ap, float r2, int i, int j, uint32_t *h) {
    const RdfTileArgs &a = *ap;
    const int b = rdf_bin_band(a.P, r2);
    if (b >= 0) {
        atomicAdd(h + b, 1u);
        return;
    }
    const int slot = atomicAdd(a.esc_count, 1);
    if (slot < a.esc_cap) {
        a.esc[slot] = make_int2(i, j);
    } else {
        const int be = exact_bin(a.T, a.bins, exact_r2_idx(a.t.bd, a.t.p_orig, i, a.t.p_orig, j));
        if (be >= 0) atomicAdd(a.hist + be, (unsigned long long)a.weight);
    }
}

// One staged candidate against the queries [0, nq) of the pass.  CENTER: the candidate
// may be one of A's own points, valid only against queries before it (tl < lim).
//
// The bin work sits behind the in-range test: about a third of the rounds have no lane
// in range (whole stencil cells lie beyond r_max of a query) and skip it.  The fast test
// is rdf_bin's; pairs that fail it go to rdf_tile_slow.
template <bool CENTER>
__device__ __forceinline__ void rdf_tile_rounds(const RdfTileArgs &a, const float4 *qs, int nq, const TileCand &c,
                                                int lim, uint32_t *h) {
    const float rhi = a.P.rmax_hi, rlo = a.P.rmin_lo;
    const float invd = a.P.invdelta, rmid = a.P.rmin_invdelta, g2h = a.P.g2h, eps = a.P.eps, r2f = a.P.r2_fast;
#pragma unroll 4
    for (int tl = 0; tl < nq; ++tl) {
        const float4 q = qs[tl];
        const float r2 = r2_f32(c.x - q.x, c.y - q.y, c.z - q.z);
        bool in = r2 < rhi && r2 >= rlo;
        if (CENTER) in = in && tl < lim;
        if (in) {
            const float inv = rsqrt_ftz(r2);
            const float x = fmaf(r2 * inv, invd, -rmid);
            const float fb = floorf(x);
            const float e = fmaf(g2h, inv, eps);
            if (r2 > r2f && fabsf((x - fb) - 0.5f) < 0.5f - e)
                atomicAdd(h + (int)fb, 1u);
            else
                rdf_tile_slow(&a, r2, __float_as_int(q.w), c.j, h);
        }
    }
}

__device__ __forceinline__ void rdf_tile_flush(uint32_t *h, int bins, unsigned long long *hist, unsigned weight) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    for (int b = lane; b < bins; b += 32) {
        const uint32_t v = h[b];
        if (v) {
            atomicAdd(hist + b, (unsigned long long)v * weight);
            h[b] = 0;
        }
    }
    __syncwarp();
}

template <int NS>
__device__ __forceinline__ void rdf_tile_body(const RdfTileArgs &a) {
    __shared__ TileStencilT<NS> sts[kRdfTileWarps];
    __shared__ float4 sq[kRdfTileWarps][kRdfTileQ];
    __shared__ float4 sbuf[kRdfTileWarps][64];  // candidates kept after the box test
    __shared__ uint8_t sown[kRdfTileWarps][kRdfOwnCap];  // owner table of the stencil
    extern __shared__ uint32_t shist[];  // kRdfTileWarps * bins
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *h = shist + warp * a.bins;
    for (int b = lane; b < a.bins; b += 32) h[b] = 0;
    __syncwarp();
    TileStencilT<NS> &ts = sts[warp];
    float4 *qs = sq[warp];
    float4 *buf = sbuf[warp];
    const unsigned lt = lanemask_lt();
    // a candidate farther than this (squared, FP32, with slack for the rounding of the
    // box distance) from the queries' bounding box cannot be in range of any of them
    const float reach2 = a.P.rmax_hi * (1.0f + 1e-5f);
    uint64_t tests = 0;  // pair tests since the last flush bound every private count
    for (;;) {
        unsigned w = 0;
        if (lane == 0) w = atomicAdd(a.work, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        const int64_t A = a.t.cell_lo + (int64_t)w;
        if (A >= a.t.ncell) break;
        const int begA = (int)__ldg(a.t.cell_start + A);
        const int nA = (int)__ldg(a.t.cell_start + A + 1) - begA;
        if (nA == 0) continue;
        int cx, cy, cz;
        cell_coords((uint32_t)A, a.t.nc, cx, cy, cz);
        __syncwarp();
        const int n = tile_stencil(a.t, cx, cy, cz, true, ts);
        const int total = ts.pre[n];
        const uint8_t *own = nullptr;
        if (total <= kRdfOwnCap) {
            tile_owners(ts, n, sown[warp]);
            own = sown[warp];
        }
        for (int qb = 0; qb < nA; qb += kRdfTileQ) {
            const int nq = min(kRdfTileQ, nA - qb);
            __syncwarp();
            if (lane < nq) qs[lane] = __ldg(a.t.pts + begA + qb + lane);
            __syncwarp();
            float3 blo, bhi;
            {
                const float4 q = qs[lane < nq ? lane : 0];
                warp_box(q.x, q.y, q.z, lane < nq, blo, bhi);
            }
            // A's own points first (they pair only with earlier queries)
            for (int base = 0; base < nA; base += 32) {
                if (tests > 0xffffffffull - 32 * kRdfTileQ) {
                    rdf_tile_flush(h, a.bins, a.hist, a.weight);
                    tests = 0;
                }
                tests += 32u * (unsigned)nq;
                const int k = base + lane;
                const TileCand c = tile_load_own(a.t, ts, own, n, nA, k);
                rdf_tile_rounds<true>(a, qs, nq, c, k < nA ? k - qb : 0, h);
            }
            // the other cells: candidates out of reach of the whole pass are dropped, the
            // rest are packed into full chunks (ballot + popc) before the query rounds
            int cnt = 0;
            for (int base = nA; base < total; base += 32) {
                const int k = base + lane;
                const TileCand c = tile_load_own(a.t, ts, own, n, total, k);
                const bool keep = k < total && box_dist2(blo, bhi, c.x, c.y, c.z) <= reach2;
                const unsigned m = __ballot_sync(0xffffffffu, keep);
                if (keep) buf[cnt + __popc(m & lt)] = make_float4(c.x, c.y, c.z, __int_as_float(c.j));
                cnt += __popc(m);
                if (cnt >= 32) {
                    __syncwarp();
                    if (tests > 0xffffffffull - 32 * kRdfTileQ) {
                        rdf_tile_flush(h, a.bins, a.hist, a.weight);
                        tests = 0;
                    }
                    tests += 32u * (unsigned)nq;
                    const float4 e = buf[lane];
                    TileCand ck;
                    ck.x = e.x, ck.y = e.y, ck.z = e.z, ck.j = __float_as_int(e.w), ck.p = 0, ck.o = 0;
                    rdf_tile_rounds<false>(a, qs, nq, ck, 0, h);
                    const float4 rest = buf[32 + lane];
                    __syncwarp();
                    if (lane < cnt - 32) buf[lane] = rest;
                    __syncwarp();
                    cnt -= 32;
                }
            }
            if (cnt > 0) {
                __syncwarp();
                tests += 32u * (unsigned)nq;
                const float4 e = lane < cnt ? buf[lane] : make_float4(kFar, kFar, kFar, __int_as_float(-1));
                TileCand ck;
                ck.x = e.x, ck.y = e.y, ck.z = e.z, ck.j = __float_as_int(e.w), ck.p = 0, ck.o = 0;
                rdf_tile_rounds<false>(a, qs, nq, ck, 0, h);
            }
        }
    }
    __syncthreads();
    // merge the warps' histograms, then one global add per bin and block
    for (int b = threadIdx.x; b < a.bins; b += blockDim.x) {
        unsigned long long v = 0;
        for (int w = 0; w < kRdfTileWarps; ++w) v += shist[w * a.bins + b];
        if (v) atomicAdd(a.hist + b, v * a.weight);
    }
}

// At most 64 registers, so eight blocks (32 warps) fit an SM: the kernel is bound by
// instruction latency, and eight blocks measured 4.01 ms at c3 against 4.17 ms for the
// unconstrained build (72 registers, seven blocks; FGB_RDF_VARIANT=0 selects it).
template <int NS>
__global__ void __launch_bounds__(kRdfTileWarps * 32, 8) k_rdf_tile(const __grid_constant__ RdfTileArgs a) {
    rdf_tile_body<NS>(a);
}

template <int NS>
__global__ void __launch_bounds__(kRdfTileWarps * 32) k_rdf_tile_r72(const __grid_constant__ RdfTileArgs a) {
    rdf_tile_body<NS>(a);
}

// Histogram of the pairs of a NeighborList.  Below 0.499 of a box length on every axis
// the defining sequence shifts by no box vector and its displacement is the plain
// difference, which the FP32 difference matches within u |d_k|: such pairs take the
// FP32 bin test with bands for that error.  Other pairs, and pairs inside a band, are
// decided with the FP64 sequence.
struct RdfListArgs {
    BoxD bd;
    const int32_t *qi, *pj;
    int64_t m;
    const float *q_orig, *p_orig;
    const double *T;
    int bins;
    BinParams P;
    float wx, wy, wz;
    unsigned long long *hist;
};

// COPIES shared histograms per block (one per warp for few bins, else one), over the
// block's contiguous range of at most 2^30 pairs so no 32-bit count can overflow;
// COPIES = 0 adds to the global counts directly (bins beyond the shared limit).
constexpr int kRdfListWarps = 8;
constexpr int kRdfListMaxBins = 16384;

template <int COPIES>
__global__ void __launch_bounds__(kRdfListWarps * 32) k_rdf_nlist(const __grid_constant__ RdfListArgs a,
                                                                  int64_t per_block) {
    extern __shared__ uint32_t lh[];
    if (COPIES > 0) {
        for (int b = threadIdx.x; b < COPIES * a.bins; b += blockDim.x) lh[b] = 0;
        __syncthreads();
    }
    uint32_t *h = lh + (COPIES > 1 ? (threadIdx.x >> 5) % COPIES : 0) * a.bins;
    const int64_t e0 = (int64_t)blockIdx.x * per_block, e1 = min(a.m, e0 + per_block);
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int i = __ldg(a.qi + e), j = __ldg(a.pj + e);
        const float *xi = a.q_orig + 3 * (int64_t)i, *xj = a.p_orig + 3 * (int64_t)j;
        const float dx = __ldg(xj) - __ldg(xi), dy = __ldg(xj + 1) - __ldg(xi + 1), dz = __ldg(xj + 2) - __ldg(xi + 2);
        int b = -2;
        if (fabsf(dx) < a.wx && fabsf(dy) < a.wy && fabsf(dz) < a.wz) b = rdf_bin(a.P, r2_f32(dx, dy, dz));
        if (b == -2) b = exact_bin(a.T, a.bins, exact_r2_idx(a.bd, a.q_orig, i, a.p_orig, j));
        if (b >= 0) {
            if (COPIES > 0)
                atomicAdd(h + b, 1u);
            else
                atomicAdd(a.hist + b, 1ull);
        }
    }
    if (COPIES > 0) {
        __syncthreads();
        for (int b = threadIdx.x; b < a.bins; b += blockDim.x) {
            unsigned long long v = 0;
            for (int c = 0; c < COPIES; ++c) v += lh[c * a.bins + b];
            if (v) atomicAdd(a.hist + b, v);
        }
    }
}

template <int COPIES>
static int launch_rdf_nlist(const RdfListArgs &a, cudaStream_t s) {
    const size_t smem = (size_t)COPIES * a.bins * sizeof(uint32_t);
    int per_sm = 8;
    if (COPIES > 0) {
        FGB_CUDA(cudaFuncSetAttribute(k_rdf_nlist<COPIES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        FGB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rdf_nlist<COPIES>, kRdfListWarps * 32, smem));
    }
    // enough blocks to fill the GPU, each over at most 2^30 pairs
    int64_t grid = std::min<int64_t>((a.m + 255) / 256, (int64_t)num_sms() * std::max(per_sm, 1));
    grid = std::max<int64_t>(grid, (a.m + ((int64_t)1 << 30) - 1) >> 30);
    const int64_t per_block = (a.m + grid - 1) / grid;
    FGB_KSCOPE("k_rdf_nlist", s);
    k_rdf_nlist<COPIES><<<(unsigned)grid, kRdfListWarps * 32, smem, s>>>(a, per_block);
    FGB_LAUNCH_CHECK();
    return FGB_OK;
}

template <class K>
static int launch_rdf_tile_k(K kern, const RdfTileArgs &ta, cudaStream_t s) {
    const size_t smem = (size_t)kRdfTileWarps * ta.bins * sizeof(uint32_t);
    int per_sm = 0;
    FGB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRdfTileWarps * 32, smem));
    const int64_t cells = ta.t.ncell - ta.t.cell_lo;
    const int64_t want = (cells + kRdfTileWarps - 1) / kRdfTileWarps;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * std::max(per_sm, 1)));
    FGB_KSCOPE("k_rdf_tile", s);
    kern<<<grid, kRdfTileWarps * 32, smem, s>>>(ta);
    return FGB_OK;
}

// FGB_RDF_VARIANT=0 launches the build without the register bound (comparisons).
static bool rdf_r72() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("FGB_RDF_VARIANT");
        v = (e && e[0] == '0') ? 1 : 0;
    }
    return v == 1;
}

template <int NS>
static int launch_rdf_tile_ns(const RdfTileArgs &ta, cudaStream_t s) {
    if (rdf_r72()) return launch_rdf_tile_k(k_rdf_tile_r72<NS>, ta, s);
    return launch_rdf_tile_k(k_rdf_tile<NS>, ta, s);
}

// Self query on the shift route, bins <= kRdfTileMaxBins, half stencil of nhalf cells.
static int launch_rdf_tile(const fgb_nq *nq, const StencilPlan &plan, double R, fgb_rdf *r, const BinParams &P,
                           int nhalf, cudaStream_t s) {
    RdfTileArgs ta;
    memset(&ta, 0, sizeof(ta));
    ta.t = tile_args(nq, plan, R, 1);
    ta.P = P;
    ta.T = r->T;
    ta.bins = r->bins;
    ta.hist = r->hist;
    ta.esc = r->esc;
    ta.esc_cap = r->esc_cap;
    ta.esc_count = r->esc_count;
    ta.weight = 2u;
    ta.work = reinterpret_cast<unsigned *>(r->esc_count + 1);
    if (nhalf <= 32) return launch_rdf_tile_ns<32>(ta, s);
    if (nhalf <= 64) return launch_rdf_tile_ns<64>(ta, s);
    return launch_rdf_tile_ns<kTileMaxStencil>(ta, s);
}

}  // namespace fgb

using namespace fgb;

extern "C" int fgb_rdf_create(int32_t bins, double r_max, double r_min, fgb_rdf **out) {
    clear_error();
    if (!out) return fail(FGB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (bins <= 0 || bins > (1 << 24)) return fail(FGB_ERR_INVALID_ARG, "bins must be in [1, 2^24]");
    if (!(r_min >= 0.0) || !(r_max > r_min) || !std::isfinite(r_max))
        return fail(FGB_ERR_INVALID_ARG, "need 0 <= r_min < r_max");
    fgb_rdf *r = new fgb_rdf();
    r->bins = bins;
    r->r_max = r_max;
    r->r_min = r_min;
    r->T_host.resize(bins + 1);
    const double delta = (r_max - r_min) / bins;
    for (int b = 0; b < bins; ++b) r->T_host[b] = sqrt_threshold(r_min + b * delta);
    r->T_host[bins] = sqrt_threshold(r_max);
    *out = r;
    return FGB_OK;
}

extern "C" void fgb_rdf_destroy(fgb_rdf *r) {
    if (!r) return;
    dfree(r->hist, r->stream);
    dfree(r->T, r->stream);
    dfree(r->esc, r->stream);
    dfree(r->esc_count, r->stream);
    dfree(r->band, r->stream);
    delete r;
}

static int rdf_ensure(fgb_rdf *r, int64_t esc_cap, cudaStream_t s) {
    if (!r->hist) {
        r->stream = s;
        FGB_TRY(dalloc_n(&r->hist, r->bins, s));
        FGB_CUDA(cudaMemsetAsync(r->hist, 0, sizeof(unsigned long long) * r->bins, s));
        FGB_TRY(dalloc_n(&r->T, r->bins + 1, s));
        FGB_CUDA(cudaMemcpyAsync(r->T, r->T_host.data(), sizeof(double) * (r->bins + 1), cudaMemcpyHostToDevice, s));
        FGB_CUDA(cudaStreamSynchronize(s));
        FGB_TRY(dalloc_n(&r->esc_count, 2, s));
    }
    if (esc_cap > r->esc_cap) {
        dfree(r->esc, s);
        r->esc = nullptr;
        r->esc_cap = 0;
        FGB_TRY(dalloc_n(&r->esc, esc_cap, s));
        r->esc_cap = (int)esc_cap;
    }
    return FGB_OK;
}

extern "C" int fgb_rdf_compute(fgb_rdf *r, fgb_nq *nq, const float *query_points, int64_t n_query,
                               const fgb_nlist *nlist, int32_t reset, void *stream) {
    clear_error();
    if (!r || !nq) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    FGB_TRY(nlist_ready(nlist));
    if (nq->kind != 0 && !nlist)
        return fail(FGB_ERR_UNSUPPORTED, "the fused RDF walks a cell list; pass a NeighborList from the tree query");
    cudaStream_t s = as_stream(stream);
    const double R = r->r_max;
    if (!(R < 0.5 * nq->box.wmin * (1.0 - 1e-5)))
        return fail(FGB_ERR_BOX_TOO_SMALL, "RDF r_max=%g must be below half the smallest box width (%g)", R,
                    0.5 * nq->box.wmin);
    const int dim = nq->box.is2d ? 2 : 3;
    if (!reset && r->dim != 0 && r->dim != dim)
        return fail(FGB_ERR_INVALID_ARG, "an RDF accumulates frames of one dimension (reset to switch)");
    QueryPoints Q;
    FGB_TRY(prepare_queries(nq, nlist ? nullptr : query_points, n_query, s, &Q));
    const int64_t nqq = nlist ? nlist->n_query : Q.n;
    // expected number of band hits is well below one per query; overflow falls back to
    // deciding in the main kernel
    int st = rdf_ensure(r, std::min<int64_t>(std::max<int64_t>(nqq * 2, 1 << 16), 1 << 27), s);
    if (st == FGB_OK && reset) {
        cudaMemsetAsync(r->hist, 0, sizeof(unsigned long long) * r->bins, s);
        r->norm = 0.0;
    }
    if (st == FGB_OK) cudaMemsetAsync(r->esc_count, 0, 2 * sizeof(int), s);  // [0] band pairs, [1] work
    if (st == FGB_OK && nlist) {
        const float *q_orig = query_points ? query_points : nq->points;
        if (nlist->n_pairs > 0) {
            // plain FP32 differences: each component within u |d_k| <= u R of the exact
            // one for pairs that matter (with slack for the FP64 reference's rounding)
            const BoxHost &b = nq->box;
            const double Lsum = std::sqrt(b.M[0][0] * b.M[0][0]) +
                                std::sqrt(b.M[0][1] * b.M[0][1] + b.M[1][1] * b.M[1][1]) +
                                std::sqrt(b.M[0][2] * b.M[0][2] + b.M[1][2] * b.M[1][2] + b.M[2][2] * b.M[2][2]);
            const double delta = r2_error_bound_eps(std::ldexp(1.0, -24) * R * 1.01, Lsum, R);
            if (!r->band) st = dalloc_n(&r->band, r->bins + 1, s);
            if (st == FGB_OK && delta != r->band_delta) {
                {
                    FGB_KSCOPE("k_band", s);
                    k_band<<<(r->bins + 256) / 256, 256, 0, s>>>(r->T, r->bins + 1, delta, r->band);
                }
                r->band_delta = delta;
            }
            if (st == FGB_OK) {
                RdfListArgs a;
                memset(&a, 0, sizeof(a));
                a.bd = b.d;
                a.qi = nlist->qi;
                a.pj = nlist->pj;
                a.m = nlist->n_pairs;
                a.q_orig = q_orig;
                a.p_orig = nq->points;
                a.T = r->T;
                a.bins = r->bins;
                a.P = bin_params(r->bins, r->r_min, r->r_max, delta, r->band, r->T_host);
                a.wx = (float)(0.499 * b.p[0]);
                a.wy = (float)(0.499 * b.p[1]);
                a.wz = (float)(0.499 * b.p[2]);
                a.hist = r->hist;
                if (r->bins <= 1024)
                    st = launch_rdf_nlist<kRdfListWarps>(a, s);
                else if (r->bins <= kRdfListMaxBins)
                    st = launch_rdf_nlist<1>(a, s);
                else
                    st = launch_rdf_nlist<0>(a, s);
            }
        }
        if (st == FGB_OK)
            st = cudaGetLastError() == cudaSuccess ? FGB_OK : fail(FGB_ERR_CUDA, "rdf nlist launch failed");
    } else if (st == FGB_OK && nqq > 0) {
        StencilPlan plan;
        st = plan_stencil(nq, R, 0, s, &plan);
        if (st == FGB_OK) {
            RdfArgs a;
            memset(&a, 0, sizeof(a));
            a.S = to_device(nq, plan);
            a.bf = nq->box.f;
            a.bd = nq->box.d;
            a.pts = nq->sorted;
            a.cell_start = nq->cell_start;
            a.qs = Q.sorted;
            a.qcell = Q.cell;
            a.nq = nqq;
            a.p_orig = nq->points;
            a.q_orig = Q.orig;
            a.exclude = Q.self ? 1 : 0;
            a.half = (Q.self && plan.mode == 0) ? 1 : 0;
            a.weight = a.half ? 2u : 1u;
            a.bins = r->bins;
            a.T = r->T;
            a.hist = r->hist;
            a.esc = r->esc;
            a.esc_cap = r->esc_cap;
            a.esc_count = r->esc_count;
            // bands around every edge (rebuilt only when the error bound changes)
            const double delta = r2_error_bound(plan, R);
            if (!r->band) st = dalloc_n(&r->band, r->bins + 1, s);
            if (st == FGB_OK && delta != r->band_delta) {
                {
                    FGB_KSCOPE("k_band", s);
                    k_band<<<(r->bins + 256) / 256, 256, 0, s>>>(r->T, r->bins + 1, delta, r->band);
                }
                r->band_delta = delta;
            }
            if (st == FGB_OK) {
                a.P = bin_params(r->bins, r->r_min, r->r_max, delta, r->band, r->T_host);
                const int nfull = (2 * plan.s[0] + 1) * (2 * plan.s[1] + 1) * (2 * plan.s[2] + 1);
                const int nhalf = (nfull + 1) / 2;
                const bool tile = a.half && nhalf <= kTileMaxStencil && r->bins <= kRdfTileMaxBins && tile_worth(nq) &&
                                  (nq->walk_set || !force_thread_kernels());
                if (tile) {
                    st = launch_rdf_tile(nq, plan, R, r, a.P, nhalf, s);
                } else {
                    const int block = 256;
                    int copies = 4;
                    while (copies > 1 && (size_t)copies * r->bins * 4 > 32 * 1024) copies >>= 1;
                    const size_t smem = (size_t)copies * r->bins * 4;
                    a.copies = copies;
                    if (smem <= 48 * 1024)
                        launch_rdf<true>(a, smem, s);
                    else
                        launch_rdf<false>(a, 0, s);
                }
                launch_rdf_escalated(a, s);
                cudaError_t e = cudaGetLastError();
                if (e != cudaSuccess) st = fail(FGB_ERR_CUDA, "rdf launch failed: %s", cudaGetErrorString(e));
            }
            dfree(plan.table, s);
        }
    }
    if (st == FGB_OK) {
        const double V = nq->box.p[0] * nq->box.p[1] * (dim == 2 ? 1.0 : nq->box.p[2]);
        r->norm += (double)nqq * (double)nq->n / V;
        r->dim = dim;
    }
    release_queries(&Q, s);
    return st;
}

extern "C" int fgb_rdf_result(fgb_rdf *r, uint64_t *counts, double *rdf_values, double *bin_centers, void *stream) {
    clear_error();
    if (!r) return fail(FGB_ERR_INVALID_ARG, "rdf is NULL");
    cudaStream_t s = as_stream(stream);
    std::vector<unsigned long long> h(r->bins, 0ull);
    if (r->hist) {
        FGB_CUDA(cudaMemcpyAsync(h.data(), r->hist, sizeof(unsigned long long) * r->bins, cudaMemcpyDeviceToHost, s));
        FGB_CUDA(cudaStreamSynchronize(s));
    }
    const double delta = (r->r_max - r->r_min) / r->bins;
    for (int b = 0; b < r->bins; ++b) {
        if (counts) counts[b] = h[b];
        const double R0 = r->r_min + b * delta;
        const double R1 = b + 1 < r->bins ? r->r_min + (b + 1) * delta : r->r_max;
        const double shell = r->dim == 2 ? M_PI * (R1 * R1 - R0 * R0) : 4.0 / 3.0 * M_PI * (R1 * R1 * R1 - R0 * R0 * R0);
        if (rdf_values) rdf_values[b] = r->norm > 0 ? (double)h[b] / (r->norm * shell) : 0.0;
        if (bin_centers) bin_centers[b] = r->r_min + (b + 0.5) * delta;
    }
    return FGB_OK;
}

extern "C" int fgb_rdf_params(const fgb_rdf *r, int32_t *bins, double *r_max, double *r_min) {
    if (!r) return fail(FGB_ERR_INVALID_ARG, "rdf is NULL");
    if (bins) *bins = r->bins;
    if (r_max) *r_max = r->r_max;
    if (r_min) *r_min = r->r_min;
    return FGB_OK;
}

extern "C" int fgb_rdf_counts_device(const fgb_rdf *r, const uint64_t **counts) {
    if (!r || !counts) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    *counts = reinterpret_cast<const uint64_t *>(r->hist);
    return FGB_OK;
}

extern "C" int fgb_rdf_escalations(fgb_rdf *r, int64_t *n, void *stream) {
    if (!r || !n) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    int v = 0;
    if (r->esc_count) {
        FGB_CUDA(cudaMemcpyAsync(&v, r->esc_count, sizeof(int), cudaMemcpyDeviceToHost, as_stream(stream)));
        FGB_CUDA(cudaStreamSynchronize(as_stream(stream)));
    }
    *n = v;
    return FGB_OK;
}

// ------------------------------------------------------------------ allocation-free RDF
//
// fgb_rdf_noalloc serves callers that must not allocate device memory while they run:
// simulation engines that call analysis from inside their time step with a fixed
// memory budget, or runtimes whose own pool owns the device and treats an outside
// cudaMalloc (which may synchronise the device) as an error.  Its whole working set
// lives in the fixed array below; the caller passes the points and the output only.

namespace fgb {
namespace noalloc {

constexpr int64_t kMaxPoints = 262144;
constexpr int kMaxBins = 8192;
constexpr int64_t kMaxCells = 4 * kMaxPoints + 64;  // grid_for keeps ncell <= 4 n + 64
constexpr int kMaxOrigin = 6 * 1024;
constexpr int kMaxOffsets = (2 * kMaxStencil + 1) * (2 * kMaxStencil + 1) * (2 * kMaxStencil + 1);
constexpr int64_t kEscCap = 2 * kMaxPoints;

constexpr size_t al(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kSortTileN = 4096;
constexpr size_t kSortWs = 2 * 4 * kMaxPoints + 4 * (2 * ((kMaxPoints + kSortTileN - 1) / kSortTileN) * 256 + 1) +
                           (((2 * ((kMaxPoints + kSortTileN - 1) / kSortTileN) * 256) + 4095) / 4096) * 12 + 256 +
                           1024 + 512;
constexpr size_t oOrigin = 0;
constexpr size_t oOffsets = oOrigin + al(sizeof(float2) * kMaxOrigin);
constexpr size_t oKeys = oOffsets + al(sizeof(float4) * kMaxOffsets);
constexpr size_t oVals = oKeys + al(4 * kMaxPoints);
constexpr size_t oLocal = oVals + al(4 * kMaxPoints);
constexpr size_t oSorted = oLocal + al(16 * kMaxPoints);
constexpr size_t oSortedCell = oSorted + al(16 * kMaxPoints);
constexpr size_t oCellStart = oSortedCell + al(4 * kMaxPoints);
constexpr size_t oSortWs = oCellStart + al(4 * (kMaxCells + 1));
constexpr size_t oT = oSortWs + al(kSortWs);
constexpr size_t oBand = oT + al(sizeof(double) * (kMaxBins + 1));
constexpr size_t oEsc = oBand + al(sizeof(float2) * (kMaxBins + 1));
constexpr size_t oEscCount = oEsc + al(sizeof(int2) * kEscCap);
constexpr size_t kBytes = oEscCount + 256;  // about 24 MB

// File-scope scratch: every GPU that loads the library holds one copy until exit.
static __device__ __align__(256) unsigned char g_scratch[kBytes];

static void *g_addr[64];
static std::mutex g_mu;

// Device address of g_scratch on the current device, looked up once per device (the
// host-side symbol is only a stand-in and must never be handed to a kernel).  The
// address stays valid for the life of the device's context: a cudaDeviceReset (which
// unloads the module) would leave it stale, so calls after a reset of a device already
// used here are not supported.
static int scratch(void **out) {
    int dev = 0;
    FGB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(FGB_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return fail(FGB_ERR_CUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return FGB_OK;
}

// Exact r^2 thresholds of the bin edges on the device (same definition as
// sqrt_threshold: smallest double whose IEEE square root reaches the edge).
__global__ void k_thresholds(int bins, double rmin, double rmax, double *T) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > bins) return;
    const double R = b == bins ? rmax : __dadd_rn(rmin, __dmul_rn((double)b, __ddiv_rn(__dsub_rn(rmax, rmin), (double)bins)));
    double t = 0.0;
    if (R > 0.0) {
        t = __dmul_rn(R, R);
        for (int it = 0; it < 64 && __dsqrt_rn(t) < R; ++it) t = nextafter(t, INFINITY);
        for (int it = 0; it < 64; ++it) {
            const double p = nextafter(t, 0.0);
            if (p >= 0.0 && __dsqrt_rn(p) >= R && p < t)
                t = p;
            else
                break;
        }
    }
    T[b] = t;
}

}  // namespace noalloc
}  // namespace fgb

extern "C" int fgb_rdf_noalloc(const fgb_box *box, const float *points, int64_t n, int32_t bins, double r_max,
                               double r_min, uint64_t *counts, void *stream) {
    using namespace fgb::noalloc;
    clear_error();
    if (!box || !counts || (n > 0 && !points)) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    if (n < 0) return fail(FGB_ERR_INVALID_ARG, "n must be >= 0");
    if (n > kMaxPoints)
        return fail(FGB_ERR_CAPACITY, "fgb_rdf_noalloc takes at most %lld points (got %lld)", (long long)kMaxPoints,
                    (long long)n);
    if (bins <= 0 || bins > kMaxBins) return fail(FGB_ERR_CAPACITY, "fgb_rdf_noalloc takes 1..%d bins", kMaxBins);
    if (!(r_min >= 0.0) || !(r_max > r_min) || !std::isfinite(r_max))
        return fail(FGB_ERR_INVALID_ARG, "need 0 <= r_min < r_max");
    cudaStream_t s = as_stream(stream);
    BoxHost bh;
    FGB_TRY(make_box(box, &bh));
    if (!(r_max < 0.5 * bh.wmin * (1.0 - 1e-5)))
        return fail(FGB_ERR_BOX_TOO_SMALL, "RDF r_max=%g must be below half the smallest box width (%g)", r_max,
                    0.5 * bh.wmin);
    GridHost g;
    FGB_TRY(grid_for(bh, r_max, n, &g));
    if (g.ncell > kMaxCells || g.nc[0] + 2 * g.nc[1] + 3 * g.nc[2] > kMaxOrigin)
        return fail(FGB_ERR_CAPACITY, "cell grid exceeds the fixed scratch");
    if (sort_ws_bytes(n) > kSortWs) return fail(FGB_ERR_CAPACITY, "sort workspace exceeds the fixed scratch");
    StencilPlan plan;
    FGB_TRY(plan_stencil_host(bh, g, r_max, 0, &plan, nullptr));
    void *base = nullptr;
    FGB_TRY(scratch(&base));
    unsigned char *w = static_cast<unsigned char *>(base);
    float2 *origin = reinterpret_cast<float2 *>(w + oOrigin);
    float4 *offsets = reinterpret_cast<float4 *>(w + oOffsets);
    uint32_t *keys = reinterpret_cast<uint32_t *>(w + oKeys);
    uint32_t *vals = reinterpret_cast<uint32_t *>(w + oVals);
    float4 *local = reinterpret_cast<float4 *>(w + oLocal);
    float4 *sorted = reinterpret_cast<float4 *>(w + oSorted);
    uint32_t *sorted_cell = reinterpret_cast<uint32_t *>(w + oSortedCell);
    uint32_t *cell_start = reinterpret_cast<uint32_t *>(w + oCellStart);
    void *sort_ws = w + oSortWs;
    double *T = reinterpret_cast<double *>(w + oT);
    float2 *band = reinterpret_cast<float2 *>(w + oBand);
    int2 *esc = reinterpret_cast<int2 *>(w + oEsc);
    int *esc_count = reinterpret_cast<int *>(w + oEscCount);
    // the output and the band-pair counter start at zero on every call
    FGB_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint64_t) * bins, s));
    FGB_CUDA(cudaMemsetAsync(esc_count, 0, sizeof(int), s));
    if (n == 0) return FGB_OK;
    if (plan.mode == 0) FGB_TRY(launch_offset_table(bh, g, plan, offsets, s));
    OriginTables org;
    FGB_TRY(bin_points_into(bh, g, points, n, origin, &org, sorted, sorted_cell, cell_start, keys, vals, local, sort_ws, s));
    {
        FGB_KSCOPE("k_thresholds", s);
        k_thresholds<<<(bins + 256) / 256, 256, 0, s>>>(bins, r_min, r_max, T);
    }
    const double G2 = r2_error_bound(plan, r_max);
    {
        FGB_KSCOPE("k_band", s);
        k_band<<<(bins + 256) / 256, 256, 0, s>>>(T, bins + 1, G2, band);
    }
    RdfArgs a;
    memset(&a, 0, sizeof(a));
    a.S = to_device(bh, g, plan, plan.mode == 0 ? offsets : nullptr);
    a.bf = bh.f;
    a.bd = bh.d;
    a.pts = sorted;
    a.cell_start = cell_start;
    a.qs = sorted;
    a.qcell = sorted_cell;
    a.nq = n;
    a.p_orig = points;
    a.q_orig = points;
    a.exclude = 1;
    a.half = plan.mode == 0 ? 1 : 0;
    a.weight = a.half ? 2u : 1u;
    a.bins = bins;
    // the two outer thresholds are recomputed on the host for the range test
    std::vector<double> Th(bins + 1, 0.0);
    Th[0] = sqrt_threshold(r_min);
    Th[bins] = sqrt_threshold(r_max);
    a.P = bin_params(bins, r_min, r_max, G2, band, Th);
    a.T = T;
    a.hist = reinterpret_cast<unsigned long long *>(counts);
    a.esc = esc;
    a.esc_cap = (int)kEscCap;
    a.esc_count = esc_count;
    int copies = 4;
    while (copies > 1 && (size_t)copies * bins * 4 > 32 * 1024) copies >>= 1;
    const size_t smem = (size_t)copies * bins * 4;
    a.copies = copies;
    if (smem <= 48 * 1024)
        launch_rdf<true>(a, smem, s);
    else
        launch_rdf<false>(a, 0, s);
    launch_rdf_escalated(a, s);
    FGB_LAUNCH_CHECK();
    return FGB_OK;
}
