// Many trajectory frames in one pass (the per-frame loops of the paper's on-the-fly and
// trajectory listings): per-frame RDF counts and per-particle q_l.
//
// All frames are binned by one kernel into one global cell array (frame f owns cells
// cell_base[f] .. cell_base[f+1]) and sorted by one radix sort.  Frames whose RDF half
// stencil and ball stencil are on the fixed-offset route take the cell-tile kernels of
// batch_tile.cu (a warp per query cell).  The others take the persistent per-point
// kernel here: blocks take work items (a frame and up to `block` consecutive sorted
// points) from an atomic counter, stage that frame's description in shared memory, and
// for every point walk (1) the RDF half stencil into a shared histogram that is flushed
// when the block moves to another frame, and (2) the ball-query stencil into the
// spherical-harmonic accumulators.  Every buffer is allocated at create time, so a run
// is a fixed launch sequence with no host synchronisation; fgb_batch_run_graph captures
// it once in a CUDA graph and replays it.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "fgb_ball.cuh"
#include "fgb_batch.cuh"
#include "fgb_ylm.cuh"

namespace fgb {

struct FrameDev {
    BallArgs ball;       // ball-query walk of this frame (q_l neighbors)
    OriginTables org;
    Stencil Sr;          // RDF stencil
    BinParams P;         // RDF binning (bands around the bins+1 edges of this frame)
    int64_t pt_off;
    uint32_t cell_base;
    int n;
    int half;            // RDF: unordered pairs via the half stencil
    int pad;
};

struct BatchArgs {
    const FrameDev *frames;
    const int64_t *frame_off;  // nframes + 1
    int nframes;
    const int4 *items;         // (frame, first sorted position, count, 0)
    int nitems;
    int *ctl;                  // [0] item counter, [1] escalation count
    const float4 *sorted;
    const uint32_t *skeys;
    const uint32_t *cell_start;
    const float *pts;
    int bins;
    const double *T;
    unsigned long long *counts;  // nframes * bins
    int copies;
    int4 *esc;
    int esc_cap;
    float *q;
    float2 *Q;
    int32_t *nn;
};

// Blocks of kBinBlock points; blk_frame[b] is the frame of block b's first point (set
// at create time), and each point finds its own by stepping forward from it (a block's
// points span few frames).
constexpr int kBinBlock = 256;

__global__ void __launch_bounds__(kBinBlock) k_batch_bin(const FrameDev *__restrict__ frames,
                                                         const int64_t *__restrict__ frame_off,
                                                         const int32_t *__restrict__ blk_frame, int nframes,
                                                         const float *__restrict__ pts, int64_t total,
                                                         uint32_t *__restrict__ keys, uint32_t *__restrict__ vals,
                                                         float4 *__restrict__ local) {
    const int64_t g = (int64_t)blockIdx.x * kBinBlock + threadIdx.x;
    if (g >= total) return;
    int lo = __ldg(blk_frame + blockIdx.x);
    while (lo + 1 < nframes && __ldg(frame_off + lo + 1) <= g) ++lo;
    const FrameDev &f = frames[lo];
    GridDev gd = {{f.ball.S.nc[0], f.ball.S.nc[1], f.ball.S.nc[2]}};
    uint32_t key;
    float4 loc;
    bin_point(f.ball.bf, f.ball.bd, gd, f.org, pts[3 * g], pts[3 * g + 1], pts[3 * g + 2], key, loc);
    loc.w = __int_as_float((int)g);
    keys[g] = f.cell_base + key;
    vals[g] = (uint32_t)g;
    local[g] = loc;
}

template <int L>
__global__ void __launch_bounds__(256) k_batch(BatchArgs a) {
    extern __shared__ uint32_t sh[];
    __shared__ FrameDev fr;
    __shared__ int s_item, s_frame;
    for (int b = threadIdx.x; b < a.bins * a.copies; b += blockDim.x) sh[b] = 0;
    if (threadIdx.x == 0) s_frame = -1;
    __syncthreads();
    uint32_t *my = sh + ((threadIdx.x >> 5) % a.copies) * a.bins;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.ctl, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= a.nitems) break;
        const int4 w = a.items[it];
        if (w.x != s_frame) {
            if (s_frame >= 0) {
                const unsigned wt = fr.half ? 2u : 1u;
                for (int b = threadIdx.x; b < a.bins; b += blockDim.x) {
                    uint32_t v = 0;
                    for (int c = 0; c < a.copies; ++c) {
                        v += sh[c * a.bins + b];
                        sh[c * a.bins + b] = 0;
                    }
                    if (v) atomicAdd(a.counts + (int64_t)s_frame * a.bins + b, (unsigned long long)v * wt);
                }
            }
            __syncthreads();
            const int *src = reinterpret_cast<const int *>(a.frames + w.x);
            int *dst = reinterpret_cast<int *>(&fr);
            for (int k = threadIdx.x; k < (int)(sizeof(FrameDev) / 4); k += blockDim.x) dst[k] = src[k];
            if (threadIdx.x == 0) s_frame = w.x;
            __syncthreads();
        }
        if ((int)threadIdx.x < w.z) {
            const int64_t t = w.y + threadIdx.x;
            const float4 p = a.sorted[t];
            const int i = __float_as_int(p.w);
            const uint32_t lc = a.skeys[t] - fr.cell_base;
            int cx, cy, cz;
            cell_coords(lc, fr.Sr.nc, cx, cy, cz);
            const uint32_t *cs = a.cell_start + fr.cell_base;
            // (1) RDF, ordered pairs (each unordered pair once with weight 2 in half mode)
            const int half = fr.half;
            for_stencil(fr.Sr, cx, cy, cz, make_float3(p.x, p.y, p.z), half != 0,
                        [&](int cell, float qx, float qy, float qz, bool center) {
                            uint32_t beg = __ldg(cs + cell);
                            const uint32_t end = __ldg(cs + cell + 1);
                            if (half && center) beg = max(beg, (uint32_t)t + 1u);
                            for (uint32_t pp = beg; pp < end; ++pp) {
                                const float4 c = __ldg(a.sorted + pp);
                                const float3 d = cand_disp(fr.Sr, fr.ball.bf, c, qx, qy, qz);
                                const float r2 = r2_f32(d.x, d.y, d.z);
                                const int b = rdf_bin(fr.P, r2);
                                if (b == -1) continue;
                                const int j = __float_as_int(c.w);
                                if (j == i) continue;
                                if (b >= 0) {
                                    atomicAdd(my + b, 1u);
                                } else {
                                    const int slot = atomicAdd(a.ctl + 1, 1);
                                    if (slot < a.esc_cap) {
                                        a.esc[slot] = make_int4(s_frame, i, j, half ? 2 : 1);
                                    } else {
                                        const double e = exact_r2_idx(fr.ball.bd, a.pts, i, a.pts, j);
                                        if (e >= a.T[0] && e < a.T[a.bins]) {
                                            int lo = 0, hi = a.bins;
                                            while (hi - lo > 1) {
                                                const int mid = (lo + hi) >> 1;
                                                if (a.T[mid] <= e)
                                                    lo = mid;
                                                else
                                                    hi = mid;
                                            }
                                            atomicAdd(a.counts + (int64_t)s_frame * a.bins + lo,
                                                      (unsigned long long)(half ? 2 : 1));
                                        }
                                    }
                                }
                            }
                        });
            // (2) q_l over the ball-query neighbors
            if constexpr (L >= 0) {
                float sr[L + 1 > 0 ? L + 1 : 1], si[L + 1 > 0 ? L + 1 : 1];
#pragma unroll
                for (int m = 0; m <= L; ++m) sr[m] = si[m] = 0.f;
                int n = 0;
                BondBuffer<L> bb;
                ball_visit(fr.ball, p, lc, i, [&](int, float3 d, float, double) {
                    ++n;
                    bb.add(d, sr, si);
                });
                bb.flush(sr, si);
                finish<L>(i, n, sr, si, a.q, a.Q, a.nn);
            }
        }
        __syncthreads();
    }
    if (s_frame >= 0) {
        const unsigned wt = fr.half ? 2u : 1u;
        for (int b = threadIdx.x; b < a.bins; b += blockDim.x) {
            uint32_t v = 0;
            for (int c = 0; c < a.copies; ++c) v += sh[c * a.bins + b];
            if (v) atomicAdd(a.counts + (int64_t)s_frame * a.bins + b, (unsigned long long)v * wt);
        }
    }
}

__global__ void k_batch_escalated(BatchArgs a) {
    const int n = min(a.ctl[1], a.esc_cap);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int4 x = a.esc[e];
        const FrameDev &f = a.frames[x.x];
        const double r2 = exact_r2_idx(f.ball.bd, a.pts, x.y, a.pts, x.z);
        if (!(r2 >= a.T[0]) || !(r2 < a.T[a.bins])) continue;
        // the bin of the FP32 guess, stepped until the FP64 thresholds bracket r2
        int lo = min(max((int)((sqrtf((float)r2) - f.P.rmin) * f.P.invdelta), 0), a.bins - 1);
        while (lo > 0 && r2 < a.T[lo]) --lo;
        while (lo + 1 < a.bins && r2 >= a.T[lo + 1]) ++lo;
        atomicAdd(a.counts + (int64_t)x.x * a.bins + lo, (unsigned long long)x.w);
    }
}

template <int L>
struct BatchLaunch {
    static void run(const BatchArgs &a, int grid, int block, size_t smem, cudaStream_t s) {
        FGB_KSCOPE("k_batch", s);
        k_batch<L><<<grid, block, smem, s>>>(a);
    }
    static int max_blocks(int block, size_t smem) {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<L>, block, smem);
        return nb;
    }
};

}  // namespace fgb

using namespace fgb;

struct fgb_batch {
    int nframes;
    std::vector<int64_t> off;
    std::vector<fgb_box> boxes;
    fgb_batch_params prm;
    int64_t total;
    int cell_div, block, copies, tile_cells, qbw;
    bool tune_div, tune_block, tune_copies, tune_tile, tune_qb;
    // configuration-dependent device state
    FrameDev *frames_d;
    float2 *origin_d;
    float4 *offset_d;
    float2 *band_d;
    int4 *items_d;
    int nitems;
    FrameTile *ft_d;      // frames on the cell-tile route
    int4 *titems_d;       // their work items
    int ntitems;
    int ntile_frames;
    bool small_r;           // every tile frame's RDF half stencil <= 64 cells
    int q_ns;               // q_l stencil capacity every tile frame fits (32, 64, 128)
    uint32_t *cell_start;
    int64_t ncell_total;
    // fixed device state
    int64_t *off_d;
    int32_t *blk_d;               // frame of the first point of each binning block
    std::vector<int32_t> blk;
    double *T_d;
    std::vector<double> T_h;
    int *ctl;
    uint32_t *keys, *vals, *skeys;
    float4 *local, *sorted;
    void *sort_ws;
    unsigned long long *counts;
    float *q;
    float2 *Q;
    int32_t *nn;
    int4 *esc;
    int esc_cap;
    unsigned long long *qesc;
    cudaGraph_t graph;
    cudaGraphExec_t gexec;
    BatchTileLaunch tl;
    const float *graph_pts;
    cudaStream_t stream;
    cudaStream_t cap_stream;  // capture needs a stream other than the legacy default
};

static void free_config(fgb_batch *b, cudaStream_t s) {
    dfree(b->frames_d, s);
    dfree(b->origin_d, s);
    dfree(b->offset_d, s);
    dfree(b->band_d, s);
    dfree(b->items_d, s);
    dfree(b->ft_d, s);
    dfree(b->titems_d, s);
    dfree(b->cell_start, s);
    b->ft_d = nullptr;
    b->titems_d = nullptr;
    b->frames_d = nullptr;
    b->origin_d = nullptr;
    b->offset_d = nullptr;
    b->band_d = nullptr;
    b->items_d = nullptr;
    b->cell_start = nullptr;
}

static void drop_graph(fgb_batch *b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
    b->graph_pts = nullptr;
}

// A frame takes the cell-tile kernels when both of its stencils are on the shift route
// with at most kTileMaxStencil cells (the RDF's half stencil) and its histogram fits a
// warp's private copy; the others take the per-point kernel.
constexpr int kBatchTileMaxBins = 1024;

// Builds every per-frame table for a cell division, a block size of the per-point kernel
// and the largest work item of the tile kernels (tile_cells < 0: no tile route), and
// the query cells per warp of the tile kernels (qbw: 1, 2, 4 or 8; a frame takes the
// largest power of two up to qbw that its grid allows); synchronises.
static int configure(fgb_batch *b, int cell_div, int block, int tile_cells, int qbw, cudaStream_t s) {
    drop_graph(b);
    free_config(b, s);
    const int F = b->nframes;
    const double rq = b->prm.r_max, rr = b->prm.rdf_r_max;
    std::vector<FrameDev> fh(F);
    std::vector<float2> org;
    std::vector<float4> offs;
    std::vector<float2> bands;
    std::vector<int4> items;
    struct Fix {
        size_t org, offq, offr, band;
    };
    std::vector<Fix> fix(F);
    std::vector<FrameTile> tiles;
    std::vector<int64_t> tile_lo, tile_hi;  // query cells of each tile frame
    bool small_r = true;
    int q_cells = 0;  // largest ball stencil (or block union) of the tile frames
    int64_t cell_base = 0;
    for (int f = 0; f < F; ++f) {
        BoxHost box;
        FGB_TRY(make_box(&b->boxes[f], &box));
        const double need = std::max(rq, rr);
        if (!(need < 0.5 * box.wmin * (1.0 - 1e-5)))
            return fail(FGB_ERR_BOX_TOO_SMALL, "frame %d: r_max %g must be below half its smallest box width %g", f, need,
                        0.5 * box.wmin);
        GridHost g;
        const int64_t nf = b->off[f + 1] - b->off[f];
        FGB_TRY(grid_for(box, rq / cell_div, nf, &g));
        FrameDev &d = fh[f];
        memset(&d, 0, sizeof(d));
        // origin tables, as in the single-frame build
        fix[f].org = org.size();
        auto put = [&](double v) {
            float hi = (float)v;
            org.push_back(make_float2(hi, (float)(v - (double)hi)));
        };
        for (int c = 0; c < g.nc[0]; ++c) put(box.M[0][0] * ((double)c / g.nc[0] - 0.5));
        for (int c = 0; c < g.nc[1]; ++c) put(box.M[0][1] * ((double)c / g.nc[1] - 0.5));
        for (int c = 0; c < g.nc[1]; ++c) put(box.M[1][1] * ((double)c / g.nc[1] - 0.5));
        for (int c = 0; c < g.nc[2]; ++c) put(box.M[0][2] * ((double)c / g.nc[2] - 0.5));
        for (int c = 0; c < g.nc[2]; ++c) put(box.M[1][2] * ((double)c / g.nc[2] - 0.5));
        for (int c = 0; c < g.nc[2]; ++c) put(box.M[2][2] * ((double)c / g.nc[2] - 0.5));
        StencilPlan pq, pr;
        std::vector<float4> tq, tr;
        FGB_TRY(plan_stencil_host(box, g, rq, 0, &pq, &tq));
        // a block of qb cells along x walks the union of their ball stencils: x offsets
        // -s .. s + qb - 1 (distinct cells while qb + 2s <= nc_x; the offset table reaches
        // s + qb - 1 when nc_x >= 2s + 2qb - 1)
        auto qb_cells = [](const StencilPlan &p, int q) {
            return (q + 2 * p.s[0]) * (2 * p.s[1] + 1) * (2 * p.s[2] + 1);
        };
        int qb_f = 1;
        if (qbw > 1 && pq.mode == 0) {
            for (int q = qbw; q > 1 && qb_f == 1; q >>= 1)
                if (g.nc[0] >= 2 * pq.s[0] + 2 * q - 1 && qb_cells(pq, q) <= kTileMaxStencil) qb_f = q;
            if (qb_f > 1) {
                StencilPlan wide;
                std::vector<float4> tw;
                FGB_TRY(plan_stencil_host(box, g, rq, pq.s[0] + qb_f - 1, &wide, &tw));
                if (wide.mode == 0 && wide.ts[0] >= wide.s[0] + qb_f - 1) {
                    pq = wide;
                    tq.swap(tw);
                } else {
                    qb_f = 1;
                }
            }
        }
        FGB_TRY(plan_stencil_host(box, g, rr, 0, &pr, &tr));
        // the same for the RDF's half stencil: a block's union lists the cells after each
        // of its cells in (z, y, x) order
        auto qbr_cells = [](const StencilPlan &p, int q) {
            const int wxq = q + 2 * p.s[0];
            return wxq * (2 * p.s[1] + 1) * p.s[2] + wxq * p.s[1] + q + p.s[0];
        };
        int qbr_f = 1;
        if (qbw > 1 && pr.mode == 0) {
            for (int q = qbw; q > 1 && qbr_f == 1; q >>= 1)
                if (g.nc[0] >= 2 * pr.s[0] + 2 * q - 1 && qbr_cells(pr, q) <= kTileMaxStencil) qbr_f = q;
            if (qbr_f > 1) {
                StencilPlan wide;
                std::vector<float4> tw;
                FGB_TRY(plan_stencil_host(box, g, rr, pr.s[0] + qbr_f - 1, &wide, &tw));
                if (wide.mode == 0 && wide.ts[0] >= wide.s[0] + qbr_f - 1) {
                    pr = wide;
                    tr.swap(tw);
                } else {
                    qbr_f = 1;
                }
            }
        }
        fix[f].offq = offs.size();
        offs.insert(offs.end(), tq.begin(), tq.end());
        fix[f].offr = offs.size();
        offs.insert(offs.end(), tr.begin(), tr.end());
        fix[f].band = bands.size();
        const double dr = r2_error_bound(pr, rr);
        d.P = bin_params(b->prm.rdf_bins, b->prm.rdf_r_min, rr, dr, nullptr, b->T_h);
        for (int e = 0; e <= b->prm.rdf_bins; ++e) {
            float lo, hi;
            band_around(b->T_h[e], dr, &lo, &hi);
            bands.push_back(make_float2(lo, hi));
        }
        BallArgs &ba = d.ball;
        ba.S = to_device(box, g, pq, nullptr);
        ba.bf = box.f;
        ba.bd = box.d;
        ba.pts = nullptr;  // fixed up below
        ba.nq = nf;
        ba.T = sqrt_threshold(rq);
        band_around(ba.T, r2_error_bound(pq, rq), &ba.band.lo, &ba.band.hi);
        ba.exclude = 1;
        d.Sr = to_device(box, g, pr, nullptr);
        d.half = pr.mode == 0 ? 1 : 0;
        d.pt_off = b->off[f];
        d.n = (int)nf;
        d.cell_base = (uint32_t)cell_base;
        cell_base += g.ncell;
        auto cells = [](const StencilPlan &p) { return (2 * p.s[0] + 1) * (2 * p.s[1] + 1) * (2 * p.s[2] + 1); };
        const bool tile = tile_cells > 0 && pq.mode == 0 && pr.mode == 0 && cells(pq) <= kTileMaxStencil &&
                          (cells(pr) + 1) / 2 <= kTileMaxStencil && b->prm.rdf_bins <= kBatchTileMaxBins;
        if (tile) {
            FrameTile ft;
            memset(&ft, 0, sizeof(ft));
            auto fill = [&](TileArgs &t, const StencilPlan &p) {
                for (int k = 0; k < 3; ++k) {
                    t.nc[k] = g.nc[k];
                    t.s[k] = p.s[k];
                    t.ts[k] = p.ts[k];
                }
                t.pts = b->sorted;
                t.ncell = g.ncell;
                t.bf = box.f;
                t.bd = box.d;
                t.exclude = 1;
            };
            fill(ft.r, pr);
            ft.r.half = 1;
            fill(ft.b, pq);
            ft.b.T = ba.T;
            ft.b.band = ba.band;
            ft.P = d.P;
            ft.f = f;
            ft.qb = qb_f;
            ft.qbr = qbr_f;
            tiles.push_back(ft);
            small_r = small_r && qbr_cells(pr, qbr_f) <= 64;
            q_cells = std::max(q_cells, qb_cells(pq, qb_f));
            // a 2D frame's points all lie in the middle one of its three z layers
            const int64_t layer = (int64_t)g.nc[0] * g.nc[1];
            tile_lo.push_back(box.is2d ? layer : 0);
            tile_hi.push_back(box.is2d ? 2 * layer : g.ncell);
        } else {
            for (int64_t s0 = 0; s0 < nf; s0 += block)
                items.push_back(make_int4(f, (int)(b->off[f] + s0), (int)std::min<int64_t>(block, nf - s0), 0));
        }
    }
    // Tile work items: frames in order, each cut into ranges of at most tile_cells cells,
    // shrinking toward the end of the list (about twice as many items left as resident
    // warps) so the last items finish together.
    std::vector<int4> titems;
    {
        int64_t left = 0;
        for (size_t k = 0; k < tiles.size(); ++k) left += tile_hi[k] - tile_lo[k];
        const int64_t w2 = 2 * (int64_t)std::max(b->tl.warps, 1);
        for (size_t k = 0; k < tiles.size(); ++k) {
            for (int64_t c = tile_lo[k]; c < tile_hi[k];) {
                int64_t chunk = std::min<int64_t>((left + w2 - 1) / w2, tile_cells);
                chunk = std::max<int64_t>(1, std::min(chunk, tile_hi[k] - c));
                titems.push_back(make_int4((int)k, (int)c, (int)(c + chunk), 0));
                c += chunk;
                left -= chunk;
            }
        }
    }
    if (cell_base >= ((int64_t)1 << 32) - 1) return fail(FGB_ERR_CAPACITY, "too many cells over all frames");
    b->ncell_total = cell_base;
    b->nitems = (int)items.size();
    b->ntitems = (int)titems.size();
    b->ntile_frames = (int)tiles.size();
    b->small_r = small_r;
    b->q_ns = q_cells <= 32 ? 32 : q_cells <= 64 ? 64 : kTileMaxStencil;
    int st = FGB_OK;
    st = st ? st : dalloc_n(&b->frames_d, F, s);
    st = st ? st : dalloc_n(&b->origin_d, std::max<size_t>(org.size(), 1), s);
    st = st ? st : dalloc_n(&b->offset_d, std::max<size_t>(offs.size(), 1), s);
    st = st ? st : dalloc_n(&b->band_d, bands.size(), s);
    st = st ? st : dalloc_n(&b->items_d, std::max<size_t>(items.size(), 1), s);
    st = st ? st : dalloc_n(&b->cell_start, cell_base + 1, s);
    st = st ? st : dalloc_n(&b->ft_d, std::max<size_t>(tiles.size(), 1), s);
    st = st ? st : dalloc_n(&b->titems_d, std::max<size_t>(titems.size(), 1), s);
    FGB_TRY(st);
    for (int f = 0; f < F; ++f) {
        FrameDev &d = fh[f];
        const float2 *o = b->origin_d + fix[f].org;
        const int nx = d.ball.S.nc[0], ny = d.ball.S.nc[1], nz = d.ball.S.nc[2];
        d.org.Tx = o;
        d.org.Txy = o + nx;
        d.org.Ty = o + nx + ny;
        d.org.Txz = o + nx + 2 * ny;
        d.org.Tyz = o + nx + 2 * ny + nz;
        d.org.Tz = o + nx + 2 * ny + 2 * nz;
        if (d.ball.S.mode == 0) d.ball.S.off = b->offset_d + fix[f].offq;
        if (d.Sr.mode == 0) d.Sr.off = b->offset_d + fix[f].offr;
        d.P.band = b->band_d + fix[f].band;
        d.ball.pts = b->sorted;
        d.ball.cell_start = b->cell_start + d.cell_base;
        d.ball.qs = b->sorted;
        d.ball.qcell = nullptr;
        d.ball.p_orig = nullptr;
        d.ball.q_orig = nullptr;
        d.ball.esc = b->qesc;
        d.ball.err = reinterpret_cast<int *>(b->qesc + 1);
    }
    for (FrameTile &ft : tiles) {
        const FrameDev &d = fh[ft.f];
        ft.r.off = b->offset_d + fix[ft.f].offr;
        ft.b.off = b->offset_d + fix[ft.f].offq;
        ft.r.cell_start = ft.b.cell_start = b->cell_start + d.cell_base;
        ft.P.band = d.P.band;
    }
    // the walks index original coordinates through the packed points, set per run
    FGB_CUDA(cudaMemcpyAsync(b->frames_d, fh.data(), sizeof(FrameDev) * F, cudaMemcpyHostToDevice, s));
    if (!org.empty())
        FGB_CUDA(cudaMemcpyAsync(b->origin_d, org.data(), sizeof(float2) * org.size(), cudaMemcpyHostToDevice, s));
    if (!offs.empty())
        FGB_CUDA(cudaMemcpyAsync(b->offset_d, offs.data(), sizeof(float4) * offs.size(), cudaMemcpyHostToDevice, s));
    FGB_CUDA(cudaMemcpyAsync(b->band_d, bands.data(), sizeof(float2) * bands.size(), cudaMemcpyHostToDevice, s));
    if (!items.empty())
        FGB_CUDA(cudaMemcpyAsync(b->items_d, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, s));
    if (!tiles.empty())
        FGB_CUDA(cudaMemcpyAsync(b->ft_d, tiles.data(), sizeof(FrameTile) * tiles.size(), cudaMemcpyHostToDevice, s));
    if (!titems.empty())
        FGB_CUDA(cudaMemcpyAsync(b->titems_d, titems.data(), sizeof(int4) * titems.size(), cudaMemcpyHostToDevice, s));
    FGB_CUDA(cudaStreamSynchronize(s));
    b->cell_div = cell_div;
    b->block = block;
    b->tile_cells = tile_cells;
    b->qbw = qbw;
    return FGB_OK;
}

// Points pointer into every frame's ball-query arguments (device-side patch).
__global__ void k_batch_set_points(FrameDev *frames, int n, const float *pts) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < n) {
        frames[f].ball.p_orig = pts;
        frames[f].ball.q_orig = pts;
    }
}

static BatchArgs batch_args(const fgb_batch *b, const float *pts) {
    BatchArgs a;
    memset(&a, 0, sizeof(a));
    a.frames = b->frames_d;
    a.frame_off = b->off_d;
    a.nframes = b->nframes;
    a.items = b->items_d;
    a.nitems = b->nitems;
    a.ctl = b->ctl;
    a.sorted = b->sorted;
    a.skeys = b->skeys;
    a.cell_start = b->cell_start;
    a.pts = pts;
    a.bins = b->prm.rdf_bins;
    a.T = b->T_d;
    a.counts = b->counts;
    a.copies = b->copies;
    a.esc = b->esc;
    a.esc_cap = b->esc_cap;
    a.q = b->q;
    a.Q = b->Q;
    a.nn = b->nn;
    return a;
}

template <int L>
struct RunBatch {
    static void run(const BatchArgs &a, int grid, int block, size_t smem, cudaStream_t s) {
        BatchLaunch<L>::run(a, grid, block, smem, s);
    }
};
template <int L>
struct MaxBlocks {
    static void run(int block, size_t smem, int *out) { *out = BatchLaunch<L>::max_blocks(block, smem); }
};

template <template <int> class F, class... Args>
static bool dispatch_batch_l(int l, Args &&...args) {
    switch (l) {
#define FGB_BL(V)                               \
    case V:                                     \
        F<V>::run(std::forward<Args>(args)...); \
        return true;
        FGB_BL(-1) FGB_BL(0) FGB_BL(1) FGB_BL(2) FGB_BL(3) FGB_BL(4) FGB_BL(5) FGB_BL(6) FGB_BL(7) FGB_BL(8) FGB_BL(9)
        FGB_BL(10) FGB_BL(11) FGB_BL(12)
#undef FGB_BL
    }
    return false;
}

static int enqueue(fgb_batch *b, const float *pts, cudaStream_t s) {
    const int64_t n = b->total;
    const int F = b->nframes;
    FGB_CUDA(cudaMemsetAsync(b->ctl, 0, 4 * sizeof(int), s));
    FGB_CUDA(cudaMemsetAsync(b->counts, 0, sizeof(unsigned long long) * F * b->prm.rdf_bins, s));
    {
        FGB_KSCOPE("k_batch_set_points", s);
        k_batch_set_points<<<(F + 127) / 128, 128, 0, s>>>(b->frames_d, F, pts);
    }
    if (n > 0) {
        {
            FGB_KSCOPE("k_batch_bin", s);
            k_batch_bin<<<(unsigned)((n + kBinBlock - 1) / kBinBlock), kBinBlock, 0, s>>>(
                b->frames_d, b->off_d, b->blk_d, F, pts, n, b->keys, b->vals, b->local);
        }
        FGB_TRY(radix_sort_cells(b->keys, b->vals, n, b->ncell_total, b->local, b->sorted, b->skeys, b->sort_ws, s));
    }
    FGB_TRY(launch_cell_start(b->skeys, n, b->ncell_total, b->cell_start, s));
    BatchArgs a = batch_args(b, pts);
    const size_t smem = (size_t)b->copies * b->prm.rdf_bins * sizeof(uint32_t);
    int per_sm = 0;
    dispatch_batch_l<MaxBlocks>(b->prm.l, b->block, smem, &per_sm);
    const int grid = std::max(1, std::min(b->nitems, num_sms() * std::max(per_sm, 1)));
    if (b->nitems > 0) dispatch_batch_l<RunBatch>(b->prm.l, a, grid, b->block, smem, s);
    if (b->ntitems > 0) {
        BatchTileArgs t;
        memset(&t, 0, sizeof(t));
        t.ft = b->ft_d;
        t.items = b->titems_d;
        t.nitems = b->ntitems;
        t.ctl = b->ctl;
        t.pts = pts;
        t.bins = b->prm.rdf_bins;
        t.T = b->T_d;
        t.counts = b->counts;
        t.esc = b->esc;
        t.esc_cap = b->esc_cap;
        t.q = b->q;
        t.Q = b->Q;
        t.nn = b->nn;
        t.qesc = b->qesc;
        FGB_TRY(batch_tile_run(t, b->prm.l, b->tl, b->small_r, b->q_ns, s));
    }
    {
        FGB_KSCOPE("k_batch_escalated", s);
        k_batch_escalated<<<num_sms() * 2, 256, 0, s>>>(a);
    }
    FGB_LAUNCH_CHECK();
    return FGB_OK;
}

extern "C" int fgb_batch_create(int32_t n_frames, const int64_t *frame_offsets, const fgb_box *boxes,
                                const fgb_batch_params *params, void *stream, fgb_batch **out) {
    clear_error();
    if (!out || !frame_offsets || !boxes || !params) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (n_frames <= 0) return fail(FGB_ERR_INVALID_ARG, "n_frames must be positive");
    const fgb_batch_params &p = *params;
    if (!(p.r_max > 0.0) || p.l < -1 || p.l > 12 || p.rdf_bins <= 0 || !(p.rdf_r_max > p.rdf_r_min) ||
        p.rdf_r_min < 0.0)
        return fail(FGB_ERR_INVALID_ARG, "invalid batch parameters");
    if (p.cell_div < 0 || p.cell_div > 2 || p.block < 0 || p.block > 512 || (p.block && p.block % 32) ||
        p.hist_copies < 0 || p.hist_copies > 4 || p.tile_cells < -1 || p.tile_cells > 4096 ||
        (p.cells_per_warp != 0 && p.cells_per_warp != 1 && p.cells_per_warp != 2 && p.cells_per_warp != 4 &&
         p.cells_per_warp != 8))
        return fail(FGB_ERR_INVALID_ARG, "invalid tuning parameters");
    if (frame_offsets[0] != 0) return fail(FGB_ERR_INVALID_ARG, "frame_offsets[0] must be 0");
    for (int f = 0; f < n_frames; ++f)
        if (frame_offsets[f + 1] < frame_offsets[f]) return fail(FGB_ERR_INVALID_ARG, "frame_offsets must not decrease");
    if (frame_offsets[n_frames] >= ((int64_t)1 << 31)) return fail(FGB_ERR_CAPACITY, "at most 2^31-1 points in total");
    cudaStream_t s = as_stream(stream);
    fgb_batch *b = new fgb_batch();
    b->nframes = n_frames;
    b->off.assign(frame_offsets, frame_offsets + n_frames + 1);
    b->boxes.assign(boxes, boxes + n_frames);
    b->prm = p;
    b->total = frame_offsets[n_frames];
    b->tune_div = p.cell_div == 0;
    b->tune_block = p.block == 0;
    b->tune_copies = p.hist_copies == 0;
    b->tune_tile = p.tile_cells == 0;
    b->tune_qb = p.cells_per_warp == 0;
    b->copies = p.hist_copies ? p.hist_copies : 2;
    b->stream = s;
    const int bins = p.rdf_bins;
    b->T_h.resize(bins + 1);
    const double delta = (p.rdf_r_max - p.rdf_r_min) / bins;
    for (int e = 0; e < bins; ++e) b->T_h[e] = sqrt_threshold(p.rdf_r_min + e * delta);
    b->T_h[bins] = sqrt_threshold(p.rdf_r_max);
    const int64_t n = b->total;
    const int L = p.l < 0 ? 0 : p.l;
    b->esc_cap = (int)std::min<int64_t>(std::max<int64_t>(n, 1 << 16), 1 << 26);
    // frame of each binning block's first point: the last frame starting at or before it
    b->blk.resize((size_t)std::max<int64_t>((n + kBinBlock - 1) / kBinBlock, 1));
    for (size_t k = 0; k < b->blk.size(); ++k) {
        const int64_t g0 = (int64_t)k * kBinBlock;
        b->blk[k] = (int32_t)(std::upper_bound(b->off.begin(), b->off.end(), g0) - b->off.begin() - 1);
        b->blk[k] = std::min(std::max(b->blk[k], 0), n_frames - 1);
    }
    int st = dalloc_n(&b->off_d, n_frames + 1, s);
    st = st ? st : dalloc_n(&b->blk_d, b->blk.size(), s);
    st = st ? st : dalloc_n(&b->T_d, bins + 1, s);
    st = st ? st : dalloc_n(&b->ctl, 4, s);
    st = st ? st : dalloc_n(&b->keys, n, s);
    st = st ? st : dalloc_n(&b->vals, n, s);
    st = st ? st : dalloc_n(&b->skeys, n, s);
    st = st ? st : dalloc_n(&b->local, n, s);
    st = st ? st : dalloc_n(&b->sorted, n, s);
    st = st ? st : dalloc(&b->sort_ws, sort_ws_bytes(n), s);
    st = st ? st : dalloc_n(&b->counts, (size_t)n_frames * bins, s);
    st = st ? st : dalloc_n(&b->q, n, s);
    st = st ? st : dalloc_n(&b->Q, (size_t)n * (L + 1), s);
    st = st ? st : dalloc_n(&b->nn, n, s);
    st = st ? st : dalloc_n(&b->esc, b->esc_cap, s);
    st = st ? st : dalloc_n(&b->qesc, 2, s);
    if (st == FGB_OK && p.l >= 0) st = ensure_consts();
    if (st == FGB_OK) st = batch_tile_init(std::min(bins, kBatchTileMaxBins), p.l, &b->tl);
    if (st == FGB_OK) {
        cudaMemcpyAsync(b->off_d, frame_offsets, sizeof(int64_t) * (n_frames + 1), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(b->blk_d, b->blk.data(), sizeof(int32_t) * b->blk.size(), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(b->T_d, b->T_h.data(), sizeof(double) * (bins + 1), cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(b->qesc, 0, 2 * sizeof(unsigned long long), s);
        st = configure(b, p.cell_div ? p.cell_div : 1, p.block ? p.block : 128, p.tile_cells ? p.tile_cells : 64,
                       p.cells_per_warp ? p.cells_per_warp : 1, s);
    }
    if (st != FGB_OK) {
        fgb_batch_destroy(b);
        return st;
    }
    *out = b;
    return FGB_OK;
}

extern "C" void fgb_batch_destroy(fgb_batch *b) {
    if (!b) return;
    cudaStream_t s = b->stream;
    drop_graph(b);
    free_config(b, s);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    dfree(b->off_d, s);
    dfree(b->blk_d, s);
    dfree(b->T_d, s);
    dfree(b->ctl, s);
    dfree(b->keys, s);
    dfree(b->vals, s);
    dfree(b->skeys, s);
    dfree(b->local, s);
    dfree(b->sorted, s);
    dfree(b->sort_ws, s);
    dfree(b->counts, s);
    dfree(b->q, s);
    dfree(b->Q, s);
    dfree(b->nn, s);
    dfree(b->esc, s);
    dfree(b->qesc, s);
    delete b;
}

extern "C" int fgb_batch_run(fgb_batch *b, const float *points, void *stream) {
    clear_error();
    if (!b || (b->total > 0 && !points)) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    return enqueue(b, points, as_stream(stream));
}

extern "C" int fgb_batch_run_graph(fgb_batch *b, const float *points, void *stream) {
    clear_error();
    if (!b || (b->total > 0 && !points)) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = as_stream(stream);
    if (!b->gexec || b->graph_pts != points) {
        drop_graph(b);
        if (!b->cap_stream) FGB_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
        FGB_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        int st = enqueue(b, points, b->cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
        if (st != FGB_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return fail(FGB_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
        b->graph = g;
        FGB_CUDA(cudaGraphInstantiate(&b->gexec, g, 0));
        b->graph_pts = points;
    }
    FGB_CUDA(cudaGraphLaunch(b->gexec, s));
    return FGB_OK;
}

extern "C" int fgb_batch_tune(fgb_batch *b, const float *points, void *stream, fgb_batch_params *chosen) {
    clear_error();
    if (!b || (b->total > 0 && !points)) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = as_stream(stream);
    std::vector<int> divs = b->tune_div ? std::vector<int>{1, 2} : std::vector<int>{b->cell_div};
    std::vector<int> tiles = b->tune_tile ? std::vector<int>{16, 64} : std::vector<int>{b->tile_cells};
    std::vector<int> blocks = b->tune_block ? std::vector<int>{64, 128, 256} : std::vector<int>{b->block};
    std::vector<int> copies = b->tune_copies ? std::vector<int>{1, 2, 4} : std::vector<int>{b->copies};
    std::vector<int> qbs = b->tune_qb ? std::vector<int>{1, 2, 4, 8} : std::vector<int>{b->qbw};
    cudaEvent_t e0, e1;
    FGB_CUDA(cudaEventCreate(&e0));
    FGB_CUDA(cudaEventCreate(&e1));
    float best = INFINITY;
    int bd = b->cell_div, bt = b->tile_cells, bb = b->block, bc = b->copies, bq = b->qbw;
    int st = FGB_OK;
    for (int dv : divs) {
        for (int tc : tiles) {
            for (int bl : blocks) {
              for (int qb : qbs) {
                st = configure(b, dv, bl, tc, qb, s);
                if (st) break;
                // settings of a kernel with no work in this division are timed once
                if (b->ntitems == 0 && (tc != tiles[0] || qb != qbs[0])) break;
                if (b->nitems == 0 && bl != blocks[0]) break;
                if (b->nitems > 0 && b->ntitems > 0 && qb != qbs[0] && bl != blocks[0]) break;
                for (int cp : copies) {
                    if (cp * 32 > bl) continue;
                    if (b->nitems == 0 && cp != copies[0]) break;
                    b->copies = cp;
                    st = enqueue(b, points, s);  // warm-up
                    if (st) break;
                    float tot = 0.f;
                    for (int r = 0; r < 3 && st == FGB_OK; ++r) {
                        cudaEventRecord(e0, s);
                        st = enqueue(b, points, s);
                        cudaEventRecord(e1, s);
                        cudaEventSynchronize(e1);
                        float ms = 0.f;
                        cudaEventElapsedTime(&ms, e0, e1);
                        tot += ms;
                    }
                    if (st == FGB_OK && tot < best) {
                        best = tot;
                        bd = dv;
                        bt = tc;
                        bb = bl;
                        bc = cp;
                        bq = qb;
                    }
                }
                if (st) break;
              }
              if (st) break;
            }
            if (st) break;
        }
        if (st) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    FGB_TRY(st);
    b->copies = bc;
    FGB_TRY(configure(b, bd, bb, bt, bq, s));
    if (chosen) {
        *chosen = b->prm;
        chosen->cell_div = bd;
        chosen->block = bb;
        chosen->hist_copies = bc;
        chosen->tile_cells = bt;
        chosen->cells_per_warp = bq;
    }
    return FGB_OK;
}

extern "C" int fgb_batch_outputs(const fgb_batch *b, const uint64_t **rdf_counts, const float **q,
                                 const int32_t **n_neighbors) {
    if (!b) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    if (rdf_counts) *rdf_counts = reinterpret_cast<const uint64_t *>(b->counts);
    if (q) *q = b->q;
    if (n_neighbors) *n_neighbors = b->nn;
    return FGB_OK;
}

extern "C" int fgb_batch_routes(const fgb_batch *b, int32_t *tile_frames, int32_t *point_frames) {
    if (!b) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    if (tile_frames) *tile_frames = b->ntile_frames;
    if (point_frames) *point_frames = b->nframes - b->ntile_frames;
    return FGB_OK;
}
