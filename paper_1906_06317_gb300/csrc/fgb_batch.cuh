// Cell-tile route of the batched frames (batch_tile.cu): per-frame arguments built by the
// batch configuration (batch.cu) and the launches of its two kernels.
#pragma once

#include "fgb_tile.cuh"

namespace fgb {

constexpr int kBatchTileWarps = 4;  // warps per block of both kernels

struct FrameTile {
    TileArgs r;   // RDF: half stencil of the RDF radius (each unordered pair once, weight 2)
    TileArgs b;   // q_l: full stencil of the ball radius, T and band of its exact test
    BinParams P;  // RDF binning of this frame (bands around its bin edges)
    int f;        // frame index (row of the counts)
    int qb;       // q_l: query cells per warp (x-adjacent cells of a row taken together)
    int qbr;      // RDF: the same for its half stencil
    int pad;
};

struct BatchTileArgs {
    const FrameTile *ft;
    const int4 *items;           // (tile frame, first cell, end cell, 0), frame-local cells
    int nitems;
    int *ctl;                    // [1] FP64 list slots, [2] RDF item counter, [3] q_l item counter
    const float *pts;            // packed caller coordinates (global indices)
    int bins;
    const double *T;             // exact squared edges, bins + 1
    unsigned long long *counts;  // nframes x bins
    int4 *esc;                   // (frame, i, j, weight) left to the FP64 pass
    int esc_cap;
    float *q;
    float2 *Q;
    int32_t *nn;
    unsigned long long *qesc;    // [0] FP64 ball re-decisions
};

// Persistent grids (blocks resident at once) of the stencil capacities: RDF [0] half
// stencil (or the union of a block's half stencils) <= 64 cells, [1] kTileMaxStencil;
// q_l [0] ball stencil (or the union of a block's stencils) <= 32 cells, [1] <= 64,
// [2] kTileMaxStencil.
struct BatchTileLaunch {
    unsigned grid_r[2], grid_q[3];
    size_t smem_r;               // dynamic shared memory of the RDF kernel (histograms)
    int warps;                   // warps of the RDF kernel resident at once
};

// Sets the kernels' shared-memory limits and Legendre constants for `bins` and `l`
// (outside any stream capture) and returns their launch shapes.
int batch_tile_init(int bins, int l, BatchTileLaunch *out);
// RDF counts, then q_l (l >= 0), of every frame on the tile route; small_r: every tile
// frame's RDF half stencil has at most 64 cells; q_ns: the q_l stencil capacity (32, 64
// or kTileMaxStencil) that every tile frame's ball stencil, or block union, fits.
int batch_tile_run(const BatchTileArgs &a, int l, const BatchTileLaunch &g, bool small_r, int q_ns, cudaStream_t s);

}  // namespace fgb
