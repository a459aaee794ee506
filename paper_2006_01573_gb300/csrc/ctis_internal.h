// Internal types shared by the host plan builder and the CUDA kernels.
//
// Both projectors are one "windowed gather" kernel. A work item names an output
// tile and a contiguous range of tasks; a task names one spot cluster applied to
// that tile: a K x K weight set and the origin of the input window it reads.
//   forward  (Eqs. 1, 8-9): output = FPA tile, input windows from f_s planes,
//            weights flipped (the cluster is applied as a convolution);
//   adjoint  (Eq. 11):      output = voxel tile of wavelength s, input windows
//            from the FPA vector r, weights as stored (a correlation).
// Tiles with more tasks than one item holds are split into chunks whose
// partial sums are added, in chunk order, by the last chunk to finish.
// Every warp is an independent worker with a static list of items, balanced
// longest-first on the host, so the kernels need no work-fetch atomics and
// no block-wide barriers.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace ctis {

constexpr int kNumStats = 4;   // flux_hf, flux_g, loglik, resid2 (see ctis.h)

struct TileDesc {        // 32 bytes
    int x0, y0;          // output origin: FPA (x, y) forward, voxel (p, r) adjoint
    int plane;           // output plane: 0 forward, wavelength s adjoint
    int nchunks;         // items covering this tile
    int scratch_base;    // first partial-sum slot (only used when nchunks > 1)
    int pad0, pad1, pad2;
};

struct ItemDesc {        // 16 bytes
    int tile;
    int chunk;           // 0 .. nchunks-1
    int task_begin;
    int task_end;
};

struct TaskDesc {        // 16 bytes
    int wx;              // window origin x, a multiple of the 16-byte element count
    int wy;              // window origin y (any integer; TMA zero-fills outside)
    int plane;           // input plane (wavelength s forward, 0 adjoint)
    int wsel;            // (weight set index << 3) | (x offset inside the first chunk)
};

enum Epilogue : int {
    kEpiRaw = 0,     // out_f32 = value                      (ctis_forward / ctis_adjoint)
    kEpiRatio = 1,   // u = g / value, 0 where value == 0   (forward inside EM)
    kEpiUpdate = 2,  // f_out = f_in * value / h_s, 0 where h_s == 0 (adjoint inside EM)
    kEpiSet = 3      // f_out = value in the plan's dtype    (H^T g initial guess)
};

struct GatherParams {
    const ItemDesc* items;
    const TileDesc* tiles;
    const TaskDesc* tasks;
    const void* weights;       // [sets][K*K] in the plan's storage type
    const int* warp_begin;     // [n_warps + 1] range of each warp in warp_items
    const int* warp_items;     // item indices in processing order, per warp
    int n_warps;
    int n_tiles;
    int out_w, out_h;          // extent of one output plane
    int mode;                  // Epilogue
    int with_stats;
    // kEpiRaw / kEpiRatio output (float32)
    float* out_f32;
    long long out_plane_stride;
    int out_pitch;
    // kEpiRatio
    const float* g;
    int g_pitch;
    // kEpiUpdate / kEpiSet (datacube in the plan's dtype)
    const void* f_in;
    void* f_out;
    int f_pitch;
    long long f_plane_stride;
    const float* h;            // [w]
    // workspace
    float* scratch;            // partial tiles, [slots][TX*TY]
    int* tickets;              // [n_tiles], zero between launches
    int* counters;             // [2] stat tiles done, [3] error flag (others unused)
    double* tile_stats;        // [n_tiles][kNumStats]
    double* stats_out;         // [kNumStats] or nullptr
};

// Compile-time configuration of one gather kernel instantiation.
struct GatherShape {
    int C;    // columns per lane
    int R;    // rows per lane
    int LX;   // lanes along x (32 / LX along y)
    int NW;   // warps per CTA (independent workers; they share nothing)
    int NS;   // TMA stages per warp
};

constexpr GatherShape kShapeMain{8, 8, 4, 1, 2};   // 32 x 64 output tile per warp

}  // namespace ctis
