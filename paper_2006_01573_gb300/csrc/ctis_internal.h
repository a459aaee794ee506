// Internal types shared by the host plan builder and the CUDA kernels.
//
// Both projectors are one "windowed gather" kernel. A work item names an output
// tile and a contiguous range of tasks; a task names one spot cluster applied to
// that tile: a K x K weight set and the origin of the input window it reads.
//   forward  (Eqs. 1, 8, 12): output = FPA tile, input windows from f_s planes,
//            weights flipped (the cluster is applied as a convolution);
//   adjoint  (Eq. 14):      output = voxel tile of wavelength s, input windows
//            from the FPA vector r, weights as stored (a correlation).
// Tiles with more tasks than one item holds are split into chunks whose
// partial sums are added, in chunk order, by the last chunk to finish. Items
// are balanced longest-first over persistent CTAs; the warps of a CTA share
// each item's tasks and add their sums in shared memory.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace ctis {

constexpr int kNumStats = 4;   // flux_hf, flux_g, loglik, resid2 (see ctis.h)
// slices (one warp each) of a frame's tile statistics in the two-level
// float64 frame reduction
constexpr int kStatSlices = 8;

struct TileDesc {        // 32 bytes (host-side bookkeeping)
    int x0, y0;          // output origin: FPA (x, y) forward, voxel (p, r) adjoint
    int plane;           // output plane: 0 forward, wavelength s adjoint
    int nchunks;         // items covering this tile
    int scratch_base;    // first partial-sum slot (only used when nchunks > 1)
    int pad0, pad1, pad2;
};

struct ItemDesc {        // 16 bytes (host-side bookkeeping)
    int tile;
    int chunk;           // 0 .. nchunks-1
    int task_begin;
    int task_end;
};

// One work item as a warp reads it (its share of the item's tasks):
// everything it needs in a single 32-byte load, stored in the order the warp
// processes its items.
struct WorkItem {
    int tile, x0, y0, plane;
    int chunk_info;      // nchunks | (chunk << 16)
    int scratch_base;
    int task_begin, task_end;
};

// Input planes are kept as NC = 4 x-shifted copies: copy q holds plane[x - q]
// at x (rows are NC - 1 elements wider than the plane; the rest is zero). A
// window whose origin x0 is not a multiple of 4 is read from copy
// q = (-x0) mod 4 at x0 + q, a multiple of 4: 16-byte aligned for float32, so
// every TMA box and shared-memory load is aligned and the kernel has a single
// code path; 8-byte aligned for bfloat16, whose box then starts at the 16-byte
// boundary below and whose lanes start 0 or 4 elements into it.
struct TaskDesc {        // 16 bytes
    int wx;              // aligned window origin x inside the chosen copy
    int wy;              // window origin y (any integer; TMA zero-fills outside)
    int plane;           // TMA depth coordinate: copy * planes + plane
    int cluster;         // weight set index
};

// A warp's start, read in one round of independent loads instead of a chain
// (item range -> first item -> first task -> next task): its items and tasks,
// its first item and its first three task descriptors (fewer are valid when
// it has fewer tasks). 96 bytes.
struct WarpHead {
    int ib, ie;                  // range in the item list
    int task_begin, task_end;    // the warp's tasks
    TaskDesc first[3];
    WorkItem item0;
};

enum Epilogue : int {
    kEpiRaw = 0,     // out_f32 = value                      (ctis_forward / ctis_adjoint)
    kEpiRatio = 1,   // u copies = g / value, 0 where value == 0  (forward inside EM)
    kEpiUpdate = 2,  // f copies = f_in * value / h_s, 0 where h_s == 0 (adjoint inside EM)
    kEpiSet = 3,     // f copies = value in the plan's dtype  (H^T g initial guess)
    kEpiGrad = 4     // no output tile: per task, the K x K sums of f_s times the
                     // task's input window (PSF-value gradient), into grad_part
};

// Update rule of the EM-style launches (kEpiRatio forward, kEpiUpdate
// adjoint); values as CTIS_SOLVER_* in ctis.h.
enum Solver : int {
    kSolverEm = 0,      // u = g / q;              f <- f * z / h            (Eq. 2)
    kSolverSart = 1,    // u = (g - q) / (H 1);    f <- max(f + relax z / h, 0)
    kSolverSmart = 2    // u = log(g / q);         f <- f * exp(relax z / h)
};

struct GatherParams {
    const WorkItem* items;     // grouped by warp, in processing order
    const int* warp_begin;     // [n_warps + 1] range of each warp in items
    const WarpHead* heads;     // [n_warps] each warp's start
    const TaskDesc* tasks;     // in item order: each warp's tasks are contiguous
    const void* weights;       // [clusters][padded K*K] in the plan's storage type
    int n_warps;
    int n_tiles;
    int out_w, out_h;          // extent of one output plane
    int mode;                  // Epilogue
    int with_stats;
    // kEpiRaw output, or the kEpiRatio u copies (float32)
    float* out_f32;
    long long out_plane_stride;  // kEpiRaw: between output planes; kEpiRatio: between frames
    int out_pitch;
    long long out_copy_stride;   // kEpiRatio: elements between u copies
    int out_copies;              // kEpiRatio: number of u copies
    // kEpiRatio (item plane = frame of a batch, 0 otherwise)
    const float* g;
    int g_pitch;
    long long g_plane_stride;    // elements between frames of g
    // frame totals of a previous forward's tile statistics, added at the start
    // of this launch by red_frames * kStatSlices warps (red_out null: none)
    const double* red_src;       // [frames][tiles][kNumStats]
    double* red_out;             // frame f's row at red_out + f * red_frame_stride
    int red_tiles_per_frame;
    int red_frames;
    long long red_frame_stride;
    double* red_part;            // [frames][kStatSlices][kNumStats] slice sums
    int* red_tickets;            // [frames], zero between launches
    // kEpiUpdate / kEpiSet (datacube copies in the plan's dtype; f_in = copy 0)
    const void* f_in;
    void* f_out;
    int f_pitch;
    long long f_plane_stride;
    long long f_copy_stride;
    int f_copies;
    const float* h;            // [w] (planes f*w + s in a batch)
    // CTIS_BOUNDARY_CLIP: h per voxel, [w][out_h][out_w] (null otherwise); a
    // batch's planes f*w + s use h_vox plane (f*w + s) % h_vox_planes
    const float* h_vox;
    int h_vox_planes;
    // kEpiRatio: write 1 - g / value instead of g / value (0 where value == 0)
    int ratio_one_minus;
    // kEpiRatio / kEpiUpdate: the solver's rule (Solver) and relaxation;
    // kSolverSart's forward divides by the row sums r = H 1, [out_h][out_w]
    // dense (single frames only)
    int solver;
    float relax;
    const float* row_sum;
    // kEpiGrad: f_in is the dense datacube [w][alpha][a] (out_w = a,
    // out_h = alpha); sums go to grad_part[(cluster * tiles_per_plane + tile
    // of the plane) * K * K + dy * K + dx]
    float* grad_part;
    int grad_tiles_per_plane;
    // workspace
    float* scratch;            // partial tiles, [slots][TX*TY]
    int* tickets;              // [n_tiles], zero between launches
    int* counters;             // [3] error flag, [8 + f] frame f's statistics ticket
    // placement probe: when set, each CTA writes its SM id to smid_out[CTA],
    // stays resident ~30 us (so the grid is placed as a real launch is) and
    // returns without touching anything else
    int* smid_out;
    // test hook (ctis_plan_set_debug): arm each copy's barrier without
    // issuing the copy, so every wait runs out through its bounded path
    int drop_copies;
    double* tile_stats;        // [n_tiles][kNumStats] written by kEpiRatio with_stats
    // host side only: launch the projector with programmatic dependent launch
    // (its prologue overlaps the tail of the stream's previous kernel)
    int overlap_launch;
};

// Compile-time configuration of one gather kernel instantiation.
struct GatherShape {
    int C;    // columns per lane
    int R;    // rows per lane
    int LX;   // lanes along x (32 / LX along y)
    int NW;   // warps per CTA (they share each item's tasks)
    int NS;   // TMA stages per warp
};

// Shapes of the two projectors. The defaults can be overridden at build time
// (-DCTIS_FWD_R=..., etc.) to sweep them.
#ifndef CTIS_FWD_R
#define CTIS_FWD_R 8
#endif
#ifndef CTIS_FWD_NS
#define CTIS_FWD_NS 2
#endif
#ifndef CTIS_FWD_NS_BF16
#define CTIS_FWD_NS_BF16 3
#endif
#ifndef CTIS_ADJ_R
#define CTIS_ADJ_R 8
#endif
#ifndef CTIS_ADJ_NS
#define CTIS_ADJ_NS 2
#endif
#ifndef CTIS_NW
#define CTIS_NW 4
#endif
constexpr GatherShape kShapeFwd{4, CTIS_FWD_R, 8, CTIS_NW, CTIS_FWD_NS};   // 32 x 32 tile
constexpr GatherShape kShapeAdj{4, CTIS_ADJ_R, 8, CTIS_NW, CTIS_ADJ_NS};   // 32 x 32 tile

#ifdef CTIS_DEBUG_BOUNDS
// Buffers the epilogues may touch, registered by debug builds only.
struct DbgRanges { const char* lo[6]; const char* hi[6]; unsigned long long* log; };
#endif

}  // namespace ctis
