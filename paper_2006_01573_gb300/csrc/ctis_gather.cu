// Windowed-gather kernels for the shift-invariant CTIS projector pair.
//
// Forward (Eqs. 1, 8-9):  (H f)(x, y) = sum_s sum_k v_{s,k} f_s(x - x_k, y - y_k)
// Adjoint (Eq. 11):     (H^T r)_s(p, r) = sum_k v_{s,k} r(x_k + p, y_k + r)
//
// The PSF nonzeros of each wavelength are grouped into K x K spot clusters.
// Applying one cluster to an output tile is a K x K correlation of a window of
// the input plane (forward: f_s, zero outside the field stop; adjoint: the FPA
// vector) with the cluster's weights (flipped for the forward). Both
// projectors are therefore gathers: every output element is owned by one
// thread, no atomics touch data, and the summation order is fixed by the plan,
// so results are bit-reproducible.
//
// GB300 mapping:
//  * persistent CTAs (one per SM slot) pull work items from an atomic counter;
//    items are sorted longest-first when the plan is built;
//  * the NW warps of a CTA share one output tile and split its task list;
//    each warp stages its own windows with TMA (cp.async.bulk.tensor) into NS
//    shared-memory stages completed on mbarriers, so warps never wait on each
//    other inside the task loop;
//  * a window is loaded as LY row slabs (one per lane row) placed at a skewed
//    stride so that the 16-byte shared-memory loads of each quarter warp hit
//    eight different bank groups; TMA fills coordinates outside the plane
//    with zeros, which is exactly the zero padding of the forward projector;
//  * each lane keeps an R x C block of outputs in registers and slides down
//    the window one input row at a time, so every staged value feeds up to
//    K*K FMAs;
//  * epilogues are fused: the EM ratio u = g / (H f) with float64 statistics,
//    and the multiplicative update f <- f * (H^T u) / h.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "ctis_internal.h"
#include "ctis_kernels.h"

namespace ctis {
namespace {

// ---------------------------------------------------------------------------
// PTX helpers: mbarrier, TMA
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after ~2^31 SM cycles (about a second), records the
// failure in the plan's error flag and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (1ll << 31)) {
            atomicOr(err, 1);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y,
                                            int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// element conversion
// ---------------------------------------------------------------------------
template <typename T>
struct Elem;
template <>
struct Elem<float> {
    static constexpr int kPerChunk = 4;   // elements per 16-byte chunk
    __device__ static __forceinline__ void load_chunk(const float* p, float* out) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
    }
    __device__ static __forceinline__ float load(const float* p) { return *p; }
    __device__ static __forceinline__ void store(float* p, float v) { *p = v; }
    __device__ static __forceinline__ float weight(const void* w, int i) {
        return __ldg(static_cast<const float*>(w) + i);
    }
};
template <>
struct Elem<__nv_bfloat16> {
    static constexpr int kPerChunk = 8;
    __device__ static __forceinline__ void load_chunk(const __nv_bfloat16* p, float* out) {
        const uint4 v = *reinterpret_cast<const uint4*>(p);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            out[2 * q] = __uint_as_float(w[q] << 16);
            out[2 * q + 1] = __uint_as_float(w[q] & 0xffff0000u);
        }
    }
    __device__ static __forceinline__ float load(const __nv_bfloat16* p) {
        return __bfloat162float(*p);
    }
    __device__ static __forceinline__ void store(__nv_bfloat16* p, float v) {
        *p = __float2bfloat16_rn(v);
    }
    __device__ static __forceinline__ float weight(const void* w, int i) {
        const unsigned short b = __ldg(static_cast<const unsigned short*>(w) + i);
        return __uint_as_float(static_cast<uint32_t>(b) << 16);
    }
};

// ---------------------------------------------------------------------------
// compile-time geometry of one instantiation
// ---------------------------------------------------------------------------
// Bank-conflict avoidance. Every slab starts on a 128-byte boundary (required
// of tensor TMA destinations), so slab strides are a multiple of eight 16-byte
// bank groups. To keep the two lane rows of a quarter warp apart, odd slabs
// are loaded SH elements further left in x: their data sits SH elements
// (a whole number of chunks) to the right in shared memory. pick_shift
// returns the smallest such SH for which the first chunks read by the 8 lanes
// of every quarter warp fall into 8 different bank groups, or -1.
constexpr int pick_shift(int LX, int C, int epc) {
    for (int sh = 0; sh < 8; ++sh) {
        bool ok = true;
        for (int ph = 0; ph < 4 && ok; ++ph) {
            int used = 0;
            for (int l = ph * 8; l < ph * 8 + 8; ++l) {
                const int tx = l % LX, ty = l / LX;
                const int ch = (tx * C / epc + ((ty & 1) ? sh : 0)) % 8;
                if (used & (1 << ch)) { ok = false; break; }
                used |= 1 << ch;
            }
        }
        if (ok) return sh * epc;
    }
    return -1;
}

template <int K_, int C_, int R_, int LX_, int NW_, int NS_, typename TIn>
struct Geo {
    static constexpr int K = K_, C = C_, R = R_, LX = LX_, NW = NW_, NS = NS_;
    static constexpr int LY = 32 / LX;
    static constexpr int TX = LX * C, TY = LY * R;
    static constexpr int ES = int(sizeof(TIn));
    static constexpr int EPC = Elem<TIn>::kPerChunk;
    // data a window row needs: TX + K - 1 elements starting up to EPC - 1 past
    // a chunk boundary
    static constexpr int BX0 = ((TX + K - 1 + EPC - 1) + EPC - 1) / EPC * EPC;
    static constexpr int SH = pick_shift(LX, C, EPC);
    static_assert(SH >= 0, "no conflict-free slab shift for this shape");
    static constexpr int BXW = BX0 + SH;   // TMA box width = smem row pitch
    static constexpr int SLAB_STRIDE = (R * BXW * ES + 127) / 128 * 128 / ES;
    static constexpr int HALO = K - 1;
    static_assert(HALO <= R, "halo rows must fit in the next slab");
    static constexpr int WINDOW_ELEMS = LY * SLAB_STRIDE + HALO * BXW;
    static constexpr int STAGE_ELEMS = (WINDOW_ELEMS * ES + 127) / 128 * 128 / ES;
    static constexpr int STAGE_BYTES = STAGE_ELEMS * ES;
    static_assert((SLAB_STRIDE * ES) % 128 == 0 && STAGE_BYTES % 128 == 0,
                  "TMA destinations must be 128-byte aligned");
    static_assert((BXW * ES) % 16 == 0 && BXW <= 256, "TMA box row");
    static constexpr uint32_t TX_BYTES = uint32_t((LY * R + HALO) * BXW * ES);
    static constexpr int TILE = TX * TY;
    static constexpr int THREADS = NW * 32;
    static constexpr int STAGES_BYTES = NW * NS * STAGE_BYTES;
    static constexpr int SMEM_BYTES = STAGES_BYTES + NW * NS * 8;
    // x offset of slab g's data relative to the window origin
    __host__ __device__ static constexpr int slab_shift(int g) { return (g & 1) ? SH : 0; }
};

// ---------------------------------------------------------------------------
// per-lane correlation of one staged window
// ---------------------------------------------------------------------------
// acc[o][c] += sum_{dy,dx} w[dy][dx] * win[o + dy][c + dx + REM]
// `win0` points at this lane's first element in its own slab (row 0), `win1`
// at the same column in the next slab (the next lane row's slab, or the halo
// slab for the last lane row), which supplies rows R .. R + K - 2.
template <class G, int REM, typename TIn>
__device__ __forceinline__ void correlate(float2 (&acc)[G::R][G::C / 2], const TIn* win0,
                                          const TIn* win1, const float (&w)[G::K * G::K]) {
    constexpr int K = G::K, C = G::C, R = G::R;
    constexpr int NE = C + K - 1 + REM;
    constexpr int NCH = (NE + G::EPC - 1) / G::EPC;
    float2 w2[K * K];
#pragma unroll
    for (int q = 0; q < K * K; ++q) w2[q] = make_float2(w[q], w[q]);
#pragma unroll
    for (int i = 0; i < R + K - 1; ++i) {
        const TIn* rowp = i < R ? win0 + i * G::BXW : win1 + (i - R) * G::BXW;
        float in[NCH * G::EPC];
#pragma unroll
        for (int q = 0; q < NCH; ++q) Elem<TIn>::load_chunk(rowp + q * G::EPC, in + q * G::EPC);
#pragma unroll
        for (int dy = 0; dy < K; ++dy) {
            const int o = i - dy;
            if (o >= 0 && o < R) {
#pragma unroll
                for (int c = 0; c < C; c += 2) {
#pragma unroll
                    for (int dx = 0; dx < K; ++dx) {
                        // two adjacent outputs per packed FP32 FMA (FFMA2)
                        const float2 x2 = make_float2(in[c + dx + REM], in[c + 1 + dx + REM]);
                        acc[o][c / 2] = __ffma2_rn(x2, w2[dy * K + dx], acc[o][c / 2]);
                    }
                }
            }
        }
    }
}

template <class G, typename TIn, int REM = 0>
__device__ __forceinline__ void correlate_dispatch(int rem, float2 (&acc)[G::R][G::C / 2],
                                                   const TIn* win0, const TIn* win1,
                                                   const float (&w)[G::K * G::K]) {
    if constexpr (REM < G::EPC) {
        if (rem == REM) {
            correlate<G, REM, TIn>(acc, win0, win1, w);
        } else {
            correlate_dispatch<G, TIn, REM + 1>(rem, acc, win0, win1, w);
        }
    }
}

// ---------------------------------------------------------------------------
// epilogues (per warp, straight from the lanes' register blocks)
// ---------------------------------------------------------------------------
// Lane (tx, ty) owns tile rows ty*R .. ty*R+R-1 and columns tx*C .. tx*C+C-1.
template <class G>
__device__ __forceinline__ int tile_elem(int tx, int ty, int o, int c) {
    return (ty * G::R + o) * G::TX + tx * G::C + c;
}

// Applies the epilogue to the lane's outputs v[o][c] of `tile`; accumulates
// the forward statistics of the lane in stat[].
template <class G, typename TF>
__device__ __forceinline__ void epilogue(const GatherParams& p, const TileDesc& tile, int tx,
                                         int ty, const float (&v)[G::R][G::C],
                                         float (&stat)[kNumStats]) {
#pragma unroll
    for (int o = 0; o < G::R; ++o) {
        const int y = tile.y0 + ty * G::R + o;
        if (y >= p.out_h) break;
#pragma unroll
        for (int c = 0; c < G::C; ++c) {
            const int x = tile.x0 + tx * G::C + c;
            if (x >= p.out_w) break;
            const float val = v[o][c];
            if (p.mode == kEpiRaw) {
                p.out_f32[tile.plane * p.out_plane_stride + (long long)y * p.out_pitch + x] = val;
            } else if (p.mode == kEpiRatio) {
                const float gv = p.g[(long long)y * p.g_pitch + x];
                p.out_f32[(long long)y * p.out_pitch + x] = val > 0.f ? gv / val : 0.f;
                if (val > 0.f) {
                    stat[0] += val;
                    stat[1] += gv;
                    stat[2] += gv * logf(val) - val;
                    const float d = gv - val;
                    stat[3] += d * d;
                }
            } else {
                const long long j = tile.plane * p.f_plane_stride + (long long)y * p.f_pitch + x;
                TF* fo = static_cast<TF*>(p.f_out);
                if (p.mode == kEpiUpdate) {
                    const float fi = Elem<TF>::load(static_cast<const TF*>(p.f_in) + j);
                    const float hs = p.h[tile.plane];
                    Elem<TF>::store(fo + j, hs != 0.f ? fi * val / hs : 0.f);
                } else {
                    Elem<TF>::store(fo + j, val);
                }
            }
        }
    }
}

// Fixed-order float64 warp sum (same tree on every run); lane 0 gets the total.
__device__ __forceinline__ double warp_sum(double d) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(0xffffffffu, d, off);
    return d;
}

// Tile statistics of the warp that finished the tile; the last tile to finish
// adds all tiles' statistics in tile order into p.stats_out.
__device__ __forceinline__ void finish_stats(const GatherParams& p, int tile_idx,
                                             const float (&stat)[kNumStats], int lane) {
    double tot[kNumStats];
#pragma unroll
    for (int q = 0; q < kNumStats; ++q) tot[q] = warp_sum(static_cast<double>(stat[q]));
    int last = 0;
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < kNumStats; ++q)
            p.tile_stats[(long long)tile_idx * kNumStats + q] = tot[q];
        __threadfence();
        last = atomicAdd(&p.counters[2], 1) == p.n_tiles - 1;
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int q = 0; q < kNumStats; ++q) {
        double t = 0.0;
        for (int i = lane; i < p.n_tiles; i += 32)
            t += __ldcg(&p.tile_stats[(long long)i * kNumStats + q]);
        t = warp_sum(t);
        if (lane == 0) p.stats_out[q] = t;
    }
    if (lane == 0) p.counters[2] = 0;
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
template <class G, typename TIn, typename TF>
__global__ void __launch_bounds__(G::THREADS)
    gather_kernel(const __grid_constant__ CUtensorMap tm_slab,
                  const __grid_constant__ CUtensorMap tm_halo, const GatherParams p) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TIn* stages = reinterpret_cast<TIn*>(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + G::STAGES_BYTES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * G::NW + warp;
    if (gw >= p.n_warps) return;
    const int tx = lane % G::LX, ty = lane / G::LX;
    TIn* my_stages = stages + warp * G::NS * G::STAGE_ELEMS;
    uint64_t* my_bars = bars + warp * G::NS;
    if (lane == 0) {
        for (int s = 0; s < G::NS; ++s) mbar_init(&my_bars[s], 1);
        fence_mbar_init();
    }
    __syncwarp();

    // this lane's first element in its own slab and in the next one
    const int lane_off0 = ty * G::SLAB_STRIDE + tx * G::C + G::slab_shift(ty);
    const int lane_off1 = (ty + 1) * G::SLAB_STRIDE + tx * G::C + G::slab_shift(ty + 1);

    const int ib = p.warp_begin[gw], ie = p.warp_begin[gw + 1];
    uint32_t issued = 0, consumed = 0;   // warp-uniform TMA counters
    bool failed = false;                 // warp-uniform

    // Issue cursor: walks the same (item, task) sequence as the compute loop,
    // up to NS tasks ahead, across item boundaries.
    int cur_item = ib, cur_task = 0, cur_end = 0;
    if (ib < ie) {
        const ItemDesc it = p.items[p.warp_items[ib]];
        cur_task = it.task_begin;
        cur_end = it.task_end;
    }
    auto issue_next = [&]() {
        while (cur_task >= cur_end) {
            if (++cur_item >= ie) return;
            const ItemDesc it = p.items[p.warp_items[cur_item]];
            cur_task = it.task_begin;
            cur_end = it.task_end;
        }
        const TaskDesc t = p.tasks[cur_task++];
        TIn* dst = my_stages + (issued % G::NS) * G::STAGE_ELEMS;
        uint64_t* bar = &my_bars[issued % G::NS];
        if (lane == 0 && !failed) {
            mbar_arrive_expect_tx(bar, G::TX_BYTES);
#pragma unroll
            for (int g = 0; g < G::LY; ++g)
                tma_load_3d(dst + g * G::SLAB_STRIDE, &tm_slab, t.wx - G::slab_shift(g),
                            t.wy + g * G::R, t.plane, bar);
            if constexpr (G::HALO > 0)
                tma_load_3d(dst + G::LY * G::SLAB_STRIDE, &tm_halo, t.wx - G::slab_shift(G::LY),
                            t.wy + G::LY * G::R, t.plane, bar);
        }
        ++issued;
    };
    for (int j = 0; j < G::NS; ++j) issue_next();

    for (int ii = ib; ii < ie; ++ii) {
        const int item_idx = p.warp_items[ii];
        const ItemDesc item = p.items[item_idx];
        const TileDesc tile = p.tiles[item.tile];

        float2 acc[G::R][G::C / 2];
#pragma unroll
        for (int o = 0; o < G::R; ++o)
#pragma unroll
            for (int c = 0; c < G::C / 2; ++c) acc[o][c] = make_float2(0.f, 0.f);

        for (int t = item.task_begin; t < item.task_end; ++t) {
            const int st = consumed % G::NS;
            if (!failed) {
                const bool ok = mbar_wait_bounded(&my_bars[st], (consumed / G::NS) & 1u,
                                                  &p.counters[3]);
                failed = __any_sync(0xffffffffu, !ok);
            }
            if (!failed) {
                const TaskDesc task = p.tasks[t];
                float w[G::K * G::K];
                const int wbase = (task.wsel >> 3) * (G::K * G::K);
#pragma unroll
                for (int q = 0; q < G::K * G::K; ++q) w[q] = Elem<TF>::weight(p.weights, wbase + q);
                const TIn* stage = my_stages + st * G::STAGE_ELEMS;
                correlate_dispatch<G, TIn>(task.wsel & 7, acc, stage + lane_off0,
                                           stage + lane_off1, w);
            }
            ++consumed;
            __syncwarp();
            issue_next();
        }

        float v[G::R][G::C];
#pragma unroll
        for (int o = 0; o < G::R; ++o)
#pragma unroll
            for (int c = 0; c < G::C / 2; ++c) {
                v[o][2 * c] = acc[o][c].x;
                v[o][2 * c + 1] = acc[o][c].y;
            }

        bool finish = true;
        if (tile.nchunks > 1) {
            float* slots = p.scratch + (long long)tile.scratch_base * G::TILE;
            float* mine = slots + (long long)item.chunk * G::TILE;
#pragma unroll
            for (int o = 0; o < G::R; ++o)
#pragma unroll
                for (int c = 0; c < G::C; c += 4)
                    __stcg(reinterpret_cast<float4*>(mine + tile_elem<G>(tx, ty, o, c)),
                           make_float4(v[o][c], v[o][c + 1], v[o][c + 2], v[o][c + 3]));
            __threadfence();
            __syncwarp();
            int old = 0;
            if (lane == 0) old = atomicAdd(&p.tickets[item.tile], 1);
            old = __shfl_sync(0xffffffffu, old, 0);
            finish = old == tile.nchunks - 1;
            if (finish) {
                __threadfence();
#pragma unroll
                for (int o = 0; o < G::R; ++o)
#pragma unroll
                    for (int c = 0; c < G::C; c += 4) {
                        const int e = tile_elem<G>(tx, ty, o, c);
                        float4 s4 = __ldcg(reinterpret_cast<const float4*>(slots + e));
                        for (int ch = 1; ch < tile.nchunks; ++ch) {
                            const float4 q4 =
                                __ldcg(reinterpret_cast<const float4*>(slots + (long long)ch * G::TILE + e));
                            s4.x += q4.x; s4.y += q4.y; s4.z += q4.z; s4.w += q4.w;
                        }
                        v[o][c] = s4.x; v[o][c + 1] = s4.y; v[o][c + 2] = s4.z; v[o][c + 3] = s4.w;
                    }
                if (lane == 0) p.tickets[item.tile] = 0;
            }
        }
        if (finish) {
            float stat[kNumStats] = {0.f, 0.f, 0.f, 0.f};
            epilogue<G, TF>(p, tile, tx, ty, v, stat);
            if (p.with_stats) finish_stats(p, item.tile, stat, lane);
        }
    }

    // Loads still in flight exist only after a failed wait: give them a bounded
    // chance to land before the warp's shared memory is released.
    if (lane == 0) {
        while (consumed < issued) {
            const int st = consumed % G::NS;
            if (!mbar_wait_bounded(&my_bars[st], (consumed / G::NS) & 1u, &p.counters[3])) break;
            ++consumed;
        }
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// small utility kernels
// ---------------------------------------------------------------------------
template <typename TF>
__global__ void fill_kernel(TF* f, int a, int rows, int pitch, float value) {
    const long long n = (long long)a * rows;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long row = i / a, col = i % a;
        Elem<TF>::store(f + row * pitch + col, value);
    }
}

// Sec. 3 embedding: datacube element j = (p, r, s) sits at FPA pixel
// (x, y) = (p, r) of the s-th stacked FPA vector.
__device__ __forceinline__ long long stacked_fpa_index(int p, int r, int s, int gamma, long long n) {
    return (long long)p + (long long)gamma * r + n * s;
}

__global__ void index_map_kernel(long long* out, int a, int alpha, int w, int gamma, long long n) {
    const long long m = (long long)a * alpha * w;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < m;
         j += (long long)gridDim.x * blockDim.x) {
        const int p = int(j % a);
        const int r = int((j / a) % alpha);
        const int s = int(j / ((long long)a * alpha));
        out[j] = stacked_fpa_index(p, r, s, gamma, n);
    }
}

template <class G, typename TIn, typename TF>
cudaError_t prepare_impl(int* blocks_per_sm) {
    auto kern = gather_kernel<G, TIn, TF>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         G::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, G::THREADS,
                                                      G::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    return *blocks_per_sm >= 1 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

template <class G, typename TIn, typename TF>
cudaError_t launch_impl(const CUtensorMap& slab, const CUtensorMap& halo, const GatherParams& p,
                        cudaStream_t stream) {
    const int grid = (p.n_warps + G::NW - 1) / G::NW;
    gather_kernel<G, TIn, TF><<<grid, G::THREADS, G::SMEM_BYTES, stream>>>(slab, halo, p);
    return cudaGetLastError();
}

template <int K, typename TIn>
using GeoMain = Geo<K, kShapeMain.C, kShapeMain.R, kShapeMain.LX, kShapeMain.NW, kShapeMain.NS, TIn>;

// Calls fn.template operator()<G, TIn, TF>() for the instantiation that serves
// (K, dtype, direction).
template <class Fn>
cudaError_t dispatch(bool forward, int K, int dtype, Fn&& fn) {
    auto by_k = [&](auto tin, auto tf) -> cudaError_t {
        using TIn = decltype(tin);
        using TF = decltype(tf);
        switch (K) {
            case 1: return fn.template operator()<GeoMain<1, TIn>, TIn, TF>();
            case 3: return fn.template operator()<GeoMain<3, TIn>, TIn, TF>();
            case 5: return fn.template operator()<GeoMain<5, TIn>, TIn, TF>();
            default: return cudaErrorInvalidValue;
        }
    };
    if (dtype == kDtypeBF16) {
        if (forward) return by_k(__nv_bfloat16{}, __nv_bfloat16{});
        return by_k(float{}, __nv_bfloat16{});
    }
    return by_k(float{}, float{});
}

}  // namespace

// ---------------------------------------------------------------------------
// host entry points used by the plan / API code
// ---------------------------------------------------------------------------
int gather_tile_w() { return kShapeMain.LX * kShapeMain.C; }
int gather_tile_h() { return (32 / kShapeMain.LX) * kShapeMain.R; }
int gather_window_rows(int K) { return (32 / kShapeMain.LX) * kShapeMain.R + K - 1; }

int gather_box_w(int K, int dtype) {
    int bw = -1;
    dispatch(true, K, dtype, [&]<class G, typename TIn, typename TF>() {
        bw = G::BXW;
        return cudaSuccess;
    });
    return bw;
}

int gather_box_w_input_f32(int K) {
    int bw = -1;
    dispatch(false, K, kDtypeF32, [&]<class G, typename TIn, typename TF>() {
        bw = G::BXW;
        return cudaSuccess;
    });
    return bw;
}

cudaError_t gather_prepare(bool forward, int K, int dtype, int* blocks_per_sm) {
    return dispatch(forward, K, dtype, [&]<class G, typename TIn, typename TF>() {
        return prepare_impl<G, TIn, TF>(blocks_per_sm);
    });
}

cudaError_t gather_launch(bool forward, int K, int dtype, const CUtensorMap& slab,
                          const CUtensorMap& halo, const GatherParams& p, cudaStream_t stream) {
    return dispatch(forward, K, dtype, [&]<class G, typename TIn, typename TF>() {
        return launch_impl<G, TIn, TF>(slab, halo, p, stream);
    });
}

int gather_warps_per_cta() { return kShapeMain.NW; }

cudaError_t launch_fill(int dtype, void* f, int a, int rows, int pitch, float value,
                        cudaStream_t stream) {
    const int threads = 256, blocks = 1024;
    if (dtype == kDtypeBF16)
        fill_kernel<__nv_bfloat16><<<blocks, threads, 0, stream>>>(
            static_cast<__nv_bfloat16*>(f), a, rows, pitch, value);
    else
        fill_kernel<float><<<blocks, threads, 0, stream>>>(static_cast<float*>(f), a, rows, pitch,
                                                           value);
    return cudaGetLastError();
}

cudaError_t launch_index_map(long long* out, int a, int alpha, int w, int gamma, long long n,
                             cudaStream_t stream) {
    index_map_kernel<<<1024, 256, 0, stream>>>(out, a, alpha, w, gamma, n);
    return cudaGetLastError();
}

}  // namespace ctis
