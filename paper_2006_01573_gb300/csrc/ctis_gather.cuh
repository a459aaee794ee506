// Windowed-gather device code for the shift-invariant CTIS projector pair,
// shared by the forward and adjoint translation units.
//
// Forward (Eqs. 1, 8, 12):  (H f)(x, y) = sum_s sum_k v_{s,k} f_s(x - x_k, y - y_k)
// Adjoint (Eq. 14):     (H^T r)_s(p, r) = sum_k v_{s,k} r(x_k + p, y_k + r)
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
//  * persistent CTAs with static item lists balanced longest-first on the
//    host; the CTA's warps share each item's tasks and add their sums in
//    shared memory (no work-fetch atomics, no global traffic for a tile that
//    one CTA finishes);
//  * lane 0 stages the input window of each task with tensor TMA
//    (cp.async.bulk.tensor) and the task's weights with a bulk copy into one
//    of NS shared-memory stages completed on an mbarrier, NS tasks ahead of
//    the compute loop, across item boundaries;
//  * a window is one dense TMA box; the 8 lanes of a quarter warp read 8
//    consecutive 16-byte chunks of a row (conflict-free); TMA fills
//    coordinates outside the plane with zeros, which is exactly the zero
//    padding of the forward projector;
//  * each lane keeps an R x C block of outputs in registers and slides down
//    the window one input row at a time, so every staged value feeds up to
//    K*K FMAs;
//  * epilogues are fused and selected at compile time: the EM ratio
//    u = g / (H f) with float64 statistics, and the multiplicative update
//    f <- f * (H^T u) / h.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <type_traits>

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

// Barrier over the CTA's warps only (id 1; id 0 is __syncthreads).
__device__ __forceinline__ void cta_barrier(int nthreads) {
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// GPU-scope release/acquire fence (lighter than the sequentially consistent
// __threadfence): orders this thread's earlier memory accesses, and those it
// has observed, before its later ones for every thread of the GPU.
__device__ __forceinline__ void fence_acq_rel_gpu() {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

// The copy-side operations (the barrier's expected bytes, a tensor-TMA box,
// a bulk copy), executed only by the lanes whose `on` is set (the warp's
// lane 0) as predicated instructions: the warp runs one instruction stream
// instead of branching around a one-lane block.
__device__ __forceinline__ void mbar_arrive_expect_tx_if(bool on, uint64_t* bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %2, 0;\n\t"
        "@p mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
        "r"(bytes), "r"(int(on))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d_if(bool on, void* dst, const CUtensorMap* map, int x,
                                               int y, int z, uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %6, 0;\n\t"
        "@p cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n\t}" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar)),
        "r"(int(on))
        : "memory");
}
__device__ __forceinline__ void bulk_load_if(bool on, void* dst, const void* src, uint32_t bytes,
                                             uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "@p cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        "\n\t}" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "r"(int(on))
        : "memory");
}

// Programmatic dependent launch. launch_dependents lets the stream's next
// kernel be scheduled once every CTA of this grid has executed it (its CTAs
// become resident as this grid's CTAs exit); grid_dependency_wait blocks
// until the stream's previous kernel has completed and its memory operations
// are visible (it returns at once when the grid was launched without the
// programmatic attribute).
__device__ __forceinline__ void launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void grid_dependency_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
// Pulls a tensor map (a __grid_constant__ kernel parameter) into the
// descriptor cache before its first TMA.
__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
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
    // the first N (< 4) elements of a 16-byte chunk, with 8- and 4-byte loads
    template <int N>
    __device__ static __forceinline__ void load_part(const float* p, float* out) {
        static_assert(N > 0 && N < 4, "a partial chunk");
        if constexpr (N >= 2) {
            const float2 v = *reinterpret_cast<const float2*>(p);
            out[0] = v.x; out[1] = v.y;
        }
        if constexpr (N % 2 == 1) out[N - 1] = p[N - 1];
    }
    __device__ static __forceinline__ float load(const float* p) { return *p; }
    __device__ static __forceinline__ void store(float* p, float v) { *p = v; }
    // weight stored as one float32 word
    using Weight = float;
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
    // the first N (even, < 8) elements of a 16-byte chunk, with 8- and 4-byte loads
    template <int N>
    __device__ static __forceinline__ void load_part(const __nv_bfloat16* p, float* out) {
        static_assert(N > 0 && N < 8 && N % 2 == 0, "a partial chunk of bfloat16 pairs");
        uint32_t w[N / 2];
        if constexpr (N >= 4) {
            const uint2 v = *reinterpret_cast<const uint2*>(p);
            w[0] = v.x; w[1] = v.y;
        }
        if constexpr (N % 4 == 2) w[N / 2 - 1] = reinterpret_cast<const uint32_t*>(p)[N / 2 - 1];
#pragma unroll
        for (int q = 0; q < N / 2; ++q) {
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
    // weight stored as a bfloat16 duplicated in both halves of a 32-bit word
    // (fma.rn.f32.bf16 takes the low half)
    using Weight = uint32_t;
};

// ---------------------------------------------------------------------------
// compile-time geometry of one instantiation
// ---------------------------------------------------------------------------
// Shared-memory layout of one stage: the task's input window as ONE dense TMA
// box of (TY + K - 1) rows x BXW elements (row pitch BXW), then the task's
// weights. Lanes are laid out LX = 8 across a row: the 8 lanes of a quarter
// warp read 8 consecutive 16-byte chunks of one row, which hit 8 different
// bank groups whatever the pitch, so the window needs no padding or skew.
template <int K_, int C_, int R_, int LX_, int NW_, int NS_, typename TIn, typename TF>
struct Geo {
    static constexpr int K = K_, C = C_, R = R_, LX = LX_, NW = NW_, NS = NS_;
    static constexpr int LY = 32 / LX;
    static constexpr int TX = LX * C, TY = LY * R;
    static constexpr int ES = int(sizeof(TIn));
    static constexpr int EPC = Elem<TIn>::kPerChunk;
    // a lane's first column is 16-byte aligned (float32: C = 4) or 8-byte
    // aligned (bfloat16 with C = 4, read with 8- and 4-byte loads)
    static_assert(C % EPC == 0 || (ES == 2 && C == 4), "a lane's columns: whole 16-byte chunks, "
                                                       "or 4 bfloat16");
    static_assert(LX >= 8, "a quarter warp must span 8 consecutive chunks of a row");
    // window row: TX + K - 1 elements from a chunk-aligned origin
    // bfloat16 inputs come in 4 x-shifted copies (8-byte alignment) while a
    // TMA box must start 16-byte aligned: the box starts at the 16-byte
    // boundary at or below the window, and the lanes start MS elements in
    // (0 or 4, the task's shift); the box is MSLACK elements wider for it
    static constexpr int MSLACK = ES == 2 ? 4 : 0;
    static constexpr int BXW = (TX + K - 1 + MSLACK + EPC - 1) / EPC * EPC;
    static constexpr int ROWS = TY + K - 1;           // TMA box height
    static_assert((BXW * ES) % 16 == 0 && BXW <= 256 && ROWS <= 256, "TMA box");
    static constexpr int WINDOW_BYTES = ROWS * BXW * ES;
    // per-cluster weights (one 32-bit word each), padded to a 16-byte
    // multiple, copied with the window
    static constexpr int WES = int(sizeof(typename Elem<TF>::Weight));
    static constexpr int WPAD = (K * K * WES + 15) / 16 * 16 / WES;
    static constexpr int WBYTES = WPAD * WES;
    static constexpr int WOFF = (WINDOW_BYTES + 15) / 16 * 16;   // bytes into the stage
    static constexpr int STAGE_BYTES = (WOFF + WBYTES + 127) / 128 * 128;
    static_assert(STAGE_BYTES % 128 == 0, "TMA destinations must be 128-byte aligned");
    static constexpr uint32_t TX_BYTES = uint32_t(WINDOW_BYTES + WBYTES);
    static constexpr int TILE = TX * TY;
    static constexpr int THREADS = NW * 32;
    static constexpr int STAGES_BYTES = NW * NS * STAGE_BYTES;
    // the CTA's tile reduction: NW - 1 partial tiles, then a flag word
    static constexpr int RED_OFF = STAGES_BYTES;
    static constexpr int RED_BYTES = (NW - 1) * TILE * 4;
    static constexpr int FLAG_OFF = RED_OFF + RED_BYTES;
    static constexpr int TSTAT_OFF = FLAG_OFF + 16;       // [NW][4] float64 tile statistics
    static constexpr int BAR_OFF = TSTAT_OFF + NW * 4 * 8;
    static constexpr int SHIFT_OFF = BAR_OFF + NW * NS * 8;     // [NW][NS] lane shift per stage
    static constexpr int HEAD_OFF = SHIFT_OFF + (NW * NS * 4 + 15) / 16 * 16;   // [NW][3] first tasks
    static constexpr int SMEM_BYTES = HEAD_OFF + NW * 3 * 16;
    static constexpr int ER = R / NW;   // epilogue rows of each lane's block per warp
    static_assert(R % NW == 0, "the epilogue splits a lane's rows evenly over the warps");
    // resident CTAs per SM the register budget must allow (4 x 4 warps = 16
    // warps per SM when the stages fit; the occupancy query has the last word)
    static constexpr int MIN_BLOCKS = (227 * 1024) / (SMEM_BYTES + 1024) >= 4 ? 4 : 1;
};

// ---------------------------------------------------------------------------
// per-lane correlation of one staged window
// ---------------------------------------------------------------------------
// The C + K - 1 elements of one window row a lane uses, from its first
// (16-byte aligned) element: whole 16-byte chunks, then the rest with 8- and
// 4-byte loads. Loading only what is used keeps the shared-memory traffic of
// the inner loop, which competes with the FMAs, at its minimum (6 of 8
// float32 for C = 4, K = 3).
template <class G, typename TIn>
__device__ __forceinline__ void load_row_elems(const TIn* rowp, float (&raw)[G::C + G::K - 1]) {
    constexpr int NE = G::C + G::K - 1, EPC = G::EPC;
    constexpr int NFULL = NE / EPC, NREST = NE - NFULL * EPC;
#pragma unroll
    for (int q = 0; q < NFULL; ++q) Elem<TIn>::load_chunk(rowp + q * EPC, raw + q * EPC);
    if constexpr (NREST > 0) Elem<TIn>::template load_part<NREST>(rowp + NFULL * EPC, raw + NFULL * EPC);
}

// acc[o][c] += sum_{dy,dx} w[dy][dx] * win[o + dy][c + dx]
// `win` points at this lane's first element (window row ty*R, column tx*C).
// Windows are chunk-aligned (shifted copies), so each row is a few aligned
// loads (load_row_elems). The multiply-adds are scalar FFMAs: packed FFMA2
// pairs would need the odd-offset operand pairs rebuilt in registers every
// row, and on this part the packed form does not raise the FMA pipe's rate
// (a measured correlation loop ran at 0.71 of the FP32 peak with scalar
// FFMAs against 0.63 with FFMA2). Both round each product-sum once, so the
// results are the same bit for bit. acc is kept as float2 pairs (c, c+1)
// for the item-end code.
// bfloat16 windows (the storage form; the lane starts 0 or 4 elements into
// the box, so 8-byte aligned): the elements stay 16-bit and feed
// fma.rn.f32.bf16, which widens both bfloat16 operands exactly and rounds the
// float32 product-sum once, as the float32 path does after widening them
// itself (same bits), without spending issue slots on the widening. The
// lane's C + K - 1 elements start 8-byte aligned: 8-byte loads, then a 4-byte
// one. wh[q] holds tap q's weight in its low 16 bits.
template <class G>
__device__ __forceinline__ void correlate_bf16(float2 (&acc)[G::R][G::C / 2], const __nv_bfloat16* win,
                                               const uint32_t (&wh)[G::K * G::K]) {
    constexpr int K = G::K, C = G::C, R = G::R;
    constexpr int NE = C + K - 1;
    static_assert(NE % 2 == 0, "whole bfloat16 pairs");
#pragma unroll
    for (int i = 0; i < R + K - 1; ++i) {
        const uint16_t* rp = reinterpret_cast<const uint16_t*>(win + i * G::BXW);
        uint16_t h[NE];
#pragma unroll
        for (int q = 0; q + 4 <= NE; q += 4) {
            const uint2 v = *reinterpret_cast<const uint2*>(rp + q);
            h[q] = uint16_t(v.x & 0xffffu);
            h[q + 1] = uint16_t(v.x >> 16);
            h[q + 2] = uint16_t(v.y & 0xffffu);
            h[q + 3] = uint16_t(v.y >> 16);
        }
        if constexpr (NE % 4 == 2) {
            const uint32_t v = *reinterpret_cast<const uint32_t*>(rp + NE - 2);
            h[NE - 2] = uint16_t(v & 0xffffu);
            h[NE - 1] = uint16_t(v >> 16);
        }
#pragma unroll
        for (int dx = 0; dx < K; ++dx) {
#pragma unroll
            for (int dy = 0; dy < K; ++dy) {
                const int o = i - dy;
                if (o >= 0 && o < R) {
                    const uint16_t wq = uint16_t(wh[dy * K + dx] & 0xffffu);
#pragma unroll
                    for (int c2 = 0; c2 < C / 2; ++c2) {
                        float d0, d1;
                        asm("fma.rn.f32.bf16 %0, %1, %2, %3;"
                            : "=f"(d0) : "h"(h[2 * c2 + dx]), "h"(wq), "f"(acc[o][c2].x));
                        asm("fma.rn.f32.bf16 %0, %1, %2, %3;"
                            : "=f"(d1) : "h"(h[2 * c2 + 1 + dx]), "h"(wq), "f"(acc[o][c2].y));
                        acc[o][c2].x = d0;
                        acc[o][c2].y = d1;
                    }
                }
            }
        }
    }
}

template <class G, typename TIn>
__device__ __forceinline__ void correlate(float2 (&acc)[G::R][G::C / 2], const TIn* win,
                                          const float2 (&w2)[G::K * G::K]) {
    constexpr int K = G::K, C = G::C, R = G::R;
    constexpr int NE = C + K - 1;                 // elements used per row
#pragma unroll
    for (int i = 0; i < R + K - 1; ++i) {
        float raw[NE];
        load_row_elems<G, TIn>(win + i * G::BXW, raw);
#pragma unroll
        for (int dx = 0; dx < K; ++dx) {
#pragma unroll
            for (int dy = 0; dy < K; ++dy) {
                const int o = i - dy;
                if (o >= 0 && o < R) {
                    const float wv = w2[dy * K + dx].x;
#pragma unroll
                    for (int c2 = 0; c2 < C / 2; ++c2) {
                        acc[o][c2].x = fmaf(raw[2 * c2 + dx], wv, acc[o][c2].x);
                        acc[o][c2].y = fmaf(raw[2 * c2 + 1 + dx], wv, acc[o][c2].y);
                    }
                }
            }
        }
    }
}

// Per-lane sums for the PSF-value gradient of one staged window:
// acc[dy*K + dx] += sum_{o,c} f[o][c] * win[o + dy][c + dx], with the lane's
// datacube block held as pairs fp[o][c/2] = (f[o][c], f[o][c+1]). The same
// sliding pass over the window as correlate(), with the lane's values in the
// place of the weights; each pair sum is finished (x + y) by the caller.
template <class G, typename TIn>
__device__ __forceinline__ void correlate_grad(float2 (&acc)[G::K * G::K], const TIn* win,
                                               const float2 (&fp)[G::R][G::C / 2]) {
    constexpr int K = G::K, C = G::C, R = G::R;
    constexpr int NE = C + K - 1;
#pragma unroll
    for (int i = 0; i < R + K - 1; ++i) {
        float raw[NE];
        load_row_elems<G, TIn>(win + i * G::BXW, raw);
#pragma unroll
        for (int dx = 0; dx < K; ++dx) {
#pragma unroll
            for (int dy = 0; dy < K; ++dy) {
                const int o = i - dy;
                if (o >= 0 && o < R) {
#pragma unroll
                    for (int c2 = 0; c2 < C / 2; ++c2) {
                        acc[dy * K + dx].x = fmaf(raw[2 * c2 + dx], fp[o][c2].x, acc[dy * K + dx].x);
                        acc[dy * K + dx].y = fmaf(raw[2 * c2 + 1 + dx], fp[o][c2].y, acc[dy * K + dx].y);
                    }
                }
            }
        }
    }
}

// Fixed-order float32 warp sum (same tree on every run); lane 0 gets the total.
__device__ __forceinline__ float warp_sum_f(float d) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(0xffffffffu, d, off);
    return d;
}

// ---------------------------------------------------------------------------
// epilogues (per warp, straight from the lanes' register blocks)
// ---------------------------------------------------------------------------
// Lane (tx, ty) owns tile rows ty*R .. ty*R+R-1 and columns tx*C .. tx*C+C-1.
template <class G>
__device__ __forceinline__ int tile_elem(int tx, int ty, int o, int c) {
    return (ty * G::R + o) * G::TX + tx * G::C + c;
}

// Optional self-check of every epilogue access against the buffer ranges the
// host registered (compiled in with -DCTIS_DEBUG_BOUNDS only): a bad access
// is counted, its address recorded, and the access still happens only when
// it is in range.
#ifdef CTIS_DEBUG_BOUNDS
__device__ DbgRanges g_dbg;
__device__ __forceinline__ bool dbg_ok(const void* ptr, int bytes) {
    const char* p0 = static_cast<const char*>(ptr);
    for (int i = 0; i < 6; ++i)
        if (g_dbg.lo[i] && p0 >= g_dbg.lo[i] && p0 + bytes <= g_dbg.hi[i]) return true;
    if (g_dbg.log) {
        if (atomicAdd(g_dbg.log, 1ull) == 0) g_dbg.log[1] = reinterpret_cast<unsigned long long>(p0);
    }
    return false;
}
#define DBG_CHECK_RANGE(ptr, n) \
    if (!dbg_ok((ptr), int(sizeof(*(ptr))) * (n))) continue
#else
#define DBG_CHECK_RANGE(ptr, n) ((void)0)
#endif

// Vector access to C consecutive elements (16 bytes of float32, or 8/16 bytes
// of bfloat16) at an address aligned to that size.
template <typename T, int C>
struct Vec;
template <>
struct Vec<float, 4> {
    __device__ static __forceinline__ void load(const float* p, float (&v)[4]) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    __device__ static __forceinline__ void store(float* p, const float (&v)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <>
struct Vec<float, 8> {
    __device__ static __forceinline__ void load(const float* p, float (&v)[8]) {
        const float4 a = reinterpret_cast<const float4*>(p)[0];
        const float4 b = reinterpret_cast<const float4*>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    }
    __device__ static __forceinline__ void store(float* p, const float (&v)[8]) {
        reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
        reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
    }
};
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&b);
}
__device__ __forceinline__ void unpack_bf16x2(uint32_t w, float& lo, float& hi) {
    lo = __uint_as_float(w << 16);
    hi = __uint_as_float(w & 0xffff0000u);
}
template <>
struct Vec<__nv_bfloat16, 4> {
    __device__ static __forceinline__ void load(const __nv_bfloat16* p, float (&v)[4]) {
        const uint2 q = *reinterpret_cast<const uint2*>(p);
        unpack_bf16x2(q.x, v[0], v[1]);
        unpack_bf16x2(q.y, v[2], v[3]);
    }
    __device__ static __forceinline__ void store(__nv_bfloat16* p, const float (&v)[4]) {
        *reinterpret_cast<uint2*>(p) = make_uint2(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]));
    }
};

template <>
struct Vec<__nv_bfloat16, 8> {
    __device__ static __forceinline__ void load(const __nv_bfloat16* p, float (&v)[8]) {
        const uint4 q = *reinterpret_cast<const uint4*>(p);
        unpack_bf16x2(q.x, v[0], v[1]);
        unpack_bf16x2(q.y, v[2], v[3]);
        unpack_bf16x2(q.z, v[4], v[5]);
        unpack_bf16x2(q.w, v[6], v[7]);
    }
    __device__ static __forceinline__ void store(__nv_bfloat16* p, const float (&v)[8]) {
        *reinterpret_cast<uint4*>(p) = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]),
                                                  pack_bf16x2(v[4], v[5]), pack_bf16x2(v[6], v[7]));
    }
};

// Reads this lane's C consecutive elements of a row starting at column x
// (tile-relative column base; `n_valid` of them inside the plane). Uses one
// vector load when the row is complete and aligned, element loads otherwise.
template <typename T, int C>
__device__ __forceinline__ void load_row(const T* p, int n_valid, bool aligned, float (&v)[C]) {
#ifdef CTIS_DEBUG_BOUNDS
    for (int c = 0; c < C; ++c) v[c] = 0.f;
    for (int c = 0; c < C && c < n_valid; ++c) {
        DBG_CHECK_RANGE(p + c, 1);
        v[c] = Elem<T>::load(p + c);
    }
    return;
#endif
    if (n_valid >= C && aligned) {
        Vec<T, C>::load(p, v);
    } else {
#pragma unroll
        for (int c = 0; c < C; ++c) v[c] = c < n_valid ? Elem<T>::load(p + c) : 0.f;
    }
}

// Stores this lane's row values v[0..C-1] (plane columns col0 + c, col0 =
// tx*C inside the tile; `tile_cols` of the tile's columns lie inside the
// plane) into the x-shifted copies: copy q holds plane column x at x + q.
// `row` points at copy 0, tile column 0, of this row. For each copy the lane
// writes the C-aligned group [col0, col0 + C) of that copy with one vector
// store; the values come from this lane and its left neighbours (warp
// shuffles, same lane row). Groups cut by the tile edge, and the q values
// that spill past the tile's right edge, are written as aligned 8- and
// 4-byte pieces in a full float32 tile, element by element otherwise.
template <typename T, int C, int LX>
__device__ __forceinline__ void store_copies(T* row, long long copy_stride, int ncopies, bool active,
                                             int tx, int tile_cols, const float (&v)[C]) {
    constexpr int NCMAX = 16 / int(sizeof(T));
    constexpr int DMAX = (NCMAX - 1 + C - 1) / C;   // lanes to the left a copy reaches
    const int col0 = tx * C;
    if constexpr (sizeof(T) == 2 && C == 4) {
        // A full bfloat16 tile with the 4 copies of the plan (uniform over
        // the warp): each value is rounded once, the lanes pass packed pairs
        // to the right, and each copy's 4 elements are two 32-bit words
        // assembled with byte permutes (the same bits as rounding per copy).
        if (tile_cols == LX * C && ncopies <= 4) {
            const uint32_t p0 = pack_bf16x2(v[0], v[1]), p1 = pack_bf16x2(v[2], v[3]);
            const uint32_t l0 = __shfl_up_sync(0xffffffffu, p0, 1);   // left lane's (e0, e1)
            const uint32_t l1 = __shfl_up_sync(0xffffffffu, p1, 1);   // left lane's (e2, e3)
            if (!active) return;
            // the high half of x and the low half of y: (x.hi, y.lo)
            auto mid = [](uint32_t x, uint32_t y) { return __byte_perm(x, y, 0x5432); };
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (q >= ncopies) break;
                uint16_t* dst = reinterpret_cast<uint16_t*>(row + q * copy_stride);
                // copy q, columns col0 .. col0 + 3: source columns col0 - q ..
                const uint32_t w0 = q == 0 ? p0 : q == 1 ? mid(l1, p0) : q == 2 ? l1 : mid(l0, l1);
                const uint32_t w1 = q == 0 ? p1 : q == 1 ? mid(p0, p1) : q == 2 ? p0 : mid(l1, p0);
                if (q == 0 || tx >= 1) {
                    DBG_CHECK_RANGE(reinterpret_cast<T*>(dst) + col0, C);
                    *reinterpret_cast<uint2*>(dst + col0) = make_uint2(w0, w1);
                } else if (q == 1) {   // left edge: columns 1..3 (e0, e1, e2)
                    DBG_CHECK_RANGE(reinterpret_cast<T*>(dst) + 1, 3);
                    dst[1] = uint16_t(w0 >> 16);
                    *reinterpret_cast<uint32_t*>(dst + 2) = w1;
                } else if (q == 2) {   // columns 2, 3 (e0, e1)
                    DBG_CHECK_RANGE(reinterpret_cast<T*>(dst) + 2, 2);
                    *reinterpret_cast<uint32_t*>(dst + 2) = w1;
                } else {               // column 3 (e0)
                    DBG_CHECK_RANGE(reinterpret_cast<T*>(dst) + 3, 1);
                    dst[3] = uint16_t(w1 >> 16);
                }
                // right edge: the last q source columns land past the tile
                if (q >= 1 && tx == LX - 1) {
                    uint16_t* sp = dst + LX * C;
                    DBG_CHECK_RANGE(reinterpret_cast<T*>(sp), q);
                    if (q == 1) {          // e3
                        sp[0] = uint16_t(p1 >> 16);
                    } else if (q == 2) {   // e2, e3
                        *reinterpret_cast<uint32_t*>(sp) = p1;
                    } else {               // e1, e2, e3
                        *reinterpret_cast<uint32_t*>(sp) = mid(p0, p1);
                        sp[2] = uint16_t(p1 >> 16);
                    }
                }
            }
            return;
        }
    }
    // The values of the DMAX lanes to the left, fetched once for all copies.
    // Every lane runs the shuffles (DMAX is uniform); lanes of rows outside
    // the plane (`active` false) store nothing.
    float left[DMAX][C];
#pragma unroll
    for (int d = 1; d <= DMAX; ++d)
#pragma unroll
        for (int j = 0; j < C; ++j) left[d - 1][j] = __shfl_up_sync(0xffffffffu, v[j], d);
    if (!active) return;
    if constexpr (sizeof(T) == 4 && C == 4) {
        // A full float32 tile (the common case; uniform over the warp): the
        // groups that straddle the tile's edges are written as aligned
        // 8- and 4-byte pieces instead of element by element.
        if (tile_cols == LX * C) {
#pragma unroll
            for (int q = 0; q < NCMAX; ++q) {
                if (q >= ncopies) break;
                T* dst = row + q * copy_stride;
                float a[C];
#pragma unroll
                for (int j = 0; j < C; ++j) a[j] = j >= q ? v[j - q] : left[0][j - q + C];
                if (q == 0 || tx >= 1) {
                    DBG_CHECK_RANGE(dst + col0, C);
                    Vec<T, C>::store(dst + col0, a);
                } else if (q == 1) {   // left edge: columns 1..3 of the group
                    DBG_CHECK_RANGE(dst + 1, 3);
                    dst[1] = v[0];
                    *reinterpret_cast<float2*>(dst + 2) = make_float2(v[1], v[2]);
                } else if (q == 2) {
                    DBG_CHECK_RANGE(dst + 2, 2);
                    *reinterpret_cast<float2*>(dst + 2) = make_float2(v[0], v[1]);
                } else {
                    DBG_CHECK_RANGE(dst + 3, 1);
                    dst[3] = v[0];
                }
                // right edge: the last q source columns land past the tile
                if (q >= 1 && tx == LX - 1) {
                    T* sp = dst + LX * C;
                    DBG_CHECK_RANGE(sp, q);
                    if (q == 1) {
                        sp[0] = v[3];
                    } else if (q == 2) {
                        *reinterpret_cast<float2*>(sp) = make_float2(v[2], v[3]);
                    } else {
                        *reinterpret_cast<float2*>(sp) = make_float2(v[1], v[2]);
                        sp[2] = v[3];
                    }
                }
            }
            return;
        }
    }
#pragma unroll
    for (int q = 0; q < NCMAX; ++q) {
        if (q >= ncopies) break;
        // destination column col0 + j of copy q holds source column col0 + j - q
        float a[C];
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const int e = j - q;
            if (e >= 0) {
                a[j] = v[e];
            } else {
                const int d = (-e + C - 1) / C;
                a[j] = left[d - 1][e + d * C];
            }
        }
        T* dst = row + q * copy_stride;
        const int dneed = (q + C - 1) / C;   // lanes to the left the group reads
        if (tx >= dneed && col0 + C - 1 - q < tile_cols) {
            DBG_CHECK_RANGE(dst + col0, C);
            Vec<T, C>::store(dst + col0, a);
        } else {
#pragma unroll
            for (int j = 0; j < C; ++j) {
                const int src = col0 + j - q;
                if (src >= 0 && src < tile_cols) {
                    DBG_CHECK_RANGE(dst + col0 + j, 1);
                    Elem<T>::store(dst + col0 + j, a[j]);
                }
            }
        }
        // spill: own source columns whose copy-q position is past the tile
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int src = col0 + c;
            if (src + q >= LX * C && src < tile_cols) {
                DBG_CHECK_RANGE(dst + src + q, 1);
                Elem<T>::store(dst + src + q, v[c]);
            }
        }
    }
}

// Applies the epilogue MODE to ER of the lane's rows (rows o0 .. o0+ER-1 of
// its block; v[o][c]) of the item's tile, with the rows' inputs ein (g for
// the ratio, f for the update) already loaded; accumulates the forward
// statistics of the lane in stat[].
template <class G, typename TF, int MODE, int ER>
__device__ __forceinline__ void epilogue(const GatherParams& p, const WorkItem& it, int tx,
                                         int ty, int o0, const float (&v)[ER][G::C],
                                         const float (&ein)[ER][G::C], float (&stat)[kNumStats],
                                         float hs) {
    constexpr int C = G::C;
    const int tile_cols = min(G::TX, p.out_w - it.x0);
    const int col0 = tx * C;
    const int n_valid = tile_cols - col0;
    float rh = 0.f;   // kEpiUpdate: 1 / h_s (0 where h_s == 0: f = 0 there)
    if constexpr (MODE == kEpiUpdate) rh = hs != 0.f ? 1.0f / hs : 0.f;
#pragma unroll
    for (int o = 0; o < ER; ++o) {
        const int y = it.y0 + ty * G::R + o0 + o;
        const bool row_ok = y < p.out_h;      // warp-divergent only at the bottom edge
        if constexpr (MODE == kEpiRaw) {
            if (!row_ok || n_valid <= 0) continue;
            float* dst = p.out_f32 + it.plane * p.out_plane_stride + (long long)y * p.out_pitch +
                         it.x0 + col0;
#ifdef CTIS_DEBUG_BOUNDS
            for (int c = 0; c < C && c < n_valid; ++c) {
                DBG_CHECK_RANGE(dst + c, 1);
                dst[c] = v[o][c];
            }
            continue;
#endif
            if (n_valid >= C && (p.out_pitch % 4) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
                Vec<float, C>::store(dst, v[o]);
            } else {
                for (int c = 0; c < C && c < n_valid; ++c) dst[c] = v[o][c];
            }
        } else if constexpr (MODE == kEpiRatio) {
            float u[C];
            const float (&gv)[C] = ein[o];   // g of this row (loaded by the caller)
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const float val = v[o][c];
                // u = g / Hf on the support of Hf (Eq. 2); the fast quotient
                // (within 2 ulp) is used for normal Hf, the IEEE one below
                u[c] = val >= 1.17549435e-38f ? __fdividef(gv[c], val) : (val > 0.f ? gv[c] / val : 0.f);
                // d/dq (q - g log q) = 1 - g / q on the support of q
                if (p.ratio_one_minus) u[c] = val > 0.f ? 1.f - u[c] : 0.f;
            }
            if (p.solver == kSolverSmart) {   // uniform; log(g / q) where both are > 0
#pragma unroll
                for (int c = 0; c < C; ++c)
                    u[c] = (gv[c] > 0.f && v[o][c] > 0.f) ? __logf(u[c]) : 0.f;
            } else if (p.solver == kSolverSart) {   // (g - q) / r where r = (H 1) > 0
                const float* rp = p.row_sum + (long long)(row_ok ? y : 0) * p.out_w + it.x0 + col0;
                float rs[C];
                load_row<float, C>(rp, row_ok ? n_valid : 0,
                                   (p.out_w % 4) == 0 && (reinterpret_cast<uintptr_t>(rp) & 15) == 0, rs);
#pragma unroll
                for (int c = 0; c < C; ++c)
                    u[c] = rs[c] > 0.f ? __fdividef(gv[c] - v[o][c], rs[c]) : 0.f;
            }
            if (p.with_stats) {   // uniform; selects instead of branches per element
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const float val = v[o][c];
                    const bool on = val > 0.f && row_ok && c < n_valid;
                    const float hv = on ? val : 0.f, gg = on ? gv[c] : 0.f;
                    stat[0] += hv;
                    stat[1] += gg;
                    stat[2] += gg * __logf(on ? val : 1.f) - hv;
                    const float dd = gg - hv;
                    stat[3] += dd * dd;
                }
            }
            // all lanes of the row take part in the shuffles; rows past the
            // plane store nothing
            float* row = p.out_f32 + it.plane * p.out_plane_stride +
                         (long long)(row_ok ? y : 0) * p.out_pitch + it.x0;
            store_copies<float, C, G::LX>(row, p.out_copy_stride, p.out_copies, row_ok, tx,
                                          tile_cols, u);
        } else {   // kEpiUpdate, or kEpiSet when p.mode says so
            const long long rowoff = it.plane * p.f_plane_stride +
                                     (long long)(row_ok ? y : 0) * p.f_pitch + it.x0;
            float fv[C];
            if (p.mode == kEpiUpdate && p.solver != kSolverEm) {
                // SART / SMART step relax * z / h (0 where h == 0: f stays)
                float rhc[C];
                if (p.h_vox) {
                    const float* hp = p.h_vox +
                                      ((long long)(it.plane % p.h_vox_planes) * p.out_h +
                                       (row_ok ? y : 0)) * p.out_w + it.x0 + col0;
                    load_row<float, C>(hp, row_ok ? n_valid : 0,
                                       (p.out_w % 4) == 0 && (reinterpret_cast<uintptr_t>(hp) & 15) == 0,
                                       rhc);
#pragma unroll
                    for (int c = 0; c < C; ++c) rhc[c] = rhc[c] != 0.f ? 1.0f / rhc[c] : 0.f;
                } else {
#pragma unroll
                    for (int c = 0; c < C; ++c) rhc[c] = rh;
                }
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const float step = p.relax * v[o][c] * rhc[c];
                    fv[c] = p.solver == kSolverSart ? fmaxf(ein[o][c] + step, 0.f)
                                                    : ein[o][c] * __expf(step);
                }
            } else if (p.mode == kEpiUpdate) {   // ein: f_in of this row (loaded by the caller)
                if (p.h_vox) {            // clipped boundary: h per voxel
                    const float* hp = p.h_vox +
                                      ((long long)(it.plane % p.h_vox_planes) * p.out_h +
                                       (row_ok ? y : 0)) * p.out_w + it.x0 + col0;
                    float hv[C];
                    load_row<float, C>(hp, row_ok ? n_valid : 0,
                                       (p.out_w % 4) == 0 && (reinterpret_cast<uintptr_t>(hp) & 15) == 0,
                                       hv);
#pragma unroll
                    for (int c = 0; c < C; ++c)
                        fv[c] = hv[c] != 0.f ? ein[o][c] * v[o][c] * (1.0f / hv[c]) : 0.f;
                } else {
#pragma unroll
                    for (int c = 0; c < C; ++c) fv[c] = ein[o][c] * v[o][c] * rh;
                }
            } else {
#pragma unroll
                for (int c = 0; c < C; ++c) fv[c] = v[o][c];
            }
            store_copies<TF, C, G::LX>(static_cast<TF*>(p.f_out) + rowoff, p.f_copy_stride,
                                       p.f_copies, row_ok, tx, tile_cols, fv);
        }
    }
}

// Fixed-order float64 warp sum (same tree on every run); lane 0 gets the total.
__device__ __forceinline__ double warp_sum(double d) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(0xffffffffu, d, off);
    return d;
}

__device__ __forceinline__ void load_stats(const double* src, double (&d)[kNumStats]) {
    const double2 a = __ldcg(reinterpret_cast<const double2*>(src));
    const double2 b = __ldcg(reinterpret_cast<const double2*>(src) + 1);
    d[0] = a.x; d[1] = a.y; d[2] = b.x; d[3] = b.y;
}

// Sum over the warp of four float32 values per lane, as a reduce-scatter
// (fixed tree, same on every run): the first two levels halve the set of
// values a lane carries (lanes with bit 4 clear keep values 0 and 1, the
// others 2 and 3; then bit 3 picks one of the two) in float32, so each lane
// holds a float32 sum of four lanes' values; that is widened to float64 and
// the last three levels add within groups of eight lanes. One conversion and
// three float64 additions per lane (float64 runs at 1/64 of the float32
// rate here); lane l ends with the total of value l >> 3 (all eight lanes of
// a group hold it).
__device__ __forceinline__ double warp_sum4(const float (&v)[kNumStats], int lane) {
    static_assert(kNumStats == 4, "four values per lane");
    const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
    const float k0 = hi16 ? v[2] : v[0], k1 = hi16 ? v[3] : v[1];
    const float s0 = hi16 ? v[0] : v[2], s1 = hi16 ? v[1] : v[3];
    const float a0 = k0 + __shfl_xor_sync(0xffffffffu, s0, 16);
    const float a1 = k1 + __shfl_xor_sync(0xffffffffu, s1, 16);
    const float m32 = (hi8 ? a1 : a0) + __shfl_xor_sync(0xffffffffu, hi8 ? a0 : a1, 8);
    double m = static_cast<double>(m32);
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) m += __shfl_xor_sync(0xffffffffu, m, off);
    return m;
}

// Statistics of one finished tile, per warp: the warp's sum (warp_sum4) of
// its lanes' float32 sums goes to tstat[warp][0..3] in shared memory. The
// CTA's warps' values are added later, in warp order, by flush_tile_stats,
// after the next CTA barrier (no barrier of its own on the tile's path); the
// frame totals are added in fixed order by reduce_frame_slice at the start
// of the next launch in stream order.
__device__ __forceinline__ void store_tile_stats(const float (&stat)[kNumStats], int warp, int lane,
                                                 double* tstat) {
    const double tot = warp_sum4(stat, lane);
    if ((lane & 7) == 0) tstat[warp * kNumStats + (lane >> 3)] = tot;
}

// Lanes 0..3 of warp 0 add the NW warps' values of `tile` in warp order and
// store the tile's four statistics. Called by every warp after a CTA barrier
// that follows all warps' store_tile_stats for the tile, and before the
// barrier after which they may write tstat again.
template <int NW>
__device__ __forceinline__ void flush_tile_stats(const GatherParams& p, int tile, int warp,
                                                 int lane, const double* tstat) {
    if (warp == 0 && lane < kNumStats) {
        double t = tstat[lane];
        for (int w = 1; w < NW; ++w) t += tstat[w * kNumStats + lane];
        __stcg(p.tile_stats + (long long)tile * kNumStats + lane, t);
    }
}

// Frame totals of a forward's tile statistics, in two fixed-order float64
// levels. Slice `slice` of frame `frame` (one warp) adds the tiles
// [slice*T/S, (slice+1)*T/S): lane l adds value l & 3 of every eighth tile
// from offset l >> 2 on, in tile order, then the eight lanes of each value
// add theirs in a fixed tree, and lanes 0..3 store the slice's four sums.
// The slice that arrives last (one ticket per frame) adds the S slice sums
// in slice order and writes the frame's row, so the result does not depend
// on which warp finishes when.
__device__ __forceinline__ void reduce_frame_slice(const double* tile_stats, int tiles, int frame,
                                                   int slice, double* part, int* tickets,
                                                   double* out, int lane) {
    const double* src = tile_stats + (long long)frame * tiles * kNumStats;
    const int b = int((long long)tiles * slice / kStatSlices);
    const int e = int((long long)tiles * (slice + 1) / kStatSlices);
    const int q = lane & 3, j = lane >> 2;
    double t = 0.0;
    constexpr int B = 4;   // loads in flight per lane
    for (int i0 = b; i0 < e; i0 += 8 * B) {
        double v[B];
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const int i = i0 + 8 * k + j;
            v[k] = i < e ? __ldcg(src + (long long)i * kNumStats + q) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < B; ++k) t += v[k];
    }
#pragma unroll
    for (int off = 4; off < 32; off <<= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    double* fpart = part + (long long)frame * kStatSlices * kNumStats;
    if (lane < kNumStats) {
        __stcg(fpart + slice * kNumStats + lane, t);
        fence_acq_rel_gpu();   // release this slice's sums
    }
    __syncwarp();
    int last = 0;
    if (lane == 0) last = atomicAdd(tickets + frame, 1) == kStatSlices - 1;
    if (!__shfl_sync(0xffffffffu, last, 0)) return;
    fence_acq_rel_gpu();       // acquire the other slices' sums
    if (lane < kNumStats) {
        double sum = __ldcg(fpart + lane);
        for (int k = 1; k < kStatSlices; ++k) sum += __ldcg(fpart + k * kNumStats + lane);
        out[lane] = sum;
    }
    if (lane == 0) tickets[frame] = 0;
}

// ---------------------------------------------------------------------------
// the kernel body (wrapped by forward_kernel / adjoint_kernel)
// ---------------------------------------------------------------------------
// The host balances work items (a tile, or a chunk of a long tile) over the
// CTAs, longest first. The NW warps of a CTA walk parallel item lists: warp w
// runs the w-th quarter of each item's tasks, then the warps add their sums
// through shared memory (fixed order), a tile split over CTAs adds its chunks
// through global memory in chunk order (the last chunk to arrive, by ticket),
// and each warp applies the epilogue to its share of the tile's rows. Each
// warp's tasks are stored contiguously, so its TMA issue cursor is a plain
// counter running NS tasks ahead of the compute loop, across item boundaries.
// Lane 0 alone issues the copies (predicated instructions, no branch); the
// warp loads the next task descriptor right after each issue, so the load's
// latency overlaps a task of compute.
template <class G, typename TIn, typename TF, int MODE>
__device__ __forceinline__ void gather_body(const CUtensorMap& tm_win, const GatherParams& p) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + G::BAR_OFF);

    if (p.smid_out) {   // placement probe
        if (threadIdx.x == 0) {
            unsigned smid;
            asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
            p.smid_out[blockIdx.x] = int(smid);
        }
        for (int i = 0; i < 16; ++i) __nanosleep(2000);
        return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * G::NW + warp;
    const bool has_work = gw < p.n_warps;   // warp-uniform
    // the warp's start: lanes 0..5 load its 96-byte head at once, then the
    // fields go to every lane by shuffles. Up to the dependency wait below
    // the kernel reads only the plan's work lists (written by host copies
    // before any launch that uses them) and its own parameters: under
    // programmatic launch this part runs while the previous projector's grid
    // drains. (That grid lets this one be scheduled only once all its CTAs
    // have finished their work: scheduled earlier, this grid's CTAs would
    // take the SM slots in the order the previous CTAs exit, not in the
    // placement the work lists were balanced for.)
    int4 hv = make_int4(0, 0, 0, 0);
    if (has_work && lane < 6) hv = __ldg(reinterpret_cast<const int4*>(p.heads + gw) + lane);
    if (threadIdx.x == 0) prefetch_tensormap(&tm_win);
    // the inputs (copies, g, f, statistics) are the previous kernel's outputs
    // and the outputs may still be its inputs
    grid_dependency_wait();
    // the previous forward's statistics: slice r of the frames' reduction on
    // warp r / gridDim.x of CTA r % gridDim.x (the CTAs' first warps first)
    if (p.red_out) {
        const int r = warp * gridDim.x + blockIdx.x;
        if (r < p.red_frames * kStatSlices) {
            const int f = r / kStatSlices;
            reduce_frame_slice(p.red_src, p.red_tiles_per_frame, f, r - f * kStatSlices, p.red_part,
                               p.red_tickets, p.red_out + f * p.red_frame_stride, lane);
        }
    }
    if (!has_work) return;
    auto from = [&](int src, int4& d) {
        d.x = __shfl_sync(0xffffffffu, hv.x, src);
        d.y = __shfl_sync(0xffffffffu, hv.y, src);
        d.z = __shfl_sync(0xffffffffu, hv.z, src);
        d.w = __shfl_sync(0xffffffffu, hv.w, src);
    };
    int4 h0, i0, i1;
    from(0, h0);
    from(4, i0);
    from(5, i1);
    const int ib = h0.x, ie = h0.y;
    if (ib >= ie) return;   // nothing issued, nothing to drain
    // the first three task descriptors wait in shared memory for lane 0
    int4* my_head = reinterpret_cast<int4*>(smem_raw + G::HEAD_OFF) + warp * 3;
    if (lane >= 1 && lane <= 3) my_head[lane - 1] = hv;
    __syncwarp();
    const int tx = lane % G::LX, ty = lane / G::LX;
    unsigned char* my_stages = smem_raw + warp * G::NS * G::STAGE_BYTES;
    uint64_t* my_bars = bars + warp * G::NS;
    int* my_shift = reinterpret_cast<int*>(smem_raw + G::SHIFT_OFF) + warp * G::NS;
    if (lane == 0) {
        for (int s = 0; s < G::NS; ++s) mbar_init(&my_bars[s], 1);
        fence_mbar_init();
    }
    __syncwarp();

    const int lane_off = ty * G::R * G::BXW + tx * G::C;   // this lane's first element
    WorkItem next_it{i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w};
    const int task_end = h0.w;                              // end of the warp's task range
    int issue_task = h0.z;                                  // next task to issue (uniform)
    int issue_stage = 0;
    int cons_stage = 0;
    uint32_t cons_phase = 0;
    int outstanding = 0;                                    // copies issued, not yet waited for
    bool failed = false;                                    // warp-uniform
    // descriptor of issue_task, held by every lane (same-address loads); the
    // first three come with the head, the later ones are loaded one issue
    // ahead
    TaskDesc nxt;
    {
        const int4 f0 = my_head[0];
        nxt = TaskDesc{f0.x, f0.y, f0.z, f0.w};
    }
    const int head_end = issue_task + 3;
    const bool leader = lane == 0;   // issues the copies

    auto issue_next = [&]() {
        if (issue_task >= task_end || failed) return;
        unsigned char* stage = my_stages + issue_stage * G::STAGE_BYTES;
        uint64_t* bar = &my_bars[issue_stage];
        // bfloat16 windows: the lanes' shift inside the box (wx is a multiple
        // of 4, the box starts at a multiple of 8), published before the
        // arrival that releases the stage to the warp (float32 windows start
        // aligned: no shift)
        if constexpr (G::EPC > 4)
            if (leader) my_shift[issue_stage] = nxt.wx & (G::EPC - 1);
        mbar_arrive_expect_tx_if(leader, bar, G::TX_BYTES);
        if (!p.drop_copies) {
            tma_load_3d_if(leader, stage, &tm_win, nxt.wx & ~(G::EPC - 1), nxt.wy, nxt.plane, bar);
            bulk_load_if(leader, stage + G::WOFF,
                         static_cast<const unsigned char*>(p.weights) +
                             (long long)nxt.cluster * G::WBYTES,
                         G::WBYTES, bar);
        }
        const int t1 = issue_task + 1;
        if (t1 < task_end) {
            if (t1 < head_end) {
                const int4 f = my_head[t1 - (head_end - 3)];
                nxt = TaskDesc{f.x, f.y, f.z, f.w};
            } else {
                nxt = p.tasks[t1];
            }
        }
        ++issue_task;
        ++outstanding;
        if (++issue_stage == G::NS) issue_stage = 0;
    };
#pragma unroll
    for (int j = 0; j < G::NS; ++j) issue_next();

    // kEpiRatio with statistics: the tile whose per-warp sums wait in tstat
    // for the CTA combine after the next barrier (-1: none; uniform)
    int stats_tile = -1;
    double* tstat = reinterpret_cast<double*>(smem_raw + G::TSTAT_OFF);
    for (int ii = ib; ii < ie; ++ii) {
        const WorkItem it = next_it;
        if (ii + 1 < ie) next_it = p.items[ii + 1];   // prefetch; used next item
        // kEpiUpdate: h_s of the item's plane, loaded now for its item end
        float hs_item = 0.f;
        if constexpr (MODE == kEpiUpdate) hs_item = __ldg(p.h + it.plane);
        // pull the epilogue's inputs toward L1 while the item's tasks run
        if constexpr (MODE == kEpiRatio || MODE == kEpiUpdate) {
            if (MODE == kEpiRatio || p.mode == kEpiUpdate) {
#pragma unroll
                for (int o = 0; o < G::ER; ++o) {
                    const int y = it.y0 + ty * G::R + warp * G::ER + o;
                    const int x = it.x0 + tx * G::C;
                    if (y < p.out_h && x < p.out_w) {
                        const void* src =
                            MODE == kEpiRatio
                                ? static_cast<const void*>(p.g + it.plane * p.g_plane_stride +
                                                           (long long)y * p.g_pitch + x)
                                : static_cast<const void*>(static_cast<const TF*>(p.f_in) +
                                                           it.plane * p.f_plane_stride +
                                                           (long long)y * p.f_pitch + x);
                        asm volatile("prefetch.global.L1 [%0];" ::"l"(src));
                    }
                }
            }
        }

        float2 acc[G::R][G::C / 2];
#pragma unroll
        for (int o = 0; o < G::R; ++o)
#pragma unroll
            for (int c = 0; c < G::C / 2; ++c) acc[o][c] = make_float2(0.f, 0.f);
        // kEpiGrad: this lane's block of the datacube plane, as pairs (zero
        // outside the field stop)
        float2 fp[G::R][G::C / 2];
        if constexpr (MODE == kEpiGrad) {
            const TF* fs = static_cast<const TF*>(p.f_in) + (long long)it.plane * p.out_w * p.out_h;
#pragma unroll
            for (int o = 0; o < G::R; ++o) {
                const int y = it.y0 + ty * G::R + o;
                float fv[G::C];
#pragma unroll
                for (int c = 0; c < G::C; ++c) {
                    const int x = it.x0 + tx * G::C + c;
                    fv[c] = (y < p.out_h && x < p.out_w) ? Elem<TF>::load(fs + (long long)y * p.out_w + x)
                                                         : 0.f;
                }
#pragma unroll
                for (int c = 0; c < G::C / 2; ++c) fp[o][c] = make_float2(fv[2 * c], fv[2 * c + 1]);
            }
        }

        for (int t = it.task_begin; t < it.task_end; ++t) {
            if (!failed) {
                // fast path: one try_wait; the bounded spin runs only when the
                // copies have not landed yet
                if (!mbar_try_wait(&my_bars[cons_stage], cons_phase)) {
                    const bool ok = mbar_wait_bounded(&my_bars[cons_stage], cons_phase, &p.counters[3]);
                    failed = __any_sync(0xffffffffu, !ok);
                }
            }
            if (!failed) {
                const unsigned char* stage = my_stages + cons_stage * G::STAGE_BYTES;
                using WP = typename Elem<TF>::Weight;
                const WP* ws = reinterpret_cast<const WP*>(stage + G::WOFF);
                if constexpr (MODE == kEpiGrad) {
                    const int cl = p.tasks[t].cluster;
                    float2 gacc[G::K * G::K];
#pragma unroll
                    for (int q = 0; q < G::K * G::K; ++q) gacc[q] = make_float2(0.f, 0.f);
                    correlate_grad<G, TIn>(gacc, reinterpret_cast<const TIn*>(stage) + lane_off, fp);
                    float* dst = p.grad_part +
                                 ((long long)cl * p.grad_tiles_per_plane +
                                  (it.tile - it.plane * p.grad_tiles_per_plane)) * (G::K * G::K);
#pragma unroll
                    for (int q = 0; q < G::K * G::K; ++q) {
                        const float sum = warp_sum_f(gacc[q].x + gacc[q].y);
                        if (lane == 0) dst[q] = sum;
                    }
                } else {
                    // the task's weights: one 32-bit word each, read 16 bytes
                    // at a time (the slot is whole 16-byte words)
                    static_assert(sizeof(WP) == 4 && G::WPAD % 4 == 0, "weight slot of 16-byte words");
                    uint32_t wq[G::WPAD];
#pragma unroll
                    for (int i = 0; i < G::WPAD / 4; ++i) {
                        const uint4 v = reinterpret_cast<const uint4*>(ws)[i];
                        wq[4 * i] = v.x;
                        wq[4 * i + 1] = v.y;
                        wq[4 * i + 2] = v.z;
                        wq[4 * i + 3] = v.w;
                    }
                    if constexpr (std::is_same_v<TIn, __nv_bfloat16>) {
                        uint32_t wh[G::K * G::K];
#pragma unroll
                        for (int q = 0; q < G::K * G::K; ++q) wh[q] = wq[q];
                        correlate_bf16<G>(acc, reinterpret_cast<const TIn*>(stage) + lane_off +
                                                   my_shift[cons_stage], wh);
                    } else {
                        float2 w2[G::K * G::K];
#pragma unroll
                        for (int q = 0; q < G::K * G::K; ++q)   // a bfloat16 weight widened exactly
                            w2[q].x = __uint_as_float(std::is_same_v<TF, __nv_bfloat16> ? wq[q] << 16 : wq[q]);
                        correlate<G, TIn>(acc, reinterpret_cast<const TIn*>(stage) + lane_off, w2);
                    }
                }
                // after a failed wait the stage and phase stay at the copy
                // that did not land, where the final drain resumes
                --outstanding;
                if (++cons_stage == G::NS) {
                    cons_stage = 0;
                    cons_phase ^= 1u;
                }
            }
            __syncwarp();   // every lane is done with the stage before it is refilled
            issue_next();
        }

        if constexpr (MODE == kEpiGrad) continue;   // every task wrote its own sums

        // The CTA's warps ran disjoint parts of this item's tasks. Warp d
        // finalises rows d*ER .. d*ER+ER-1 of every lane's block: each warp
        // publishes in shared memory the rows the other warps finalise, and
        // each warp adds its rows over the warps in order, p0 + p1 + p2 + p3.
        constexpr int NW = G::NW, ER = G::ER, C = G::C;
        float* pub = reinterpret_cast<float*>(smem_raw + G::RED_OFF);
        auto pub_at = [&](int w, int d, int o) {   // warp w's copy of warp d's row o
            const int slot = d < w ? d : d - 1;
            return pub + (((w * (NW - 1) + slot) * ER + o) * 32 + lane) * C;
        };
        // this warp's epilogue inputs, loaded now so their latency overlaps
        // the reduction (rows beyond the plane read as zero and are not used)
        float ein[ER][C];
        if constexpr (MODE == kEpiRatio || MODE == kEpiUpdate) {
            const int tile_cols = min(G::TX, p.out_w - it.x0);
            const int n_valid = tile_cols - tx * C;
#pragma unroll
            for (int o = 0; o < ER; ++o) {
                const int y = it.y0 + ty * G::R + warp * ER + o;
                const bool row_ok = y < p.out_h;
                if constexpr (MODE == kEpiRatio) {
                    const float* gp = p.g + it.plane * p.g_plane_stride +
                                      (long long)(row_ok ? y : 0) * p.g_pitch + it.x0 + tx * C;
                    load_row<float, C>(gp, row_ok ? n_valid : 0,
                                       (p.g_pitch % 4) == 0 && (reinterpret_cast<uintptr_t>(gp) & 15) == 0,
                                       ein[o]);
                } else {
                    if (p.mode == kEpiUpdate) {
                        const long long rowoff = it.plane * p.f_plane_stride +
                                                 (long long)(row_ok ? y : 0) * p.f_pitch + it.x0;
                        load_row<TF, C>(static_cast<const TF*>(p.f_in) + rowoff + tx * C,
                                        row_ok ? n_valid : 0, true, ein[o]);
                    }
                }
            }
        }
#pragma unroll
        for (int d = 0; d < NW; ++d) {
            if (d == warp) continue;
#pragma unroll
            for (int o = 0; o < ER; ++o) {
                float row[C];
#pragma unroll
                for (int c = 0; c < C / 2; ++c) {
                    row[2 * c] = acc[d * ER + o][c].x;
                    row[2 * c + 1] = acc[d * ER + o][c].y;
                }
                Vec<float, C>::store(pub_at(warp, d, o), row);
            }
        }
        cta_barrier(G::THREADS);
        if constexpr (MODE == kEpiRatio) {
            if (stats_tile >= 0) {   // the previous finished tile's statistics
                flush_tile_stats<G::NW>(p, stats_tile, warp, lane, tstat);
                stats_tile = -1;
            }
        }
        float ve[ER][C];
#pragma unroll
        for (int o = 0; o < ER; ++o) {
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                float row[C];
                if (w == warp) {
#pragma unroll
                    for (int c = 0; c < C / 2; ++c) {
                        row[2 * c] = acc[warp * ER + o][c].x;
                        row[2 * c + 1] = acc[warp * ER + o][c].y;
                    }
                } else {
                    Vec<float, C>::load(pub_at(w, warp, o), row);
                }
#pragma unroll
                for (int c = 0; c < C; ++c) ve[o][c] = w == 0 ? row[c] : ve[o][c] + row[c];
            }
        }
        cta_barrier(G::THREADS);   // the published rows are free for the next item

        // Tiles longer than one item are split over CTAs: chunk sums go
        // through global memory, each warp its own rows, and the last chunk
        // to arrive (one ticket per chunk) adds them in chunk order.
        const int nchunks = it.chunk_info & 0xffff;
        bool finish = true;
        if (nchunks > 1) {
            const int chunk = it.chunk_info >> 16;
            float* slots = p.scratch + (long long)it.scratch_base * G::TILE;
#pragma unroll
            for (int o = 0; o < ER; ++o)
#pragma unroll
                for (int c = 0; c < C; c += 4)
                    __stcg(reinterpret_cast<float4*>(slots + (long long)chunk * G::TILE +
                                                     tile_elem<G>(tx, ty, warp * ER + o, c)),
                           make_float4(ve[o][c], ve[o][c + 1], ve[o][c + 2], ve[o][c + 3]));
            fence_acq_rel_gpu();   // publish this warp's rows (release)
            cta_barrier(G::THREADS);
            int* flag = reinterpret_cast<int*>(smem_raw + G::FLAG_OFF);
            if (warp == 0 && lane == 0) {   // release every warp's rows, then the ticket
                fence_acq_rel_gpu();
                *flag = atomicAdd(&p.tickets[it.tile], 1) == nchunks - 1 ? 1 : 0;
            }
            cta_barrier(G::THREADS);
            finish = *flag != 0;
            cta_barrier(G::THREADS);   // the flag is free for the next item
            if (finish) {
                fence_acq_rel_gpu();   // acquire the other chunks' sums
#pragma unroll
                for (int o = 0; o < ER; ++o)
#pragma unroll
                    for (int c = 0; c < C; c += 4) {
                        const int e = tile_elem<G>(tx, ty, warp * ER + o, c);
                        float4 s4 = __ldcg(reinterpret_cast<const float4*>(slots + e));
                        for (int ch = 1; ch < nchunks; ++ch) {
                            const float4 q4 = __ldcg(
                                reinterpret_cast<const float4*>(slots + (long long)ch * G::TILE + e));
                            s4.x += q4.x; s4.y += q4.y; s4.z += q4.z; s4.w += q4.w;
                        }
                        ve[o][c] = s4.x; ve[o][c + 1] = s4.y; ve[o][c + 2] = s4.z; ve[o][c + 3] = s4.w;
                    }
                if (warp == 0 && lane == 0) p.tickets[it.tile] = 0;
            }
        }
        if (finish) {
            float stat[kNumStats] = {0.f, 0.f, 0.f, 0.f};
            epilogue<G, TF, MODE, ER>(p, it, tx, ty, warp * ER, ve, ein, stat, hs_item);
            if constexpr (MODE == kEpiRatio) {
                if (p.with_stats) {   // uniform over the launch
                    store_tile_stats(stat, warp, lane, tstat);
                    stats_tile = it.tile;
                }
            }
        }
    }
    if constexpr (MODE == kEpiRatio) {
        if (stats_tile >= 0) {   // the last finished tile's statistics
            cta_barrier(G::THREADS);
            flush_tile_stats<G::NW>(p, stats_tile, warp, lane, tstat);
        }
    }

    // this CTA's work is done: once every CTA is here (or gone) the next
    // projector of the stream may be scheduled (it waits for this grid
    // before touching data)
    launch_dependents();
    // Copies still in flight exist only after a failed wait: give them a
    // bounded chance to land before the warp's shared memory is released.
    if (lane == 0) {
        while (outstanding > 0) {
            if (!mbar_wait_bounded(&my_bars[cons_stage], cons_phase, &p.counters[3])) break;
            --outstanding;
            if (++cons_stage == G::NS) {
                cons_stage = 0;
                cons_phase ^= 1u;
            }
        }
    }
    __syncwarp();
}

// Tile shapes: C = 4 columns per lane, 8 lanes across (32 columns). Shape 0
// (every adjoint, and the forward by default): R = 8 rows per lane, 32 x 32
// tiles. Shape 1 (a forward alternative for small field stops, whose
// footprints waste less of 16-row tiles): R = 4, 32 x 16 tiles, whose windows
// are half as tall, so a third TMA stage fits. The forward of a bfloat16 plan
// reads bfloat16 windows, half the bytes of a float32 window, and spends the
// freed shared memory on a third TMA stage per warp (a deeper look-ahead on
// the window stream at the same 4 CTAs per SM).
constexpr int kFwdShapes = 2;

template <bool FWD, typename TIn, int SHAPE>
constexpr GatherShape shape_of() {
    GatherShape s = FWD ? kShapeFwd : kShapeAdj;
    if (FWD && SHAPE == 1) {
        s.R = 4;
        s.NS = 3;
    }
    if (FWD && sizeof(TIn) == 2) s.NS = CTIS_FWD_NS_BF16;
    return s;
}

template <int K, typename TIn, typename TF, bool FWD, int SHAPE = 0>
using GeoOf = Geo<K, shape_of<FWD, TIn, SHAPE>().C, shape_of<FWD, TIn, SHAPE>().R,
                  shape_of<FWD, TIn, SHAPE>().LX, shape_of<FWD, TIn, SHAPE>().NW,
                  shape_of<FWD, TIn, SHAPE>().NS, TIn, TF>;

template <class G, class Kern>
cudaError_t prepare_kernel(Kern kern, int* blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         G::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, G::THREADS,
                                                      G::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    return *blocks_per_sm >= 1 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

template <class G, class Kern>
cudaError_t launch_kernel(Kern kern, const CUtensorMap& win, const GatherParams& p,
                          cudaStream_t stream) {
    const int grid = (p.n_warps + G::NW - 1) / G::NW;
    if (!p.overlap_launch) {
        kern<<<grid, G::THREADS, G::SMEM_BYTES, stream>>>(win, p);
        return cudaGetLastError();
    }
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(G::THREADS);
    cfg.dynamicSmemBytes = G::SMEM_BYTES;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, win, p);
}

}  // namespace
}  // namespace ctis
