// Plan construction and the C-ABI entry points of libctis.
//
// A plan turns the calibration PSFs (Sec. 2: one image per wavelength, the
// response to field-stop pixel (0,0)) into everything the gather kernels need:
//   * merged nonzeros (duplicates added in float64, rounded once to the
//     storage type) and h = H^T 1 (Eq. 2), which under the on-FPA bounds rule
//     is, for every voxel of wavelength s, the sum of that wavelength's values;
//   * spot clusters: 8-connected groups of nonzeros, each covered by K x K
//     boxes (K the smallest supported side that fits the largest group);
//   * work lists: for the forward projector every FPA tile lists the clusters
//     whose footprint (a + K - 1) x (alpha + K - 1) meets it; for the adjoint
//     every voxel tile of wavelength s lists the clusters of s. Long lists are
//     split into chunks; items are ordered longest first.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <unordered_map>
#include <vector>

#include "ctis.h"
#include "ctis_internal.h"
#include "ctis_kernels.h"

using namespace ctis;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(CTIS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CTIS_CUDA(call)                                              \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);          \
    } while (0)

// Round a float to bfloat16, round to nearest even (finite, nonnegative input).
uint16_t to_bf16_bits(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    return static_cast<uint16_t>(u >> 16);
}

float bf16_bits_to_float(uint16_t b) {
    const uint32_t u = static_cast<uint32_t>(b) << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }
int64_t floor_div(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
int64_t floor_mod(int64_t a, int64_t b) { return a - floor_div(a, b) * b; }

struct Cluster {
    int s, X, Y;
};

struct ProjTables {
    std::vector<TileDesc> tiles;
    std::vector<ItemDesc> items;
    std::vector<TaskDesc> tasks;   // warp order (what the kernel reads)
    std::vector<TaskDesc> tile_tasks;       // tile order, the input of schedule()
    std::vector<int> tile_task_begin;       // [tiles + 1]
    std::vector<int> warp_begin;   // [n_warps + 1]
    std::vector<WarpHead> heads;   // [n_warps] each warp's start (warp_begin, first item/tasks)
    std::vector<int> cta_begin;    // [CTAs + 1]
    std::vector<int> cta_items;    // item indices, grouped by CTA
    int nw = 4;                    // warps per CTA of the projector's kernel
    std::vector<WorkItem> witems;  // the items in warp order, as the kernel reads them
    int tile_w = 0, tile_h = 0;
    int64_t scratch_slots = 0;
    int per_item = 0;              // chunk size of the longest-first schedule (0: split)
    int split_q = 0;               // balanced split: item overhead in quarter tasks (0: chunks)
    int skew_pm = 0;               // CTA priority skew of the schedule (permille)
    std::vector<int> block_sm;     // SM of each CTA in a launch of this grid (probed; may be empty)
    std::vector<std::pair<int, int>> witem_src;   // each warp item's range in tile_tasks
    int n_warps = 0;
    double max_warp_load = 0.0;    // LPT estimate of the busiest CTA, tasks per warp
    TaskDesc* d_tasks = nullptr;
    int* d_warp_begin = nullptr;
    WarpHead* d_heads = nullptr;
    WorkItem* d_witems = nullptr;
    void* d_weights = nullptr;
    int blocks_per_sm = 0;
};

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    });
    return fn;
}

static_assert(CTIS_SOLVER_EM == kSolverEm && CTIS_SOLVER_SART == kSolverSart &&
                  CTIS_SOLVER_SMART == kSolverSmart,
              "the C ABI's solver codes are the kernels'");

struct GraphKey {
    const void* g = nullptr;
    const void* f = nullptr;
    const void* stats = nullptr;
    int k = -1, flags = 0, solver = 0;
    float relax = 1.f;
    bool profiling = false;
    bool operator==(const GraphKey& o) const {
        return g == o.g && f == o.f && stats == o.stats && k == o.k && flags == o.flags &&
               solver == o.solver && relax == o.relax && profiling == o.profiling;
    }
};

}  // namespace

namespace {
struct BatchState;
void free_batch(BatchState* B);
void drop_batched_graph_of(const ctis_plan* P);
}  // namespace

struct ctis_plan {
    int a = 0, alpha = 0, w = 0, gamma = 0, xi = 0, dtype = 0;
    int64_t m = 0, n = 0;
    int device = 0, num_sms = 0, K = 1;
    int a_pitch = 0;      // row pitch of the internal datacube copies (elements)
    int g_pitch = 0;      // row pitch of the internal FPA copies (elements)
    int f_copies = 4, u_copies = 4;
    int64_t f_copy_stride = 0, u_copy_stride = 0;   // elements between copies
    std::vector<int32_t> tap_s, tap_x, tap_y;
    std::vector<float> tap_v;   // stored values widened to float32
    std::vector<float> h;       // [w]
    std::vector<Cluster> clusters;
    std::vector<int32_t> tap_slot;   // cluster * K*K + dy*K + dx of every stored tap
    ProjTables fwd, adj;
    int fwd_shape = 0;               // forward tile shape (0: 32 x 32, 1: 32 x 16)
    int adj_tiles_per_plane = 0;
    int* d_tap_slot = nullptr;
    int* d_tap_s = nullptr;
    float* d_grad_part = nullptr;    // [clusters][adjoint tiles per plane][K*K]
    // unrolled-EM gradient workspace (grown on demand)
    int ck_steps = -1;               // checkpoints held: ck_steps + 1 iterates
    float* d_ck = nullptr;
    float* d_work = nullptr;         // q, gu (n each); z, gfd, gb, hq, a (m each)
    double* d_gwork = nullptr;       // vjp partials [w][blocks], dh [w], stats [4]
    BatchState* batch = nullptr;     // frames of ctis_reconstruct_batched (grown on demand)
    float* d_h = nullptr;
    float* d_u = nullptr;        // u_copies x-shifted copies of the FPA input of the adjoint
    void* d_fwork = nullptr;     // f_copies x-shifted copies of the datacube (forward input)
    float* d_scratch = nullptr;
    int64_t scratch_capacity = 0;    // float elements of d_scratch
    int* d_tickets = nullptr;
    size_t tickets_capacity = 0;      // ints in d_tickets
    int* d_counters = nullptr;   // [3] error flag, [8] the frame reduction's ticket
    double* d_tile_stats = nullptr;
    size_t tile_stats_capacity = 0;   // forward tiles d_tile_stats holds
    double* d_red_part = nullptr;   // [kStatSlices][kNumStats] frame reduction slices
    int64_t device_bytes = 0;
    cudaStream_t cap_stream = nullptr;
    GraphKey gkey;
    cudaGraphExec_t gexec = nullptr;
    bool profiling = false;
    int forced_per_item = 0;          // 0: chosen by schedule()
    int forced_split_q = 0;           // 0: chosen by schedule()
    int forced_skew_pm = 0;           // CTA priority skew of the model's schedule
    int host_ctas = 0;                // > 0: host-only tables for this many CTAs (no device)
    bool clip = false;                // CTIS_BOUNDARY_CLIP: shifted nonzeros off the FPA dropped
    bool wrap = false;                // CTIS_BOUNDARY_WRAP: stored as the clip reading of the
                                      // PSF and its wrapped images (clip is set too)
    float* d_hvox = nullptr;          // clip: h = H^T 1 per voxel [w][alpha][a]
    float* d_rowsum = nullptr;        // SART: r = H 1 per pixel [xi][gamma], built on first use
    bool rowsum_valid = false;
    bool drop_copies = false;         // CTIS_DEBUG_DROP_COPIES (test hook)
    bool overlap_launch = true;       // programmatic dependent launch of the projectors
    FftForm* fft = nullptr;           // the paper's FFT form, built on first use
    float* d_fft_u = nullptr;         // its EM ratio [n]
    float* d_shard_q = nullptr;       // wavelength-sharded EM: the summed H f [n]
    double* d_shard_part = nullptr;   // its statistics' block sums
    std::vector<cudaEvent_t> events;                  // pool, pairs (start, stop)
    std::vector<std::pair<int, int>> prof_fwd, prof_adj;   // event index pairs of the last call
};

namespace {

int dmalloc(ctis_plan* P, void** ptr, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CTIS_ERR_NOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    P->device_bytes += static_cast<int64_t>(bytes);
    return CTIS_OK;
}

template <typename T>
int upload(ctis_plan* P, T** dst, const std::vector<T>& src) {
    int rc = dmalloc(P, reinterpret_cast<void**>(dst), src.size() * sizeof(T));
    if (rc) return rc;
    if (!src.empty())
        CTIS_CUDA(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return CTIS_OK;
}

void free_tables(ProjTables& t) {
    cudaFree(t.d_tasks);
    cudaFree(t.d_warp_begin);
    cudaFree(t.d_heads);
    t.d_heads = nullptr;
    cudaFree(t.d_weights);
    cudaFree(t.d_witems);
    t.d_tasks = nullptr;
    t.d_warp_begin = nullptr;
    t.d_weights = nullptr;
    t.d_witems = nullptr;
}

void destroy(ctis_plan* P) {
    if (!P) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(P->device);
    cudaDeviceSynchronize();
    drop_batched_graph_of(P);
    free_batch(P->batch);
    if (P->gexec) cudaGraphExecDestroy(P->gexec);
    if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
    for (cudaEvent_t e : P->events) cudaEventDestroy(e);
    free_tables(P->fwd);
    free_tables(P->adj);
    cudaFree(P->d_h);
    cudaFree(P->d_u);
    cudaFree(P->d_fwork);
    cudaFree(P->d_scratch);
    cudaFree(P->d_tickets);
    cudaFree(P->d_counters);
    cudaFree(P->d_tile_stats);
    cudaFree(P->d_red_part);
    cudaFree(P->d_hvox);
    cudaFree(P->d_rowsum);
    fft_form_destroy(P->fft);
    cudaFree(P->d_fft_u);
    cudaFree(P->d_shard_q);
    cudaFree(P->d_shard_part);
    cudaFree(P->d_tap_slot);
    cudaFree(P->d_tap_s);
    cudaFree(P->d_grad_part);
    cudaFree(P->d_ck);
    cudaFree(P->d_work);
    cudaFree(P->d_gwork);
    cudaSetDevice(cur);
    delete P;
}

// Cost of an item in tasks per warp: the CTA's warps share its tasks, then
// wait for each other, add their sums in shared memory and run the epilogue
// (measured on GB300: about three tasks' time), and a tile split over CTAs
// pays the chunk sums' round trip through global memory (about three more).
constexpr double kItemCost = 3.0, kChunkCost = 3.0;
double item_cost(int tasks, int nw, bool chunked) {
    return (tasks + nw - 1) / nw + (chunked ? kChunkCost : 0.0) + kItemCost;
}

// Splits every tile's task range into chunks of at most `per_item` tasks and
// fills the item list and the scratch slot bases.
void make_items(ProjTables& T, const std::vector<int>& tile_task_begin, int per_item) {
    T.items.clear();
    T.scratch_slots = 0;
    for (size_t t = 0; t < T.tiles.size(); ++t) {
        const int b = tile_task_begin[t], e = tile_task_begin[t + 1];
        const int cnt = e - b;
        const int nch = std::max(1, (cnt + per_item - 1) / per_item);
        T.tiles[t].nchunks = nch;
        T.tiles[t].scratch_base = 0;
        if (nch > 1) {
            T.tiles[t].scratch_base = static_cast<int>(T.scratch_slots);
            T.scratch_slots += nch;
        }
        for (int c = 0; c < nch; ++c) {
            ItemDesc it;
            it.tile = static_cast<int>(t);
            it.chunk = c;
            it.task_begin = b + static_cast<int>(static_cast<int64_t>(cnt) * c / nch);
            it.task_end = b + static_cast<int>(static_cast<int64_t>(cnt) * (c + 1) / nch);
            T.items.push_back(it);
        }
    }
}

// Writes the CTAs' item lists. The SM's warp schedulers favour the warps of
// the CTAs that became resident first (the lower block indices), so those run
// their tasks faster while all CTAs are active, and an SM finishes with its
// last CTA. Without a placement map the lists go to the CTAs in order of
// decreasing estimated load (ties: original order). With the probed map of
// CTAs to SMs, the lists, heaviest first, go to the SM with the least load
// that still has a free CTA (ties: lower SM id), so the SMs' totals are
// balanced, and each SM's lists go to its CTAs heaviest first in block order.
// Either way every list runs exactly once: the map only decides which CTA.
void place_ctas(ProjTables& T, const std::vector<std::vector<int>>& per_cta,
                const std::vector<double>& load) {
    const int n = static_cast<int>(per_cta.size());
    std::vector<int> ord(n);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return load[x] > load[y]; });
    std::vector<int> list_of(n);   // block -> list
    if (static_cast<int>(T.block_sm.size()) == n) {
        std::map<int, std::vector<int>> blocks;   // SM -> its blocks, ascending
        for (int b = 0; b < n; ++b) blocks[T.block_sm[b]].push_back(b);
        struct Sm {
            std::vector<int> blocks, lists;
            double load = 0.0;
        };
        std::vector<Sm> sms;
        for (auto& kv : blocks) sms.push_back({kv.second, {}, 0.0});
        for (int l : ord) {
            int best = -1;
            for (int k = 0; k < static_cast<int>(sms.size()); ++k) {
                if (sms[k].lists.size() >= sms[k].blocks.size()) continue;
                if (best < 0 || sms[k].load < sms[best].load - 1e-9) best = k;
            }
            sms[best].lists.push_back(l);   // lists arrive heaviest first
            sms[best].load += load[l];
        }
        for (const Sm& sm : sms)
            for (size_t k = 0; k < sm.blocks.size(); ++k) list_of[sm.blocks[k]] = sm.lists[k];
    } else {
        for (int b = 0; b < n; ++b) list_of[b] = ord[b];
    }
    T.cta_begin.assign(1, 0);
    T.cta_items.clear();
    for (int b = 0; b < n; ++b) {
        const std::vector<int>& items = per_cta[list_of[b]];
        T.cta_items.insert(T.cta_items.end(), items.begin(), items.end());
        T.cta_begin.push_back(static_cast<int>(T.cta_items.size()));
    }
}

// Relative speed of CTA c of n under a priority skew of skew_pm permille:
// the SM's warp schedulers favour the warps of the CTAs that became resident
// first (the lower block indices), so while all CTAs are active CTA c runs
// about 1 + skew (1 - 2 c / (n - 1)) times the mean rate.
double cta_speed(int c, int n, int skew_pm) {
    if (n <= 1 || skew_pm == 0) return 1.0;
    return 1.0 + skew_pm / 1000.0 * (1.0 - 2.0 * c / (n - 1));
}

// Longest-processing-time-first assignment of the items to n_ctas CTAs: each
// item, largest first, goes to the CTA with the earliest estimated finish
// (load / speed; ties: the lower index). Returns the latest estimated finish
// (tasks per warp at the mean rate); fills cta_begin / cta_items.
double assign_ctas(ProjTables& T, int n_ctas, int skew_pm) {
    std::vector<int> order(T.items.size());
    std::iota(order.begin(), order.end(), 0);
    auto cost = [&](int i) {
        const ItemDesc& it = T.items[i];
        return item_cost(it.task_end - it.task_begin, T.nw, T.tiles[it.tile].nchunks > 1);
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
    std::vector<double> speed(n_ctas);
    for (int c = 0; c < n_ctas; ++c) speed[c] = cta_speed(c, n_ctas, skew_pm);
    using Slot = std::pair<double, int>;   // (estimated finish, CTA)
    std::vector<Slot> heap;
    heap.reserve(n_ctas);
    for (int c = 0; c < n_ctas; ++c) heap.emplace_back(0.0, c);
    auto cmp = [](const Slot& x, const Slot& y) {
        return x.first != y.first ? x.first > y.first : x.second > y.second;
    };
    std::make_heap(heap.begin(), heap.end(), cmp);
    std::vector<std::vector<int>> per_cta(n_ctas);
    std::vector<double> load(n_ctas, 0.0);
    double max_finish = 0.0;
    for (int i : order) {
        std::pop_heap(heap.begin(), heap.end(), cmp);
        Slot& sl = heap.back();
        const int c = sl.second;
        per_cta[c].push_back(i);
        load[c] += cost(i);
        sl.first = load[c] / speed[c];
        max_finish = std::max(max_finish, sl.first);
        std::push_heap(heap.begin(), heap.end(), cmp);
    }
    place_ctas(T, per_cta, load);
    return max_finish;
}

// Balanced contiguous split: the tiles' tasks, in tile order, are cut into
// runs of nearly equal estimated cost, one run per CTA. A piece of a tile
// costs the warps' share of its tasks plus `e` (the shared-memory sum and
// the epilogue, in tasks per warp); a tile cut by a run boundary becomes
// chunks on consecutive CTAs, and each of its pieces also pays the chunk
// sums' round trip. The per-CTA budget is the smallest (bisection) for which
// the greedy fill needs at most n_ctas CTAs. Fills items (chunk order within
// a tile), cta_begin / cta_items and the tiles' chunk counts; returns the
// busiest CTA's estimate.
double split_items(ProjTables& T, int n_ctas, double e, int skew_pm) {
    const std::vector<int>& begin = T.tile_task_begin;
    const int nw = T.nw;
    const int ntiles = static_cast<int>(T.tiles.size());
    struct Piece {
        int tile, b, e, cta;
    };
    std::vector<Piece> pieces;
    auto share = [nw](int n) { return static_cast<double>((n + nw - 1) / nw); };
    // CTAs the greedy fill under budget B needs (n_ctas + 1 when it needs more)
    std::vector<double> speed(n_ctas);
    for (int c = 0; c < n_ctas; ++c) speed[c] = cta_speed(c, n_ctas, skew_pm);
    // CTA c's budget is B * speed[c]; the estimate is the latest finish
    auto fill = [&](double B, double* max_finish) -> int {
        pieces.clear();
        int cta = 0;
        double load = 0.0, top = 0.0;
        for (int t = 0; t < ntiles; ++t) {
            int pos = begin[t];
            const int end = begin[t + 1];
            bool cut = false;
            for (;;) {
                const double cap = B * speed[cta];
                const double whole = share(end - pos) + e + (cut ? kChunkCost : 0.0);
                if (load + whole <= cap) {
                    pieces.push_back({t, pos, end, cta});
                    load += whole;
                    top = std::max(top, load / speed[cta]);
                    break;
                }
                // a piece of it here, the rest on the next CTAs
                const double room = cap - load - e - kChunkCost;
                const int n = room >= 1.0 ? std::min(end - pos, static_cast<int>(room) * nw) : 0;
                if (n > 0 && n < end - pos) {
                    pieces.push_back({t, pos, pos + n, cta});
                    top = std::max(top, (load + share(n) + e + kChunkCost) / speed[cta]);
                    pos += n;
                    cut = true;
                }
                if (++cta >= n_ctas) return n_ctas + 1;
                load = 0.0;
            }
        }
        if (max_finish) *max_finish = top;
        return load > 0.0 ? cta + 1 : cta;
    };
    double total = 0.0;
    for (int t = 0; t < ntiles; ++t) total += share(begin[t + 1] - begin[t]) + e;
    double min_speed = 1.0;
    for (double v : speed) min_speed = std::min(min_speed, v);
    double lo = std::max(total / n_ctas, e + kChunkCost + 1.0);
    double hi = (total + e + kChunkCost + 1.0) / min_speed;
    if (fill(lo, nullptr) > n_ctas) {
        for (int i = 0; i < 60 && hi - lo > 1e-3; ++i) {
            const double mid = 0.5 * (lo + hi);
            (fill(mid, nullptr) <= n_ctas ? hi : lo) = mid;
        }
    } else {
        hi = lo;
    }
    double max_load = 0.0;
    fill(hi, &max_load);
    // items, chunk numbering and scratch slots
    T.items.clear();
    T.scratch_slots = 0;
    for (auto& td : T.tiles) {
        td.nchunks = 0;
        td.scratch_base = 0;
    }
    for (const Piece& pc : pieces) T.tiles[pc.tile].nchunks++;
    for (auto& td : T.tiles) {
        if (td.nchunks > 1) {
            td.scratch_base = static_cast<int>(T.scratch_slots);
            T.scratch_slots += td.nchunks;
        }
    }
    std::vector<int> next_chunk(T.tiles.size(), 0);
    std::vector<std::vector<int>> per_cta(n_ctas);
    std::vector<double> load(n_ctas, 0.0);
    for (const Piece& pc : pieces) {
        ItemDesc it;
        it.tile = pc.tile;
        it.chunk = next_chunk[pc.tile]++;
        it.task_begin = pc.b;
        it.task_end = pc.e;
        per_cta[pc.cta].push_back(static_cast<int>(T.items.size()));
        load[pc.cta] += share(pc.e - pc.b) + e + (T.tiles[pc.tile].nchunks > 1 ? kChunkCost : 0.0);
        T.items.push_back(it);
    }
    place_ctas(T, per_cta, load);
    return max_load;
}

void layout_warps(ProjTables& T);

// Picks the work schedule: `forced_split_q` > 0 forces the balanced split
// with a per-item overhead of forced_split_q / 4 tasks, `forced` > 0 the
// longest-first assignment of chunks of at most `forced` tasks; otherwise the
// candidate (chunk sizes, and the balanced split with the model's item
// overhead) with the smallest estimate of the latest CTA. CTA speeds follow
// the priority skew skew_pm (permille; see cta_speed). Then lays out the
// warps' lists (layout_warps).
void schedule(ProjTables& T, int n_warps, int forced, int forced_split_q, int skew_pm) {
    const std::vector<int>& begin = T.tile_task_begin;
    const int nw = T.nw;
    const int n_ctas = n_warps / nw;
    T.n_warps = n_ctas * nw;
    constexpr int kModelSplitQ = 12;   // the item overhead of item_cost, in quarter tasks
    int split_q = 0;
    if (forced_split_q > 0) {
        split_q = forced_split_q;
    } else {
        std::vector<int> cands;
        if (forced > 0) {
            cands.push_back(forced);
        } else {
            for (int c : {256, 192, 128, 96, 64, 48, 32, 24, 16, 12, 8}) cands.push_back(c);
        }
        int best = cands[0];
        double best_load = -1.0;
        for (int c : cands) {
            make_items(T, begin, c);
            const double load = assign_ctas(T, n_ctas, skew_pm);
            if (best_load < 0 || load < best_load - 1e-9) {
                best_load = load;
                best = c;
            }
        }
        if (forced <= 0 &&
            split_items(T, n_ctas, kModelSplitQ / 4.0, skew_pm) < best_load - 1e-9) {
            split_q = kModelSplitQ;
        } else {
            make_items(T, begin, best);
            T.max_warp_load = assign_ctas(T, n_ctas, skew_pm);
            T.per_item = best;
        }
    }
    if (split_q > 0) {
        T.max_warp_load = split_items(T, n_ctas, split_q / 4.0, skew_pm);
        T.per_item = 0;
    }
    T.split_q = split_q;
    T.skew_pm = skew_pm;
    layout_warps(T);
}

// Lays out, for every warp, its part of each of its CTA's items (from
// cta_begin / cta_items): warp w of a CTA runs tasks [b + w*n/NW,
// b + (w+1)*n/NW) of an item of n tasks; the warps' item lists are parallel
// (same tiles, same order) and every warp's tasks are stored contiguously.
void layout_warps(ProjTables& T) {
    const int nw = T.nw;
    const int n_ctas = static_cast<int>(T.cta_begin.size()) - 1;
    T.witems.clear();
    T.witem_src.clear();
    T.warp_begin.assign(1, 0);
    std::vector<TaskDesc> wt;
    wt.reserve(T.tile_tasks.size());
    for (int c = 0; c < n_ctas; ++c)
        for (int w = 0; w < nw; ++w) {
            for (int k = T.cta_begin[c]; k < T.cta_begin[c + 1]; ++k) {
                const ItemDesc& it = T.items[T.cta_items[k]];
                const TileDesc& td = T.tiles[it.tile];
                const int n = it.task_end - it.task_begin;
                const int tb = it.task_begin + static_cast<int>(static_cast<int64_t>(n) * w / nw);
                const int te = it.task_begin + static_cast<int>(static_cast<int64_t>(n) * (w + 1) / nw);
                WorkItem wi;
                wi.tile = it.tile;
                wi.x0 = td.x0;
                wi.y0 = td.y0;
                wi.plane = td.plane;
                wi.chunk_info = td.nchunks | (it.chunk << 16);
                wi.scratch_base = td.scratch_base;
                wi.task_begin = static_cast<int>(wt.size());
                wt.insert(wt.end(), T.tile_tasks.begin() + tb, T.tile_tasks.begin() + te);
                wi.task_end = static_cast<int>(wt.size());
                T.witems.push_back(wi);
                T.witem_src.push_back({tb, te});
            }
            T.warp_begin.push_back(static_cast<int>(T.witems.size()));
        }
    T.tasks = std::move(wt);
    T.heads.assign(T.warp_begin.size() - 1, WarpHead{});
    for (size_t w = 0; w + 1 < T.warp_begin.size(); ++w) {
        WarpHead& h = T.heads[w];
        h.ib = T.warp_begin[w];
        h.ie = T.warp_begin[w + 1];
        if (h.ib >= h.ie) continue;
        h.task_begin = T.witems[h.ib].task_begin;
        h.task_end = T.witems[h.ie - 1].task_end;
        for (int j = 0; j < 3 && h.task_begin + j < h.task_end; ++j)
            h.first[j] = T.tasks[h.task_begin + j];
        h.item0 = T.witems[h.ib];
    }
}

// h = H^T 1 (Eq. 2): under the on-FPA rule every voxel of wavelength s sees
// all of that wavelength's taps, so h_s is the float64 sum of its stored
// values, rounded once to float32.
void compute_h(ctis_plan* P) {
    std::vector<double> hs(P->w, 0.0);
    for (size_t k = 0; k < P->tap_v.size(); ++k) {
        // under the wrap reading the images off the FPA repeat an original
        if (P->wrap && (P->tap_x[k] < 0 || P->tap_y[k] < 0)) continue;
        hs[P->tap_s[k]] += static_cast<double>(P->tap_v[k]);
    }
    P->h.assign(P->w, 0.f);
    for (int s = 0; s < P->w; ++s) P->h[s] = static_cast<float>(hs[s]);
}

// Device image of one projector's weight table: per cluster its K x K values
// (adjoint orientation: [dy][dx] as on the FPA; forward: flipped, since the
// forward applies the cluster as a convolution), one 32-bit word each (float32,
// or a bfloat16 duplicated in both halves), padded to the kernel's 16-byte
// weight slot.
std::vector<unsigned char> weight_table(const ctis_plan* P, bool forward) {
    const int K = P->K, KK = K * K;
    const int64_t ncl = static_cast<int64_t>(P->clusters.size());
    std::vector<float> wts(static_cast<size_t>(ncl) * KK, 0.f);
    for (size_t k = 0; k < P->tap_v.size(); ++k) {
        const int64_t sl = P->tap_slot[k];
        const int64_t c = sl / KK, e = sl % KK;
        wts[c * KK + (forward ? KK - 1 - e : e)] = P->tap_v[k];
    }
    const int pad = gather_weight_pad(forward, K, P->dtype);
    std::vector<unsigned char> out;
    if (P->dtype == kDtypeBF16) {
        std::vector<uint32_t> b(static_cast<size_t>(ncl) * pad, 0);
        for (int64_t c = 0; c < ncl; ++c)
            for (int e = 0; e < KK; ++e) {
                const uint32_t h = to_bf16_bits(wts[c * KK + e]);
                b[c * pad + e] = h | (h << 16);
            }
        out.resize(b.size() * sizeof(uint32_t));
        std::memcpy(out.data(), b.data(), out.size());
    } else {
        std::vector<float> f(static_cast<size_t>(ncl) * pad, 0.f);
        for (int64_t c = 0; c < ncl; ++c)
            for (int e = 0; e < KK; ++e) f[c * pad + e] = wts[c * KK + e];
        out.resize(f.size() * sizeof(float));
        std::memcpy(out.data(), f.data(), out.size());
    }
    return out;
}

// Writes both weight tables and h to the device; allocates them the first time.
int write_values(ctis_plan* P, bool allocate) {
    for (ProjTables* T : {&P->fwd, &P->adj}) {
        const std::vector<unsigned char> img = weight_table(P, T == &P->fwd);
        if (allocate) {
            int rc = dmalloc(P, &T->d_weights, img.size());
            if (rc) return rc;
        }
        if (!img.empty())
            CTIS_CUDA(cudaMemcpy(T->d_weights, img.data(), img.size(), cudaMemcpyHostToDevice));
    }
    if (allocate) {
        int rc = dmalloc(P, reinterpret_cast<void**>(&P->d_h), sizeof(float) * P->w);
        if (rc) return rc;
    }
    CTIS_CUDA(cudaMemcpy(P->d_h, P->h.data(), sizeof(float) * P->w, cudaMemcpyHostToDevice));
    // a copy from pageable host memory may still be in flight when cudaMemcpy
    // returns; kernels on other streams must not read the tables before it lands
    CTIS_CUDA(cudaDeviceSynchronize());
    return CTIS_OK;
}

// Host-only validation of the PSF values and of the boundary rule: under
// REJECT every shifted copy of every nonzero must stay on the FPA (Sec. 2),
// under WRAP every nonzero must lie on it (an entry of c_s, Eq. 7).
int validate_psf(int a, int al, int w, int ga, int xi, const int32_t* psf_ptr,
                 const int32_t* psf_x, const int32_t* psf_y, const float* psf_val, int boundary) {
    const bool clip = boundary == CTIS_BOUNDARY_CLIP;
    const int64_t nnz_in = psf_ptr[w];
    for (int64_t k = 0; k < nnz_in; ++k) {
        const float v = psf_val[k];
        if (!std::isfinite(v) || v < 0.f)
            return fail(CTIS_ERR_INVALID_ARG, "psf_val[%lld] = %g is not finite and >= 0",
                        (long long)k, (double)v);
        const int64_t x = psf_x[k], y = psf_y[k];
        if (clip) {   // any position; the shifted copies off the FPA are dropped
            if (x < -(int64_t{1} << 24) || x >= (int64_t{1} << 24) || y < -(int64_t{1} << 24) ||
                y >= (int64_t{1} << 24))
                return fail(CTIS_ERR_INVALID_ARG, "PSF nonzero %lld at (%lld, %lld) out of range",
                            (long long)k, (long long)x, (long long)y);
            continue;
        }
        if (boundary == CTIS_BOUNDARY_WRAP) {
            if (x < 0 || y < 0 || x >= ga || y >= xi)
                return fail(CTIS_ERR_OUT_OF_BOUNDS,
                            "PSF nonzero %lld at (%lld, %lld) is off the %dx%d FPA", (long long)k,
                            (long long)x, (long long)y, ga, xi);
            continue;
        }
        if (x < 0 || y < 0 || x + a - 1 >= ga || y + al - 1 >= xi)
            return fail(CTIS_ERR_OUT_OF_BOUNDS,
                        "PSF nonzero %lld at (%lld, %lld) leaves the %dx%d FPA when shifted "
                        "across the %dx%d field stop",
                        (long long)k, (long long)x, (long long)y, ga, xi, a, al);
    }
    return CTIS_OK;
}

// A map key for an FPA position, unique for any coordinates in [-2^31, 2^31).
int64_t pos_key(int64_t x, int64_t y) {
    return static_cast<int64_t>((static_cast<uint64_t>(y) << 32) ^ static_cast<uint32_t>(x));
}

// Forward work lists (FPA tiles of the plan's forward tile shape x clusters
// whose footprint meets them) and their schedule over warps_fwd warps.
void build_forward_lists(ctis_plan* P, int warps_fwd) {
    const int K = P->K, a = P->a, al = P->alpha, w = P->w, ga = P->gamma, xi = P->xi;
    const int64_t ncl = static_cast<int64_t>(P->clusters.size());
    ProjTables& T = P->fwd;
    T.tiles.clear();
    T.items.clear();
    T.tile_tasks.clear();
    const int TX = T.tile_w = gather_tile_w(true, P->dtype, P->fwd_shape);
    const int TY = T.tile_h = gather_tile_h(true, P->dtype, P->fwd_shape);
    T.nw = gather_warps_per_cta(true);
    const int ntx = (ga + TX - 1) / TX, nty = (xi + TY - 1) / TY;
    const int fw = a + K - 1, fh = al + K - 1;   // footprint of one cluster
    std::vector<std::vector<int>> per_tile(static_cast<size_t>(ntx) * nty);
    for (int64_t c = 0; c < ncl; ++c) {
        const Cluster& cl = P->clusters[c];
        // the tiles that the footprint's part on the FPA meets (under
        // clipping the footprint may reach past any edge, or miss the FPA
        // altogether; a cluster box may also reach past its last tap)
        const int64_t fx0 = std::max<int64_t>(0, cl.X);
        const int64_t fx1 = std::min<int64_t>(ga, int64_t{cl.X} + fw);
        const int64_t fy0 = std::max<int64_t>(0, cl.Y);
        const int64_t fy1 = std::min<int64_t>(xi, int64_t{cl.Y} + fh);
        if (fx0 >= fx1 || fy0 >= fy1) continue;
        const int64_t tx0 = fx0 / TX, tx1 = (fx1 - 1) / TX;
        const int64_t ty0 = fy0 / TY, ty1 = (fy1 - 1) / TY;
        for (int64_t ty = ty0; ty <= ty1; ++ty)
            for (int64_t tx = tx0; tx <= tx1; ++tx)
                per_tile[static_cast<size_t>(ty) * ntx + tx].push_back(static_cast<int>(c));
    }
    // Tiles no footprint meets hold H f = 0 whatever f is: they are left out
    // of the lists (the raw forward zeroes its output first; the ratio's
    // u copies and the tile statistics are zero there).
    std::vector<int> begin{0};
    for (int ty = 0; ty < nty; ++ty)
        for (int tx = 0; tx < ntx; ++tx) {
            if (per_tile[static_cast<size_t>(ty) * ntx + tx].empty()) continue;
            TileDesc td{};
            td.x0 = tx * TX;
            td.y0 = ty * TY;
            td.plane = 0;
            T.tiles.push_back(td);
            std::vector<TaskDesc> tl;
            for (int c : per_tile[static_cast<size_t>(ty) * ntx + tx]) {
                const Cluster& cl = P->clusters[c];
                const int64_t px = static_cast<int64_t>(td.x0) - cl.X - (K - 1);
                const int64_t py = static_cast<int64_t>(td.y0) - cl.Y - (K - 1);
                const int64_t q = floor_mod(-px, P->f_copies);   // copy holding px aligned
                TaskDesc t;
                t.wx = static_cast<int>(px + q);
                t.wy = static_cast<int>(py);
                t.plane = static_cast<int>(q) * w + cl.s;   // copy * w + s
                t.cluster = c;
                tl.push_back(t);
            }
            T.tile_tasks.insert(T.tile_tasks.end(), tl.begin(), tl.end());
            begin.push_back(static_cast<int>(T.tile_tasks.size()));
        }
    T.tile_task_begin = std::move(begin);
    schedule(T, warps_fwd, P->forced_per_item, P->forced_split_q, P->forced_skew_pm);
}

int build(ctis_plan* P, const int32_t* psf_ptr, const int32_t* psf_x, const int32_t* psf_y,
          const float* psf_val) {
    const int a = P->a, al = P->alpha, w = P->w, ga = P->gamma, xi = P->xi;

    // ---- merge duplicates, sort by (s, y, x)
    std::vector<double> merged_v;
    std::vector<int64_t> order;
    for (int s = 0; s < w; ++s) {
        const int64_t b = psf_ptr[s], e = psf_ptr[s + 1];
        order.resize(e - b);
        std::iota(order.begin(), order.end(), b);
        std::sort(order.begin(), order.end(), [&](int64_t i, int64_t j) {
            return psf_y[i] != psf_y[j] ? psf_y[i] < psf_y[j] : psf_x[i] < psf_x[j];
        });
        for (size_t q = 0; q < order.size(); ++q) {
            const int64_t k = order[q];
            if (!P->tap_s.empty() && P->tap_s.back() == s && P->tap_x.back() == psf_x[k] &&
                P->tap_y.back() == psf_y[k]) {
                merged_v.back() += static_cast<double>(psf_val[k]);
            } else {
                P->tap_s.push_back(s);
                P->tap_x.push_back(psf_x[k]);
                P->tap_y.push_back(psf_y[k]);
                merged_v.push_back(static_cast<double>(psf_val[k]));
            }
        }
    }
    const int64_t nnz = static_cast<int64_t>(merged_v.size());
    std::vector<uint16_t> tap_bf16;
    P->tap_v.resize(nnz);
    for (int64_t k = 0; k < nnz; ++k) {
        const float f = static_cast<float>(merged_v[k]);
        if (P->dtype == kDtypeBF16) {
            tap_bf16.push_back(to_bf16_bits(f));
            P->tap_v[k] = bf16_bits_to_float(tap_bf16.back());
        } else {
            P->tap_v[k] = f;
        }
    }

    // ---- h = H^T 1 per wavelength, float64 sum of the stored values
    compute_h(P);

    // ---- clusters: 8-connected components, covered by K x K boxes
    std::vector<int64_t> s_begin(w + 1, 0);
    for (int64_t k = 0; k < nnz; ++k) s_begin[P->tap_s[k] + 1]++;
    for (int s = 0; s < w; ++s) s_begin[s + 1] += s_begin[s];
    std::vector<int64_t> parent(nnz);
    std::iota(parent.begin(), parent.end(), 0);
    auto find = [&](int64_t i) {
        while (parent[i] != i) i = parent[i] = parent[parent[i]];
        return i;
    };
    for (int s = 0; s < w; ++s) {
        std::unordered_map<int64_t, int64_t> at;
        for (int64_t k = s_begin[s]; k < s_begin[s + 1]; ++k)
            at[pos_key(P->tap_x[k], P->tap_y[k])] = k;
        for (int64_t k = s_begin[s]; k < s_begin[s + 1]; ++k) {
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int64_t x = P->tap_x[k] + dx, y = P->tap_y[k] + dy;
                    auto it = at.find(pos_key(x, y));
                    if (it != at.end()) {
                        const int64_t r1 = find(k), r2 = find(it->second);
                        if (r1 != r2) parent[std::max(r1, r2)] = std::min(r1, r2);
                    }
                }
        }
    }
    struct Box { int s, x0, y0, x1, y1; };
    std::unordered_map<int64_t, Box> comp;
    int max_side = 1;
    for (int64_t k = 0; k < nnz; ++k) {
        const int64_t r = find(k);
        auto it = comp.find(r);
        if (it == comp.end()) {
            comp[r] = Box{P->tap_s[k], P->tap_x[k], P->tap_y[k], P->tap_x[k], P->tap_y[k]};
        } else {
            Box& b = it->second;
            b.x0 = std::min(b.x0, P->tap_x[k]);
            b.x1 = std::max(b.x1, P->tap_x[k]);
            b.y0 = std::min(b.y0, P->tap_y[k]);
            b.y1 = std::max(b.y1, P->tap_y[k]);
        }
    }
    for (auto& kv : comp)
        max_side = std::max(max_side, std::max(kv.second.x1 - kv.second.x0 + 1,
                                               kv.second.y1 - kv.second.y0 + 1));
    const int K = max_side <= 1 ? 1 : (max_side <= 3 ? 3 : 5);
    P->K = K;
    std::vector<Box> boxes;
    for (auto& kv : comp) boxes.push_back(kv.second);
    std::sort(boxes.begin(), boxes.end(), [](const Box& x, const Box& y) {
        if (x.s != y.s) return x.s < y.s;
        if (x.y0 != y.y0) return x.y0 < y.y0;
        return x.x0 < y.x0;
    });
    // Cover every component with K x K boxes. Every tap belongs to the first
    // box (in this order) that contains it, whatever its value: tap_slot[k] =
    // box * K*K + dy*K + dx. Boxes of one wavelength may overlap where two
    // components' bounding boxes do; a tap is never claimed twice.
    const int KK = K * K;
    P->tap_slot.assign(nnz, -1);
    for (int s = 0; s < w; ++s) {
        std::unordered_map<int64_t, int64_t> at;
        for (int64_t k = s_begin[s]; k < s_begin[s + 1]; ++k)
            at[pos_key(P->tap_x[k], P->tap_y[k])] = k;
        for (const Box& b : boxes) {
            if (b.s != s) continue;
            for (int by = b.y0; by <= b.y1; by += K)
                for (int bx = b.x0; bx <= b.x1; bx += K) {
                    std::vector<std::pair<int64_t, int>> mine;   // (tap, slot in the box)
                    for (int dy = 0; dy < K; ++dy)
                        for (int dx = 0; dx < K; ++dx) {
                            const int64_t x = bx + dx, y = by + dy;
                            if (x > b.x1 || y > b.y1) continue;
                            auto it = at.find(pos_key(x, y));
                            if (it == at.end() || P->tap_slot[it->second] >= 0) continue;
                            mine.emplace_back(it->second, dy * K + dx);
                        }
                    if (mine.empty()) continue;
                    const int64_t c = static_cast<int64_t>(P->clusters.size());
                    P->clusters.push_back(Cluster{s, bx, by});
                    for (const auto& te : mine) P->tap_slot[te.first] = c * KK + te.second;
                }
        }
    }
    for (int64_t k = 0; k < nnz; ++k)
        if (P->tap_slot[k] < 0)
            return fail(CTIS_ERR_INVALID_ARG, "internal: tap %lld not covered by a cluster",
                        (long long)k);
    const int64_t ncl = static_cast<int64_t>(P->clusters.size());

    int warps_fwd = P->host_ctas * gather_warps_per_cta(true);
    int warps_adj = P->host_ctas * gather_warps_per_cta(false);
    if (P->host_ctas == 0) {
        CTIS_CUDA(gather_prepare(true, K, P->dtype, &P->fwd.blocks_per_sm, P->fwd_shape));
        CTIS_CUDA(gather_prepare(false, K, P->dtype, &P->adj.blocks_per_sm));
        int grad_blocks = 0;   // runs on the adjoint's work lists and warp count
        CTIS_CUDA(psf_grad_prepare(K, P->dtype, &grad_blocks));
        warps_fwd = P->num_sms * P->fwd.blocks_per_sm * gather_warps_per_cta(true);
        warps_adj = P->num_sms * P->adj.blocks_per_sm * gather_warps_per_cta(false);
    }

    build_forward_lists(P, warps_fwd);

    // ---- adjoint work lists: voxel tiles of wavelength s x clusters of s
    {
        ProjTables& T = P->adj;
        const int TX = T.tile_w = gather_tile_w(false, P->dtype), TY = T.tile_h = gather_tile_h(false, P->dtype);
        T.nw = gather_warps_per_cta(false);
        std::vector<int64_t> c_begin(w + 1, 0);
        for (int64_t c = 0; c < ncl; ++c) c_begin[P->clusters[c].s + 1]++;
        for (int s = 0; s < w; ++s) c_begin[s + 1] += c_begin[s];
        std::vector<int> begin{0};
        const int ntx = (a + TX - 1) / TX, nty = (al + TY - 1) / TY;
        P->adj_tiles_per_plane = ntx * nty;
        for (int s = 0; s < w; ++s)
            for (int ty = 0; ty < nty; ++ty)
                for (int tx = 0; tx < ntx; ++tx) {
                    TileDesc td{};
                    td.x0 = tx * TX;
                    td.y0 = ty * TY;
                    td.plane = s;
                    T.tiles.push_back(td);
                    std::vector<TaskDesc> tl;
                    for (int64_t c = c_begin[s]; c < c_begin[s + 1]; ++c) {
                        const Cluster& cl = P->clusters[c];
                        const int64_t px = static_cast<int64_t>(cl.X) + td.x0;
                        const int64_t py = static_cast<int64_t>(cl.Y) + td.y0;
                        // clipped boundary: a window wholly off the FPA adds nothing
                        if (P->clip && (px >= ga || py >= xi || px + TX + K - 1 <= 0 ||
                                        py + TY + K - 1 <= 0))
                            continue;
                        const int64_t q = floor_mod(-px, P->u_copies);
                        TaskDesc t;
                        t.wx = static_cast<int>(px + q);
                        t.wy = static_cast<int>(py);
                        t.plane = static_cast<int>(q);   // copy index
                        t.cluster = static_cast<int>(c);
                        tl.push_back(t);
                    }
                    T.tile_tasks.insert(T.tile_tasks.end(), tl.begin(), tl.end());
                    begin.push_back(static_cast<int>(T.tile_tasks.size()));
                }
        T.tile_task_begin = std::move(begin);
        schedule(T, warps_adj, P->forced_per_item, P->forced_split_q, P->forced_skew_pm);
    }

    if (P->host_ctas > 0) return CTIS_OK;   // host-only tables

    // ---- device buffers
    for (ProjTables* T : {&P->fwd, &P->adj}) {
        int rc = upload(P, &T->d_tasks, T->tasks);
        if (!rc) rc = upload(P, &T->d_warp_begin, T->warp_begin);
        if (!rc) rc = upload(P, &T->d_heads, T->heads);
        if (!rc) rc = upload(P, &T->d_witems, T->witems);
        if (rc) return rc;
    }
    int rc = write_values(P, true);
    if (!rc) rc = upload(P, &P->d_tap_slot, P->tap_slot);
    if (!rc) rc = upload(P, &P->d_tap_s, P->tap_s);
    if (!rc) rc = dmalloc(P, reinterpret_cast<void**>(&P->d_grad_part),
                          sizeof(float) * static_cast<size_t>(ncl) * P->adj_tiles_per_plane * K * K);
    if (rc) return rc;
    const size_t es = P->dtype == kDtypeBF16 ? 2 : 4;
    P->u_copy_stride = static_cast<int64_t>(P->g_pitch) * xi;
    P->f_copy_stride = static_cast<int64_t>(P->a_pitch) * al * w;
    rc = dmalloc(P, reinterpret_cast<void**>(&P->d_u),
                 sizeof(float) * static_cast<size_t>(P->u_copy_stride) * P->u_copies);
    if (!rc) rc = dmalloc(P, &P->d_fwork, es * static_cast<size_t>(P->f_copy_stride) * P->f_copies);
    const int64_t scratch_elems =
        std::max(P->fwd.scratch_slots * P->fwd.tile_w * P->fwd.tile_h,
                 P->adj.scratch_slots * P->adj.tile_w * P->adj.tile_h);
    if (!rc) rc = dmalloc(P, reinterpret_cast<void**>(&P->d_scratch),
                          sizeof(float) * static_cast<size_t>(scratch_elems));
    P->scratch_capacity = scratch_elems;
    // tickets: one per tile (chunked tiles); statistics: per forward tile
    const size_t ntiles = std::max(P->fwd.tiles.size(), P->adj.tiles.size());
    if (!rc) rc = dmalloc(P, reinterpret_cast<void**>(&P->d_tickets), sizeof(int) * ntiles);
    // counters: [3] the bounded waits' error flag, [8] the frame reduction's ticket
    if (!rc) rc = dmalloc(P, reinterpret_cast<void**>(&P->d_counters), sizeof(int) * 16);
    if (!rc) rc = dmalloc(P, reinterpret_cast<void**>(&P->d_tile_stats),
                          sizeof(double) * kNumStats * P->fwd.tiles.size());
    P->tickets_capacity = ntiles;
    P->tile_stats_capacity = P->fwd.tiles.size();
    if (!rc) rc = dmalloc(P, reinterpret_cast<void**>(&P->d_red_part),
                          sizeof(double) * kNumStats * kStatSlices);
    if (rc) return rc;
    // copies start zeroed: the elements past each copy's shifted end are never
    // written and must read as zero
    CTIS_CUDA(cudaMemset(P->d_u, 0, sizeof(float) * static_cast<size_t>(P->u_copy_stride) * P->u_copies));
    CTIS_CUDA(cudaMemset(P->d_fwork, 0, es * static_cast<size_t>(P->f_copy_stride) * P->f_copies));
    CTIS_CUDA(cudaMemset(P->d_tickets, 0, sizeof(int) * ntiles));
    CTIS_CUDA(cudaMemset(P->d_counters, 0, sizeof(int) * 16));
    CTIS_CUDA(cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking));
    CTIS_CUDA(cudaDeviceSynchronize());
    return CTIS_OK;
}

// The work lists are about to change: drops the cached graphs and the batch
// state built on the old ones (the caller has synchronised the device).
void drop_table_users(ctis_plan* P) {
    if (P->gexec) {
        cudaGraphExecDestroy(P->gexec);
        P->gexec = nullptr;
        P->gkey = GraphKey{};
    }
    drop_batched_graph_of(P);
    free_batch(P->batch);
    P->batch = nullptr;
}

// Replaces the device copies of a projector's work lists after a new
// schedule (and grows the chunk scratch when the schedule needs more).
int reupload_tables(ctis_plan* P, ProjTables& T) {
    cudaFree(T.d_tasks);
    cudaFree(T.d_warp_begin);
    cudaFree(T.d_heads);
    cudaFree(T.d_witems);
    T.d_tasks = nullptr;
    T.d_warp_begin = nullptr;
    T.d_heads = nullptr;
    T.d_witems = nullptr;
    int r = upload(P, &T.d_tasks, T.tasks);
    if (!r) r = upload(P, &T.d_warp_begin, T.warp_begin);
    if (!r) r = upload(P, &T.d_heads, T.heads);
    if (!r) r = upload(P, &T.d_witems, T.witems);
    if (r) return r;
    const int64_t need = T.scratch_slots * T.tile_w * T.tile_h;
    if (need > P->scratch_capacity) {
        cudaFree(P->d_scratch);
        P->d_scratch = nullptr;
        P->scratch_capacity = 0;
        r = dmalloc(P, reinterpret_cast<void**>(&P->d_scratch), sizeof(float) * need);
        if (r) return r;
        P->scratch_capacity = need;
    }
    // the uploads above come from pageable host memory and may still be in
    // flight; the next launch may be on any stream
    CTIS_CUDA(cudaDeviceSynchronize());
    return CTIS_OK;
}

int check_plan(const ctis_plan* P) {
    if (!P) return fail(CTIS_ERR_INVALID_ARG, "plan is NULL");
    int cur = -1;
    CTIS_CUDA(cudaGetDevice(&cur));
    if (cur != P->device)
        return fail(CTIS_ERR_INVALID_ARG, "plan belongs to device %d, current device is %d",
                    P->device, cur);
    return CTIS_OK;
}

// L2 sector promotion of the window maps' loads (a build-time option; the
// default was kept after measuring the others on the realistic workload)
#ifndef CTIS_TMA_L2_PROMOTION
#define CTIS_TMA_L2_PROMOTION CU_TENSOR_MAP_L2_PROMOTION_L2_128B
#endif

int make_map(CUtensorMap* map, const void* base, int dtype, int width, int height, int depth,
             int64_t pitch, int64_t plane, int box_w, int box_h) {
    EncodeFn fn = encode_fn();
    if (!fn) return fail(CTIS_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    const int64_t es = dtype == kDtypeBF16 ? 2 : 4;
    cuuint64_t dims[3] = {(cuuint64_t)width, (cuuint64_t)height, (cuuint64_t)depth};
    cuuint64_t strides[2] = {(cuuint64_t)(pitch * es), (cuuint64_t)(plane * es)};
    cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map,
                          dtype == kDtypeBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                              : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                          3, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CTIS_TMA_L2_PROMOTION, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(CTIS_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for %dx%dx%d box %dx%d",
                    (int)r, width, height, depth, box_w, box_h);
    return CTIS_OK;
}

GatherParams base_params(const ctis_plan* P, const ProjTables& T) {
    GatherParams p{};
    p.items = T.d_witems;
    p.tasks = T.d_tasks;
    p.weights = T.d_weights;
    p.warp_begin = T.d_warp_begin;
    p.heads = T.d_heads;
    p.n_warps = T.n_warps;
    p.n_tiles = static_cast<int>(T.tiles.size());
    p.scratch = P->d_scratch;
    p.tickets = P->d_tickets;
    p.counters = P->d_counters;
    p.tile_stats = P->d_tile_stats;
    p.h = P->d_h;
    p.h_vox = P->d_hvox;
    p.h_vox_planes = P->w;
    p.drop_copies = P->drop_copies;
    p.overlap_launch = P->overlap_launch;
    return p;
}

// Forward pass from the plan's datacube copies.
// The raw forward's output outside the listed tiles (no footprint meets
// them, H f = 0 there) is zeroed before the launch.
int zero_raw_output(const GatherParams& p, cudaStream_t st) {
    CTIS_CUDA(cudaMemset2DAsync(p.out_f32, sizeof(float) * static_cast<size_t>(p.out_pitch), 0,
                                sizeof(float) * static_cast<size_t>(p.out_w),
                                static_cast<size_t>(p.out_h), st));
    return CTIS_OK;
}

int enqueue_forward(const ctis_plan* P, GatherParams p, cudaStream_t st) {
    if (p.mode == kEpiRaw) {
        const int rc = zero_raw_output(p, st);
        if (rc) return rc;
    }
    CUtensorMap win;
    const int64_t plane = static_cast<int64_t>(P->a_pitch) * P->alpha;
    int rc = make_map(&win, P->d_fwork, P->dtype, P->a + P->f_copies - 1, P->alpha,
                      P->w * P->f_copies, P->a_pitch, plane, gather_box_w(true, P->K, P->dtype, P->fwd_shape),
                      gather_window_rows(true, P->K, P->dtype, P->fwd_shape));
    if (rc) return rc;
    CTIS_CUDA(gather_launch(true, P->K, P->dtype, win, p, st, P->fwd_shape));
    return CTIS_OK;
}

// Adjoint pass from the plan's FPA copies.
int enqueue_adjoint(const ctis_plan* P, GatherParams p, cudaStream_t st) {
    CUtensorMap win;
    int rc = make_map(&win, P->d_u, kDtypeF32, P->gamma + P->u_copies - 1, P->xi, P->u_copies,
                      P->g_pitch, P->u_copy_stride, gather_box_w(false, P->K, P->dtype),
                      gather_window_rows(false, P->K, P->dtype));
    if (rc) return rc;
    CTIS_CUDA(gather_launch(false, P->K, P->dtype, win, p, st));
    return CTIS_OK;
}

// Records which SM each CTA of the projector's launch lands on: one launch of
// the EM kernel itself (same resources, so the same placement) in probe mode.
// The map is only a scheduling hint; on any failure it is left empty.
void probe_placement(ctis_plan* P, ProjTables& T, bool forward) {
    T.block_sm.clear();
    const int n = T.n_warps / T.nw;
    int* d = nullptr;
    if (n <= 0 || cudaMalloc(&d, sizeof(int) * n) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    GatherParams p = base_params(P, T);
    p.mode = forward ? kEpiRatio : kEpiUpdate;   // the EM loop's instantiations
    p.smid_out = d;
    const int rc = forward ? enqueue_forward(P, p, nullptr) : enqueue_adjoint(P, p, nullptr);
    std::vector<int> h(n, -1);
    if (rc == CTIS_OK && cudaMemcpy(h.data(), d, sizeof(int) * n, cudaMemcpyDeviceToHost) == cudaSuccess) {
        bool ok = true;
        for (int v : h) ok = ok && v >= 0 && v < 4096;
        if (ok) T.block_sm = std::move(h);
    }
    cudaGetLastError();
    cudaFree(d);
}

// Switches the forward projector to tile shape `shape`: its kernel's launch
// resources, its work lists (same schedule parameters), the tile tickets and
// statistics grown to the new tile count, and its probed placement. The
// caller has synchronised the device and dropped the tables' users.
int set_forward_shape(ctis_plan* P, int shape) {
    P->fwd_shape = shape;
    CTIS_CUDA(gather_prepare(true, P->K, P->dtype, &P->fwd.blocks_per_sm, shape));
    P->fwd.block_sm.clear();
    build_forward_lists(P, P->num_sms * P->fwd.blocks_per_sm * gather_warps_per_cta(true));
    const size_t ntiles = std::max(P->fwd.tiles.size(), P->adj.tiles.size());
    if (ntiles > P->tickets_capacity) {
        cudaFree(P->d_tickets);
        P->d_tickets = nullptr;
        P->tickets_capacity = 0;
        const int rc = dmalloc(P, reinterpret_cast<void**>(&P->d_tickets), sizeof(int) * ntiles);
        if (rc) return rc;
        CTIS_CUDA(cudaMemset(P->d_tickets, 0, sizeof(int) * ntiles));
        P->tickets_capacity = ntiles;
    }
    if (P->fwd.tiles.size() > P->tile_stats_capacity) {
        cudaFree(P->d_tile_stats);
        P->d_tile_stats = nullptr;
        P->tile_stats_capacity = 0;
        const int rc = dmalloc(P, reinterpret_cast<void**>(&P->d_tile_stats),
                               sizeof(double) * kNumStats * P->fwd.tiles.size());
        if (rc) return rc;
        P->tile_stats_capacity = P->fwd.tiles.size();
    }
    int rc = reupload_tables(P, P->fwd);
    if (rc) return rc;
    probe_placement(P, P->fwd, true);
    if (P->fwd.block_sm.empty()) return CTIS_OK;
    schedule(P->fwd, P->fwd.n_warps, P->fwd.per_item, P->fwd.split_q, P->fwd.skew_pm);
    return reupload_tables(P, P->fwd);
}

// Probes both projectors' placements and, when the maps came back, lays the
// work lists out again with them (same schedule parameters) and re-uploads.
int place_by_probe(ctis_plan* P) {
    for (ProjTables* T : {&P->fwd, &P->adj}) {
        probe_placement(P, *T, T == &P->fwd);
        if (T->block_sm.empty()) continue;
        schedule(*T, T->n_warps, T->per_item, T->split_q, T->skew_pm);
        const int rc = reupload_tables(P, *T);
        if (rc) return rc;
    }
    return CTIS_OK;
}

// PSF-value gradient pass: the FPA input r already sits in the plan's FPA
// copies; f_dense is a dense datacube of the plan's dtype. Writes (or adds
// to) dval one value per stored tap, plus extra[s] for taps of wavelength s
// when extra is given.
int enqueue_psf_grad(const ctis_plan* P, const void* f_dense, float* dval, bool accumulate,
                     const double* extra, cudaStream_t st) {
    CUtensorMap win;
    int rc = make_map(&win, P->d_u, kDtypeF32, P->gamma + P->u_copies - 1, P->xi, P->u_copies,
                      P->g_pitch, P->u_copy_stride, gather_box_w(false, P->K, P->dtype),
                      gather_window_rows(false, P->K, P->dtype));
    if (rc) return rc;
    GatherParams p = base_params(P, P->adj);
    p.mode = kEpiGrad;
    p.out_w = P->a;
    p.out_h = P->alpha;
    p.f_in = f_dense;
    p.grad_part = P->d_grad_part;
    p.grad_tiles_per_plane = P->adj_tiles_per_plane;
    CTIS_CUDA(psf_grad_launch(P->K, P->dtype, win, p, st));
    CTIS_CUDA(launch_grad_reduce(dval, P->d_grad_part, P->d_tap_slot, P->d_tap_s, extra,
                                 static_cast<int>(P->tap_v.size()), P->K * P->K,
                                 P->adj_tiles_per_plane, accumulate, st));
    return CTIS_OK;
}

// Fills the datacube copies from a dense caller datacube (src_dtype) or, when
// src is null, with `value`.
int scatter_f(const ctis_plan* P, const void* src, int src_dtype, float value, cudaStream_t st) {
    CTIS_CUDA(launch_scatter_copies(P->dtype, P->d_fwork, P->f_copy_stride, P->f_copies,
                                    P->a_pitch, static_cast<int64_t>(P->a_pitch) * P->alpha, src,
                                    src_dtype, P->a, static_cast<int64_t>(P->a) * P->alpha, P->a,
                                    P->alpha, P->w, value, st));
    return CTIS_OK;
}

// Fills the FPA copies from a dense float32 caller image (value everywhere
// when src is NULL).
int scatter_u(const ctis_plan* P, const float* src, cudaStream_t st, float value = 0.f) {
    CTIS_CUDA(launch_scatter_copies(kDtypeF32, P->d_u, P->u_copy_stride, P->u_copies, P->g_pitch,
                                    P->u_copy_stride, src, kDtypeF32, P->gamma,
                                    static_cast<int64_t>(P->gamma) * P->xi, P->gamma, P->xi, 1,
                                    value, st));
    return CTIS_OK;
}

// Zeroes the FPA copies (the ratio forward leaves the pixels outside every
// footprint untouched; they must read as zero, whatever an earlier call
// scattered there).
int zero_u(const ctis_plan* P, cudaStream_t st) {
    CTIS_CUDA(cudaMemsetAsync(P->d_u, 0,
                              sizeof(float) * static_cast<size_t>(P->u_copy_stride) * P->u_copies, st));
    return CTIS_OK;
}

void set_f_copies(const ctis_plan* P, GatherParams& p) {
    p.f_in = P->d_fwork;
    p.f_out = P->d_fwork;
    p.f_pitch = P->a_pitch;
    p.f_plane_stride = static_cast<int64_t>(P->a_pitch) * P->alpha;
    p.f_copy_stride = P->f_copy_stride;
    p.f_copies = P->f_copies;
}

// Records event `idx` of the plan's pool on `st` (an event-record node when
// the stream is being captured).
int record(ctis_plan* P, int idx, cudaStream_t st) {
    CTIS_CUDA(cudaEventRecordWithFlags(P->events[idx], st, cudaEventRecordExternal));
    return CTIS_OK;
}

// CTIS_BOUNDARY_CLIP: h = H^T 1 per voxel (Eq. 2's normaliser; the light of
// voxels near the field stop's edges partly leaves the FPA), as the adjoint
// of an all-ones FPA image: the copies hold 1 on the FPA and 0 around it.
int compute_hvox(ctis_plan* P, cudaStream_t st) {
    if (!P->clip) return CTIS_OK;
    if (!P->d_hvox) {
        const int rc = dmalloc(P, reinterpret_cast<void**>(&P->d_hvox), sizeof(float) * P->m);
        if (rc) return rc;
    }
    int rc = zero_u(P, st);
    if (!rc) rc = scatter_u(P, nullptr, st, 1.0f);
    if (rc) return rc;
    GatherParams p = base_params(P, P->adj);
    p.mode = kEpiRaw;
    p.out_w = P->a;
    p.out_h = P->alpha;
    p.out_f32 = P->d_hvox;
    p.out_pitch = P->a;
    p.out_plane_stride = static_cast<long long>(P->a) * P->alpha;
    p.h_vox = nullptr;
    rc = enqueue_adjoint(P, p, st);
    if (rc) return rc;
    CTIS_CUDA(cudaStreamSynchronize(st));
    return CTIS_OK;
}

// SART's row sums r = H 1 (per FPA pixel, from the stored values), as the
// forward projection of an all-ones datacube; built once per set of values.
// Synchronous (it uses the plan's datacube copies).
int ensure_rowsum(ctis_plan* P) {
    if (P->rowsum_valid) return CTIS_OK;
    CTIS_CUDA(cudaDeviceSynchronize());   // queued work may still use the copies
    if (!P->d_rowsum) {
        const int rc = dmalloc(P, reinterpret_cast<void**>(&P->d_rowsum), sizeof(float) * P->n);
        if (rc) return rc;
    }
    int rc = scatter_f(P, nullptr, P->dtype, 1.0f, nullptr);
    if (rc) return rc;
    GatherParams p = base_params(P, P->fwd);
    p.mode = kEpiRaw;
    p.out_w = P->gamma;
    p.out_h = P->xi;
    p.out_f32 = P->d_rowsum;
    p.out_pitch = P->gamma;
    p.out_plane_stride = 0;
    rc = enqueue_forward(P, p, nullptr);
    if (rc) return rc;
    CTIS_CUDA(cudaDeviceSynchronize());
    P->rowsum_valid = true;
    return CTIS_OK;
}

// Enqueues the whole reconstruction on `st`: k updates of `solver` (Solver)
// with relaxation `relax` (EM ignores it).
int enqueue_reconstruct(ctis_plan* P, const float* g, void* f, int k, int flags,
                        double* stats, cudaStream_t st, int solver = kSolverEm,
                        float relax = 1.f) {
    int rc = zero_u(P, st);   // the ratio writes u only where H f can be nonzero
    if (rc) return rc;
    if (flags & CTIS_INIT_ONES) {
        rc = scatter_f(P, nullptr, P->dtype, 1.0f, st);
    } else if (flags & CTIS_INIT_HTG) {
        rc = scatter_u(P, g, st);
        if (rc) return rc;
        GatherParams p = base_params(P, P->adj);
        p.mode = kEpiSet;
        p.out_w = P->a;
        p.out_h = P->alpha;
        set_f_copies(P, p);
        rc = enqueue_adjoint(P, p, st);
    } else {
        rc = scatter_f(P, f, P->dtype, 0.f, st);
    }
    if (rc) return rc;
    GatherParams pf = base_params(P, P->fwd);
    pf.mode = kEpiRatio;
    pf.out_w = P->gamma;
    pf.out_h = P->xi;
    pf.out_f32 = P->d_u;
    pf.out_pitch = P->g_pitch;
    pf.out_copy_stride = P->u_copy_stride;
    pf.out_copies = P->u_copies;
    pf.g = g;
    pf.g_pitch = P->gamma;
    pf.solver = solver;
    pf.relax = relax;
    pf.row_sum = P->d_rowsum;
    GatherParams pa = base_params(P, P->adj);
    pa.mode = kEpiUpdate;
    pa.out_w = P->a;
    pa.out_h = P->alpha;
    pa.solver = solver;
    pa.relax = relax;
    set_f_copies(P, pa);
    P->prof_fwd.clear();
    P->prof_adj.clear();
    int ev = 0;
    if (P->profiling) {
        const size_t need = 4 * static_cast<size_t>(k + 1);
        while (P->events.size() < need) {
            cudaEvent_t e;
            CTIS_CUDA(cudaEventCreate(&e));
            P->events.push_back(e);
        }
    }
    auto timed = [&](std::vector<std::pair<int, int>>& log, auto&& body) -> int {
        if (!P->profiling) return body();
        int r = record(P, ev, st);
        if (!r) r = body();
        if (!r) r = record(P, ev + 1, st);
        if (!r) log.emplace_back(ev, ev + 1);
        ev += 2;
        return r;
    };
    pf.with_stats = stats != nullptr;
    const int ftiles = static_cast<int>(P->fwd.tiles.size());
    for (int it = 0; it <= k; ++it) {
        if (it == k && !stats) break;
        rc = timed(P->prof_fwd, [&] { return enqueue_forward(P, pf, st); });
        if (rc) return rc;
        if (it == k) break;
        if (stats) {   // the adjoint adds this forward's tile statistics first
            pa.red_src = P->d_tile_stats;
            pa.red_out = stats + static_cast<int64_t>(it) * kNumStats;
            pa.red_tiles_per_frame = ftiles;
            pa.red_frames = 1;
            pa.red_part = P->d_red_part;
            pa.red_tickets = P->d_counters + 8;
        }
        rc = timed(P->prof_adj, [&] { return enqueue_adjoint(P, pa, st); });
        if (rc) return rc;
    }
    if (stats)
        CTIS_CUDA(launch_stats_reduce(stats + static_cast<int64_t>(k) * kNumStats, P->d_tile_stats,
                                      ftiles, 1, 0, P->d_red_part, P->d_counters + 8, st));
    CTIS_CUDA(launch_gather_copy0(P->dtype, f, P->d_fwork, P->a_pitch,
                                  static_cast<int64_t>(P->a_pitch) * P->alpha, P->a, P->alpha,
                                  P->w, st));
    return CTIS_OK;
}

// ---------------------------------------------------------------------------
// batches of frames (ctis_reconstruct_batched)
// ---------------------------------------------------------------------------
// F frames of one plan's geometry run as F more copies of its work lists, so
// one launch per projector covers them all: every warp keeps its item list
// and runs it once per frame. Frame f's datacube planes are planes f*w + s of
// the copies, its FPA image in FPA copy q is plane q*F + f of the adjoint's
// window map (so a window past the FPA's first or last row reads zeros, not
// a neighbouring frame), and its tiles are tiles f*T + t, each frame with its
// own partial-sum slots and statistics.
struct BatchTables {
    WorkItem* d_witems = nullptr;
    TaskDesc* d_tasks = nullptr;
    int* d_warp_begin = nullptr;
    WarpHead* d_heads = nullptr;
    int n_warps = 0;
    int n_tiles = 0;
    int64_t scratch_slots = 0;   // chunk partial-sum slots of the joint schedule
};

struct BatchState {
    int F = 0;
    BatchTables fwd, adj;
    void* d_fwork = nullptr;       // datacube copies, planes f*w + s
    float* d_u = nullptr;          // FPA copies: copy q of frame f at (q*F + f) * xi rows
    float* d_scratch = nullptr;
    int* d_tickets = nullptr;
    int* d_counters = nullptr;     // [3] error flag, [8 + f] frame f's reduction ticket
    double* d_tile_stats = nullptr;
    double* d_red_part = nullptr;  // [F][kStatSlices][kNumStats]
    float* d_h = nullptr;          // h for every plane f*w + s
    float* d_g = nullptr;          // the frames' g, contiguous
    void** d_ptrs = nullptr;       // [F] g pointers, [F] f pointers
    int* d_gid = nullptr;          // [F] position of each frame in the caller's order
    double* d_stats = nullptr;     // [F][k+1][4]
    int stats_rows = 0;
    int64_t f_copy_stride = 0, u_copy_stride = 0;
};

void free_tables(BatchTables& t) {
    cudaFree(t.d_witems);
    cudaFree(t.d_tasks);
    cudaFree(t.d_warp_begin);
    cudaFree(t.d_heads);
    t = BatchTables{};
}

void free_batch(BatchState* B) {
    if (!B) return;
    free_tables(B->fwd);
    free_tables(B->adj);
    cudaFree(B->d_fwork);
    cudaFree(B->d_u);
    cudaFree(B->d_scratch);
    cudaFree(B->d_tickets);
    cudaFree(B->d_counters);
    cudaFree(B->d_tile_stats);
    cudaFree(B->d_red_part);
    cudaFree(B->d_h);
    cudaFree(B->d_g);
    cudaFree(B->d_ptrs);
    cudaFree(B->d_gid);
    cudaFree(B->d_stats);
    delete B;
}

// The work lists of F frames, scheduled as one problem. The joint tiles are
// frame f's tiles f*T + t (so tickets and tile statistics stay frame-major),
// their tasks the plan's with frame f's planes (forward: datacube planes
// f*w + s of the copies; adjoint: FPA planes q*F + f of copy q),
// and the joint items are the plan's items (same tiles, chunks and task
// ranges) of every frame, assigned longest first over the CTAs with the
// plan's priority skew and CTA-to-SM map. Each tile is therefore summed
// exactly as in a single-frame call (bit-identical results), while small
// frames no longer give every warp a few tasks per frame.
int replicate(ctis_plan* P, const ProjTables& T, bool forward, int F, BatchTables& B) {
    ProjTables J;
    J.nw = T.nw;
    J.tile_w = T.tile_w;
    J.tile_h = T.tile_h;
    J.block_sm = T.block_sm;
    J.n_warps = T.n_warps;
    const int ntiles = static_cast<int>(T.tiles.size());
    const int64_t ntasks = static_cast<int64_t>(T.tile_tasks.size());
    if (ntasks * F > (int64_t{1} << 31) - 1 || static_cast<int64_t>(ntiles) * F > (int64_t{1} << 30))
        return fail(CTIS_ERR_UNSUPPORTED, "too many frames for one batch");
    J.tiles.reserve(static_cast<size_t>(ntiles) * F);
    J.tile_tasks.reserve(static_cast<size_t>(ntasks) * F);
    J.tile_task_begin.assign(1, 0);
    for (int f = 0; f < F; ++f)
        for (int t = 0; t < ntiles; ++t) {
            TileDesc td = T.tiles[t];
            td.plane = forward ? f : f * P->w + td.plane;
            if (td.nchunks > 1) td.scratch_base += static_cast<int>(f * T.scratch_slots);
            J.tiles.push_back(td);
            for (int k = T.tile_task_begin[t]; k < T.tile_task_begin[t + 1]; ++k) {
                TaskDesc d = T.tile_tasks[k];
                if (forward) {   // copies' plane q*w + s -> q*(F*w) + f*w + s
                    const int q = d.plane / P->w, sw = d.plane % P->w;
                    d.plane = q * (F * P->w) + f * P->w + sw;
                } else {         // copy q's plane -> plane q*F + f of the frames' FPAs
                    d.plane = d.plane * F + f;
                }
                J.tile_tasks.push_back(d);
            }
            J.tile_task_begin.push_back(static_cast<int>(J.tile_tasks.size()));
        }
    J.items.reserve(T.items.size() * F);
    for (int f = 0; f < F; ++f)
        for (const ItemDesc& it : T.items) {
            ItemDesc j = it;
            j.tile = f * ntiles + it.tile;
            j.task_begin = static_cast<int>(it.task_begin + f * ntasks);
            j.task_end = static_cast<int>(it.task_end + f * ntasks);
            J.items.push_back(j);
        }
    J.scratch_slots = T.scratch_slots * F;
    assign_ctas(J, J.n_warps / J.nw, T.skew_pm);
    // each CTA runs its items frame by frame, so the CTAs move through the
    // frames together and the frames in flight stay in L2
    for (size_t c = 0; c + 1 < J.cta_begin.size(); ++c)
        std::stable_sort(J.cta_items.begin() + J.cta_begin[c], J.cta_items.begin() + J.cta_begin[c + 1],
                         [&](int x, int y) { return J.items[x].tile / ntiles < J.items[y].tile / ntiles; });
    layout_warps(J);
    B.n_warps = J.n_warps;
    B.n_tiles = ntiles * F;
    B.scratch_slots = J.scratch_slots;
    int rc = upload(P, &B.d_witems, J.witems);
    if (!rc) rc = upload(P, &B.d_tasks, J.tasks);
    if (!rc) rc = upload(P, &B.d_warp_begin, J.warp_begin);
    if (!rc) rc = upload(P, &B.d_heads, J.heads);
    return rc;
}

// Makes P->batch hold exactly F frames (and statistics rows for k).
int ensure_batch(ctis_plan* P, int F, int k) {
    BatchState* B = P->batch;
    if (B && B->F == F) {
        if (B->stats_rows < k + 1) {
            cudaFree(B->d_stats);
            B->d_stats = nullptr;
            B->stats_rows = 0;
            int rc = dmalloc(P, reinterpret_cast<void**>(&B->d_stats),
                             sizeof(double) * kNumStats * static_cast<size_t>(F) * (k + 1));
            if (rc) return rc;
            B->stats_rows = k + 1;
        }
        return CTIS_OK;
    }
    CTIS_CUDA(cudaDeviceSynchronize());
    drop_batched_graph_of(P);
    free_batch(P->batch);
    P->batch = nullptr;
    B = new (std::nothrow) BatchState();
    if (!B) return fail(CTIS_ERR_NOMEM, "host allocation failed");
    P->batch = B;
    B->F = F;
    int rc = replicate(P, P->fwd, true, F, B->fwd);
    if (!rc) rc = replicate(P, P->adj, false, F, B->adj);
    if (rc) return rc;
    const size_t es = P->dtype == kDtypeBF16 ? 2 : 4;
    B->f_copy_stride = static_cast<int64_t>(P->a_pitch) * P->alpha * P->w * F;
    B->u_copy_stride = static_cast<int64_t>(P->g_pitch) * P->xi * F;
    const size_t fbytes = es * static_cast<size_t>(B->f_copy_stride) * P->f_copies;
    const size_t ubytes = sizeof(float) * static_cast<size_t>(B->u_copy_stride) * P->u_copies;
    const int64_t scratch = std::max(B->fwd.scratch_slots * P->fwd.tile_w * P->fwd.tile_h,
                                     B->adj.scratch_slots * P->adj.tile_w * P->adj.tile_h);
    const size_t tpf = P->fwd.tiles.size();
    const size_t ntick = std::max(tpf * F, P->adj.tiles.size() * F);
    rc = dmalloc(P, &B->d_fwork, fbytes);
    if (!rc) rc = dmalloc(P, reinterpret_cast<void**>(&B->d_u), ubytes);
    if (!rc) rc = dmalloc(P, reinterpret_cast<void**>(&B->d_scratch),
                          sizeof(float) * static_cast<size_t>(scratch));
    if (!rc) rc = dmalloc(P, reinterpret_cast<void**>(&B->d_tickets), sizeof(int) * ntick);
    if (!rc) rc = dmalloc(P, reinterpret_cast<void**>(&B->d_counters), sizeof(int) * (8 + F));
    if (!rc) rc = dmalloc(P, reinterpret_cast<void**>(&B->d_tile_stats),
                          sizeof(double) * kNumStats * tpf * F);
    if (!rc) rc = dmalloc(P, reinterpret_cast<void**>(&B->d_red_part),
                          sizeof(double) * kNumStats * kStatSlices * F);
    if (!rc) rc = dmalloc(P, reinterpret_cast<void**>(&B->d_h), sizeof(float) * P->w * F);
    if (!rc) rc = dmalloc(P, reinterpret_cast<void**>(&B->d_g), sizeof(float) * P->n * F);
    if (!rc) rc = dmalloc(P, reinterpret_cast<void**>(&B->d_ptrs), sizeof(void*) * 2 * F);
    if (!rc) rc = dmalloc(P, reinterpret_cast<void**>(&B->d_gid), sizeof(int) * F);
    if (!rc) rc = dmalloc(P, reinterpret_cast<void**>(&B->d_stats),
                          sizeof(double) * kNumStats * static_cast<size_t>(F) * (k + 1));
    if (rc) return rc;
    B->stats_rows = k + 1;
    CTIS_CUDA(cudaMemset(B->d_fwork, 0, fbytes));
    CTIS_CUDA(cudaMemset(B->d_u, 0, ubytes));
    CTIS_CUDA(cudaMemset(B->d_tickets, 0, sizeof(int) * ntick));
    CTIS_CUDA(cudaMemset(B->d_counters, 0, sizeof(int) * (8 + F)));
    std::vector<float> hx(static_cast<size_t>(P->w) * F);
    for (int f = 0; f < F; ++f) std::copy(P->h.begin(), P->h.end(), hx.begin() + f * P->w);
    CTIS_CUDA(cudaMemcpy(B->d_h, hx.data(), sizeof(float) * hx.size(), cudaMemcpyHostToDevice));
    // the tables and h come from pageable host memory (copies that may still
    // be in flight when cudaMemcpy returns); the batch runs on any stream
    CTIS_CUDA(cudaDeviceSynchronize());
    return CTIS_OK;
}

GatherParams batch_params(const ctis_plan* P, const BatchState* B, bool forward) {
    const ProjTables& T = forward ? P->fwd : P->adj;
    const BatchTables& BT = forward ? B->fwd : B->adj;
    GatherParams p{};
    p.items = BT.d_witems;
    p.warp_begin = BT.d_warp_begin;
    p.heads = BT.d_heads;
    p.tasks = BT.d_tasks;
    p.weights = T.d_weights;
    p.n_warps = BT.n_warps;
    p.n_tiles = BT.n_tiles;
    p.scratch = B->d_scratch;
    p.tickets = B->d_tickets;
    p.counters = B->d_counters;
    p.tile_stats = B->d_tile_stats;
    p.h = B->d_h;
    p.h_vox = P->d_hvox;
    p.h_vox_planes = P->w;
    p.drop_copies = P->drop_copies;
    p.overlap_launch = P->overlap_launch;
    return p;
}

int batch_forward(const ctis_plan* P, const BatchState* B, GatherParams p, cudaStream_t st) {
    CUtensorMap win;
    const int64_t plane = static_cast<int64_t>(P->a_pitch) * P->alpha;
    int rc = make_map(&win, B->d_fwork, P->dtype, P->a + P->f_copies - 1, P->alpha,
                      P->w * B->F * P->f_copies, P->a_pitch, plane,
                      gather_box_w(true, P->K, P->dtype, P->fwd_shape), gather_window_rows(true, P->K, P->dtype, P->fwd_shape));
    if (rc) return rc;
    CTIS_CUDA(gather_launch(true, P->K, P->dtype, win, p, st, P->fwd_shape));
    return CTIS_OK;
}

int batch_adjoint(const ctis_plan* P, const BatchState* B, GatherParams p, cudaStream_t st) {
    CUtensorMap win;
    // copy q of frame f starts at (q*F + f) * xi * g_pitch (u_copy_stride = F * xi * g_pitch)
    int rc = make_map(&win, B->d_u, kDtypeF32, P->gamma + P->u_copies - 1, P->xi,
                      P->u_copies * B->F, P->g_pitch, static_cast<int64_t>(P->g_pitch) * P->xi,
                      gather_box_w(false, P->K, P->dtype), gather_window_rows(false, P->K, P->dtype));
    if (rc) return rc;
    CTIS_CUDA(gather_launch(false, P->K, P->dtype, win, p, st));
    return CTIS_OK;
}

// One plan's part of a batched reconstruction, as separate phases so that the
// caller can interleave the plans: setup (g, initial f), iteration it, finish.
struct BatchRun {
    ctis_plan* P;
    BatchState* B;
    GatherParams pf, pa;
    bool stats;
    int solver = kSolverEm;
    float relax = 1.f;
};

int batch_setup(BatchRun& r, int flags, cudaStream_t st) {
    ctis_plan* P = r.P;
    BatchState* B = r.B;
    const int F = B->F;
    const float* const* gptrs = reinterpret_cast<const float* const*>(B->d_ptrs);
    void* const* fptrs = B->d_ptrs + F;
    CTIS_CUDA(launch_frames_gather(B->d_g, gptrs, P->n, F, st));
    const int64_t fplane = static_cast<int64_t>(P->a_pitch) * P->alpha;
    if (flags & CTIS_INIT_HTG) {
        // the frames' g into the tall FPA copies, then f = H^T g per frame
        CTIS_CUDA(launch_scatter_copies(kDtypeF32, B->d_u, B->u_copy_stride, P->u_copies,
                                        P->g_pitch, static_cast<int64_t>(P->g_pitch) * P->xi,
                                        B->d_g, kDtypeF32, P->gamma, P->n, P->gamma, P->xi, F,
                                        0.f, st));
        GatherParams p = batch_params(P, B, false);
        p.mode = kEpiSet;
        p.out_w = P->a;
        p.out_h = P->alpha;
        p.f_in = B->d_fwork;
        p.f_out = B->d_fwork;
        p.f_pitch = P->a_pitch;
        p.f_plane_stride = fplane;
        p.f_copy_stride = B->f_copy_stride;
        p.f_copies = P->f_copies;
        int rc = batch_adjoint(P, B, p, st);
        if (rc) return rc;
    } else {
        CTIS_CUDA(launch_frames_scatter_copies(
            P->dtype, B->d_fwork, B->f_copy_stride, P->f_copies, P->a_pitch, fplane,
            (flags & CTIS_INIT_ONES) ? nullptr : const_cast<const void* const*>(fptrs), 1.0f,
            P->a, P->alpha, P->w, F, st));
    }
    GatherParams& pf = r.pf;
    pf = batch_params(P, B, true);
    pf.mode = kEpiRatio;
    pf.out_w = P->gamma;
    pf.out_h = P->xi;
    pf.out_f32 = B->d_u;
    pf.out_pitch = P->g_pitch;
    pf.out_plane_stride = static_cast<long long>(P->g_pitch) * P->xi;   // between frames
    pf.out_copy_stride = B->u_copy_stride;
    pf.out_copies = P->u_copies;
    pf.g = B->d_g;
    pf.g_pitch = P->gamma;
    pf.g_plane_stride = P->n;
    GatherParams& pa = r.pa;
    pa = batch_params(P, B, false);
    pa.mode = kEpiUpdate;
    pa.out_w = P->a;
    pa.out_h = P->alpha;
    pa.f_in = B->d_fwork;
    pa.f_out = B->d_fwork;
    pa.f_pitch = P->a_pitch;
    pa.f_plane_stride = fplane;
    pa.f_copy_stride = B->f_copy_stride;
    pa.f_copies = P->f_copies;
    pf.solver = pa.solver = r.solver;   // the rules of ctis_reconstruct_solver
    pf.relax = pa.relax = r.relax;
    pf.row_sum = P->d_rowsum;           // per pixel, the same for every frame
    return CTIS_OK;
}

int batch_forward_step(BatchRun& r, cudaStream_t st) {
    GatherParams p = r.pf;
    p.with_stats = r.stats ? 1 : 0;
    return batch_forward(r.P, r.B, p, st);
}

// The adjoint of iteration it; it first adds the frames' statistics of that
// iteration's forward (one warp per frame; a separate launch when the batch
// has more frames than the adjoint has warps).
int batch_adjoint_step(BatchRun& r, int it, int k, cudaStream_t st) {
    GatherParams p = r.pa;
    const int tiles = static_cast<int>(r.P->fwd.tiles.size());
    double* out = r.B->d_stats + static_cast<int64_t>(it) * kNumStats;
    const long long stride = static_cast<long long>(k + 1) * kNumStats;
    if (r.stats && static_cast<int64_t>(r.B->F) * kStatSlices <= p.n_warps) {
        p.red_src = r.B->d_tile_stats;
        p.red_out = out;
        p.red_tiles_per_frame = tiles;
        p.red_frames = r.B->F;
        p.red_frame_stride = stride;
        p.red_part = r.B->d_red_part;
        p.red_tickets = r.B->d_counters + 8;
    } else if (r.stats) {
        CTIS_CUDA(launch_stats_reduce(out, r.B->d_tile_stats, tiles, r.B->F, stride,
                                      r.B->d_red_part, r.B->d_counters + 8, st));
    }
    return batch_adjoint(r.P, r.B, p, st);
}

int batch_finish(BatchRun& r, int k, double* stats_dev, cudaStream_t st) {
    ctis_plan* P = r.P;
    BatchState* B = r.B;
    CTIS_CUDA(launch_frames_copy0_out(P->dtype, B->d_ptrs + B->F, B->d_fwork, P->a_pitch,
                                      static_cast<int64_t>(P->a_pitch) * P->alpha, P->a, P->alpha,
                                      P->w, B->F, st));
    if (r.stats) {   // the last forward's statistics, then every frame's rows to the caller
        CTIS_CUDA(launch_stats_reduce(B->d_stats + static_cast<int64_t>(k) * kNumStats,
                                      B->d_tile_stats, static_cast<int>(P->fwd.tiles.size()), B->F,
                                      static_cast<long long>(k + 1) * kNumStats, B->d_red_part,
                                      B->d_counters + 8, st));
        CTIS_CUDA(launch_rows_scatter(stats_dev, B->d_stats, B->d_gid, (k + 1) * kNumStats, B->F, st));
    }
    return CTIS_OK;
}

// The cached graph of the last batched call (one entry, keyed by every input).
struct BatchedKey {
    std::vector<const ctis_plan*> plans;
    std::vector<int> plan_idx;
    std::vector<const void*> g, f;
    int k = -1, flags = 0, solver = 0;
    float relax = 1.f;
    const void* stats = nullptr;
    bool operator==(const BatchedKey& o) const {
        return plans == o.plans && plan_idx == o.plan_idx && g == o.g && f == o.f && k == o.k &&
               flags == o.flags && solver == o.solver && relax == o.relax && stats == o.stats;
    }
};
std::mutex g_batched_mu;
BatchedKey g_batched_key;
cudaGraphExec_t g_batched_exec = nullptr;
cudaStream_t g_batched_stream = nullptr;
int g_batched_device = -1;

void drop_batched_graph_of(const ctis_plan* P) {
    std::lock_guard<std::mutex> lock(g_batched_mu);
    if (!g_batched_exec) return;
    for (const ctis_plan* q : g_batched_key.plans)
        if (q == P) {
            cudaGraphExecDestroy(g_batched_exec);
            g_batched_exec = nullptr;
            g_batched_key = BatchedKey{};
            return;
        }
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* ctis_status_string(int status) {
    switch (status) {
        case CTIS_OK: return "CTIS_OK";
        case CTIS_ERR_INVALID_ARG: return "CTIS_ERR_INVALID_ARG";
        case CTIS_ERR_OUT_OF_BOUNDS: return "CTIS_ERR_OUT_OF_BOUNDS";
        case CTIS_ERR_NOMEM: return "CTIS_ERR_NOMEM";
        case CTIS_ERR_CUDA: return "CTIS_ERR_CUDA";
        case CTIS_ERR_TIMEOUT: return "CTIS_ERR_TIMEOUT";
        case CTIS_ERR_UNSUPPORTED: return "CTIS_ERR_UNSUPPORTED";
        default: return "CTIS_ERR_UNKNOWN";
    }
}

const char* ctis_last_error(void) { return g_last_error.c_str(); }

int ctis_plan_create(ctis_plan** out, int a, int alpha, int w, int gamma, int xi,
                     const int32_t* psf_ptr, const int32_t* psf_x, const int32_t* psf_y,
                     const float* psf_val, int dtype) {
    return ctis_plan_create_ex(out, a, alpha, w, gamma, xi, psf_ptr, psf_x, psf_y, psf_val,
                               dtype, nullptr);
}

}  // extern "C"

namespace {

// Validates the arguments of a plan and allocates it (host fields only).
int new_plan(ctis_plan** out, int a, int alpha, int w, int gamma, int xi, const int32_t* psf_ptr,
             const int32_t* psf_x, const int32_t* psf_y, const float* psf_val, int dtype,
             const ctis_plan_options* opt) {
    if (!out) return fail(CTIS_ERR_INVALID_ARG, "out is NULL");
    int forced_per_item = 0, forced_split_q = 0, forced_skew_pm = 0, boundary = 0;
    int forward_tile = CTIS_TILE_32X32;
    if (opt) {
        if (opt->struct_size != static_cast<int>(sizeof(ctis_plan_options)))
            return fail(CTIS_ERR_INVALID_ARG, "ctis_plan_options.struct_size mismatch");
        for (int r : opt->reserved)
            if (r != 0) return fail(CTIS_ERR_INVALID_ARG, "reserved option fields must be 0");
        if (opt->tasks_per_item < 0 || opt->tasks_per_item > 1 << 20)
            return fail(CTIS_ERR_INVALID_ARG, "tasks_per_item out of range");
        if (opt->item_overhead_q < 0 || opt->item_overhead_q > 1 << 16)
            return fail(CTIS_ERR_INVALID_ARG, "item_overhead_q out of range");
        if (opt->tasks_per_item > 0 && opt->item_overhead_q > 0)
            return fail(CTIS_ERR_INVALID_ARG, "tasks_per_item and item_overhead_q are exclusive");
        if (opt->cta_skew_permille < 0 || opt->cta_skew_permille > 900)
            return fail(CTIS_ERR_INVALID_ARG, "cta_skew_permille out of range [0, 900]");
        if (opt->boundary != CTIS_BOUNDARY_REJECT && opt->boundary != CTIS_BOUNDARY_CLIP &&
            opt->boundary != CTIS_BOUNDARY_WRAP)
            return fail(CTIS_ERR_INVALID_ARG,
                        "boundary must be CTIS_BOUNDARY_REJECT, _CLIP or _WRAP");
        if (opt->forward_tile != CTIS_TILE_32X32 && opt->forward_tile != CTIS_TILE_32X16)
            return fail(CTIS_ERR_INVALID_ARG, "forward_tile must be CTIS_TILE_32X32 or CTIS_TILE_32X16");
        forward_tile = opt->forward_tile;
        boundary = opt->boundary;
        forced_per_item = opt->tasks_per_item;
        forced_split_q = opt->item_overhead_q;
        forced_skew_pm = opt->cta_skew_permille;
    }
    *out = nullptr;
    if (a < 1 || alpha < 1 || w < 1 || gamma < 1 || xi < 1)
        return fail(CTIS_ERR_INVALID_ARG, "sizes must be >= 1 (a=%d alpha=%d w=%d gamma=%d xi=%d)",
                    a, alpha, w, gamma, xi);
    if (a > gamma || alpha > xi)
        return fail(CTIS_ERR_OUT_OF_BOUNDS, "field stop %dx%d larger than FPA %dx%d", a, alpha,
                    gamma, xi);
    if ((int64_t)gamma * xi > (int64_t)1 << 31 || (int64_t)a * alpha * w > (int64_t)1 << 31)
        return fail(CTIS_ERR_UNSUPPORTED, "problem larger than 2^31 elements");
    if (dtype != CTIS_F32 && dtype != CTIS_BF16)
        return fail(CTIS_ERR_INVALID_ARG, "dtype must be CTIS_F32 or CTIS_BF16");
    if (!psf_ptr) return fail(CTIS_ERR_INVALID_ARG, "psf_ptr is NULL");
    if (psf_ptr[0] != 0) return fail(CTIS_ERR_INVALID_ARG, "psf_ptr[0] must be 0");
    for (int s = 0; s < w; ++s)
        if (psf_ptr[s + 1] < psf_ptr[s])
            return fail(CTIS_ERR_INVALID_ARG, "psf_ptr must be non-decreasing (at %d)", s);
    if (psf_ptr[w] > 0 && (!psf_x || !psf_y || !psf_val))
        return fail(CTIS_ERR_INVALID_ARG, "PSF arrays are NULL");
    // (the wrap reading stores up to four entries per nonzero)
    if ((int64_t)psf_ptr[w] * (boundary == CTIS_BOUNDARY_WRAP ? 32 : 8) > (int64_t)1 << 31)
        return fail(CTIS_ERR_UNSUPPORTED, "too many PSF nonzeros");
    {
        const int rc = validate_psf(a, alpha, w, gamma, xi, psf_ptr, psf_x, psf_y, psf_val,
                                    boundary);
        if (rc) return rc;
    }

    ctis_plan* P = new (std::nothrow) ctis_plan();
    if (!P) return fail(CTIS_ERR_NOMEM, "host allocation failed");
    P->a = a;
    P->alpha = alpha;
    P->w = w;
    P->gamma = gamma;
    P->xi = xi;
    P->dtype = dtype;
    P->m = (int64_t)a * alpha * w;
    P->n = (int64_t)gamma * xi;
    P->f_copies = gather_input_copies(true, dtype);
    P->u_copies = gather_input_copies(false, dtype);
    P->forced_per_item = forced_per_item;
    P->forced_split_q = forced_split_q;
    P->forced_skew_pm = forced_skew_pm;
    P->clip = boundary != CTIS_BOUNDARY_REJECT;
    P->wrap = boundary == CTIS_BOUNDARY_WRAP;
    P->fwd_shape = forward_tile;
    // copies are NC - 1 elements wider than the plane (see TaskDesc)
    // (a multiple of 16 bytes: the window map's row stride)
    P->a_pitch = static_cast<int>(round_up(a + P->f_copies - 1, dtype == CTIS_BF16 ? 8 : 4));
    P->g_pitch = static_cast<int>(round_up(gamma + P->u_copies - 1, 4));
    *out = P;
    return CTIS_OK;
}

// The PSF the plan stores: the caller's, or under the wrap reading the
// caller's together with, for each nonzero (x, y), its images at
// (x - gamma, y + 1), (x, y - xi) and (x - gamma, y + 1 - xi) whose shifted
// copies can meet the FPA. A shifted copy (x + p, y + r), p < a <= gamma,
// r < alpha <= xi, of a nonzero on the FPA has row index
// (x + p + gamma (y + r)) mod n (Eq. 7); when it leaves the FPA it re-enters
// at exactly one image's shifted copy, so the clip reading of this PSF is the
// wrap reading of the caller's.
struct StoredPsf {
    std::vector<int32_t> ptr, x, y;
    std::vector<float> v;
};

StoredPsf wrap_images(const ctis_plan* P, const int32_t* psf_ptr, const int32_t* psf_x,
                      const int32_t* psf_y, const float* psf_val) {
    const int ga = P->gamma, xi = P->xi;
    StoredPsf out;
    out.ptr.assign(1, 0);
    for (int s = 0; s < P->w; ++s) {
        for (int64_t k = psf_ptr[s]; k < psf_ptr[s + 1]; ++k) {
            const int x = psf_x[k], y = psf_y[k];
            const bool past_x = x + P->a - 1 >= ga;       // some copy passes the right edge
            const bool past_y = y + P->alpha - 1 >= xi;   // some copy passes the last row
            auto add = [&](int xx, int yy) {
                out.x.push_back(xx);
                out.y.push_back(yy);
                out.v.push_back(psf_val[k]);
            };
            add(x, y);
            if (past_x && y + 1 < xi) add(x - ga, y + 1);
            if (past_y) add(x, y - xi);
            // copies past the right edge of the last row re-enter at the top
            if (past_x && y + P->alpha >= xi) add(x - ga, y + 1 - xi);
        }
        out.ptr.push_back(static_cast<int32_t>(out.x.size()));
    }
    return out;
}

}  // namespace

extern "C" {

int ctis_plan_create_ex(ctis_plan** out, int a, int alpha, int w, int gamma, int xi,
                        const int32_t* psf_ptr, const int32_t* psf_x, const int32_t* psf_y,
                        const float* psf_val, int dtype, const ctis_plan_options* opt) {
    if (!out) return fail(CTIS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    ctis_plan* P = nullptr;
    const int rc0 = new_plan(&P, a, alpha, w, gamma, xi, psf_ptr, psf_x, psf_y, psf_val, dtype, opt);
    if (rc0) return rc0;
    cudaError_t e = cudaGetDevice(&P->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device);
    if (e != cudaSuccess) {
        delete P;
        return cuda_fail(e, "no usable CUDA device");
    }
    StoredPsf images;
    if (P->wrap) {
        images = wrap_images(P, psf_ptr, psf_x, psf_y, psf_val);
        psf_ptr = images.ptr.data();
        psf_x = images.x.data();
        psf_y = images.y.data();
        psf_val = images.v.data();
    }
    int rc = build(P, psf_ptr, psf_x, psf_y, psf_val);
    if (!rc) rc = place_by_probe(P);
    if (!rc) rc = compute_hvox(P, nullptr);
    if (!rc) {
        const cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = cuda_fail(e, "placing the work lists");
    }
    if (rc) {
        destroy(P);
        return rc;
    }
    *out = P;
    return CTIS_OK;
}

int ctis_tables_inspect(int a, int alpha, int w, int gamma, int xi, const int32_t* psf_ptr,
                        const int32_t* psf_x, const int32_t* psf_y, const float* psf_val, int dtype,
                        const ctis_plan_options* opt, int forward, int n_ctas,
                        const int32_t* block_sm, ctis_tables_info* info, int32_t* clusters,
                        int32_t* tile_xyp, int32_t* tile_task_ptr, int32_t* task_cluster,
                        int32_t* warp_begin, int32_t* item_tile, int32_t* item_chunk,
                        int32_t* item_range) {
    if (!info || info->struct_size != static_cast<int>(sizeof(ctis_tables_info)))
        return fail(CTIS_ERR_INVALID_ARG, "info is NULL or its struct_size mismatches");
    if (n_ctas < 1 || n_ctas > 1 << 16) return fail(CTIS_ERR_INVALID_ARG, "n_ctas out of range");
    if (block_sm)
        for (int b = 0; b < n_ctas; ++b)
            if (block_sm[b] < 0 || block_sm[b] >= 4096)
                return fail(CTIS_ERR_INVALID_ARG, "block_sm[%d] = %d out of range", b, block_sm[b]);
    ctis_plan* P = nullptr;
    int rc = new_plan(&P, a, alpha, w, gamma, xi, psf_ptr, psf_x, psf_y, psf_val, dtype, opt);
    if (rc) return rc;
    P->host_ctas = n_ctas;
    if (block_sm) {
        (forward ? P->fwd : P->adj).block_sm.assign(block_sm, block_sm + n_ctas);
    }
    StoredPsf images;
    if (P->wrap) {
        images = wrap_images(P, psf_ptr, psf_x, psf_y, psf_val);
        psf_ptr = images.ptr.data();
        psf_x = images.x.data();
        psf_y = images.y.data();
        psf_val = images.v.data();
    }
    rc = build(P, psf_ptr, psf_x, psf_y, psf_val);
    if (rc) {
        delete P;   // host-only: nothing on the device
        return rc;
    }
    const ProjTables& T = forward ? P->fwd : P->adj;
    info->clusters = static_cast<int64_t>(P->clusters.size());
    info->cluster_k = P->K;
    info->tiles = static_cast<int64_t>(T.tiles.size());
    info->tasks = static_cast<int64_t>(T.tile_tasks.size());
    info->witems = static_cast<int64_t>(T.witems.size());
    info->warps = T.n_warps;
    info->warps_per_cta = T.nw;
    info->tile_w = T.tile_w;
    info->tile_h = T.tile_h;
    info->chunk = T.per_item;
    info->split_q = T.split_q;
    info->skew_pm = T.skew_pm;
    info->load_milli = static_cast<int64_t>(T.max_warp_load * 1000.0);
    if (clusters)
        for (size_t c = 0; c < P->clusters.size(); ++c) {
            clusters[3 * c] = P->clusters[c].s;
            clusters[3 * c + 1] = P->clusters[c].X;
            clusters[3 * c + 2] = P->clusters[c].Y;
        }
    if (tile_xyp)
        for (size_t t = 0; t < T.tiles.size(); ++t) {
            tile_xyp[3 * t] = T.tiles[t].x0;
            tile_xyp[3 * t + 1] = T.tiles[t].y0;
            tile_xyp[3 * t + 2] = T.tiles[t].plane;
        }
    if (tile_task_ptr) std::copy(T.tile_task_begin.begin(), T.tile_task_begin.end(), tile_task_ptr);
    if (task_cluster)
        for (size_t k = 0; k < T.tile_tasks.size(); ++k) task_cluster[k] = T.tile_tasks[k].cluster;
    if (warp_begin) std::copy(T.warp_begin.begin(), T.warp_begin.end(), warp_begin);
    for (size_t i = 0; i < T.witems.size(); ++i) {
        const WorkItem& wi = T.witems[i];
        if (item_tile) item_tile[i] = wi.tile;
        if (item_chunk) {
            item_chunk[2 * i] = wi.chunk_info >> 16;
            item_chunk[2 * i + 1] = wi.chunk_info & 0xffff;
        }
        if (item_range) {
            item_range[2 * i] = T.witem_src[i].first;
            item_range[2 * i + 1] = T.witem_src[i].second;
        }
    }
    delete P;
    return CTIS_OK;
}

int ctis_plan_destroy(ctis_plan* plan) {
    destroy(plan);
    return CTIS_OK;
}

int ctis_plan_get_info(const ctis_plan* P, ctis_plan_info* info) {
    if (!P || !info) return fail(CTIS_ERR_INVALID_ARG, "NULL argument");
    info->a = P->a;
    info->alpha = P->alpha;
    info->w = P->w;
    info->gamma = P->gamma;
    info->xi = P->xi;
    info->m = P->m;
    info->n = P->n;
    info->nnz = static_cast<int64_t>(P->tap_v.size());
    info->clusters = static_cast<int64_t>(P->clusters.size());
    info->cluster_k = P->K;
    info->fwd_tiles = static_cast<int64_t>(P->fwd.tiles.size());
    info->fwd_tasks = static_cast<int64_t>(P->fwd.tasks.size());
    info->fwd_items = static_cast<int64_t>(P->fwd.items.size());
    info->adj_tiles = static_cast<int64_t>(P->adj.tiles.size());
    info->adj_tasks = static_cast<int64_t>(P->adj.tasks.size());
    info->adj_items = static_cast<int64_t>(P->adj.items.size());
    info->scratch_bytes = P->device_bytes;
    info->dtype = P->dtype;
    info->fwd_warps = P->fwd.n_warps;
    info->adj_warps = P->adj.n_warps;
    info->fwd_chunk = P->fwd.per_item;
    info->adj_chunk = P->adj.per_item;
    info->fwd_load_milli = static_cast<int64_t>(P->fwd.max_warp_load * 1000.0);
    info->adj_load_milli = static_cast<int64_t>(P->adj.max_warp_load * 1000.0);
    info->fwd_split_q = P->fwd.split_q;
    info->adj_split_q = P->adj.split_q;
    info->fwd_skew_pm = P->fwd.skew_pm;
    info->adj_skew_pm = P->adj.skew_pm;
    info->boundary = P->wrap ? CTIS_BOUNDARY_WRAP
                             : (P->clip ? CTIS_BOUNDARY_CLIP : CTIS_BOUNDARY_REJECT);
    info->fwd_tile_w = P->fwd.tile_w;
    info->fwd_tile_h = P->fwd.tile_h;
    return CTIS_OK;
}

int ctis_plan_export_taps(const ctis_plan* P, int32_t* s, int32_t* x, int32_t* y, float* val,
                          float* h) {
    if (!P) return fail(CTIS_ERR_INVALID_ARG, "plan is NULL");
    const size_t n = P->tap_v.size();
    if (s) std::memcpy(s, P->tap_s.data(), n * sizeof(int32_t));
    if (x) std::memcpy(x, P->tap_x.data(), n * sizeof(int32_t));
    if (y) std::memcpy(y, P->tap_y.data(), n * sizeof(int32_t));
    if (val) std::memcpy(val, P->tap_v.data(), n * sizeof(float));
    if (h) std::memcpy(h, P->h.data(), P->h.size() * sizeof(float));
    return CTIS_OK;
}

int ctis_index_map(const ctis_plan* P, int64_t* out_dev, void* stream) {
    int rc = check_plan(P);
    if (rc) return rc;
    if (!out_dev) return fail(CTIS_ERR_INVALID_ARG, "out_dev is NULL");
    CTIS_CUDA(launch_index_map(reinterpret_cast<long long*>(out_dev), P->a, P->alpha, P->w,
                               P->gamma, P->n, static_cast<cudaStream_t>(stream)));
    return CTIS_OK;
}

int ctis_forward(const ctis_plan* P, const void* f_dev, float* hf_dev, void* stream) {
    int rc = check_plan(P);
    if (rc) return rc;
    if (!f_dev || !hf_dev) return fail(CTIS_ERR_INVALID_ARG, "NULL device pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rc = scatter_f(P, f_dev, P->dtype, 0.f, st);
    if (rc) return rc;
    GatherParams p = base_params(P, P->fwd);
    p.mode = kEpiRaw;
    p.out_w = P->gamma;
    p.out_h = P->xi;
    p.out_f32 = hf_dev;
    p.out_pitch = P->gamma;
    p.out_plane_stride = 0;
    return enqueue_forward(P, p, st);
}

int ctis_adjoint(const ctis_plan* P, const float* r_dev, float* out_dev, void* stream) {
    int rc = check_plan(P);
    if (rc) return rc;
    if (!r_dev || !out_dev) return fail(CTIS_ERR_INVALID_ARG, "NULL device pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rc = scatter_u(P, r_dev, st);
    if (rc) return rc;
    GatherParams p = base_params(P, P->adj);
    p.mode = kEpiRaw;
    p.out_w = P->a;
    p.out_h = P->alpha;
    p.out_f32 = out_dev;
    p.out_pitch = P->a;
    p.out_plane_stride = static_cast<long long>(P->a) * P->alpha;
    return enqueue_adjoint(P, p, st);
}

#ifdef CTIS_DEBUG_BOUNDS
// Debug builds: register the buffers of a call for the epilogue range checks.
int ctis_debug_arm(const ctis_plan* P, const void* user0, size_t bytes0, const void* user1,
                   size_t bytes1, unsigned long long* log_dev) {
    const size_t es = P->dtype == kDtypeBF16 ? 2 : 4;
    const void* lo[6] = {P->d_u, P->d_fwork, P->d_scratch, user0, user1, nullptr};
    const size_t bytes[6] = {sizeof(float) * static_cast<size_t>(P->u_copy_stride) * P->u_copies,
                             es * static_cast<size_t>(P->f_copy_stride) * P->f_copies,
                             sizeof(float) * static_cast<size_t>(std::max(
                                 P->fwd.scratch_slots * P->fwd.tile_w * P->fwd.tile_h,
                                 P->adj.scratch_slots * P->adj.tile_w * P->adj.tile_h)),
                             bytes0, bytes1, 0};
    CTIS_CUDA(debug_arm(lo, bytes, log_dev));
    return CTIS_OK;
}
#endif

int ctis_reconstruct(const ctis_plan* Pc, const float* g_dev, void* f_dev, int k, int flags,
                     double* stats_dev, void* stream) {
    return ctis_reconstruct_solver(Pc, g_dev, f_dev, k, flags, CTIS_SOLVER_EM, 1.0f, stats_dev,
                                   stream);
}

int ctis_reconstruct_solver(const ctis_plan* Pc, const float* g_dev, void* f_dev, int k, int flags,
                            int solver, float relax, double* stats_dev, void* stream) {
    int rc = check_plan(Pc);
    if (rc) return rc;
    ctis_plan* P = const_cast<ctis_plan*>(Pc);
    if (!g_dev || !f_dev) return fail(CTIS_ERR_INVALID_ARG, "NULL device pointer");
    if (k < 0) return fail(CTIS_ERR_INVALID_ARG, "k must be >= 0");
    if (flags & ~(CTIS_INIT_ONES | CTIS_INIT_HTG) ||
        (flags & CTIS_INIT_ONES && flags & CTIS_INIT_HTG))
        return fail(CTIS_ERR_INVALID_ARG, "bad flags 0x%x", flags);
    if (solver != CTIS_SOLVER_EM && solver != CTIS_SOLVER_SART && solver != CTIS_SOLVER_SMART)
        return fail(CTIS_ERR_INVALID_ARG, "solver must be CTIS_SOLVER_EM, _SART or _SMART");
    if (!(relax > 0.f && relax <= 2.f))
        return fail(CTIS_ERR_INVALID_ARG, "relax = %g is not in (0, 2]", (double)relax);
    if (solver == CTIS_SOLVER_EM) relax = 1.f;   // unused: one graph for every value
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CTIS_CUDA(cudaStreamIsCapturing(st, &cap));
    if (solver == CTIS_SOLVER_SART && !P->rowsum_valid) {
        if (cap != cudaStreamCaptureStatusNone)
            return fail(CTIS_ERR_INVALID_ARG,
                        "SART's row sums are built by the first uncaptured call");
        rc = ensure_rowsum(P);
        if (rc) return rc;
    }
    if (cap != cudaStreamCaptureStatusNone)   // caller is building its own graph
        return enqueue_reconstruct(P, g_dev, f_dev, k, flags, stats_dev, st, solver, relax);

    GraphKey key;
    key.g = g_dev;
    key.f = f_dev;
    key.stats = stats_dev;
    key.k = k;
    key.flags = flags;
    key.solver = solver;
    key.relax = relax;
    key.profiling = P->profiling;
    if (!(P->gexec && P->gkey == key)) {
        if (P->gexec) {
            cudaGraphExecDestroy(P->gexec);
            P->gexec = nullptr;
        }
        CTIS_CUDA(cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal));
        rc = enqueue_reconstruct(P, g_dev, f_dev, k, flags, stats_dev, P->cap_stream, solver,
                                 relax);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(P->cap_stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&P->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            P->gexec = nullptr;
            return cuda_fail(e, "cudaGraphInstantiate");
        }
        P->gkey = key;
    }
    CTIS_CUDA(cudaGraphLaunch(P->gexec, st));
    return CTIS_OK;
}

int ctis_plan_set_debug(ctis_plan* P, int flags) {
    if (!P) return fail(CTIS_ERR_INVALID_ARG, "plan is NULL");
    if (flags & ~(CTIS_DEBUG_DROP_COPIES | CTIS_DEBUG_SERIAL_LAUNCH))
        return fail(CTIS_ERR_INVALID_ARG, "bad flags 0x%x", flags);
    CTIS_CUDA(cudaDeviceSynchronize());   // cached graphs hold the old parameters
    drop_table_users(P);
    P->drop_copies = (flags & CTIS_DEBUG_DROP_COPIES) != 0;
    P->overlap_launch = (flags & CTIS_DEBUG_SERIAL_LAUNCH) == 0;
    return CTIS_OK;
}

int ctis_plan_set_profiling(ctis_plan* P, int enable) {
    if (!P) return fail(CTIS_ERR_INVALID_ARG, "plan is NULL");
    P->profiling = enable != 0;
    return CTIS_OK;
}

int ctis_plan_kernel_times(const ctis_plan* P, double* fwd_ms, int* n_fwd, double* adj_ms,
                           int* n_adj) {
    int rc = check_plan(P);
    if (rc) return rc;
    auto sum = [&](const std::vector<std::pair<int, int>>& log, double* ms, int* n) -> int {
        double t = 0.0;
        for (const auto& pr : log) {
            CTIS_CUDA(cudaEventSynchronize(P->events[pr.second]));
            float x = 0.f;
            CTIS_CUDA(cudaEventElapsedTime(&x, P->events[pr.first], P->events[pr.second]));
            t += x;
        }
        if (ms) *ms = t;
        if (n) *n = static_cast<int>(log.size());
        return CTIS_OK;
    };
    rc = sum(P->prof_fwd, fwd_ms, n_fwd);
    if (!rc) rc = sum(P->prof_adj, adj_ms, n_adj);
    return rc;
}

int ctis_forward_static_scratch(const ctis_plan* P, const void* f_dev, float* hf_dev,
                                void* stream) {
    int rc = check_plan(P);
    if (rc) return rc;
    if (!f_dev || !hf_dev) return fail(CTIS_ERR_INVALID_ARG, "NULL device pointer");
    // Pieces of the static array, each 256-byte aligned: tile tickets, chunk
    // partial sums, the x-shifted copies of f. The bounded waits' error flag
    // stays the plan's own (ctis_plan_check reports it).
    const size_t es = P->dtype == kDtypeBF16 ? 2 : 4;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = static_cast<size_t>(round_up(static_cast<int64_t>(off + bytes), 256));
        return o;
    };
    const size_t o_tickets = take(P->fwd.tiles.size() * sizeof(int));
    const size_t o_partials = take(sizeof(float) * static_cast<size_t>(P->fwd.scratch_slots) *
                                   P->fwd.tile_w * P->fwd.tile_h);
    const size_t copies_bytes = es * static_cast<size_t>(P->f_copy_stride) * P->f_copies;
    const size_t o_copies = take(copies_bytes);
    if (off > static_scratch_bytes())
        return fail(CTIS_ERR_UNSUPPORTED,
                    "this plan's forward projection needs %zu bytes of scratch; the static "
                    "scratch array holds %zu bytes (use ctis_forward)",
                    off, static_scratch_bytes());
    void* base_v = nullptr;
    CTIS_CUDA(static_scratch_ptr(&base_v));
    unsigned char* base = static_cast<unsigned char*>(base_v);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // The array keeps the previous call's contents. The tile tickets must
    // start at zero (the kernel leaves them at zero, but a call whose waits
    // gave up may not have), and so must the columns of each copy that the
    // scatter below leaves unwritten and the window map still reads: copy q
    // holds f at columns [q, a + q) of its rows, so [0, q) and the row's rest
    // from a + q on are cleared (every row of a copy is a_pitch apart, across
    // the planes too).
    CTIS_CUDA(cudaMemsetAsync(base + o_tickets, 0, o_partials - o_tickets, st));
    const size_t rows = static_cast<size_t>(P->alpha) * P->w;
    const size_t pitch_b = es * static_cast<size_t>(P->a_pitch);
    for (int q = 0; q < P->f_copies; ++q) {
        unsigned char* cq = base + o_copies + es * static_cast<size_t>(P->f_copy_stride) * q;
        if (q > 0) CTIS_CUDA(cudaMemset2DAsync(cq, pitch_b, 0, es * q, rows, st));
        const size_t right = static_cast<size_t>(P->a_pitch - P->a - q);
        if (right > 0)
            CTIS_CUDA(cudaMemset2DAsync(cq + es * static_cast<size_t>(P->a + q), pitch_b, 0,
                                        es * right, rows, st));
    }
    void* copies = base + o_copies;
    const int64_t plane = static_cast<int64_t>(P->a_pitch) * P->alpha;
    CTIS_CUDA(launch_scatter_copies(P->dtype, copies, P->f_copy_stride, P->f_copies, P->a_pitch,
                                    plane, f_dev, P->dtype, P->a,
                                    static_cast<int64_t>(P->a) * P->alpha, P->a, P->alpha, P->w,
                                    0.f, st));
    CUtensorMap win;
    rc = make_map(&win, copies, P->dtype, P->a + P->f_copies - 1, P->alpha, P->w * P->f_copies,
                  P->a_pitch, plane, gather_box_w(true, P->K, P->dtype, P->fwd_shape),
                  gather_window_rows(true, P->K, P->dtype, P->fwd_shape));
    if (rc) return rc;
    GatherParams p = base_params(P, P->fwd);
    p.scratch = reinterpret_cast<float*>(base + o_partials);
    p.tickets = reinterpret_cast<int*>(base + o_tickets);
    p.tile_stats = nullptr;
    p.mode = kEpiRaw;
    p.out_w = P->gamma;
    p.out_h = P->xi;
    p.out_f32 = hf_dev;
    p.out_pitch = P->gamma;
    p.out_plane_stride = 0;
    rc = zero_raw_output(p, st);
    if (rc) return rc;
    CTIS_CUDA(gather_launch(true, P->K, P->dtype, win, p, st, P->fwd_shape));
    return CTIS_OK;
}

}  // extern "C"

namespace {

// Builds the plan's FFT form on first use: the calibration images c_s of the
// merged nonzeros on the FPA (under the wrap reading the stored images off
// it repeat those), d_s = F c_s, h per wavelength.
int ensure_fft(ctis_plan* P) {
    if (P->fft) return CTIS_OK;
    if (P->clip && !P->wrap)
        return fail(CTIS_ERR_UNSUPPORTED,
                    "the FFT form needs CTIS_BOUNDARY_REJECT or _WRAP (Eq. 7's circulant wraps)");
    if (P->dtype != kDtypeF32) return fail(CTIS_ERR_UNSUPPORTED, "the FFT form needs a float32 plan");
    const int64_t n = P->n;
    std::vector<float> calib(static_cast<size_t>(n) * P->w, 0.f);
    for (size_t k = 0; k < P->tap_v.size(); ++k) {
        if (P->tap_x[k] < 0 || P->tap_y[k] < 0) continue;
        calib[static_cast<size_t>(P->tap_s[k]) * n + P->tap_x[k] +
              static_cast<int64_t>(P->gamma) * P->tap_y[k]] += P->tap_v[k];
    }
    int rc = dmalloc(P, reinterpret_cast<void**>(&P->d_fft_u), sizeof(float) * n);
    if (rc) return rc;
    CTIS_CUDA(fft_form_create(&P->fft, P->a, P->alpha, P->w, P->gamma, P->xi, calib.data(),
                              P->h.data()));
    return CTIS_OK;
}

}  // namespace

extern "C" {

int ctis_fft_forward(ctis_plan* P, const float* f_dev, float* hf_dev, void* stream) {
    int rc = check_plan(P);
    if (rc) return rc;
    if (!f_dev || !hf_dev) return fail(CTIS_ERR_INVALID_ARG, "NULL device pointer");
    rc = ensure_fft(P);
    if (rc) return rc;
    CTIS_CUDA(fft_form_forward(P->fft, f_dev, hf_dev, static_cast<cudaStream_t>(stream)));
    return CTIS_OK;
}

int ctis_fft_adjoint(ctis_plan* P, const float* r_dev, float* out_dev, void* stream) {
    int rc = check_plan(P);
    if (rc) return rc;
    if (!r_dev || !out_dev) return fail(CTIS_ERR_INVALID_ARG, "NULL device pointer");
    rc = ensure_fft(P);
    if (rc) return rc;
    CTIS_CUDA(fft_form_adjoint(P->fft, r_dev, out_dev, static_cast<cudaStream_t>(stream)));
    return CTIS_OK;
}

int ctis_fft_reconstruct(ctis_plan* P, const float* g_dev, float* f_dev, int k, int flags,
                         void* stream) {
    int rc = check_plan(P);
    if (rc) return rc;
    if (!g_dev || !f_dev) return fail(CTIS_ERR_INVALID_ARG, "NULL device pointer");
    if (k < 0) return fail(CTIS_ERR_INVALID_ARG, "k must be >= 0");
    if (flags & ~CTIS_INIT_ONES) return fail(CTIS_ERR_INVALID_ARG, "bad flags 0x%x", flags);
    rc = ensure_fft(P);
    if (rc) return rc;
    CTIS_CUDA(fft_form_reconstruct(P->fft, g_dev, f_dev, P->d_fft_u, k, (flags & CTIS_INIT_ONES) != 0,
                                   static_cast<cudaStream_t>(stream)));
    return CTIS_OK;
}

int ctis_plan_set_values(ctis_plan* P, const float* vals) {
    int rc = check_plan(P);
    if (rc) return rc;
    if (P->wrap)
        return fail(CTIS_ERR_UNSUPPORTED,
                    "new values under CTIS_BOUNDARY_WRAP (each image keeps its original's value)");
    const size_t nnz = P->tap_v.size();
    if (!vals && nnz) return fail(CTIS_ERR_INVALID_ARG, "vals is NULL");
    for (size_t k = 0; k < nnz; ++k)
        if (!std::isfinite(vals[k]) || vals[k] < 0.f)
            return fail(CTIS_ERR_INVALID_ARG, "vals[%zu] = %g is not finite and >= 0", k,
                        (double)vals[k]);
    // work already queued on any stream may still read the old tables
    CTIS_CUDA(cudaDeviceSynchronize());
    for (size_t k = 0; k < nnz; ++k)
        P->tap_v[k] = P->dtype == kDtypeBF16 ? bf16_bits_to_float(to_bf16_bits(vals[k])) : vals[k];
    compute_h(P);
    P->rowsum_valid = false;   // rebuilt from the new values on SART's next use
    rc = write_values(P, false);
    if (!rc) rc = compute_hvox(P, nullptr);
    fft_form_destroy(P->fft);   // rebuilt from the new values on its next use
    P->fft = nullptr;
    return rc;
}

int ctis_psf_grad(const ctis_plan* P, const void* f_dev, const float* r_dev, float* dval_dev,
                  void* stream) {
    int rc = check_plan(P);
    if (rc) return rc;
    if (!f_dev || !r_dev || !dval_dev) return fail(CTIS_ERR_INVALID_ARG, "NULL device pointer");
    if (P->wrap)
        return fail(CTIS_ERR_UNSUPPORTED,
                    "the PSF-value gradient under CTIS_BOUNDARY_WRAP (images share values)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rc = scatter_u(P, r_dev, st);
    if (rc) return rc;
    return enqueue_psf_grad(P, f_dev, dval_dev, false, nullptr, st);
}

int ctis_unrolled_nll_grad(ctis_plan* P, const float* g_dev, const float* f0_dev, int k,
                           double* nll_dev, float* dval_dev, float* df0_dev, void* stream) {
    int rc = check_plan(P);
    if (rc) return rc;
    if (P->dtype != kDtypeF32)
        return fail(CTIS_ERR_UNSUPPORTED, "the unrolled EM gradient needs a float32 plan");
    if (P->wrap)
        return fail(CTIS_ERR_UNSUPPORTED,
                    "the unrolled EM gradient under CTIS_BOUNDARY_WRAP (images share values)");
    if (!g_dev || !nll_dev || !dval_dev) return fail(CTIS_ERR_INVALID_ARG, "NULL device pointer");
    if (k < 0 || k > 4096) return fail(CTIS_ERR_INVALID_ARG, "k must be in [0, 4096]");
    const int64_t m = P->m, n = P->n;
    const int a = P->a, al = P->alpha, w = P->w, ga = P->gamma, xi = P->xi;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // ---- workspace: k + 1 checkpoints of f, the dense vectors of a step
    if (P->ck_steps < k) {
        CTIS_CUDA(cudaStreamSynchronize(st));
        cudaFree(P->d_ck);
        P->d_ck = nullptr;
        P->ck_steps = -1;
        rc = dmalloc(P, reinterpret_cast<void**>(&P->d_ck), sizeof(float) * m * (k + 1));
        if (rc) return rc;
        P->ck_steps = k;
    }
    const int vb = voxel_vjp_blocks();
    if (!P->d_work) {
        rc = dmalloc(P, reinterpret_cast<void**>(&P->d_work), sizeof(float) * (2 * n + 6 * m));
        if (!rc)
            rc = dmalloc(P, reinterpret_cast<void**>(&P->d_gwork),
                         sizeof(double) * (static_cast<size_t>(w) * vb + w + kNumStats));
        if (rc) return rc;
    }
    float* q = P->d_work;
    float* gu = q + n;
    float* z = gu + n;
    float* gfd = z + m;
    float* gb = gfd + m;
    float* hq = gb + m;
    float* adense = hq + m;
    float* dh_vox = adense + m;   // clipped boundary: dL/dh per voxel
    double* vjp_part = P->d_gwork;
    double* dh = vjp_part + static_cast<size_t>(w) * vb;
    double* stats = dh + w;
    auto ck = [&](int t) { return P->d_ck + static_cast<int64_t>(t) * m; };
    const int64_t fplane = static_cast<int64_t>(P->a_pitch) * al;

    auto copy_out = [&](float* dst) -> int {   // f copies (copy 0) -> dense
        CTIS_CUDA(launch_gather_copy0(kDtypeF32, dst, P->d_fwork, P->a_pitch, fplane, a, al, w, st));
        return CTIS_OK;
    };
    auto forward_raw = [&](float* out) -> int {
        GatherParams p = base_params(P, P->fwd);
        p.mode = kEpiRaw;
        p.out_w = ga;
        p.out_h = xi;
        p.out_f32 = out;
        p.out_pitch = ga;
        return enqueue_forward(P, p, st);
    };
    auto adjoint_raw = [&](float* out) -> int {
        GatherParams p = base_params(P, P->adj);
        p.mode = kEpiRaw;
        p.out_w = a;
        p.out_h = al;
        p.out_f32 = out;
        p.out_pitch = a;
        p.out_plane_stride = static_cast<long long>(a) * al;
        return enqueue_adjoint(P, p, st);
    };

    // ---- k EM updates (Eq. 2) from f0 or ones, keeping every iterate
    rc = zero_u(P, st);
    if (!rc)
        rc = f0_dev ? scatter_f(P, f0_dev, kDtypeF32, 0.f, st) : scatter_f(P, nullptr, kDtypeF32, 1.f, st);
    if (rc) return rc;
    GatherParams pf = base_params(P, P->fwd);
    pf.mode = kEpiRatio;
    pf.out_w = ga;
    pf.out_h = xi;
    pf.out_f32 = P->d_u;
    pf.out_pitch = P->g_pitch;
    pf.out_copy_stride = P->u_copy_stride;
    pf.out_copies = P->u_copies;
    pf.g = g_dev;
    pf.g_pitch = ga;
    GatherParams pa = base_params(P, P->adj);
    pa.mode = kEpiUpdate;
    pa.out_w = a;
    pa.out_h = al;
    set_f_copies(P, pa);
    for (int t = 0; t < k; ++t) {
        rc = copy_out(ck(t));
        if (!rc) rc = enqueue_forward(P, pf, st);
        if (!rc) rc = enqueue_adjoint(P, pa, st);
        if (rc) return rc;
    }
    rc = copy_out(ck(k));
    if (rc) return rc;

    // ---- L = sum (q - g log q) over q = H f^(k) > 0; dL/dq = 1 - g/q there
    GatherParams pl = pf;
    pl.ratio_one_minus = 1;
    pl.with_stats = 1;
    rc = enqueue_forward(P, pl, st);             // 1 - g/q into the FPA copies
    if (rc) return rc;
    CTIS_CUDA(launch_stats_reduce(stats, P->d_tile_stats, static_cast<int>(P->fwd.tiles.size()), 1,
                                  0, P->d_red_part, P->d_counters + 8, st));
    rc = adjoint_raw(gb);                        // dL/df^(k) = H^T (1 - g/q)
    if (!rc) rc = enqueue_psf_grad(P, ck(k), dval_dev, false, nullptr, st);
    if (rc) return rc;
    CTIS_CUDA(launch_negate(nll_dev, stats + CTIS_STAT_LOGLIK, st));

    // ---- back through the updates f' = f * H^T(g / H f) / h, newest first
    for (int t = k - 1; t >= 0; --t) {
        rc = scatter_f(P, ck(t), kDtypeF32, 0.f, st);
        if (!rc) rc = forward_raw(q);                                   // q = H f
        if (rc) return rc;
        CTIS_CUDA(launch_fpa_to_copies(P->d_u, P->u_copy_stride, P->u_copies, P->g_pitch, q, g_dev,
                                       nullptr, ga, xi, 0, st));       // u = g / q
        rc = adjoint_raw(z);                                            // z = H^T u
        if (rc) return rc;
        CTIS_CUDA(launch_voxel_vjp(adense, static_cast<float*>(P->d_fwork), P->f_copy_stride,
                                   P->f_copies, P->a_pitch, fplane, gfd, vjp_part, gb, ck(t), z,
                                   P->d_h, a, al, w, P->clip ? P->d_hvox : nullptr, dh_vox,
                                   st));                                // a, gfd, dL/dh parts
        if (!P->clip) CTIS_CUDA(launch_dh_finish(dh, vjp_part, P->d_h, w, st));
        rc = forward_raw(gu);                                           // dL/du = H a
        if (!rc) rc = enqueue_psf_grad(P, adense, dval_dev, true, nullptr, st);   // via H^T u
        if (rc) return rc;
        CTIS_CUDA(launch_fpa_to_copies(P->d_u, P->u_copy_stride, P->u_copies, P->g_pitch, q, g_dev,
                                       gu, ga, xi, 1, st));            // dL/dq = -gu g / q^2
        rc = adjoint_raw(hq);                                           // H^T dL/dq
        if (!rc) rc = enqueue_psf_grad(P, ck(t), dval_dev, true, P->clip ? nullptr : dh, st);
        if (rc) return rc;                                              // via H f (and h_s)
        if (P->clip) {   // via h_j = sum of the taps whose copy for voxel j lands on the FPA:
                         // dh_j/dv_t = 1 there, the adjoint of an all-ones FPA image
            rc = scatter_u(P, nullptr, st, 1.0f);
            if (!rc) rc = enqueue_psf_grad(P, dh_vox, dval_dev, true, nullptr, st);
            if (rc) return rc;
        }
        CTIS_CUDA(launch_add(gb, gfd, hq, m, st));                      // dL/df
    }
    if (df0_dev)
        CTIS_CUDA(cudaMemcpyAsync(df0_dev, gb, sizeof(float) * m, cudaMemcpyDeviceToDevice, st));
    return CTIS_OK;
}

int ctis_reconstruct_batched(ctis_plan* const* plans, int nplans, int nframes,
                             const int* plan_idx, const float* const* g_dev, void* const* f_dev,
                             int k, int flags, double* stats_dev, void* stream) {
    return ctis_reconstruct_batched_solver(plans, nplans, nframes, plan_idx, g_dev, f_dev, k,
                                           flags, CTIS_SOLVER_EM, 1.0f, stats_dev, stream);
}

int ctis_reconstruct_batched_solver(ctis_plan* const* plans, int nplans, int nframes,
                                    const int* plan_idx, const float* const* g_dev,
                                    void* const* f_dev, int k, int flags, int solver, float relax,
                                    double* stats_dev, void* stream) {
    if (!plans || nplans < 1 || nframes < 1 || !plan_idx || !g_dev || !f_dev)
        return fail(CTIS_ERR_INVALID_ARG, "NULL array or empty batch");
    if (k < 0) return fail(CTIS_ERR_INVALID_ARG, "k must be >= 0");
    if (flags & ~(CTIS_INIT_ONES | CTIS_INIT_HTG) ||
        (flags & CTIS_INIT_ONES && flags & CTIS_INIT_HTG))
        return fail(CTIS_ERR_INVALID_ARG, "bad flags 0x%x", flags);
    if (solver != CTIS_SOLVER_EM && solver != CTIS_SOLVER_SART && solver != CTIS_SOLVER_SMART)
        return fail(CTIS_ERR_INVALID_ARG, "solver must be CTIS_SOLVER_EM, _SART or _SMART");
    if (!(relax > 0.f && relax <= 2.f))
        return fail(CTIS_ERR_INVALID_ARG, "relax = %g is not in (0, 2]", (double)relax);
    if (solver == CTIS_SOLVER_EM) relax = 1.f;
    for (int p = 0; p < nplans; ++p) {
        int rc = check_plan(plans[p]);
        if (rc) return rc;
        for (int q = 0; q < p; ++q)
            if (plans[q] == plans[p])
                return fail(CTIS_ERR_INVALID_ARG, "plan %d appears twice in plans[]", p);
    }
    std::vector<std::vector<int>> frames(nplans);
    for (int i = 0; i < nframes; ++i) {
        if (plan_idx[i] < 0 || plan_idx[i] >= nplans)
            return fail(CTIS_ERR_INVALID_ARG, "plan_idx[%d] = %d out of range", i, plan_idx[i]);
        if (!g_dev[i] || !f_dev[i])
            return fail(CTIS_ERR_INVALID_ARG, "frame %d has a NULL pointer", i);
        frames[plan_idx[i]].push_back(i);
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<int> used;
    for (int p = 0; p < nplans; ++p) {
        if (frames[p].empty()) continue;
        int rc = ensure_batch(plans[p], static_cast<int>(frames[p].size()), k);
        if (!rc && solver == CTIS_SOLVER_SART) rc = ensure_rowsum(plans[p]);
        if (rc) return rc;
        used.push_back(p);
    }
    // per-frame pointers and caller positions, ordered on the stream
    for (int p : used) {
        BatchState* B = plans[p]->batch;
        const int F = B->F;
        std::vector<const void*> ptrs(2 * F);
        std::vector<int> gid(F);
        for (int j = 0; j < F; ++j) {
            ptrs[j] = g_dev[frames[p][j]];
            ptrs[F + j] = f_dev[frames[p][j]];
            gid[j] = frames[p][j];
        }
        CTIS_CUDA(cudaMemcpyAsync(B->d_ptrs, ptrs.data(), sizeof(void*) * 2 * F,
                                  cudaMemcpyHostToDevice, st));
        CTIS_CUDA(cudaMemcpyAsync(B->d_gid, gid.data(), sizeof(int) * F, cudaMemcpyHostToDevice, st));
    }

    BatchedKey key;
    key.plans.assign(plans, plans + nplans);
    key.plan_idx.assign(plan_idx, plan_idx + nframes);
    key.g.assign(g_dev, g_dev + nframes);
    key.f.assign(f_dev, f_dev + nframes);
    key.k = k;
    key.flags = flags;
    key.solver = solver;
    key.relax = relax;
    key.stats = stats_dev;
    std::lock_guard<std::mutex> lock(g_batched_mu);
    int dev = 0;
    CTIS_CUDA(cudaGetDevice(&dev));
    if (!(g_batched_exec && g_batched_key == key && g_batched_device == dev)) {
        if (g_batched_exec) {
            cudaGraphExecDestroy(g_batched_exec);
            g_batched_exec = nullptr;
            g_batched_key = BatchedKey{};
        }
        if (g_batched_stream && g_batched_device != dev) {
            cudaStreamDestroy(g_batched_stream);
            g_batched_stream = nullptr;
        }
        if (!g_batched_stream) {
            CTIS_CUDA(cudaStreamCreateWithFlags(&g_batched_stream, cudaStreamNonBlocking));
            g_batched_device = dev;
        }
        cudaStream_t cs = g_batched_stream;
        std::vector<BatchRun> runs;
        for (int p : used)
            runs.push_back(BatchRun{plans[p], plans[p]->batch, {}, {}, stats_dev != nullptr, solver,
                                    relax});
        CTIS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        int rc = CTIS_OK;
        for (BatchRun& r : runs)
            if (!rc) rc = batch_setup(r, flags, cs);
        for (int it = 0; it <= k && !rc; ++it) {
            if (it == k && !stats_dev) break;
            for (BatchRun& r : runs)
                if (!rc) rc = batch_forward_step(r, cs);
            if (it == k) break;
            for (BatchRun& r : runs)
                if (!rc) rc = batch_adjoint_step(r, it, k, cs);
        }
        for (BatchRun& r : runs)
            if (!rc) rc = batch_finish(r, k, stats_dev, cs);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&g_batched_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            g_batched_exec = nullptr;
            return cuda_fail(e, "cudaGraphInstantiate");
        }
        g_batched_key = key;
    }
    CTIS_CUDA(cudaGraphLaunch(g_batched_exec, st));
    return CTIS_OK;
}

int ctis_plan_set_schedule(ctis_plan* P, int forward, int tasks_per_item, int item_overhead_q,
                           int cta_skew_permille) {
    int rc = check_plan(P);
    if (rc) return rc;
    if (tasks_per_item < 0 || tasks_per_item > 1 << 20)
        return fail(CTIS_ERR_INVALID_ARG, "tasks_per_item out of range");
    if (item_overhead_q < 0 || item_overhead_q > 1 << 16)
        return fail(CTIS_ERR_INVALID_ARG, "item_overhead_q out of range");
    if (tasks_per_item > 0 && item_overhead_q > 0)
        return fail(CTIS_ERR_INVALID_ARG, "tasks_per_item and item_overhead_q are exclusive");
    if (cta_skew_permille < 0 || cta_skew_permille > 900)
        return fail(CTIS_ERR_INVALID_ARG, "cta_skew_permille out of range [0, 900]");
    CTIS_CUDA(cudaDeviceSynchronize());
    drop_table_users(P);
    ProjTables& T = forward ? P->fwd : P->adj;
    schedule(T, T.n_warps, tasks_per_item, item_overhead_q, cta_skew_permille);
    rc = reupload_tables(P, T);
    if (rc) return rc;
    CTIS_CUDA(cudaDeviceSynchronize());
    return CTIS_OK;
}

int ctis_plan_autotune(ctis_plan* P, const float* g_dev, void* stream) {
    int rc = check_plan(P);
    if (rc) return rc;
    if (!g_dev) return fail(CTIS_ERR_INVALID_ARG, "g_dev is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CTIS_CUDA(cudaDeviceSynchronize());
    drop_table_users(P);
    // realistic operands: f = 1 in the datacube copies, g in the FPA copies
    rc = scatter_f(P, nullptr, P->dtype, 1.0f, st);
    if (!rc) rc = scatter_u(P, g_dev, st);
    if (rc) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CTIS_CUDA(cudaEventCreate(&e0));
    {
        const cudaError_t e = cudaEventCreate(&e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            return cuda_fail(e, "cudaEventCreate");
        }
    }
    auto reupload = [&](ProjTables& T) -> int { return reupload_tables(P, T); };
    // the EM launches (ratio with statistics; update) on the candidate tables
    auto run = [&](bool forward) -> int {
        if (forward) {
            GatherParams p = base_params(P, P->fwd);
            p.mode = kEpiRatio;
            p.out_w = P->gamma;
            p.out_h = P->xi;
            p.out_f32 = P->d_u;
            p.out_pitch = P->g_pitch;
            p.out_copy_stride = P->u_copy_stride;
            p.out_copies = P->u_copies;
            p.g = g_dev;
            p.g_pitch = P->gamma;
            p.with_stats = 1;   // tile statistics, as inside the EM loop
            return enqueue_forward(P, p, st);
        }
        GatherParams p = base_params(P, P->adj);
        p.mode = kEpiUpdate;
        p.out_w = P->a;
        p.out_h = P->alpha;
        set_f_copies(P, p);
        return enqueue_adjoint(P, p, st);
    };
    // candidates: the model's choice, chunks of 16..192 tasks (longest-first),
    // and the balanced split with item overheads of 0.5..6 tasks
    struct Cand {
        int chunk, split_q, skew_pm;
    };
    std::vector<Cand> cands{{0, 0, 0}};
    for (int c : {16, 24, 32, 48, 64, 96, 128, 192}) cands.push_back({c, 0, 0});
    for (int q : {2, 4, 8, 12, 16, 24}) cands.push_back({0, q, 0});
    for (int skew : {100, 200, 300}) {   // the CTA priority skew, on the likeliest shapes
        for (int c : {64, 96, 128}) cands.push_back({c, 0, skew});
        for (int q : {12, 16, 20}) cands.push_back({0, q, skew});
    }
    int result = CTIS_OK;
    // milliseconds per launch of the projector's current tables over `reps`
    // launches (after two warm-up launches); < 0 when something failed
    // (result is set)
    auto time_now = [&](bool forward, int reps) -> float {
        for (int r = 0; r < 2 && !result; ++r) result = run(forward);   // warm-up
        cudaError_t e = result ? cudaSuccess : cudaEventRecord(e0, st);
        for (int r = 0; r < reps && !result && e == cudaSuccess; ++r) result = run(forward);
        if (!result && e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (!result && e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (!result && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (!result && e != cudaSuccess) result = cuda_fail(e, "timing a candidate schedule");
        return result ? -1.f : ms / reps;
    };
    auto time_cand = [&](ProjTables* T, const Cand& c, int reps) -> float {
        schedule(*T, T->n_warps, c.chunk, c.split_q, c.skew_pm);
        result = reupload(*T);
        return result ? -1.f : time_now(T == &P->fwd, reps);
    };
    // The best schedule of the projector's current tables: a first pass over
    // all candidates, then the four fastest again, interleaved over three
    // rounds of 10 launches, to keep the timing noise out of the choice.
    auto tune = [&](ProjTables* T) -> Cand {
        std::vector<std::pair<float, Cand>> timed;
        for (const Cand& c : cands) {
            const float ms = time_cand(T, c, 5);
            if (ms < 0.f) break;
            timed.push_back({ms, {T->per_item, T->split_q, T->skew_pm}});
        }
        if (result) return Cand{};
        std::stable_sort(timed.begin(), timed.end(),
                         [](const auto& x, const auto& y) { return x.first < y.first; });
        timed.resize(std::min<size_t>(timed.size(), 4));
        std::vector<float> total(timed.size(), 0.f);
        for (int round = 0; round < 3 && !result; ++round)
            for (size_t i = 0; i < timed.size() && !result; ++i) {
                const float ms = time_cand(T, timed[i].second, 10);
                if (ms >= 0.f) total[i] += ms;
            }
        size_t bi = 0;
        for (size_t i = 1; i < timed.size(); ++i)
            if (total[i] < total[bi]) bi = i;
        return timed.empty() ? Cand{} : timed[bi].second;
    };
    // Forward: every tile shape with its own best schedule, then the shapes'
    // winners against each other, interleaved over three rounds.
    const int nshapes = gather_fwd_shapes();
    std::vector<Cand> shape_best(nshapes);
    for (int sh = 0; sh < nshapes && !result; ++sh) {
        result = set_forward_shape(P, sh);
        if (!result) shape_best[sh] = tune(&P->fwd);
    }
    int best_shape = 0;
    if (!result && nshapes > 1) {
        std::vector<float> total(nshapes, 0.f);
        for (int round = 0; round < 3 && !result; ++round)
            for (int sh = 0; sh < nshapes && !result; ++sh) {
                if (P->fwd_shape != sh) result = set_forward_shape(P, sh);
                const float ms = result ? -1.f : time_cand(&P->fwd, shape_best[sh], 10);
                if (ms >= 0.f) total[sh] += ms;
            }
        for (int sh = 1; sh < nshapes; ++sh)
            if (total[sh] < total[best_shape]) best_shape = sh;
    }
    if (!result && P->fwd_shape != best_shape) result = set_forward_shape(P, best_shape);
    if (!result) {
        const Cand& b = shape_best[best_shape];
        schedule(P->fwd, P->fwd.n_warps, b.chunk, b.split_q, b.skew_pm);
        result = reupload(P->fwd);
    }
    // adjoint: one tile shape
    if (!result) {
        const Cand b = tune(&P->adj);
        if (!result) {
            schedule(P->adj, P->adj.n_warps, b.chunk, b.split_q, b.skew_pm);
            result = reupload(P->adj);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result) return result;
    CTIS_CUDA(cudaStreamSynchronize(st));
    return CTIS_OK;
}

int ctis_reconstruct_sharded(ctis_plan* P, const float* g_dev, void* f_dev, int k, int flags,
                             double* stats_dev, ctis_reduce_fn reduce, void* reduce_ctx,
                             void* stream) {
    int rc = check_plan(P);
    if (rc) return rc;
    if (!g_dev || !f_dev) return fail(CTIS_ERR_INVALID_ARG, "NULL device pointer");
    if (k < 0) return fail(CTIS_ERR_INVALID_ARG, "k must be >= 0");
    if ((flags & CTIS_INIT_ONES) && (flags & CTIS_INIT_HTG))
        return fail(CTIS_ERR_INVALID_ARG, "CTIS_INIT_ONES and CTIS_INIT_HTG are exclusive");
    if (flags & ~(CTIS_INIT_ONES | CTIS_INIT_HTG))
        return fail(CTIS_ERR_INVALID_ARG, "unknown flags 0x%x", flags);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!P->d_shard_q) {
        rc = dmalloc(P, reinterpret_cast<void**>(&P->d_shard_q), sizeof(float) * static_cast<size_t>(P->n));
        if (!rc)
            rc = dmalloc(P, reinterpret_cast<void**>(&P->d_shard_part),
                         sizeof(double) * kNumStats * shard_ratio_blocks());
        if (rc) return rc;
    }
    rc = zero_u(P, st);
    if (rc) return rc;
    if (flags & CTIS_INIT_ONES) {
        rc = scatter_f(P, nullptr, P->dtype, 1.0f, st);
    } else if (flags & CTIS_INIT_HTG) {
        rc = scatter_u(P, g_dev, st);
        if (rc) return rc;
        GatherParams p = base_params(P, P->adj);
        p.mode = kEpiSet;
        p.out_w = P->a;
        p.out_h = P->alpha;
        set_f_copies(P, p);
        rc = enqueue_adjoint(P, p, st);
    } else {
        rc = scatter_f(P, f_dev, P->dtype, 0.f, st);
    }
    if (rc) return rc;
    GatherParams pq = base_params(P, P->fwd);   // the slice's partial image
    pq.mode = kEpiRaw;
    pq.out_w = P->gamma;
    pq.out_h = P->xi;
    pq.out_f32 = P->d_shard_q;
    pq.out_pitch = P->gamma;
    pq.out_plane_stride = 0;
    GatherParams pa = base_params(P, P->adj);
    pa.mode = kEpiUpdate;
    pa.out_w = P->a;
    pa.out_h = P->alpha;
    set_f_copies(P, pa);
    for (int it = 0; it <= k; ++it) {
        if (it == k && !stats_dev) break;
        rc = enqueue_forward(P, pq, st);
        if (rc) return rc;
        if (reduce) {
            const int r = reduce(P->d_shard_q, P->n, reduce_ctx, stream);
            if (r != 0)
                return fail(CTIS_ERR_CUDA, "the reduction callback returned %d at iteration %d", r, it);
        }
        CTIS_CUDA(launch_shard_ratio(P->d_u, P->u_copy_stride, P->u_copies, P->g_pitch,
                                     P->d_shard_q, g_dev, P->gamma, P->xi, P->d_shard_part,
                                     stats_dev ? stats_dev + static_cast<int64_t>(it) * kNumStats
                                               : nullptr,
                                     st));
        if (it == k) break;
        rc = enqueue_adjoint(P, pa, st);
        if (rc) return rc;
    }
    CTIS_CUDA(launch_gather_copy0(P->dtype, f_dev, P->d_fwork, P->a_pitch,
                                  static_cast<int64_t>(P->a_pitch) * P->alpha, P->a, P->alpha,
                                  P->w, st));
    return CTIS_OK;
}

int ctis_plan_time_launches(ctis_plan* P, const float* g_dev, int reps, double* fwd_ms,
                            double* adj_ms, void* stream) {
    int rc = check_plan(P);
    if (rc) return rc;
    if (!g_dev || reps < 1 || !fwd_ms || !adj_ms)
        return fail(CTIS_ERR_INVALID_ARG, "g_dev, fwd_ms or adj_ms is NULL, or reps < 1");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CTIS_CUDA(cudaStreamSynchronize(st));
    // the EM loop's operands: f = 1 in the datacube copies, u from g
    rc = scatter_f(P, nullptr, P->dtype, 1.0f, st);
    if (!rc) rc = zero_u(P, st);
    if (!rc) rc = scatter_u(P, g_dev, st);
    if (rc) return rc;
    auto launch = [&](bool forward) -> int {
        if (forward) {
            GatherParams p = base_params(P, P->fwd);
            p.mode = kEpiRatio;
            p.out_w = P->gamma;
            p.out_h = P->xi;
            p.out_f32 = P->d_u;
            p.out_pitch = P->g_pitch;
            p.out_copy_stride = P->u_copy_stride;
            p.out_copies = P->u_copies;
            p.g = g_dev;
            p.g_pitch = P->gamma;
            p.with_stats = 1;   // tile statistics, as inside the EM loop
            return enqueue_forward(P, p, st);
        }
        GatherParams p = base_params(P, P->adj);
        p.mode = kEpiUpdate;
        p.out_w = P->a;
        p.out_h = P->alpha;
        set_f_copies(P, p);
        return enqueue_adjoint(P, p, st);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CTIS_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(CTIS_ERR_CUDA, "cudaEventCreate failed");
    }
    for (int side = 0; side < 2 && !rc; ++side) {
        const bool forward = side == 0;
        for (int r = 0; r < 2 && !rc; ++r) rc = launch(forward);   // warm-up
        cudaError_t e = rc ? cudaSuccess : cudaEventRecord(e0, st);
        for (int r = 0; r < reps && !rc && e == cudaSuccess; ++r) rc = launch(forward);
        if (!rc && e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (!rc && e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (!rc && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (!rc && e != cudaSuccess) rc = cuda_fail(e, "timing back-to-back launches");
        (forward ? *fwd_ms : *adj_ms) = static_cast<double>(ms) / reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

int ctis_plan_check(const ctis_plan* P, void* stream) {
    int rc = check_plan(P);
    if (rc) return rc;
    CTIS_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int flag = 0;
    CTIS_CUDA(cudaMemcpy(&flag, P->d_counters + 3, sizeof(int), cudaMemcpyDeviceToHost));
    if (P->batch) {   // the batched launches keep their own counters
        int bflag = 0;
        CTIS_CUDA(cudaMemcpy(&bflag, P->batch->d_counters + 3, sizeof(int), cudaMemcpyDeviceToHost));
        if (bflag) CTIS_CUDA(cudaMemset(P->batch->d_counters + 3, 0, sizeof(int)));
        flag |= bflag;
    }
    if (flag) {
        CTIS_CUDA(cudaMemset(P->d_counters + 3, 0, sizeof(int)));
        return fail(CTIS_ERR_TIMEOUT, "a kernel's bounded wait gave up (flag %d)", flag);
    }
    return CTIS_OK;
}

}  // extern "C"
