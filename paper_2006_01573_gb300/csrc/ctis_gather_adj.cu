// Adjoint projector kernels (Eq. 14): voxel tiles of one wavelength, input
// windows from the x-shifted FPA copies, cluster weights as stored.
// Epilogues: H^T r as is (ctis_adjoint), or the EM update
// f <- f * (H^T u) / h (Eq. 2) written into the datacube copies, which with
// no previous f sets f = H^T g (the initial guess).
#include "ctis_gather.cuh"

namespace ctis {
namespace {

template <class G, typename TIn, typename TF, int MODE>
__global__ void __launch_bounds__(G::THREADS, G::MIN_BLOCKS)
    adjoint_kernel(const __grid_constant__ CUtensorMap tm_win, const GatherParams p) {
    gather_body<G, TIn, TF, MODE>(tm_win, p);
}

// Calls fn(kernel, G{}) for the instantiation serving (K, dtype, mode); the
// initial-guess mode shares the update instantiation.
template <class Fn>
cudaError_t dispatch_adj(int K, int dtype, int mode, Fn&& fn) {
    auto by_k = [&](auto tin, auto tf) -> cudaError_t {
        using TIn = decltype(tin);
        using TF = decltype(tf);
        auto by_mode = [&](auto geo) -> cudaError_t {
            using G = decltype(geo);
            if (mode == kEpiUpdate || mode == kEpiSet)
                return fn(adjoint_kernel<G, TIn, TF, kEpiUpdate>, geo);
            if (mode == kEpiRaw) return fn(adjoint_kernel<G, TIn, TF, kEpiRaw>, geo);
            return cudaErrorInvalidValue;
        };
        switch (K) {
            case 1: return by_mode(GeoOf<1, TIn, TF, false>{});
            case 3: return by_mode(GeoOf<3, TIn, TF, false>{});
            case 5: return by_mode(GeoOf<5, TIn, TF, false>{});
            default: return cudaErrorInvalidValue;
        }
    };
    // the adjoint reads the float32 FPA copies; bfloat16 plans store f in bfloat16
    if (dtype == kDtypeBF16) return by_k(float{}, __nv_bfloat16{});
    return by_k(float{}, float{});
}

}  // namespace

cudaError_t gather_prepare_adj(int K, int dtype, int* blocks_per_sm) {
    int lo = 1 << 30;
    for (int mode : {kEpiRaw, kEpiUpdate}) {
        int b = 0;
        const cudaError_t e = dispatch_adj(K, dtype, mode, [&](auto kern, auto geo) {
            return prepare_kernel<decltype(geo)>(kern, &b);
        });
        if (e != cudaSuccess) return e;
        lo = b < lo ? b : lo;
    }
    *blocks_per_sm = lo;
    return cudaSuccess;
}

cudaError_t gather_launch_adj(int K, int dtype, const CUtensorMap& win, const GatherParams& p,
                              cudaStream_t stream) {
    return dispatch_adj(K, dtype, p.mode, [&](auto kern, auto geo) {
        return launch_kernel<decltype(geo)>(kern, win, p, stream);
    });
}

#ifdef CTIS_DEBUG_BOUNDS
cudaError_t debug_arm_adj(const DbgRanges& r) { return cudaMemcpyToSymbol(g_dbg, &r, sizeof r); }
#endif

}  // namespace ctis
