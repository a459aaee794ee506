// Forward projector kernels (Eqs. 1, 8, 12): FPA tiles, input windows from the
// x-shifted datacube copies, flipped cluster weights. Epilogues: H f as is
// (ctis_forward), or the EM ratio u = g / H f (Eq. 2) written into the FPA
// copies, with float64 statistics of the iteration.
#include "ctis_gather.cuh"

namespace ctis {
namespace {

template <class G, typename TIn, typename TF, int MODE>
__global__ void __launch_bounds__(G::THREADS, G::MIN_BLOCKS)
    forward_kernel(const __grid_constant__ CUtensorMap tm_win, const GatherParams p) {
    gather_body<G, TIn, TF, MODE>(tm_win, p);
}

// Calls fn(kernel, G{}) for the instantiation serving (K, dtype, mode, tile
// shape).
template <class Fn>
cudaError_t dispatch_fwd(int K, int dtype, int mode, int shape, Fn&& fn) {
    auto by_k = [&](auto tin, auto tf) -> cudaError_t {
        using TIn = decltype(tin);
        using TF = decltype(tf);
        auto by_mode = [&](auto geo) -> cudaError_t {
            using G = decltype(geo);
            if (mode == kEpiRatio) return fn(forward_kernel<G, TIn, TF, kEpiRatio>, geo);
            if (mode == kEpiRaw) return fn(forward_kernel<G, TIn, TF, kEpiRaw>, geo);
            return cudaErrorInvalidValue;
        };
        auto by_shape = [&](auto kc) -> cudaError_t {
            constexpr int KK = decltype(kc)::value;
            if (shape == 1) return by_mode(GeoOf<KK, TIn, TF, true, 1>{});
            if (shape == 0) return by_mode(GeoOf<KK, TIn, TF, true, 0>{});
            return cudaErrorInvalidValue;
        };
        switch (K) {
            case 1: return by_shape(std::integral_constant<int, 1>{});
            case 3: return by_shape(std::integral_constant<int, 3>{});
            case 5: return by_shape(std::integral_constant<int, 5>{});
            default: return cudaErrorInvalidValue;
        }
    };
    if (dtype == kDtypeBF16) return by_k(__nv_bfloat16{}, __nv_bfloat16{});
    return by_k(float{}, float{});
}

}  // namespace

cudaError_t gather_prepare_fwd(int K, int dtype, int shape, int* blocks_per_sm) {
    int lo = 1 << 30;
    for (int mode : {kEpiRaw, kEpiRatio}) {
        int b = 0;
        const cudaError_t e = dispatch_fwd(K, dtype, mode, shape, [&](auto kern, auto geo) {
            return prepare_kernel<decltype(geo)>(kern, &b);
        });
        if (e != cudaSuccess) return e;
        lo = b < lo ? b : lo;
    }
    *blocks_per_sm = lo;
    return cudaSuccess;
}

cudaError_t gather_launch_fwd(int K, int dtype, int shape, const CUtensorMap& win,
                              const GatherParams& p, cudaStream_t stream) {
    return dispatch_fwd(K, dtype, p.mode, shape, [&](auto kern, auto geo) {
        return launch_kernel<decltype(geo)>(kern, win, p, stream);
    });
}

#ifdef CTIS_DEBUG_BOUNDS
cudaError_t debug_arm_fwd(const DbgRanges& r) { return cudaMemcpyToSymbol(g_dbg, &r, sizeof r); }
#endif

}  // namespace ctis
