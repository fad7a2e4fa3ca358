// Bounds-checked copies of the one-code decode kernels (one and two shots per
// thread; plain, Momentum, AdaGrad and EWAInit BP; one or two nodes per
// thread; every table layout), compiled with BPQ_DEBUG into namespace
// bpq::dk_debug.  bpq_set_debug_checks selects them.
#define BPQ_DEBUG 1
#define dk dk_debug
#include "decode_kernel.cuh"
#include "decode_pair.cuh"
#undef dk

namespace bpq {

namespace {

template <int V>
DecodeKernelFn pick_debug_v(int npt, bool pairs, int layout) {
    if (pairs) {
        if (layout == 2) return npt == 1 ? dk_debug::decode_pair_kernel<V, 1, true> : dk_debug::decode_pair_kernel<V, 2, true>;
        if (layout == 1) return npt == 1 ? dk_debug::decode_pair_kernel<V, 1, false> : dk_debug::decode_pair_kernel<V, 2, false>;
        return nullptr;
    }
    switch (layout) {
        case 2: return npt == 1 ? dk_debug::decode_kernel<V, 1, false, true, true> : dk_debug::decode_kernel<V, 2, false, true, true>;
        case 1: return npt == 1 ? dk_debug::decode_kernel<V, 1, false, true, false> : dk_debug::decode_kernel<V, 2, false, true, false>;
        default: return npt == 1 ? dk_debug::decode_kernel<V, 1, false, false, false> : dk_debug::decode_kernel<V, 2, false, false, false>;
    }
}

}  // namespace

DecodeKernelFn pick_debug(int variant, int npt, bool pairs, int layout) {
    if (npt < 1 || npt > 2) return nullptr;
    switch (variant) {
        case BPQ_PLAIN: return pick_debug_v<BPQ_PLAIN>(npt, pairs, layout);
        case BPQ_MOMENTUM: return pick_debug_v<BPQ_MOMENTUM>(npt, pairs, layout);
        case BPQ_ADAGRAD: return pick_debug_v<BPQ_ADAGRAD>(npt, pairs, layout);
        case BPQ_EWAINIT: return pick_debug_v<BPQ_EWAINIT>(npt, pairs, layout);
    }
    return nullptr;
}

}  // namespace bpq
