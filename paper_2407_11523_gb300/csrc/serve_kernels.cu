// Instantiations of the slot-granular serving kernel for the four variants
// (a translation unit of its own so that it compiles in parallel with the
// decode kernels).
#include "serve_kernel.cuh"

namespace bpq {

ServeKernelFn pick_serve_kernel(int variant) {
    switch (variant) {
        case BPQ_PLAIN: return dk::decode_serve_kernel<BPQ_PLAIN, 2>;
        case BPQ_MOMENTUM: return dk::decode_serve_kernel<BPQ_MOMENTUM, 2>;
        case BPQ_ADAGRAD: return dk::decode_serve_kernel<BPQ_ADAGRAD, 2>;
        case BPQ_EWAINIT: return dk::decode_serve_kernel<BPQ_EWAINIT, 2>;
    }
    return nullptr;
}

}  // namespace bpq
