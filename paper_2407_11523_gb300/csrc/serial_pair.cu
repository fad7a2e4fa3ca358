// Two-shots-per-warp serial-schedule kernels (serial_kernel.cuh), in a
// translation unit of their own so that they compile in parallel with the
// one-shot kernels.
#include "serial_kernel.cuh"

namespace bpq {
namespace sk {

SerialKernelFn pick_serial_pair(int variant, int layout) {
#define BPQ_SERIAL_PAIR_CASE(V)                                                        \
    case V:                                                                            \
        return layout == 2   ? serial_pair_kernel<V, true, true>                       \
               : layout == 1 ? serial_pair_kernel<V, true, false>                      \
                             : serial_pair_kernel<V, false, false>;
    switch (variant) {
        BPQ_SERIAL_PAIR_CASE(BPQ_PLAIN)
        BPQ_SERIAL_PAIR_CASE(BPQ_MOMENTUM)
        BPQ_SERIAL_PAIR_CASE(BPQ_ADAGRAD)
        BPQ_SERIAL_PAIR_CASE(BPQ_EWAINIT)
    }
#undef BPQ_SERIAL_PAIR_CASE
    return nullptr;
}

}  // namespace sk
}  // namespace bpq
