// Decode kernels of the momentum variant for split tables without padding
// (bpq_tanner::full), in a translation unit of their own.
#include "decode_kernel.cuh"

namespace bpq {
BPQ_DEFINE_PICK_FULL(pick_momentum_full, BPQ_MOMENTUM)
}  // namespace bpq
