// Decode kernels of the momentum variant (one translation unit per variant so
// that they compile in parallel).
#include "decode_kernel.cuh"

namespace bpq {
BPQ_DEFINE_PICK(pick_momentum, BPQ_MOMENTUM)
}  // namespace bpq
