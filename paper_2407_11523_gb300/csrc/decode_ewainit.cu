// Decode kernels of the ewainit variant (one translation unit per variant so
// that they compile in parallel).
#include "decode_kernel.cuh"

namespace bpq {
BPQ_DEFINE_PICK(pick_ewainit, BPQ_EWAINIT)
}  // namespace bpq
