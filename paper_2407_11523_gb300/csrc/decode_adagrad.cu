// Decode kernels of the adagrad variant (one translation unit per variant so
// that they compile in parallel).
#include "decode_kernel.cuh"

namespace bpq {
BPQ_DEFINE_PICK(pick_adagrad, BPQ_ADAGRAD)
}  // namespace bpq
