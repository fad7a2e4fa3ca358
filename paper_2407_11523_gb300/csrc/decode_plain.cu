// Decode kernels of the plain variant (one translation unit per variant so
// that they compile in parallel).
#include "decode_kernel.cuh"

namespace bpq {
BPQ_DEFINE_PICK(pick_plain, BPQ_PLAIN)
}  // namespace bpq
