// Decode kernels of the plain variant for split tables without padding
// (bpq_tanner::full), in a translation unit of their own.
#include "decode_kernel.cuh"

namespace bpq {
BPQ_DEFINE_PICK_FULL(pick_plain_full, BPQ_PLAIN)
}  // namespace bpq
