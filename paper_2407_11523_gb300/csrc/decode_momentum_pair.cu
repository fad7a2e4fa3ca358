// Two-shots-per-thread decode kernels of the momentum variant (split tables, with
// and without padding), in a translation unit of their own.
#include "decode_pair.cuh"

namespace bpq {
BPQ_DEFINE_PICK_PAIR(pick_momentum_pair, BPQ_MOMENTUM, false)
BPQ_DEFINE_PICK_PAIR(pick_momentum_pair_full, BPQ_MOMENTUM, true)
}  // namespace bpq
