// Two-shots-per-thread decode kernels of the plain variant (split tables, with
// and without padding), in a translation unit of their own.
#include "decode_pair.cuh"

namespace bpq {
BPQ_DEFINE_PICK_PAIR(pick_plain_pair, BPQ_PLAIN, false)
BPQ_DEFINE_PICK_PAIR(pick_plain_pair_full, BPQ_PLAIN, true)
}  // namespace bpq
