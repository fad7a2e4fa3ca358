// Two-shots-per-thread decode kernels of the ewainit variant (split tables, with
// and without padding), in a translation unit of their own.
#include "decode_pair.cuh"

namespace bpq {
BPQ_DEFINE_PICK_PAIR(pick_ewainit_pair, BPQ_EWAINIT, false)
BPQ_DEFINE_PICK_PAIR(pick_ewainit_pair_full, BPQ_EWAINIT, true)
}  // namespace bpq
