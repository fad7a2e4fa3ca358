// Two-shots-per-thread decode kernels of the adagrad variant (split tables, with
// and without padding), in a translation unit of their own.
#include "decode_pair.cuh"

namespace bpq {
BPQ_DEFINE_PICK_PAIR(pick_adagrad_pair, BPQ_ADAGRAD, false)
BPQ_DEFINE_PICK_PAIR(pick_adagrad_pair_full, BPQ_ADAGRAD, true)
}  // namespace bpq
