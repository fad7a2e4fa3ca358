// The batched many-code kernel of plain BP (decode_kernel.cuh).
#include "decode_kernel.cuh"

namespace bpq {
BPQ_DEFINE_PICK_BATCH(pick_plain_batch, BPQ_PLAIN)
}  // namespace bpq
