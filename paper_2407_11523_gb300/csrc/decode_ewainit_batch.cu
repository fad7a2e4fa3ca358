// The batched many-code kernel of EWAInit-BP (decode_kernel.cuh).
#include "decode_kernel.cuh"

namespace bpq {
BPQ_DEFINE_PICK_BATCH(pick_ewainit_batch, BPQ_EWAINIT)
}  // namespace bpq
