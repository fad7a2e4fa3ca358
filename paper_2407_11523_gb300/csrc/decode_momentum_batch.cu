// The batched many-code kernel of Momentum-BP (decode_kernel.cuh).
#include "decode_kernel.cuh"

namespace bpq {
BPQ_DEFINE_PICK_BATCH(pick_momentum_batch, BPQ_MOMENTUM)
}  // namespace bpq
