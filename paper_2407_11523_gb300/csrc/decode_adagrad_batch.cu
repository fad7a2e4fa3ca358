// The batched many-code kernel of AdaGrad-BP (decode_kernel.cuh).
#include "decode_kernel.cuh"

namespace bpq {
BPQ_DEFINE_PICK_BATCH(pick_adagrad_batch, BPQ_ADAGRAD)
}  // namespace bpq
