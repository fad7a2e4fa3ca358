// Decode kernels of AEWA-BP (the adaptive EWAInit-BP of Appendix C), one
// translation unit so that they compile in parallel with the others.
#include "decode_kernel.cuh"

namespace bpq {
BPQ_DEFINE_PICK_AEWA(pick_aewa)
}  // namespace bpq
