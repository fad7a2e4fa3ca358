"""GB300-native GF(4) belief-propagation decoding of surface-code syndromes:
plain LLR-BP4, Momentum-BP, AdaGrad-BP and EWAInit-BP under the flooding
schedule, AEWA-BP, and the serial schedule (Chen, Yi, Liang, Wang,
"Improved Belief Propagation Decoding Algorithms for Surface Codes").

The compute lives in libbpq.so (CUDA for sm_103a, C ABI in include/bpq.h);
this package is its thin Python binding.
"""
from ._binding import (  # noqa: F401
    ADAGRAD, AEWA, CODES, EWAINIT, MOMENTUM, PLAIN, PLANAR, TORIC, VARIANTS, XZZX,
    BPQError, BatchPlan, Params, Server, Tanner, autotune, autotune_batch, check_logical, decode, decode_host,
    decode_host_bytes, decode_status,
    decode_trace, default_params, lib, make_params, prior_rows, prior_tensor, probe_peak, sample, unrolled_loss,
    unrolled_posterior, workspace,
)
