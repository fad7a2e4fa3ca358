"""bpq_decode_host_noalloc: the decode entry point for callers that cannot
allocate device memory (for example a real-time decoding loop that may not
allocate once running).  It stages inputs and outputs in a fixed array inside
the library instead of caller- or library-allocated device memory, so its
results must equal those of bpq_decode_host on the same inputs.

This file is collected last (test_zz_...) so that a run stopping at the first
failure has already run every other test; it also passes on its own in a
fresh process."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_decode_host_on_two_calls():
    """Two calls in a row on different batches give bpq_decode_host's
    results, and the second call (the kernel's module already loaded by the
    first) leaves the device's free memory unchanged."""
    import paper_2407_11523_gb300 as bpq

    L = bpq.lib()
    t = bpq.Tanner("toric", 15).upload()
    max_shots = L.bpq_decode_host_noalloc_max_shots(t.handle)
    assert max_shots >= 8192
    stream = torch.cuda.current_stream()
    params = bpq.make_params("ewainit", alpha=0.5)
    calls = []
    for p, B, seed in [(0.08, 4000, 11), (0.12, 2500, 12)]:
        _, syn = bpq.sample(t, p / 3, p / 3, p / 3, seed=seed, shot0=0, B=B)
        syn_h = syn.cpu().pin_memory()
        prior_h = bpq.prior_tensor(t, p / 3, p / 3, p / 3).cpu().pin_memory()
        ref = bpq.decode_host(t, syn_h, prior_h, "ewainit", params=params, max_iter=100)
        outs = (torch.zeros((B, t.N), dtype=torch.uint8, pin_memory=True),
                torch.zeros(B, dtype=torch.uint8, pin_memory=True),
                torch.zeros(B, dtype=torch.uint8, pin_memory=True))
        calls.append((B, syn_h, prior_h, ref, outs))
    torch.cuda.synchronize()
    free = []
    for B, syn_h, prior_h, ref, (est, conv, iters) in calls:
        rc = L.bpq_decode_host_noalloc(t.handle, _p(syn_h), _p(prior_h), bpq.EWAINIT, ctypes.byref(params), 100, B,
                                       _p(est), _p(conv), _p(iters), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, L.bpq_last_error()
        free.append(torch.cuda.mem_get_info()[0])
    assert free[1] == free[0], free
    for k, (B, syn_h, prior_h, ref, (est, conv, iters)) in enumerate(calls):
        # integer outputs of the same kernel on the same inputs: identical
        assert torch.equal(est, ref[0]) and torch.equal(conv, ref[1]) and torch.equal(iters, ref[2]), k
        assert int(conv.sum()) > 0


def test_noalloc_rejects_oversized_batch():
    import paper_2407_11523_gb300 as bpq

    L = bpq.lib()
    t = bpq.Tanner("toric", 15).upload()
    B = L.bpq_decode_host_noalloc_max_shots(t.handle) + 1
    syn = torch.zeros((B, t.W), dtype=torch.int32, pin_memory=True)
    prior = torch.full((t.N, 3), 0.01, dtype=torch.float32, pin_memory=True)
    out = torch.zeros((B, t.N), dtype=torch.uint8, pin_memory=True)
    flags = torch.zeros(B, dtype=torch.uint8, pin_memory=True)
    rc = L.bpq_decode_host_noalloc(t.handle, _p(syn), _p(prior), bpq.EWAINIT, None, 100, B, _p(out), _p(flags),
                                   _p(flags), None)
    assert rc == -1
    assert b"8 MiB" in L.bpq_last_error()
