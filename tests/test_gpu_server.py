"""Continuous-batching server: a Poisson trace of single-shot requests over
several codes; each request's result is the same as decoding it alone, and
completion follows arrival."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bpq():
    import paper_2407_11523_gb300 as bpq
    return bpq


def make_trace(bpq, codes, R, rate, seed):
    rng = np.random.default_rng(seed)
    ch = oracle.depolarizing(0.05)
    code_of = rng.integers(0, len(codes), size=R)
    arrival = np.cumsum(rng.exponential(1.0 / rate, size=R))
    arrival -= arrival[0]
    syn_list = [None] * R
    for c, t in enumerate(codes):
        idx = np.nonzero(code_of == c)[0]
        if idx.size:
            _, syn = bpq.sample(t, *ch, seed=seed + c, shot0=0, B=int(idx.size))
            s = syn.cpu().numpy().view(np.uint32)
            for k, r in enumerate(idx):
                syn_list[r] = s[k]
    return code_of, arrival, syn_list


@pytest.mark.parametrize("rate,lanes,max_batch", [(2e4, 2, 64), (5e5, 4, 1024)])
def test_server_results_equal_alone(bpq, rate, lanes, max_batch):
    codes = [bpq.Tanner("planar", 5), bpq.Tanner("planar", 9), bpq.Tanner("xzzx", 7), bpq.Tanner("planar", 17)]
    ch = oracle.depolarizing(0.05)
    priors = [bpq.prior_tensor(t, *ch) for t in codes]
    srv = bpq.Server(codes, priors, "ewainit", max_iter=100, n_lanes=lanes, max_batch=max_batch)
    R = 3000
    code_of, arrival, syn_list = make_trace(bpq, codes, R, rate, seed=21)
    ests, conv, iters, done, used = srv.replay(code_of, arrival, syn_list)
    assert (done >= arrival).all() and used >= 1
    # every dispatch is one batched launch, of at most max_batch requests
    assert -(-R // max_batch) <= srv.launches() <= R
    # each request alone: a launch of one shot per request for a sample, and
    # the per-code batch (shot results are independent of the batch) for all
    for c, t in enumerate(codes):
        idx = np.nonzero(code_of == c)[0]
        syn = torch.from_numpy(np.stack([syn_list[r] for r in idx]).view(np.int32)).cuda()
        e, cv, it = (x.cpu().numpy() for x in bpq.decode(t, syn, priors[c], "ewainit", max_iter=100))
        for k, r in enumerate(idx):
            assert (ests[r] == e[k]).all() and conv[r] == cv[k] and iters[r] == it[k]
        for k in range(0, idx.size, max(1, idx.size // 10)):
            e1, c1, i1 = bpq.decode(t, syn[k:k + 1].contiguous(), priors[c], "ewainit", max_iter=100)
            assert (e1.cpu().numpy()[0] == ests[idx[k]]).all()
