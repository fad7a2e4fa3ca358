"""Decoding servers: Poisson traces of single-shot requests over several
codes.  Lane server (micro-batches per stream) and slot server (a persistent
kernel whose shot groups take the next request as soon as they finish a
shot): each request's result is the same as decoding it alone, completion
follows arrival, and served results agree with the FP64 oracle."""
import os

import numpy as np
import pytest
import torch

import oracle
from oracle import codes as codes_mod

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


def check_alone(bpq, codes, priors, code_of, syn_list, ests, conv, iters):
    """Every served result equals bpq_decode's result for that syndrome."""
    for c, t in enumerate(codes):
        idx = np.nonzero(code_of == c)[0]
        if idx.size == 0:
            continue
        syn = torch.from_numpy(np.stack([syn_list[r] for r in idx]).view(np.int32)).cuda()
        e, cv, it = (x.cpu().numpy() for x in bpq.decode(t, syn, priors[c], "ewainit", max_iter=100))
        for k, r in enumerate(idx):
            assert (ests[r] == e[k]).all() and conv[r] == cv[k] and iters[r] == it[k], (c, r)


@pytest.mark.parametrize("rate,slots", [(2e4, 64), (5e5, 1024), (1e7, 4)])
def test_slot_server_results_equal_alone(bpq, rate, slots):
    """Slot-granular serving: each request is taken by the next shot group
    that finishes a shot; results equal decoding each syndrome alone, also
    with rings of only 4 slots per code (admission waits for free slots)."""
    codes = [bpq.Tanner("planar", 5), bpq.Tanner("planar", 9), bpq.Tanner("xzzx", 7), bpq.Tanner("planar", 17)]
    ch = oracle.depolarizing(0.05)
    priors = [bpq.prior_tensor(t, *ch) for t in codes]
    srv = bpq.Server(codes, priors, "ewainit", max_iter=100, mode="slots", slots_per_code=slots)
    R = 3000
    code_of, arrival, syn_list = make_trace(bpq, codes, R, rate, seed=31)
    ests, conv, iters, done, ctas = srv.replay(code_of, arrival, syn_list)
    assert (done >= arrival).all() and ctas >= 152
    assert srv.launches() >= 1
    check_alone(bpq, codes, priors, code_of, syn_list, ests, conv, iters)
    # a second trace on the same server (rings and counters start afresh)
    code_of, arrival, syn_list = make_trace(bpq, codes, 500, rate, seed=32)
    ests, conv, iters, done, _ = srv.replay(code_of, arrival, syn_list)
    check_alone(bpq, codes, priors, code_of, syn_list, ests, conv, iters)


def test_slot_server_direct_and_ring_outputs_agree(bpq):
    """Page-locked outputs at 16-byte aligned offsets (the kernel writes each
    result in place) and pageable outputs (results through the rings, copied
    by the host) give the same results, equal to decoding alone; planar
    d = 17 and 9 have N = 545 and 145, so estimates end in a partial
    16-byte chunk."""
    codes = [bpq.Tanner("planar", 17), bpq.Tanner("xzzx", 5), bpq.Tanner("planar", 9)]
    ch = oracle.depolarizing(0.05)
    priors = [bpq.prior_tensor(t, *ch) for t in codes]
    srv = bpq.Server(codes, priors, "ewainit", max_iter=100, mode="slots", slots_per_code=32)
    code_of, arrival, syn_list = make_trace(bpq, codes, 1500, 2e5, seed=35)
    direct = srv.replay(code_of, arrival, syn_list, pinned=True)
    ring = srv.replay(code_of, arrival, syn_list, pinned=False)
    for r in range(code_of.size):
        assert (direct[0][r] == ring[0][r]).all()
    assert (direct[1] == ring[1]).all() and (direct[2] == ring[2]).all()
    check_alone(bpq, codes, priors, code_of, syn_list, *direct[:3])


def test_slot_server_unaligned_outputs_use_the_rings(bpq):
    """Page-locked outputs whose estimate buffer starts one byte past a
    16-byte boundary, at offsets that are multiples of 16: the kernel's
    16-byte stores there would be misaligned, so the server takes the rings
    (the host copies the results out).  Called through the C ABI, since the
    binding allocates aligned buffers; the results equal the in-place ones."""
    import ctypes

    from paper_2407_11523_gb300 import _binding as B

    codes = [bpq.Tanner("planar", 9), bpq.Tanner("xzzx", 5)]
    ch = oracle.depolarizing(0.05)
    priors = [bpq.prior_tensor(t, *ch) for t in codes]
    srv = bpq.Server(codes, priors, "ewainit", max_iter=100, mode="slots", slots_per_code=32)
    code_of, arrival, syn_list = make_trace(bpq, codes, 600, 2e5, seed=36)
    ref = srv.replay(code_of, arrival, syn_list, pinned=True)
    R = code_of.size
    Ns = [codes[c].N for c in code_of]
    stride = [(n + 15) & ~15 for n in Ns]
    est_off = np.zeros(R, dtype=np.int64)
    est_off[1:] = np.cumsum(stride)[:-1]
    syn_off = np.zeros(R, dtype=np.int64)
    syn_off[1:] = np.cumsum([len(x) for x in syn_list])[:-1]
    syn = np.ascontiguousarray(np.concatenate(syn_list).astype(np.uint32))
    n_est = int(sum(stride))
    base = torch.zeros(n_est + 16, dtype=torch.uint8, pin_memory=True).numpy()
    assert base.ctypes.data % 16 == 0
    est = base[1:1 + n_est]
    conv = torch.zeros(R, dtype=torch.uint8, pin_memory=True).numpy()
    iters = torch.zeros(R, dtype=torch.uint8, pin_memory=True).numpy()
    done = np.zeros(R, dtype=np.float64)
    code32 = np.ascontiguousarray(code_of, dtype=np.int32)
    arr = np.ascontiguousarray(arrival, dtype=np.float64)
    used = ctypes.c_int()
    rc = B.lib().bpq_server_replay(srv._h, R, B._ptr(code32), B._ptr(arr), B._ptr(syn), B._ptr(syn_off), B._ptr(est),
                                   B._ptr(est_off), n_est, B._ptr(conv), B._ptr(iters), B._ptr(done),
                                   ctypes.byref(used))
    assert rc == 0, B.lib().bpq_last_error()
    for r in range(R):
        assert (est[est_off[r]:est_off[r] + Ns[r]] == ref[0][r]).all()
    assert (conv == ref[1]).all() and (iters == ref[2]).all()


def test_slot_server_relaunches_after_idle(bpq):
    """With a 50 us idle limit and 3 ms gaps between bursts, the serving
    kernel returns (a bounded wait, status 2) between bursts and the host
    relaunches it; every request is still served with its alone result."""
    codes = [bpq.Tanner("planar", 7), bpq.Tanner("xzzx", 5)]
    ch = oracle.depolarizing(0.05)
    priors = [bpq.prior_tensor(t, *ch) for t in codes]
    srv = bpq.Server(codes, priors, "ewainit", max_iter=100, mode="slots", slots_per_code=256, idle_timeout_us=50)
    rng = np.random.default_rng(3)
    R = 400
    code_of = rng.integers(0, 2, size=R)
    arrival = (np.arange(R) // 50) * 3e-3 + (np.arange(R) % 50) * 1e-6
    syn_list = [None] * R
    for c, t in enumerate(codes):
        idx = np.nonzero(code_of == c)[0]
        _, syn = bpq.sample(t, *ch, seed=40 + c, shot0=0, B=int(idx.size))
        for k, r in enumerate(idx):
            syn_list[r] = syn.cpu().numpy().view(np.uint32)[k]
    ests, conv, iters, done, _ = srv.replay(code_of, arrival, syn_list)
    assert srv.launches() >= 3
    check_alone(bpq, codes, priors, code_of, syn_list, ests, conv, iters)


def test_slot_server_results_match_oracle(bpq):
    """Served results against the FP64 oracle's decode of each syndrome, on a
    Poisson trace over planar and XZZX codes of distance 5 to 15 at p = 0.05
    (EWAInit-BP, at most 100 iterations).  On the precision-robust requests
    (the oracle's binary32-storage build agrees with FP64) that the oracle
    converges, convergence and logical outcome equal on at least 99.9 % and
    estimates on at least 99.5 %."""
    kinds = [(k, d) for k in ("planar", "xzzx") for d in (5, 7, 9, 11, 13, 15)]
    codes = [bpq.Tanner(k, d) for k, d in kinds]
    ch = oracle.depolarizing(0.05)
    priors = [bpq.prior_tensor(t, *ch) for t in codes]
    srv = bpq.Server(codes, priors, "ewainit", max_iter=100, mode="slots", slots_per_code=128)
    R = 1200
    rng = np.random.default_rng(51)
    code_of = rng.integers(0, len(codes), size=R)
    arrival = np.cumsum(rng.exponential(1.0 / 2e5, size=R))
    syn_list, err_of = [None] * R, [None] * R
    for c, t in enumerate(codes):
        idx = np.nonzero(code_of == c)[0]
        if idx.size == 0:
            continue
        err, syn = bpq.sample(t, *ch, seed=600 + c, shot0=0, B=int(idx.size))
        s, e = syn.cpu().numpy().view(np.uint32), err.cpu().numpy()
        for k, r in enumerate(idx):
            syn_list[r], err_of[r] = s[k], e[k]
    ests, conv, iters, done, _ = srv.replay(code_of, arrival, syn_list)
    robust_conv = same_conv = same_fail = same_est = 0
    nthreads = os.cpu_count() or 4
    for c, t in enumerate(codes):
        idx = np.nonzero(code_of == c)[0]
        if idx.size == 0:
            continue
        H = t.dense()
        bits = np.stack([np.unpackbits(syn_list[r].view(np.uint8), bitorder="little")[:t.M] for r in idx])
        prior = np.tile(np.asarray(ch, dtype=np.float32).astype(np.float64), (t.N, 1))
        e64, c64, _ = oracle.decode(H, bits, prior, "ewainit", max_iter=100, nthreads=nthreads)
        e32, c32, _ = oracle.decode(H, bits, prior, "ewainit", max_iter=100, nthreads=nthreads, precision="f32")
        errs = np.stack([err_of[r] for r in idx])
        f64 = codes_mod.logical_failure(H, errs, e64)[0]
        f32 = codes_mod.logical_failure(H, errs, e32)[0]
        served = np.stack([ests[r] for r in idx])
        fs = codes_mod.logical_failure(H, errs, served)[0]
        rob = c64 & c32 & (f64 == f32) & (e64 == e32).all(axis=1)
        cs = conv[idx].astype(bool)
        robust_conv += int(rob.sum())
        same_conv += int((cs[rob]).sum())
        same_fail += int((fs[rob] == f64[rob]).sum())
        same_est += int((served[rob] == e64[rob]).all(axis=1).sum())
    assert robust_conv >= 0.9 * R
    assert same_conv >= 0.999 * robust_conv and same_fail >= 0.999 * robust_conv
    assert same_est >= 0.995 * robust_conv
