"""Parity of the serial-schedule CUDA decoder (bpq_decode_serial) with the
FP64 oracle's serial schedule on identical inputs: messages within 1e-4 for
five sweeps, decisions on >= 99.9 % of shots, LERs inside each other's
2-sigma intervals (the same bars as the parallel decoder's)."""
import numpy as np
import pytest
import torch

import oracle
from inputs import random_priors, random_syndromes, random_tree_code, trapping_set_code
from oracle import codes
from test_gpu_parity import MSG_TOL, NTHREADS, f32, gpu_inputs, ler_interval

pytestmark = pytest.mark.gpu

VARIANTS = ["plain", "momentum", "adagrad", "ewainit"]


@pytest.fixture(scope="module")
def bpq():
    import paper_2407_11523_gb300 as bpq
    assert torch.cuda.is_available()
    return bpq


def sensitivity(H, s, prior, variant, T, b):
    """Largest change of any serial oracle message under an 8-ulp prior
    perturbation (three sign patterns): the method's own conditioning."""
    rng = np.random.default_rng(2000 + b)
    r0 = oracle.trace(H, s, f32(prior), variant=variant, T=T, schedule="serial")
    worst = 0.0
    for _ in range(3):
        pp = f32(prior) * (1 + 2.0 ** -20 * rng.choice([-1.0, 1.0], size=np.shape(prior)))
        r1 = oracle.trace(H, s, pp, variant=variant, T=T, schedule="serial")
        worst = max(worst, np.abs(r0["m_v2c"] - r1["m_v2c"]).max(), np.abs(r0["m_c2v"] - r1["m_c2v"]).max())
    return worst


def check_messages(bpq, t, H, syn_bits, prior, variant, T=5, min_strict=1.0):
    syn, pri = gpu_inputs(bpq, t, syn_bits, prior)
    rec = {k: v.cpu().numpy() for k, v in bpq.decode_trace(t, syn, pri, variant=variant, T=T,
                                                            schedule="serial").items()}
    strict = 0
    for b in range(syn_bits.shape[0]):
        ref = oracle.trace(H, syn_bits[b], f32(prior), variant=variant, T=T, schedule="serial")
        d = max(np.abs(rec["m_v2c"][b] - ref["m_v2c"]).max(), np.abs(rec["m_c2v"][b] - ref["m_c2v"]).max())
        tol = MSG_TOL
        if variant == "adagrad" and d > MSG_TOL:
            # AdaGrad's boosted step amplifies rounding where G ~ 0 (see the
            # parallel decoder's tests): bound by 10 x the oracle's own sensitivity
            tol = MSG_TOL + 10.0 * sensitivity(H, syn_bits[b], prior, variant, T, b)
        assert d <= tol, (variant, b, d, tol)
        if d <= MSG_TOL:
            strict += 1
            q = np.abs(rec["Q"][b] - ref["Q"])
            assert (q <= 4 * MSG_TOL + 1e-6 * np.abs(ref["Q"])).all(), (variant, b, q.max())
            assert (rec["dec"][b] == ref["dec"]).mean() >= 0.99
    need = 1.0 if variant != "adagrad" else min_strict
    assert strict >= need * syn_bits.shape[0], (variant, strict)


@pytest.mark.parametrize("variant", VARIANTS)
def test_serial_messages_planar_d5(bpq, variant):
    t = bpq.Tanner("planar", 5)
    H = t.dense()
    ch = oracle.depolarizing(0.05)
    _, s = oracle.sample(H, *ch, seed=0x5E0, shot0=0, B=200)
    check_messages(bpq, t, H, s, np.tile(ch, (t.N, 1)), variant, min_strict=0.8)


@pytest.mark.parametrize("variant", VARIANTS)
def test_serial_messages_toric_and_xzzx(bpq, variant):
    t = bpq.Tanner("toric", 8)
    H = t.dense()
    ch = oracle.depolarizing(0.1)
    _, s = oracle.sample(H, *ch, seed=0x5E1, shot0=0, B=24)
    check_messages(bpq, t, H, s, np.tile(ch, (t.N, 1)), variant, min_strict=0.0)
    t = bpq.Tanner("xzzx", 7)
    H = t.dense()
    _, s = oracle.sample(H, *oracle.biased(0.08, 10.0), seed=0x5E2, shot0=0, B=24)
    check_messages(bpq, t, H, s, random_priors(t.N, seed=12, lo=0.005, hi=0.1), variant, min_strict=0.25)


@pytest.mark.parametrize("variant", VARIANTS)
def test_serial_messages_trees_and_trapping_set(bpq, variant):
    for seed in range(4):
        H = random_tree_code(8, seed=710 + seed)
        t = bpq.Tanner(H=H)
        check_messages(bpq, t, H, random_syndromes(H.shape[0], 8, seed=910 + seed),
                       random_priors(8, seed=810 + seed), variant, min_strict=0.5)
    H = trapping_set_code()
    t = bpq.Tanner(H=H)
    check_messages(bpq, t, H, np.array([[1, 0, 1, 0]], dtype=np.uint8), np.tile(oracle.depolarizing(0.01), (4, 1)),
                   variant, min_strict=0.0)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("spw", [1, 2])
def test_serial_decode_planar_d5_10k_shots(bpq, variant, spw):
    """Config C1 under the serial schedule, one and two shots per warp:
    decisions, flags, LER."""
    t = bpq.Tanner("planar", 5)
    t.set_serial_shots_per_warp(spw)
    H = t.dense()
    ch = oracle.depolarizing(0.05)
    B = 10000
    err_g, syn_g = bpq.sample(t, *ch, seed=0xB9E00000, shot0=0, B=B)
    est, conv, iters = bpq.decode(t, syn_g, bpq.prior_tensor(t, *ch), variant=variant, max_iter=50,
                                  schedule="serial")
    fail_g = bpq.check_logical(t, err_g, est)
    torch.cuda.synchronize()
    est, conv, iters, fail_g = (x.cpu().numpy() for x in (est, conv, iters, fail_g))
    e_ref, s_ref = oracle.sample(H, *ch, seed=0xB9E00000, shot0=0, B=B)
    prior = f32(np.tile(ch, (t.N, 1)))
    est_r, conv_r, iters_r = oracle.decode(H, s_ref, prior, variant=variant, max_iter=50, nthreads=NTHREADS,
                                           schedule="serial")
    same = (est == est_r).all(axis=1)
    if variant == "adagrad":
        rng = np.random.default_rng(7)
        stable = np.ones(B, dtype=bool)
        for _ in range(3):
            pp = prior * (1 + 2.0 ** -20 * rng.choice([-1.0, 1.0], size=prior.shape))
            stable &= (oracle.decode(H, s_ref, pp, variant, max_iter=50, nthreads=NTHREADS,
                                     schedule="serial")[0] == est_r).all(axis=1)
        assert stable.mean() >= 0.95
        assert same[stable].mean() >= 0.999, (same[stable].mean(), same.mean())
    else:
        assert same.mean() >= 0.999, (variant, same.mean())
    assert (conv.astype(bool) == conv_r).mean() >= (0.99 if variant == "adagrad" else 0.999)
    assert (iters[conv == 1] == iters_r[conv == 1]).mean() >= 0.99
    fail_r, _ = codes.logical_failure(H, e_ref, est_r)
    pg, sg = ler_interval(fail_g > 0)
    pr, sr = ler_interval(fail_r)
    assert abs(pg - pr) <= max(sg, sr), (variant, pg, pr)
    assert ((iters >= 1) & (iters <= 50)).all() and (iters[conv == 0] == 50).all()
    assert (fail_g[conv == 1] != 1).all() and (fail_g[conv == 0] == 1).all()


def test_serial_converges_in_fewer_sweeps_than_parallel_iterations(bpq):
    """Sec. II-B: the serial schedule converges faster; toric d = 8, p = 0.06."""
    t = bpq.Tanner("toric", 8)
    ch = oracle.depolarizing(0.06)
    _, syn = bpq.sample(t, *ch, seed=31, shot0=0, B=20000)
    prior = bpq.prior_tensor(t, *ch)
    _, c_s, i_s = bpq.decode(t, syn, prior, "plain", max_iter=50, schedule="serial")
    _, c_p, i_p = bpq.decode(t, syn, prior, "plain", max_iter=50)
    both = (c_s == 1) & (c_p == 1)
    assert i_s[both].float().mean() < i_p[both].float().mean()


def test_serial_partition_invariance_and_refusals(bpq):
    t = bpq.Tanner("planar", 9)
    ch = oracle.depolarizing(0.08)
    _, syn = bpq.sample(t, *ch, seed=2, shot0=0, B=3000)
    prior = bpq.prior_tensor(t, *ch)
    whole = bpq.decode(t, syn, prior, "ewainit", max_iter=60, schedule="serial")
    a = bpq.decode(t, syn[:1234].contiguous(), prior, "ewainit", max_iter=60, schedule="serial")
    b = bpq.decode(t, syn[1234:].contiguous(), prior, "ewainit", max_iter=60, schedule="serial")
    for w, x, y in zip(whole, a, b):
        assert torch.equal(w, torch.cat([x, y]))
    with pytest.raises(bpq.BPQError):
        bpq.decode(t, syn, prior, "aewa", max_iter=60, schedule="serial")
    empty = bpq.decode(t, syn[:0].contiguous(), prior, "ewainit", max_iter=60, schedule="serial")
    assert empty[0].shape == (0, t.N)


def serial_codes(bpq):
    """Split-layout codes (planar, toric without padding, XZZX) and codes in
    the generic layout (a tree code, a trapping set, a planar code with Y
    entries)."""
    from test_gpu_batch import y_rotated
    H7 = bpq.Tanner("planar", 7).dense()
    rng = np.random.default_rng(9)
    return [bpq.Tanner("planar", 5), bpq.Tanner("toric", 8), bpq.Tanner("xzzx", 7), bpq.Tanner("planar", 13),
            bpq.Tanner(H=random_tree_code(8, seed=5)), bpq.Tanner(H=trapping_set_code()),
            bpq.Tanner(H=y_rotated(H7, rng.choice(H7.shape[1], 30, replace=False)))]


@pytest.mark.parametrize("variant", VARIANTS)
def test_serial_two_shots_per_warp_equal_one(bpq, variant):
    """Two shots per warp give the one-shot kernel's results bit for bit
    (every step rounds alike), on split and generic layouts, with a ragged
    batch, max_iter 1 and 60, and a single shot (one half of the warp
    idle)."""
    ch = oracle.depolarizing(0.07)
    for k, t in enumerate(serial_codes(bpq)):
        _, syn = bpq.sample(t, *ch, seed=700 + k, shot0=0, B=1501)
        prior = bpq.prior_tensor(t, *ch)
        for max_iter, B in ((60, 1501), (1, 333), (60, 1)):
            s = syn[:B].contiguous()
            t.set_serial_shots_per_warp(1)
            one = bpq.decode(t, s, prior, variant, max_iter=max_iter, schedule="serial")
            t.set_serial_shots_per_warp(2)
            two = bpq.decode(t, s, prior, variant, max_iter=max_iter, schedule="serial")
            t.set_serial_shots_per_warp(0)
            for x, y in zip(one, two):
                assert torch.equal(x, y), (t.N, variant, max_iter, B)

