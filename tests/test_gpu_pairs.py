"""Two shots per thread (bpq_set_shots_per_thread): every thread works on the
same nodes of two shots, whose messages share float2 shared-memory slots and
packed f32x2 arithmetic, and each lane takes the next shot from the queue as
soon as its own shot stops.  Each lane rounds as the one-shot kernel's scalar
arithmetic, so per-shot outputs must equal those of one shot per thread bit
for bit: for every variant, for codes with and without padding slots, for
both node counts per thread, for several groups per CTA, and for batches
whose size leaves one lane idle."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu
VARIANTS = ["plain", "momentum", "adagrad", "ewainit"]


@pytest.fixture(scope="module")
def bpq():
    import paper_2407_11523_gb300 as bpq
    assert torch.cuda.is_available()
    return bpq


def decode_with(bpq, t, syn, prior, variant, k, shape=(0, 0), max_iter=60):
    t.set_launch(0, 0)
    t.set_shots_per_thread(k)
    t.set_launch(*shape)
    assert t.shots_per_thread(variant) == k
    out = bpq.decode(t, syn, prior, variant, max_iter=max_iter)
    torch.cuda.synchronize()
    t.set_shots_per_thread(0)
    t.set_launch(0, 0)
    return [x.cpu() for x in out]


@pytest.mark.parametrize("kind,d,p", [("toric", 6, 0.06), ("toric", 15, 0.08), ("planar", 5, 0.06),
                                      ("planar", 9, 0.08), ("xzzx", 7, 0.07)])
@pytest.mark.parametrize("variant", VARIANTS)
def test_two_shots_per_thread_equal_one(bpq, kind, d, p, variant):
    t = bpq.Tanner(kind, d)
    ch = oracle.depolarizing(p)
    _, syn = bpq.sample(t, *ch, seed=0x9A1F + d, shot0=0, B=3001)
    prior = bpq.prior_tensor(t, *ch)
    one = decode_with(bpq, t, syn, prior, variant, 1)
    nodes = max(t.N, t.M)
    shapes = [(0, 0), (((nodes + 1) // 2 + 31) // 32 * 32, 2), ((nodes + 31) // 32 * 32, 2)]
    for shape in shapes:
        if shape[0] > 1024 or shape[0] * shape[1] > 1024:
            continue
        two = decode_with(bpq, t, syn, prior, variant, 2, shape)
        for a, b in zip(one, two):
            assert torch.equal(a, b), (kind, d, variant, shape)
    assert int(one[1].sum()) > 0


def test_two_shots_per_thread_edge_cases(bpq):
    """One shot (the second lane idle from the start), zero syndromes
    (converged at iteration 1), max_iter = 1 and 255, and an empty batch."""
    t = bpq.Tanner("toric", 9)
    ch = oracle.depolarizing(0.1)
    prior = bpq.prior_tensor(t, *ch)
    _, syn = bpq.sample(t, *ch, seed=7, shot0=0, B=5)
    for B in (1, 2, 3, 5):
        for mi in (1, 7, 255):
            a = decode_with(bpq, t, syn[:B].contiguous(), prior, "ewainit", 1, max_iter=mi)
            b = decode_with(bpq, t, syn[:B].contiguous(), prior, "ewainit", 2, max_iter=mi)
            for x, y in zip(a, b):
                assert torch.equal(x, y), (B, mi)
    zero = torch.zeros((7, t.W), dtype=torch.int32, device="cuda")
    for v in VARIANTS:
        est, conv, iters = decode_with(bpq, t, zero, prior, v, 2)
        assert (est == 0).all() and (conv == 1).all() and (iters == 1).all()
    empty = torch.zeros((0, t.W), dtype=torch.int32, device="cuda")
    est, conv, iters = decode_with(bpq, t, empty, prior, "plain", 2)
    assert est.shape == (0, t.N)
    work = bpq.workspace()
    bpq.decode(t, syn, prior, "ewainit", work=work)
    assert bpq.decode_status(work) == 0
