"""Bounds-checked decode kernels (bpq_set_debug_checks): copies of the
one-code kernels with checks on the shared-memory layout, every slot index
and table offset, and every output index, which set the device error word
instead of trapping.  On small codes of every table layout (the (4,0)
trapping set, planar d = 3, toric d = 4, XZZX d = 3), for every variant, with
one and with two shots per thread, no check fails (bpq_decode_status = 0) and
the results equal the unchecked kernels' bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from inputs import trapping_set_code

pytestmark = pytest.mark.gpu
VARIANTS = ["plain", "momentum", "adagrad", "ewainit"]


@pytest.fixture(scope="module")
def bpq():
    import paper_2407_11523_gb300 as bpq
    assert torch.cuda.is_available()
    return bpq


def codes(bpq):
    H = bpq.Tanner("toric", 4).dense()
    Hy = H.copy()
    Hy[0, np.nonzero(H[0])[0][0]] = 2  # a Y entry: the generic table layout
    return [("trapping", bpq.Tanner(H=trapping_set_code())), ("planar3", bpq.Tanner("planar", 3)),
            ("toric4", bpq.Tanner("toric", 4)), ("xzzx3", bpq.Tanner("xzzx", 3)), ("toric4y", bpq.Tanner(H=Hy))]


@pytest.mark.parametrize("variant", VARIANTS)
def test_bounds_checked_kernels_pass_and_match(bpq, variant):
    ch = oracle.depolarizing(0.08)
    for name, t in codes(bpq):
        prior = bpq.prior_tensor(t, *ch)
        if name == "trapping":
            syn = torch.tensor([[0b0101]] * 3, dtype=torch.int32, device="cuda")
        else:
            _, syn = bpq.sample(t, *ch, seed=91, shot0=0, B=777)
        for k in ([1, 2] if t.layout() else [1]):
            t.set_shots_per_thread(k)
            ref = [x.cpu() for x in bpq.decode(t, syn, prior, variant, max_iter=40)]
            t.set_debug_checks(True)
            work = bpq.workspace()
            got = [x.cpu() for x in bpq.decode(t, syn, prior, variant, max_iter=40, work=work)]
            assert bpq.decode_status(work) == 0, (name, variant, k)
            t.set_debug_checks(False)
            for a, b in zip(ref, got):
                assert torch.equal(a, b), (name, variant, k)
        t.set_shots_per_thread(0)


def test_bounds_checked_kernels_refuse_other_launches(bpq):
    """AEWA-BP and traces have no checked copy: refused, not run unchecked."""
    t = bpq.Tanner("planar", 3)
    prior = bpq.prior_tensor(t, *oracle.depolarizing(0.05))
    _, syn = bpq.sample(t, *oracle.depolarizing(0.05), seed=1, shot0=0, B=4)
    t.set_debug_checks(True)
    with pytest.raises(bpq.BPQError):
        bpq.decode(t, syn, prior, "aewa", max_iter=20)
    t.set_debug_checks(False)
    bpq.decode(t, syn, prior, "aewa", max_iter=20)
