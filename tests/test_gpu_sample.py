"""GPU Philox sampler vs the oracle sampler: errors and packed syndromes are
bit-identical, for every code family, channel and shot offset."""
import numpy as np
import pytest
import torch

import oracle
from inputs import pack_bits, trapping_set_code

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bpq():
    import paper_2407_11523_gb300 as bpq
    assert torch.cuda.is_available()
    return bpq


CASES = [
    ("planar", 5, oracle.depolarizing(0.05), 0xB9E00000, 0, 3000),
    ("toric", 15, oracle.depolarizing(0.16), 0xB9E00001, 0, 600),
    ("toric", 15, oracle.depolarizing(0.02), 0xB9E00001, 123456, 257),
    ("xzzx", 7, oracle.biased(0.06, 10.0), 7, 99, 1000),
    ("planar", 31, oracle.depolarizing(0.05), 11, 5, 64),
    ("toric", 3, (0.2, 0.0, 0.3), 1, 2**40, 100),
]


@pytest.mark.parametrize("kind,d,ch,seed,shot0,B", CASES)
def test_sampler_bit_exact(bpq, kind, d, ch, seed, shot0, B):
    t = bpq.Tanner(kind, d)
    err, syn = bpq.sample(t, *ch, seed=seed, shot0=shot0, B=B)
    torch.cuda.synchronize()
    e_ref, s_ref = oracle.sample(t.dense(), *ch, seed=seed, shot0=shot0, B=B)
    assert (err.cpu().numpy() == e_ref).all()
    assert (syn.cpu().numpy().view(np.uint32) == pack_bits(s_ref)).all()


def test_sampler_partition_invariance(bpq):
    t = bpq.Tanner("toric", 9)
    e1, s1 = bpq.sample(t, 0.03, 0.03, 0.03, seed=5, shot0=0, B=1000)
    e2, s2 = bpq.sample(t, 0.03, 0.03, 0.03, seed=5, shot0=317, B=400)
    assert torch.equal(e1[317:717], e2) and torch.equal(s1[317:717], s2)


def test_sampler_custom_graph_and_empty(bpq):
    H = trapping_set_code()
    t = bpq.Tanner(H=H)
    err, syn = bpq.sample(t, 0.1, 0.1, 0.1, seed=3, shot0=0, B=50)
    e_ref, s_ref = oracle.sample(H, 0.1, 0.1, 0.1, seed=3, shot0=0, B=50)
    assert (err.cpu().numpy() == e_ref).all()
    assert (syn.cpu().numpy().view(np.uint32) == pack_bits(s_ref)).all()
    err, syn = bpq.sample(t, 0.1, 0.1, 0.1, seed=3, shot0=0, B=0)
    assert err.shape[0] == 0
    with pytest.raises(bpq.BPQError):
        bpq.sample(t, 0.5, 0.3, 0.3, seed=3, shot0=0, B=5)
