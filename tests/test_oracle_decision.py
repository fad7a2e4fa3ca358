"""Pins of the hard decision and the stopping rule (Sec. II-B1; Algorithms 1
and 2)."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import codes

# (Q_X, Q_Y, Q_Z) -> expected Pauli.  "I if all LLRs are greater than 0,
# otherwise the Pauli with the smallest LLR"; equal minima go to the first
# of X, Y, Z (a reading: the paper does not say).
TABLE = [
    ((1.0, 2.0, 3.0), 0),
    ((1e-300, 5.0, 5.0), 0),
    ((0.0, 1.0, 1.0), 1),
    ((1.0, 0.0, 1.0), 2),
    ((1.0, 1.0, 0.0), 3),
    ((0.0, 0.0, 0.0), 1),
    ((1.0, 0.0, 0.0), 2),
    ((-1.0, -1.0, 2.0), 1),
    ((2.0, -1.0, -1.0), 2),
    ((-3.0, -1.0, -2.0), 1),
    ((4.0, 3.0, -0.5), 3),
    ((-0.5, 3.0, 4.0), 1),
]


@pytest.mark.parametrize("q,want", TABLE)
def test_decision_table(q, want):
    assert oracle.hard_decision(q) == want


def test_decision_exhaustive_patterns():
    vals = [-2.0, -1.0, 0.0, 1.0, 2.0]
    for q in itertools.product(vals, repeat=3):
        d = oracle.hard_decision(q)
        if all(v > 0 for v in q):
            assert d == 0
        else:
            assert d in (1, 2, 3)
            assert q[d - 1] == min(q)
            assert all(q[k] > min(q) for k in range(d - 1))


@pytest.mark.parametrize("kind,L", [("planar", 5), ("toric", 5), ("xzzx", 5)])
@pytest.mark.parametrize("variant", ["plain", "momentum", "adagrad", "ewainit"])
def test_stopping_rule_invariants(kind, L, variant):
    H, _ = codes.build_code(kind, L)
    prior = np.tile(oracle.depolarizing(0.07), (H.shape[1], 1))
    err, syn = oracle.sample(H, *oracle.depolarizing(0.07), seed=9, shot0=0, B=300)
    est, conv, iters = oracle.decode(H, syn, prior, variant=variant, max_iter=30, nthreads=4)
    assert ((iters >= 1) & (iters <= 30)).all()
    assert (iters[~conv] == 30).all()
    s_est = codes.syndrome(H, est)
    assert (s_est[conv] == syn[conv]).all()
    assert (s_est[~conv] != syn[~conv]).any(axis=1).all()


def test_zero_syndrome_converges_at_first_iteration():
    H, _ = codes.build_code("toric", 5)
    prior = np.tile(oracle.depolarizing(0.1), (H.shape[1], 1))
    syn = np.zeros((3, H.shape[0]), dtype=np.uint8)
    for v in ("plain", "momentum", "adagrad", "ewainit"):
        est, conv, iters = oracle.decode(H, syn, prior, variant=v, max_iter=10)
        assert conv.all() and (iters == 1).all() and (est == 0).all()


def test_batch_threads_do_not_change_results():
    H, _ = codes.build_code("planar", 5)
    prior = np.tile(oracle.depolarizing(0.06), (H.shape[1], 1))
    _, syn = oracle.sample(H, *oracle.depolarizing(0.06), seed=1, shot0=0, B=64)
    a = oracle.decode(H, syn, prior, "ewainit", nthreads=1)
    b = oracle.decode(H, syn, prior, "ewainit", nthreads=5)
    for x, y in zip(a, b):
        assert (x == y).all()
