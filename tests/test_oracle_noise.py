"""Pins of the oracle's Philox4x64-10 generator and Pauli-channel sampler.

The generator is checked against numpy's independent Philox implementation
(numpy.random.Philox, a 4x64 Philox with 10 rounds whose raw stream first
increments the 256-bit counter and then encrypts it)."""
import numpy as np
import pytest

import oracle
from oracle import codes


def numpy_block(counter, key):
    c = np.array(counter, dtype=np.uint64)
    # numpy increments before encrypting: start one below (with borrow)
    c0 = int(c[0])
    prev = [(c0 - 1) % 2**64, int(c[1]) - (1 if c0 == 0 else 0), int(c[2]), int(c[3])]
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(prev, dtype=np.uint64))
    return bg.random_raw(4)


def test_philox_matches_numpy():
    rng = np.random.default_rng(1234)
    for _ in range(200):
        ctr = [int(x) for x in rng.integers(1, 2**63, size=4, dtype=np.uint64)]
        key = [int(x) for x in rng.integers(0, 2**63, size=2, dtype=np.uint64)]
        ours = oracle.philox4x64_10(ctr, key)
        assert (ours == numpy_block(ctr, key)).all()
    # the counters the sampler uses: (shot, j/4, 0, 0), key (seed, 0)
    for shot in [1, 7, 123456789]:
        for blk in [0, 1, 112]:
            assert (oracle.philox4x64_10([shot, blk, 0, 0], [99, 0]) == numpy_block([shot, blk, 0, 0], [99, 0])).all()


def test_sampler_uses_documented_stream():
    H, _ = codes.build_code("planar", 3)
    px, py, pz = 0.1, 0.05, 0.2
    err, _ = oracle.sample(H, px, py, pz, seed=5, shot0=10, B=3)
    tx, ty, tz = (int(np.ldexp(c, 64)) for c in (px, px + py, px + py + pz))
    for b in range(3):
        for j in range(H.shape[1]):
            u = int(numpy_block([10 + b, j // 4, 0, 0], [5, 0])[j % 4])
            want = 1 if u < tx else 2 if u < ty else 3 if u < tz else 0
            assert err[b, j] == want


def test_shot_offsets_are_consistent():
    H, _ = codes.build_code("toric", 5)
    e1, s1 = oracle.sample(H, 0.02, 0.02, 0.02, seed=77, shot0=0, B=40)
    e2, s2 = oracle.sample(H, 0.02, 0.02, 0.02, seed=77, shot0=13, B=27)
    assert (e1[13:] == e2).all() and (s1[13:] == s2).all()


def test_channel_frequencies():
    H, _ = codes.build_code("planar", 9)
    N = H.shape[1]
    px, py, pz = oracle.biased(0.06, 10.0)
    err, _ = oracle.sample(H, px, py, pz, seed=2024, shot0=0, B=4000)
    n = err.size
    for code, p in [(1, px), (2, py), (3, pz), (0, 1 - px - py - pz)]:
        f = (err == code).mean()
        assert abs(f - p) < 5 * np.sqrt(p * (1 - p) / n), (code, f, p)


def test_syndrome_is_symplectic_product():
    for kind in ["planar", "toric", "xzzx"]:
        H, _ = codes.build_code(kind, 5)
        err, syn = oracle.sample(H, 0.05, 0.03, 0.04, seed=3, shot0=0, B=200)
        assert (syn == codes.syndrome(H, err)).all()
    # a stabilizer as "error" has the zero syndrome
    assert not codes.syndrome(H, H).any()


def test_depolarizing_and_biased_channels():
    assert oracle.depolarizing(0.06) == pytest.approx((0.02, 0.02, 0.02))
    px, py, pz = oracle.biased(0.06, 10.0)
    assert px + py + pz == pytest.approx(0.06)
    assert pz / (px + py) == pytest.approx(10.0)
    # the paper's own example p_z = 2/3 p, p_x = p_y = 1/6 p is eta = 2 (Sec. IV-B3)
    px, py, pz = oracle.biased(0.06, 2.0)
    assert (px, py, pz) == pytest.approx((0.01, 0.01, 0.04))
