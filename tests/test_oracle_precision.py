"""Which decoding results the working precision decides.

EWAInit-BP cannot leave an exactly symmetric state under the parallel
schedule (Sec. IV-A: the recursion of every node of a trapping set stays
symmetric).  With the paper's uniform priors (Sec. IV, depolarising p/3 per
Pauli) the toric and planar codes put many trapping sets into a nearly
symmetric oscillation, which breaks only through the small asymmetries that
the rest of the syndrome feeds in.  EWAInit-BP's state forgets its past as
(1 - alpha)^t (eq. (EWAInit)), and once that transient falls below the
working precision the oscillation freezes.  Whether such a shot converges
within max_iter is therefore decided by the precision the decoder computes
in, not by the method.  These tests pin that with the oracle alone, built
at three precisions from one source:

* at uniform priors the fraction of unconverged shots falls as the
  precision rises, and the FP64 oracle and its long-double build already
  disagree on more than 0.1 % of the shots;
* every shot that the FP64 oracle converges within 24 iterations (binary32
  has a 24-bit significand, and (1 - alpha)^24 = 2^-24 at alpha = 0.5) gets
  the same convergence flag, logical outcome and estimate at every precision;
* priors jittered by 2^-16 per qubit (reading 19 of the design notes) break
  the ties in the input, and the three builds then agree on the convergence
  flag and the logical outcome of every shot but a handful.

No GPU is used."""
import os

import numpy as np
import pytest

import oracle
from inputs import jittered_priors
from oracle import codes

NTHREADS = os.cpu_count() or 4
ROBUST_ITERS = 24
PRECISIONS = ("f32", "f64", "ext")


@pytest.fixture(scope="module")
def toric15_p02():
    H, _ = codes.build_code("toric", 15)
    ch = oracle.depolarizing(0.02)
    err, syn = oracle.sample(H, *ch, seed=0xB9E00001, shot0=0, B=4000)
    return H, ch, err, syn


def run_all(H, err, syn, prior):
    out = {}
    for prec in PRECISIONS:
        est, conv, iters = oracle.decode(H, syn, prior, "ewainit", max_iter=100, alpha=0.5, nthreads=NTHREADS,
                                         precision=prec)
        fail, _ = codes.logical_failure(H, err, est)
        out[prec] = (est, conv, iters, fail)
    return out


def test_builds_share_the_update_rules():
    """On a random tree code with moderate messages the three builds give the
    same messages up to their working precision (same rules, same order)."""
    from inputs import random_priors, random_syndromes, random_tree_code
    H = random_tree_code(9, seed=31)
    prior = random_priors(9, seed=32)
    s = random_syndromes(H.shape[0], 1, seed=33)[0]
    ref = oracle.trace(H, s, prior, "ewainit", T=6, precision="f64")
    ext = oracle.trace(H, s, prior, "ewainit", T=6, precision="ext")
    f32 = oracle.trace(H, s, prior, "ewainit", T=6, precision="f32")
    assert np.abs(ext["m_v2c"] - ref["m_v2c"]).max() < 1e-12
    assert np.abs(ext["Q"] - ref["Q"]).max() < 1e-12
    d32 = max(np.abs(f32["m_v2c"] - ref["m_v2c"]).max(), np.abs(f32["Q"] - ref["Q"]).max())
    assert 0 < d32 < 1e-4
    assert np.array_equal(f32["dec"], ref["dec"])


def test_uniform_priors_low_p_is_precision_decided(toric15_p02):
    """Toric d = 15, p = 0.02, 4000 shots, EWAInit-BP (alpha = 0.5), at most
    100 iterations, uniform priors."""
    H, ch, err, syn = toric15_p02
    prior = np.asarray(ch, dtype=np.float32).astype(np.float64)
    r = run_all(H, err, syn, prior)
    unconv = {p: 1.0 - r[p][1].mean() for p in PRECISIONS}
    # more precision, fewer shots left in a frozen oscillation
    assert unconv["f32"] > unconv["f64"] + 0.01, unconv
    assert unconv["f64"] > unconv["ext"] + 0.002, unconv
    # so the FP64 oracle and a more precise build of itself miss a 99.9 % bar
    assert (r["f64"][1] == r["ext"][1]).mean() < 0.999
    # the shots that converge before the EWA transient drops below binary32
    # resolution have a precision-independent answer
    est, conv, iters, fail = r["f64"]
    robust = conv & (iters <= ROBUST_ITERS)
    assert robust.mean() >= 0.9, robust.mean()
    for p in ("f32", "ext"):
        e, c, _, f = r[p]
        assert c[robust].all(), p
        assert np.array_equal(f[robust], fail[robust]), p
        assert (e[robust] == est[robust]).all(axis=1).mean() >= 0.999, p
    # every precision-decided shot is one that converges late or never
    decided = np.zeros_like(conv)
    for p in ("f32", "ext"):
        decided |= (r[p][1] != conv) | (r[p][3] != fail)
    assert not (decided & robust).any()


def test_jittered_priors_are_precision_robust(toric15_p02):
    """The same shots on priors jittered by 2^-16 per qubit: the three builds
    agree on the convergence flag and the logical outcome of at least 99.9 %
    of the shots and on every robust one."""
    H, ch, err, syn = toric15_p02
    prior = jittered_priors(H.shape[1], *ch, 2.0 ** -16).astype(np.float64)
    r = run_all(H, err, syn, prior)
    est, conv, iters, fail = r["f64"]
    assert conv.mean() >= 0.99
    robust = conv & (iters <= ROBUST_ITERS)
    for p in ("f32", "ext"):
        e, c, _, f = r[p]
        assert (c == conv).mean() >= 0.999, p
        assert (f == fail).mean() >= 0.999, p
        assert c[robust].all() and np.array_equal(f[robust], fail[robust]), p
