"""Decoding-outcome parity with the FP64 oracle across the bench's toric
d = 15 sweep (Sec. IV-B2: toric code, parallel schedule, at most 100
iterations), for plain BP, Momentum-BP, AdaGrad-BP and EWAInit-BP at the
paper's parameters, 1000 shots at each of p = 0.02, 0.06, 0.10, 0.14.

The oracle's outcomes come from tests/golden/toric15_sweep_oracle.npz,
written by tests/golden/make_oracle_outcomes.py (which calls only oracle/);
an FP64 oracle run of this size would take many minutes on the test host,
whose long double is software binary128.  test_oracle_outcomes_file.py
re-derives a sample of the file on the CPU.

A shot is precision-robust when the oracle's binary32-storage build and
three FP64 runs on priors perturbed by 8 binary32 ulps all give the same
convergence flag, logical outcome and (if converged) estimate as the FP64
run; its answer is then the method's, not the rounding's.  On the robust
shots that the oracle converges the GPU must agree on at least 99.9 % of
convergence flags and logical outcomes, and on the estimates to the bound
of MIN_SAME_ESTIMATE (degenerate equivalents aside); on the robust shots that
the oracle runs to max_iter (no unique outcome after 100 oscillating
iterations) it may converge on at most 0.5 % of the batch; and the logical error
rates on the robust shots must lie inside each other's 2-sigma binomial
interval.  The fraction of shots that are not precision-robust is bounded by
what the oracle itself measures (plain BP: none), and every
GPU output must be valid (a converged shot satisfies its syndrome, an
unconverged one ran max_iter iterations)."""
import hashlib
import os

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "toric15_sweep_oracle.npz")
P_SWEEP = (0.02, 0.06, 0.10, 0.14)
K_OF_P = {0.02: 0, 0.06: 2, 0.10: 4, 0.14: 6}
SHOTS = 1000
# the largest fraction of shots whose oracle outcome the rounding decides,
# per variant, as the oracle itself measures it on this workload (binary32
# storage and three 8-ulp prior perturbations against FP64): plain BP none,
# Momentum-BP 1.9 % (p = 0.02), AdaGrad-BP 17.5 % (p = 0.06, where its boosted
# step is ill-conditioned), EWAInit-BP 9.9 % (p = 0.14; the near-symmetric
# trapping-set oscillations of Sec. IV-A)
MAX_UNROBUST = {"plain": 0.0, "momentum": 0.02, "adagrad": 0.18, "ewainit": 0.10}
# a converged estimate is unique only up to a stabilizer: where the update is
# ill-conditioned (AdaGrad-BP's boosted step with G ~ 0) or near-symmetric
# (EWAInit-BP's trapping sets) the kernel's rounding can settle on a
# degenerate equivalent that none of the oracle's witnesses picked.  The
# logical outcome is held to 99.9 % on every variant; equal estimates to
# 99.9 % for plain BP and Momentum-BP (measured: 100 %), 99.5 % for
# EWAInit-BP (measured: at least 99.89 %) and 98.5 % for AdaGrad-BP
# (measured: 99.0-99.8 %).
MIN_SAME_ESTIMATE = {"plain": 0.999, "momentum": 0.999, "adagrad": 0.985, "ewainit": 0.995}


def row_hashes(est: np.ndarray) -> np.ndarray:
    est = np.ascontiguousarray(est, dtype=np.uint8)
    return np.array([int.from_bytes(hashlib.blake2b(r.tobytes(), digest_size=4).digest(), "little") for r in est],
                    dtype=np.uint32)


@pytest.fixture(scope="module")
def golden():
    return np.load(GOLDEN)


@pytest.fixture(scope="module")
def bpq():
    import paper_2407_11523_gb300 as bpq
    assert torch.cuda.is_available()
    return bpq


def ler_interval(fails):
    n = max(fails.size, 1)
    p = fails.mean() if fails.size else 0.0
    return p, 2 * np.sqrt(max(p * (1 - p), 1.0 / n) / n)


@pytest.mark.parametrize("p", P_SWEEP)
@pytest.mark.parametrize("variant", ["plain", "momentum", "adagrad", "ewainit"])
def test_sweep_outcomes_match_oracle(bpq, golden, variant, p):
    key = f"{variant}_p{p:.2f}"
    unpack = lambda a: np.unpackbits(golden[key + a])[:SHOTS].astype(bool)
    conv_r, fail_r, robust = unpack("_conv"), unpack("_fail"), unpack("_robust")
    est_h = golden[key + "_est"]

    t = bpq.Tanner("toric", 15)
    ch = (p / 3, p / 3, p / 3)
    err, syn = bpq.sample(t, *ch, seed=0xB9E00001 + K_OF_P[p], shot0=0, B=SHOTS)
    est, conv, iters = bpq.decode(t, syn, bpq.prior_tensor(t, *ch), variant, max_iter=100)
    fail = bpq.check_logical(t, err, est)
    torch.cuda.synchronize()
    est, conv, iters, fail = (x.cpu().numpy() for x in (est, conv, iters, fail))
    conv = conv.astype(bool)

    # every output is valid
    assert (fail[conv] != 1).all() and (fail[~conv] == 1).all()
    assert ((iters >= 1) & (iters <= 100)).all() and (iters[~conv] == 100).all()

    assert 1.0 - robust.mean() <= MAX_UNROBUST[variant] + 1e-9, (key, robust.mean())
    R = robust
    bad = np.nonzero(R & ((conv != conv_r) | ((fail > 0) != fail_r)))[0]
    if bad.size:
        print(f"{key}: robust shots that differ: {bad.tolist()} oracle iters {golden[key + '_iters'][bad].tolist()} "
              f"conv {conv_r[bad].astype(int).tolist()}; GPU iters {iters[bad].tolist()} conv {conv[bad].astype(int).tolist()}")
    # robust shots the oracle converges: a unique answer, held to the strict bar
    RC = R & conv_r
    assert conv[RC].mean() >= 0.999, (key, conv[RC].mean())
    assert ((fail[RC] > 0) == fail_r[RC]).mean() >= 0.999, key
    both = RC & conv
    if both.any():
        same = row_hashes(est[both]) == est_h[both]
        assert same.mean() >= MIN_SAME_ESTIMATE[variant], (key, same.mean())
    # robust shots the oracle runs to max_iter: 100 iterations of an
    # oscillating or chaotic trajectory have no unique outcome; the GPU may
    # stumble on a syndrome-satisfying decision on a few of them (1-3 of the
    # 1000 shots measured for AdaGrad-BP and EWAInit-BP from p = 0.06), on at
    # most 0.5 % of the batch (which bounds their effect on the LER)
    RU = R & ~conv_r
    assert (RU & conv).sum() <= 0.005 * SHOTS, (key, int((RU & conv).sum()))
    pg, sg = ler_interval(fail[R] > 0)
    pr, sr = ler_interval(fail_r[R])
    assert abs(pg - pr) <= max(sg, sr), (key, pg, pr)
    print(f"{key}: robust {R.mean():.3f}, GPU LER {(fail > 0).mean():.4f} (on robust {pg:.4f}), "
          f"oracle LER {fail_r.mean():.4f} (on robust {pr:.4f}), converged GPU {conv.mean():.3f} oracle "
          f"{conv_r.mean():.3f}")
