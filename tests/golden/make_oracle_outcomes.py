"""Write the FP64 oracle's decoding outcomes that the GPU parity tests compare
with, for workloads whose oracle run would take minutes on the test host.

Calls only oracle/ (its decoder, its Philox sampler, its logical-failure
test) and hashlib.  Run from the repository root:

    python tests/golden/make_oracle_outcomes.py

Files (numpy .npz, one group of arrays per workload <key>):
  toric15_sweep_oracle.npz  toric d = 15, depolarising p in {0.02, 0.06,
      0.10, 0.14} (the k = 0, 2, 4, 6 points of the 8-step sweep 0.02..0.16,
      seed 0xB9E00001 + k, shots 0..999), plain BP, Momentum-BP (alpha 0.5,
      gamma 0), AdaGrad-BP (alpha 5) and EWAInit-BP (alpha 0.5), at most 100
      iterations (Sec. IV-B2).
  lowp_ewainit_oracle.npz  EWAInit-BP (alpha 0.5), uniform priors, toric
      d = 10 and 15 and planar d = 15 at p = 0.02 (seed 0xB9E00001) and
      p = 0.04 (seed 0xB9E00002), shots 0..3999, at most 100 iterations.

Per workload: <key>_conv and <key>_fail (bit-packed bools: converged, and
the residual is not a stabilizer, Sec. IV), <key>_iters (uint8),
<key>_est (uint32: the first four bytes of blake2b(estimate row), so that
estimates can be compared without storing them), <key>_robust (bit-packed,
sweep file only): the shot's outcome does not depend on the rounding, i.e.
the binary32-storage build of the oracle and three FP64 runs on priors
perturbed by 8 binary32 ulps (each probability scaled by 1 +- 2^-20, random
signs) all give the same convergence flag, logical outcome and, for
converged shots, estimate as the FP64 run.
"""
from __future__ import annotations

import hashlib
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle import codes  # noqa: E402

SWEEP_P = (0.02, 0.06, 0.10, 0.14)
SWEEP_K = {0.02: 0, 0.06: 2, 0.10: 4, 0.14: 6}
SWEEP_VARIANTS = ("plain", "momentum", "adagrad", "ewainit")
SWEEP_SHOTS = 1000
LOWP_CODES = (("toric", 15), ("toric", 10), ("planar", 15))
LOWP_P = {0.02: 0xB9E00001, 0.04: 0xB9E00002}
LOWP_SHOTS = 4000
MAX_ITER = 100


def row_hashes(est: np.ndarray) -> np.ndarray:
    est = np.ascontiguousarray(est, dtype=np.uint8)
    return np.array([int.from_bytes(hashlib.blake2b(r.tobytes(), digest_size=4).digest(), "little") for r in est],
                    dtype=np.uint32)


def sweep_key(variant: str, p: float) -> str:
    return f"{variant}_p{p:.2f}"


def lowp_key(kind: str, d: int, p: float) -> str:
    return f"{kind}{d}_p{p:.2f}"


PERTURBATIONS = 3


def perturbed(prior: np.ndarray, n_qubits: int, seed: int, r: int) -> np.ndarray:
    """(N, 3) priors with every probability scaled by 1 +- 2^-20 (8 ulps of
    binary32), signs from numpy's seeded generator."""
    rows = np.tile(np.asarray(prior, dtype=np.float64).reshape(1, 3), (n_qubits, 1))
    rng = np.random.default_rng([seed, r])
    return rows * (1 + 2.0 ** -20 * rng.choice([-1.0, 1.0], size=rows.shape))


def same_outcome(a, b):
    est_a, conv_a, _, fail_a = a
    est_b, conv_b, _, fail_b = b
    return (conv_a == conv_b) & (fail_a == fail_b) & (~conv_a | (est_a == est_b).all(axis=1))


def outcomes(H, err, syn, prior, variant, precision, nthreads):
    est, conv, iters = oracle.decode(H, syn, prior, variant, max_iter=MAX_ITER, nthreads=nthreads,
                                     precision=precision)
    fail, _ = codes.logical_failure(H, err, est)
    return est, conv, iters, fail


def main() -> None:
    nthreads = os.cpu_count() or 4
    out = {}
    H, _ = codes.build_code("toric", 15)
    for p in SWEEP_P:
        ch = oracle.depolarizing(p)
        err, syn = oracle.sample(H, *ch, seed=0xB9E00001 + SWEEP_K[p], shot0=0, B=SWEEP_SHOTS)
        prior = np.asarray(ch, dtype=np.float32).astype(np.float64)
        for vi, v in enumerate(SWEEP_VARIANTS):
            ref = outcomes(H, err, syn, prior, v, "f64", nthreads)
            est, conv, iters, fail = ref
            robust = same_outcome(ref, outcomes(H, err, syn, prior, v, "f32", nthreads))
            for r in range(PERTURBATIONS):
                pp = perturbed(prior, H.shape[1], seed=1000 * vi + SWEEP_K[p], r=r)
                robust &= same_outcome(ref, outcomes(H, err, syn, pp, v, "f64", nthreads))
            k = sweep_key(v, p)
            out[k + "_conv"] = np.packbits(conv)
            out[k + "_fail"] = np.packbits(fail)
            out[k + "_robust"] = np.packbits(robust)
            out[k + "_iters"] = iters.astype(np.uint8)
            out[k + "_est"] = row_hashes(est)
            print(f"{k}: converged {conv.mean():.3f}, LER {fail.mean():.4f}, robust {robust.mean():.4f}", flush=True)
    np.savez_compressed(os.path.join(HERE, "toric15_sweep_oracle.npz"), **out)

    out = {}
    for kind, d in LOWP_CODES:
        H, _ = codes.build_code(kind, d)
        for p, seed in LOWP_P.items():
            ch = oracle.depolarizing(p)
            err, syn = oracle.sample(H, *ch, seed=seed, shot0=0, B=LOWP_SHOTS)
            prior = np.asarray(ch, dtype=np.float32).astype(np.float64)
            est, conv, iters, fail = outcomes(H, err, syn, prior, "ewainit", "f64", nthreads)
            k = lowp_key(kind, d, p)
            out[k + "_conv"] = np.packbits(conv)
            out[k + "_fail"] = np.packbits(fail)
            out[k + "_iters"] = iters.astype(np.uint8)
            out[k + "_est"] = row_hashes(est)
            print(f"{k}: converged {conv.mean():.4f}, LER {fail.mean():.5f}", flush=True)
    np.savez_compressed(os.path.join(HERE, "lowp_ewainit_oracle.npz"), **out)


if __name__ == "__main__":
    main()
