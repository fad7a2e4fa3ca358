"""The stored oracle outcomes (tests/golden/*_oracle.npz, written by
tests/golden/make_oracle_outcomes.py) are the oracle's: a sample of shots is
decoded again here and must give the stored convergence flags, logical
outcomes, iteration counts and estimate hashes.  The files were written on
x86-64, where long double is the x87 80-bit format; on other hosts the
oracle's long-double check update rounds differently, so there only the
precision-robust shots are required to match.  No GPU is used."""
import os
import platform
import sys

import numpy as np
import pytest

import oracle
from oracle import codes

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_oracle_outcomes as mk  # noqa: E402

EXACT = platform.machine() in ("x86_64", "AMD64")
SAMPLE = 120


def check(g, key, H, err, syn, prior, variant, robust):
    est, conv, iters = oracle.decode(H, syn, prior, variant, max_iter=mk.MAX_ITER, nthreads=os.cpu_count() or 4)
    fail, _ = codes.logical_failure(H, err, est)
    n = syn.shape[0]
    got = dict(conv=conv, fail=fail, iters=iters.astype(np.uint8), est=mk.row_hashes(est))
    want = dict(conv=np.unpackbits(g[key + "_conv"])[:n].astype(bool),
                fail=np.unpackbits(g[key + "_fail"])[:n].astype(bool),
                iters=g[key + "_iters"][:n], est=g[key + "_est"][:n])
    sel = np.ones(n, dtype=bool) if EXACT else robust[:n]
    for f in want:
        assert np.array_equal(got[f][sel], want[f][sel]), (key, f)


@pytest.mark.parametrize("variant,p", [("plain", 0.06), ("ewainit", 0.02), ("adagrad", 0.06), ("momentum", 0.10)])
def test_sweep_file_matches_oracle(variant, p):
    g = np.load(os.path.join(HERE, "golden", "toric15_sweep_oracle.npz"))
    key = mk.sweep_key(variant, p)
    H, _ = codes.build_code("toric", 15)
    ch = oracle.depolarizing(p)
    err, syn = oracle.sample(H, *ch, seed=0xB9E00001 + mk.SWEEP_K[p], shot0=0, B=SAMPLE)
    prior = np.asarray(ch, dtype=np.float32).astype(np.float64)
    robust = np.unpackbits(g[key + "_robust"]).astype(bool)
    check(g, key, H, err, syn, prior, variant, robust)
    assert g[key + "_iters"].shape == (mk.SWEEP_SHOTS,)


@pytest.mark.parametrize("kind,d,p", [("toric", 10, 0.02), ("planar", 15, 0.04)])
def test_lowp_file_matches_oracle(kind, d, p):
    g = np.load(os.path.join(HERE, "golden", "lowp_ewainit_oracle.npz"))
    key = mk.lowp_key(kind, d, p)
    H, _ = codes.build_code(kind, d)
    ch = oracle.depolarizing(p)
    err, syn = oracle.sample(H, *ch, seed=mk.LOWP_P[p], shot0=0, B=SAMPLE)
    prior = np.asarray(ch, dtype=np.float32).astype(np.float64)
    conv = np.unpackbits(g[key + "_conv"]).astype(bool)
    robust = conv & (g[key + "_iters"] <= 24)
    check(g, key, H, err, syn, prior, "ewainit", robust)
    assert g[key + "_iters"].shape == (mk.LOWP_SHOTS,)
