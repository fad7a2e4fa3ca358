"""Whole-decoder pins: exact maximum-likelihood decoding of the d = 3 planar
code bounds every BP variant's logical error rate from below (Sec. II-B1,
eq. (qecobject)); and the (4,0) trapping set of Sec. IV-A / Table I."""
import os

import numpy as np
import pytest

import oracle
from inputs import trapping_set_code
from oracle import codes

GOLDEN_TS = os.path.join(os.path.dirname(__file__), "golden", "trapping_set.txt")


def ml_tables(H, logicals, prior4):
    """P(syndrome, logical class) summed over all 4^N errors, by splitting the
    qubits into two halves and combining their (syndrome, class, weight)
    tables (both syndrome and class are XOR-linear in the error)."""
    M, N = H.shape
    anti = np.array([[0, 0, 0, 0], [0, 0, 1, 1], [0, 1, 0, 1], [0, 1, 1, 0]], dtype=np.int64)
    rows = np.vstack([H, logicals])
    split = N // 2

    def half(qubits):
        grid = np.array(np.meshgrid(*[np.arange(4)] * len(qubits), indexing="ij")).reshape(len(qubits), -1).T
        key = np.zeros(grid.shape[0], dtype=np.int64)
        for r in range(rows.shape[0]):
            bit = anti[grid, rows[r, qubits][None, :]].sum(axis=1) % 2
            key |= bit << r
        w = np.prod(prior4[np.array(qubits)[None, :], grid], axis=1)
        return key, w

    klo, wlo = half(list(range(split)))
    khi, whi = half(list(range(split, N)))
    nkeys = 1 << rows.shape[0]
    table = np.zeros(nkeys)
    for k2, w2 in zip(khi, whi):
        table += np.bincount(klo ^ k2, weights=wlo * w2, minlength=nkeys)
    return _by_syndrome(table, M, logicals.shape[0])


def _by_syndrome(table, M, L):
    """table[key] with key = syndrome bits | class bits << M -> (2^M, 2^L)."""
    out = np.zeros((1 << M, 1 << L))
    keys = np.arange(table.size)
    np.add.at(out, (keys & ((1 << M) - 1), keys >> M), table)
    return out


@pytest.mark.slow
def test_ml_lower_bound_planar_d3():
    H, _ = codes.build_code("planar", 3)
    M, N = H.shape
    lg = codes.logical_operators(H)
    p = 0.09
    prior4 = np.tile([1 - p, p / 3, p / 3, p / 3], (N, 1))
    P = ml_tables(H, lg, prior4)
    assert P.sum() == pytest.approx(1.0, abs=1e-12)
    ler_ml = 1.0 - P.max(axis=1).sum()

    B = 20000
    err, syn = oracle.sample(H, *oracle.depolarizing(p), seed=31, shot0=0, B=B)
    # Monte Carlo of the ML decoder itself agrees with the exact value
    anti = np.array([[0, 0, 0, 0], [0, 0, 1, 1], [0, 1, 0, 1], [0, 1, 1, 0]])
    sidx = (syn.astype(np.int64) << np.arange(M)).sum(axis=1)
    cls = np.zeros(B, dtype=np.int64)
    for r in range(lg.shape[0]):
        cls |= (anti[err, lg[r][None, :]].sum(axis=1) % 2) << r
    mc_fail = (P[sidx].argmax(axis=1) != cls).mean()
    sigma = np.sqrt(ler_ml * (1 - ler_ml) / B)
    assert abs(mc_fail - ler_ml) < 4 * sigma
    # no BP variant beats maximum likelihood
    prior = np.tile(oracle.depolarizing(p), (N, 1))
    group = codes.StabilizerGroup(H)
    for v in ("plain", "momentum", "adagrad", "ewainit"):
        est, conv, _ = oracle.decode(H, syn, prior, variant=v, max_iter=50, nthreads=8)
        fail, _ = codes.logical_failure(H, err, est, group)
        assert fail.mean() >= ler_ml - 2 * sigma, (v, fail.mean(), ler_ml)
        # non-converged shots are failures (detected errors)
        assert fail[~conv].all()


def read_golden():
    kv = {}
    for line in open(GOLDEN_TS):
        line = line.split("#")[0].strip()
        if line:
            k, *v = line.split()
            kv[k] = v
    return kv


@pytest.mark.parametrize("per_pauli", [False, True])
def test_trapping_set_parallel_never_converges(per_pauli):
    g = read_golden()
    H = trapping_set_code()
    err = np.zeros(4, dtype=np.uint8)
    for q in g["error_qubits"]:
        err[int(q) - 1] = 1  # X
    syn = codes.syndrome(H, err)
    assert syn.tolist() == [int(x) for x in g["syndrome"]]
    p = float(g["prior"][0])
    prior = np.full((4, 3), p) if per_pauli else np.tile(oracle.depolarizing(p), (4, 1))
    T = int(g["max_iter"][0])
    for v, key in (("plain", "plain_parallel_converges"), ("ewainit", "ewainit_parallel_converges")):
        _, conv, iters = oracle.decode(H, syn[None], prior, variant=v, max_iter=T)
        assert g[key] == ["no"]
        assert not conv[0] and iters[0] == T
        tr = oracle.trace(H, syn, prior, variant=v, T=T)
        # the 8-cycle is symmetric under a syndrome-preserving automorphism:
        # all four decisions are equal at every iteration
        assert (tr["dec"] == tr["dec"][:, :1]).all()
    # plain BP oscillates between all-I and all-X (Sec. IV-A)
    tr = oracle.trace(H, syn, prior, variant="plain", T=T)
    seen = {tuple(r) for r in tr["dec"]}
    assert (0, 0, 0, 0) in seen and (1, 1, 1, 1) in seen


def test_prior_jitter_breaks_the_exact_symmetry():
    """Under the parallel schedule EWAInit-BP cannot leave the symmetric
    (4,0) trapping set by itself (Sec. IV-A); any asymmetry in the input priors
    is amplified by the prior re-initialisation of eq. (EWAInit) until the
    decisions split and satisfy the syndrome.  Plain BP has no such
    amplification and keeps oscillating."""
    from inputs import jittered_priors
    H = trapping_set_code()
    syn = np.array([[1, 0, 1, 0]], dtype=np.uint8)
    prior = jittered_priors(4, *oracle.depolarizing(0.01), 2.0 ** -16).astype(np.float64)
    est, conv, iters = oracle.decode(H, syn, prior, variant="ewainit", max_iter=50)
    assert conv[0] and iters[0] < 50
    assert np.array_equal(codes.syndrome(H, est[0]), syn[0])
    assert len(set(est[0].tolist())) == 2  # the decisions are no longer all equal
    _, conv, _ = oracle.decode(H, syn, prior, variant="plain", max_iter=50)
    assert not conv[0]


def test_uniform_priors_leave_tie_failures_on_the_toric_code():
    """Toric d = 6 at p = 0.02: every EWAInit-BP non-convergence with uniform
    priors is an exact-symmetry tie.  A relative per-qubit jitter of 2^-16
    converts all of them to converged estimates and loses no shot that
    converged before."""
    from inputs import jittered_priors
    H, _ = codes.build_code("toric", 6)
    ch = oracle.depolarizing(0.02)
    _, syn = oracle.sample(H, *ch, seed=0xB9E00001, shot0=0, B=2000)
    conv = {}
    for rel in (0.0, 2.0 ** -16):
        prior = jittered_priors(H.shape[1], *ch, rel).astype(np.float64)
        _, conv[rel], _ = oracle.decode(H, syn, prior, variant="ewainit", max_iter=100)
    assert (~conv[0.0]).sum() >= 5
    assert conv[2.0 ** -16].all()
