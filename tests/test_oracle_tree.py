"""Pin of the whole plain decoder: on a Tanner graph without cycles, BP
computes the exact posterior marginals (Sec. II-B2: it is the cycles that
break exactness).  The oracle's posterior LLRs are compared with brute-force
enumeration of all 4^n errors."""
import itertools

import numpy as np
import pytest

import oracle
from inputs import random_priors, random_syndromes, random_tree_code


def brute_force_posterior_llr(H, prior, syn):
    """ln P(E_j = I | s) / P(E_j = W | s) by enumerating every Pauli error.
    The syndrome bit of check i is the parity of the entries of E that
    anticommute with row i (written here from the Pauli multiplication
    table, independently of the oracle)."""
    M, N = H.shape
    errs = np.array(list(itertools.product(range(4), repeat=N)), dtype=np.int64)
    anti = np.zeros((4, 4), dtype=np.int64)
    for a in range(1, 4):
        for b in range(1, 4):
            anti[a, b] = int(a != b)
    synd = np.zeros((errs.shape[0], M), dtype=np.int64)
    for i in range(M):
        synd[:, i] = anti[errs, H[i][None, :]].sum(axis=1) % 2
    ok = (synd == syn[None, :]).all(axis=1)
    p4 = np.concatenate([(1 - prior.sum(axis=1))[:, None], prior], axis=1)
    w = np.prod(p4[np.arange(N)[None, :], errs], axis=1) * ok
    Q = np.zeros((N, 3))
    for j in range(N):
        PI = w[errs[:, j] == 0].sum()
        for W in range(1, 4):
            Q[j, W - 1] = np.log(PI / w[errs[:, j] == W].sum())
    return Q


@pytest.mark.parametrize("seed", range(12))
def test_plain_bp_is_exact_on_trees(seed):
    n = 4 + seed % 5
    H = random_tree_code(n, seed=100 + seed)
    prior = random_priors(n, seed=200 + seed)
    for syn in random_syndromes(H.shape[0], 3, seed=300 + seed):
        T = 2 * n
        tr = oracle.trace(H, syn, prior, variant="plain", T=T)
        assert np.abs(tr["m_c2v"]).max() < 29.0  # the clip never binds here
        want = brute_force_posterior_llr(H, prior, syn)
        assert np.allclose(tr["Q"][-1], want, rtol=0, atol=1e-9)
        # the hard decision is the per-qubit MAP of the exact marginals
        for j in range(n):
            q = want[j]
            expect = 0 if (q > 0).all() else 1 + int(np.argmin(q))
            if np.min(np.abs(q)) > 1e-6:
                assert tr["dec"][-1][j] == expect


@pytest.mark.parametrize("seed", range(4))
def test_variant_reductions_to_plain_on_trees(seed):
    """EWAInit-BP with alpha = 1 is plain BP exactly (eq. (EWAInit)); Momentum-BP
    with alpha = 1, gamma = 0 is plain BP (Sec. III-A1, text after (mombp3))."""
    n = 6
    H = random_tree_code(n, seed=400 + seed)
    prior = random_priors(n, seed=500 + seed)
    syn = random_syndromes(H.shape[0], 1, seed=600 + seed)[0]
    ref = oracle.trace(H, syn, prior, variant="plain", T=10)
    ewa = oracle.trace(H, syn, prior, variant="ewainit", alpha=1.0, T=10)
    for k in ("m_v2c", "m_c2v", "Q", "S"):
        assert (ewa[k] == ref[k]).all()
    mom = oracle.trace(H, syn, prior, variant="momentum", alpha=1.0, gamma=0.0, T=10)
    for k in ("m_v2c", "m_c2v", "Q"):
        assert np.allclose(mom[k], ref[k], rtol=0, atol=1e-9)
