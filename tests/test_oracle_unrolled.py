"""Pins of the differentiable unrolled EWAInit-BP oracle (oracle/unrolled.py):
at the paper's parameters it is EWAInit-BP (checked against the C oracle,
which is itself pinned by Theorem 1 and tree exactness); alpha = 1 is plain
BP; beta = 1 freezes the variable-to-check messages; autograd gradients
agree with central finite differences."""
import numpy as np
import pytest
import torch

import oracle
from oracle import codes, unrolled


@pytest.fixture(scope="module")
def case():
    H, _ = codes.build_code("planar", 5)
    ch = oracle.depolarizing(0.06)
    err, syn = oracle.sample(H, *ch, seed=77, shot0=0, B=6)
    prior = np.tile(ch, (H.shape[1], 1))
    return H, err, syn, prior


@pytest.mark.parametrize("variant,alpha", [("ewainit", 0.5), ("ewainit", 0.3), ("plain", 1.0)])
def test_matches_c_oracle_trace(case, variant, alpha):
    """Same posterior as the C oracle (literal tanh/atanh in long double),
    also once messages saturate at the clip (they do by iteration 5)."""
    H, err, syn, prior = case
    T = 9
    g = unrolled.Graph(H)
    E = g.E
    Q = unrolled.forward(g, syn, prior, torch.full((T,), alpha, dtype=torch.float64),
                         torch.zeros(T, dtype=torch.float64), torch.ones(E, dtype=torch.float64), T)
    for b in range(syn.shape[0]):
        tr = oracle.trace(H, syn[b], prior, variant="ewainit", alpha=alpha, T=T)
        # near saturation the 64-bit-mantissa long double of the C oracle
        # limits the agreement to ~1e-6
        assert np.allclose(Q[b].numpy(), tr["Q"][-1], rtol=1e-8, atol=1e-5)


def test_full_damping_freezes_messages(case):
    """beta_t = 1: the variable-to-check messages stay at eq. (init), so
    every iteration sees the same check messages and with alpha = 1 the
    posterior is the same at every iteration."""
    H, err, syn, prior = case
    g = unrolled.Graph(H)
    args = (torch.ones(4, dtype=torch.float64), torch.ones(4, dtype=torch.float64),
            torch.ones(g.E, dtype=torch.float64))
    Q1 = unrolled.forward(g, syn, prior, args[0][:1], args[1][:1], args[2], 1)
    Q4 = unrolled.forward(g, syn, prior, *args, 4)
    assert torch.allclose(Q1, Q4, atol=1e-12)


def test_gradients_match_finite_differences(case):
    H, err, syn, prior = case
    T = 6
    g = unrolled.Graph(H)
    rng = np.random.default_rng(3)
    alpha = 0.5 + 0.2 * rng.standard_normal(T)
    beta = 0.1 * np.abs(rng.standard_normal(T))
    w = 1.0 + 0.1 * rng.standard_normal(g.E)
    L, ga, gb, gw = unrolled.loss_and_grads(H, syn[:2], err[:2], prior, alpha, beta, w, T)

    def f(a, b, ww):
        return float(unrolled.loss(unrolled.forward(g, syn[:2], prior, torch.tensor(a), torch.tensor(b),
                                                    torch.tensor(ww), T), err[:2]))

    h = 1e-6
    for k in [0, 2, T - 1]:
        d = np.zeros(T); d[k] = h
        assert (f(alpha + d, beta, w) - f(alpha - d, beta, w)) / (2 * h) == pytest.approx(ga[k], rel=1e-5, abs=1e-9)
        assert (f(alpha, beta + d, w) - f(alpha, beta - d, w)) / (2 * h) == pytest.approx(gb[k], rel=1e-5, abs=1e-9)
    for e in [0, 17, g.E - 1]:
        d = np.zeros(g.E); d[e] = h
        assert (f(alpha, beta, w + d) - f(alpha, beta, w - d)) / (2 * h) == pytest.approx(gw[e], rel=1e-5, abs=1e-9)


@pytest.mark.parametrize("alpha,gamma", [(0.5, 0.0), (0.7, 0.3)])
def test_momentum_model_matches_c_oracle_trace(case, alpha, gamma):
    """The Momentum model at constant alpha, gamma, beta = 0, w = 1 is
    Momentum-BP (eqs. (mombp1), (mombp2), (mombp5)): same posterior as the
    C oracle."""
    H, err, syn, prior = case
    T = 8
    g = unrolled.Graph(H)
    Q = unrolled.forward(g, syn, prior, torch.full((T,), alpha, dtype=torch.float64), torch.zeros(T, dtype=torch.float64),
                         torch.ones(g.E, dtype=torch.float64), T, model="momentum",
                         gamma=torch.full((T,), gamma, dtype=torch.float64))
    for b in range(syn.shape[0]):
        tr = oracle.trace(H, syn[b], prior, variant="momentum", alpha=alpha, gamma=gamma, T=T)
        assert np.allclose(Q[b].numpy(), tr["Q"][-1], rtol=1e-8, atol=1e-5)


def test_momentum_model_gradients_match_finite_differences(case):
    H, err, syn, prior = case
    T = 6
    g = unrolled.Graph(H)
    rng = np.random.default_rng(4)
    alpha = 0.6 + 0.1 * rng.standard_normal(T)
    gamma = 0.3 + 0.1 * rng.standard_normal(T)
    beta = 0.1 * np.abs(rng.standard_normal(T))
    w = 1.0 + 0.1 * rng.standard_normal(g.E)
    L, ga, gb, gw, gg = unrolled.loss_and_grads(H, syn[:2], err[:2], prior, alpha, beta, w, T, model="momentum",
                                                gamma=gamma)

    def f(a, b, ww, gm):
        return float(unrolled.loss(unrolled.forward(g, syn[:2], prior, torch.tensor(a), torch.tensor(b),
                                                    torch.tensor(ww), T, model="momentum", gamma=torch.tensor(gm)),
                                   err[:2]))

    h = 1e-6
    for k in [0, 2, T - 1]:
        d = np.zeros(T); d[k] = h
        assert (f(alpha + d, beta, w, gamma) - f(alpha - d, beta, w, gamma)) / (2 * h) == pytest.approx(
            ga[k], rel=1e-5, abs=1e-9)
        assert (f(alpha, beta, w, gamma + d) - f(alpha, beta, w, gamma - d)) / (2 * h) == pytest.approx(
            gg[k], rel=1e-5, abs=1e-9)
        assert (f(alpha, beta + d, w, gamma) - f(alpha, beta - d, w, gamma)) / (2 * h) == pytest.approx(
            gb[k], rel=1e-5, abs=1e-9)
    for e in [0, 17, g.E - 1]:
        d = np.zeros(g.E); d[e] = h
        assert (f(alpha, beta, w + d, gamma) - f(alpha, beta, w - d, gamma)) / (2 * h) == pytest.approx(
            gw[e], rel=1e-5, abs=1e-9)


# ---------------------------------------------------------------- coset loss


def brute_force_coset_term(pi, R, target):
    """-log P(<E^, R> = target) for one operator R by enumerating every
    assignment of Paulis to its support under the product distribution pi
    (N, 4) of (I, X, Y, Z)."""
    import itertools
    supp = np.nonzero(R)[0]
    P = 0.0
    for ops in itertools.product(range(4), repeat=supp.size):
        pr = np.prod([pi[j, o] for j, o in zip(supp, ops)])
        par = sum(int(o != 0 and o != R[j]) for j, o in zip(supp, ops)) % 2
        if par == target:
            P += pr
    return -np.log(P)


def test_coset_loss_matches_brute_force_enumeration():
    """Planar d = 3: every check's and logical's parity probability under
    random posterior marginals equals the sum over all 4^w assignments of
    its support (the parity convolution is exact), for two iterations."""
    H, _ = codes.build_code("planar", 3)
    Lg = codes.logical_operators(H)
    rng = np.random.default_rng(11)
    B, N = 2, H.shape[1]
    err = rng.integers(0, 4, size=(B, N)).astype(np.uint8)
    syn = codes.syndrome(H, err).astype(np.uint8)
    Qs = [torch.tensor(rng.normal(2.0, 2.5, size=(B, N, 3))) for _ in range(2)]
    got = float(unrolled.coset_loss(Qs, H, syn, err, Lg))
    total = 0.0
    for Q in Qs:
        for b in range(B):
            z = np.concatenate([np.zeros((N, 1)), -Q[b].numpy()], 1)
            pi = np.exp(z - z.max(1, keepdims=True))
            pi /= pi.sum(1, keepdims=True)
            chk = np.mean([brute_force_coset_term(pi, H[i], syn[b, i]) for i in range(H.shape[0])])
            tl = [int(sum(int(err[b, j] != 0 and Lg[l, j] != 0 and err[b, j] != Lg[l, j]) for j in range(N)) % 2)
                  for l in range(Lg.shape[0])]
            log = np.mean([brute_force_coset_term(pi, Lg[l], tl[l]) for l in range(Lg.shape[0])])
            total += chk + log
    assert got == pytest.approx(total / (len(Qs) * B), rel=1e-12)


def test_coset_loss_vanishes_on_a_certain_correct_posterior():
    """A posterior concentrated on the true error (or on any error of its
    coset with the same syndrome) gives P = 1 for every check and logical."""
    H, _ = codes.build_code("planar", 5)
    Lg = codes.logical_operators(H)
    ch = oracle.depolarizing(0.08)
    err, syn = oracle.sample(H, *ch, seed=5, shot0=0, B=4)
    B, N = err.shape
    Q = torch.full((B, N, 3), 60.0, dtype=torch.float64)
    for b in range(B):
        for j in range(N):
            if err[b, j]:
                Q[b, j, :] = 0.0
                Q[b, j, err[b, j] - 1] = -60.0
    assert float(unrolled.coset_loss([Q], H, syn, err, Lg)) < 1e-20
    # a logical error flips a logical parity: the loss is then large
    e2 = err.copy()
    e2[0] = codes.from_symplectic(codes.to_symplectic(err[0]) ^ codes.to_symplectic(Lg[0]))
    assert float(unrolled.coset_loss([Q[:1]], H, syn[:1], e2[:1], Lg)) > 10.0


def test_coset_loss_gradients_match_finite_differences(case):
    H, err, syn, prior = case
    Lg = codes.logical_operators(H)
    T = 5
    g = unrolled.Graph(H)
    rng = np.random.default_rng(8)
    alpha = 0.5 + 0.2 * rng.standard_normal(T)
    beta = 0.1 * np.abs(rng.standard_normal(T))
    w = 1.0 + 0.1 * rng.standard_normal(g.E)
    L, ga, gb, gw = unrolled.loss_and_grads(H, syn[:3], err[:3], prior, alpha, beta, w, T, kind="coset",
                                            logicals=Lg)

    def f(a, b, ww):
        Qs = unrolled.forward(g, syn[:3], prior, torch.tensor(a), torch.tensor(b), torch.tensor(ww), T, every=True)
        return float(unrolled.coset_loss(Qs, H, syn[:3], err[:3], Lg))

    assert f(alpha, beta, w) == pytest.approx(L, rel=1e-12)
    h = 1e-6
    for k in [0, 2, T - 1]:
        d = np.zeros(T); d[k] = h
        assert (f(alpha + d, beta, w) - f(alpha - d, beta, w)) / (2 * h) == pytest.approx(ga[k], rel=1e-5, abs=1e-9)
        assert (f(alpha, beta + d, w) - f(alpha, beta - d, w)) / (2 * h) == pytest.approx(gb[k], rel=1e-5, abs=1e-9)
    for e in [0, 17, g.E - 1]:
        d = np.zeros(g.E); d[e] = h
        assert (f(alpha, beta, w + d) - f(alpha, beta, w - d)) / (2 * h) == pytest.approx(gw[e], rel=1e-5, abs=1e-9)
