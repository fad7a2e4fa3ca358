"""Pins of the oracle's Momentum-BP, AdaGrad-BP and EWAInit-BP posterior
updates against the closed forms the paper derives (Theorem 1 and
Appendix B), the stated reductions (Sec. III-A1) and AdaGrad invariants.

Index convention of the closed forms: the sums run over k = 0 .. t-1 (the
printed upper limit t refers to a check message S^(0) that does not exist;
taking S^(0) = 0 gives the same value)."""
import numpy as np
import pytest

import oracle
from oracle import codes


@pytest.fixture(scope="module")
def shots():
    H, _ = codes.build_code("planar", 5)
    err, syn = oracle.sample(H, *oracle.depolarizing(0.08), seed=42, shot0=0, B=24)
    # keep shots with a nontrivial syndrome
    keep = syn.any(axis=1)
    return H, syn[keep][:12], np.tile(oracle.depolarizing(0.08), (H.shape[1], 1))


def pi0(prior):
    pI = 1 - prior.sum(axis=1, keepdims=True)
    return np.log(pI / prior)


@pytest.mark.parametrize("alpha", [0.3, 0.5, 0.8])
def test_theorem1_ewainit_closed_form(shots, alpha):
    H, syns, prior = shots
    P = pi0(prior)
    for syn in syns:
        tr = oracle.trace(H, syn, prior, variant="ewainit", alpha=alpha, T=10)
        S, Q = tr["S"], tr["Q"]
        for t in range(1, 11):
            want = P + sum((1 - alpha) ** k * S[t - k - 1] for k in range(t))
            assert np.allclose(Q[t - 1], want, rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("alpha", [0.3, 0.5, 0.7])
def test_momentum_closed_form_gamma0(shots, alpha):
    """Appendix B: with gamma = 0, Q^(t) = Pi + alpha sum_k (1-alpha)^k S^(t-k),
    and eq. (mombp4): Q^(t) = alpha (Pi + S^(t)) + (1 - alpha) Q^(t-1)."""
    H, syns, prior = shots
    P = pi0(prior)
    for syn in syns:
        tr = oracle.trace(H, syn, prior, variant="momentum", alpha=alpha, gamma=0.0, T=10)
        S, Q = tr["S"], tr["Q"]
        for t in range(1, 11):
            want = P + alpha * sum((1 - alpha) ** k * S[t - k - 1] for k in range(t))
            assert np.allclose(Q[t - 1], want, rtol=1e-12, atol=1e-10)
            prev = P if t == 1 else Q[t - 2]
            assert np.allclose(Q[t - 1], alpha * (P + S[t - 1]) + (1 - alpha) * prev, atol=1e-10)


@pytest.mark.parametrize("gamma", [0.3, 0.6])
def test_momentum_alpha1_form(shots, gamma):
    """Second form of eq. (mombp3) at alpha = 1:
    Q^(t) = gamma (Q^(t-1) - g^(t-1)) + (1 - gamma)(Pi + S^(t))."""
    H, syns, prior = shots
    P = pi0(prior)
    for syn in syns[:6]:
        tr = oracle.trace(H, syn, prior, variant="momentum", alpha=1.0, gamma=gamma, T=8)
        S, Q, g = tr["S"], tr["Q"], tr["aux"]
        for t in range(1, 9):
            Qp = P if t == 1 else Q[t - 2]
            gp = np.zeros_like(P) if t == 1 else g[t - 2]
            want = gamma * (Qp - gp) + (1 - gamma) * (P + S[t - 1])
            assert np.allclose(Q[t - 1], want, atol=1e-10)


def test_reductions_to_plain(shots):
    H, syns, prior = shots
    for syn in syns[:6]:
        ref = oracle.trace(H, syn, prior, variant="plain", T=8)
        ewa = oracle.trace(H, syn, prior, variant="ewainit", alpha=1.0, T=8)
        for k in ("m_v2c", "m_c2v", "Q", "dec"):
            assert (ewa[k] == ref[k]).all()
        mom = oracle.trace(H, syn, prior, variant="momentum", alpha=1.0, gamma=0.0, T=8)
        assert np.allclose(mom["Q"], ref["Q"], atol=1e-8)
        assert (mom["dec"] == ref["dec"]).all()


def test_ewainit_prior_refresh(shots):
    """Algorithm 2: Pi^(1) = Pi^(0) and Pi^(t) = alpha Pi^(0) + (1-alpha) Q^(t-1)."""
    H, syns, prior = shots
    P = pi0(prior)
    tr = oracle.trace(H, syns[0], prior, variant="ewainit", alpha=0.5, T=6)
    assert np.allclose(tr["aux"][0], P, atol=1e-12)
    for t in range(2, 7):
        assert np.allclose(tr["aux"][t - 1], 0.5 * P + 0.5 * tr["Q"][t - 2], atol=1e-12)


@pytest.mark.parametrize("from_iter1", [1, 0])
def test_adagrad_invariants(shots, from_iter1):
    """Sec. III-A2: (boost) takes effect after the first iteration, so
    iteration 1 equals plain BP; because G^(t) contains g'^(t)^2, every
    boosted step moves Q by at most alpha; G never decreases."""
    H, syns, prior = shots
    alpha = 5.0
    for syn in syns:
        ref = oracle.trace(H, syn, prior, variant="plain", T=1)
        tr = oracle.trace(H, syn, prior, variant="adagrad", alpha=alpha, T=12,
                          adagrad_g_from_iter1=from_iter1)
        assert np.allclose(tr["Q"][0], ref["Q"][0], atol=1e-12)
        assert np.allclose(tr["m_v2c"][:2], ref["m_v2c"][:2], atol=1e-12)
        steps = np.abs(np.diff(tr["Q"], axis=0))
        assert steps.max() <= alpha * (1 + 1e-12)
        G = tr["aux"]
        assert (np.diff(G, axis=0) >= 0).all()
        if from_iter1:
            assert np.allclose(G[0], tr["S"][0] ** 2, atol=1e-9)  # g'^(1) = -S^(1)
        else:
            assert (G[0] == 0).all()


def test_adagrad_small_rate_freezes_posterior(shots):
    """With a vanishing boost rate the posterior stays at Q^(1)."""
    H, syns, prior = shots
    tr = oracle.trace(H, syns[0], prior, variant="adagrad", alpha=1e-9, T=6)
    assert np.allclose(tr["Q"][1:], tr["Q"][0][None], atol=1e-7)


@pytest.fixture(scope="module")
def aewa_runs():
    """Planar d = 7 at depolarising p = 0.08 (one of the Appendix C
    workloads): AEWA-BP and EWAInit-BP at each of its eleven alphas."""
    H, _ = codes.build_code("planar", 7)
    ch = oracle.depolarizing(0.08)
    _, syn = oracle.sample(H, *ch, seed=77, shot0=0, B=600)
    prior = np.tile(ch, (H.shape[1], 1))
    aewa = oracle.decode(H, syn, prior, variant="aewa", max_iter=60, nthreads=4)
    runs = [oracle.decode(H, syn, prior, variant="ewainit", alpha=1.0 - 0.1 * k, max_iter=60, nthreads=4)
            for k in range(11)]
    plain = oracle.decode(H, syn, prior, variant="plain", max_iter=60, nthreads=4)
    return aewa, runs, plain


def test_aewa_takes_the_first_converging_alpha(aewa_runs):
    """Appendix C: alpha = 1.0, 0.9, ..., 0.0 is tried in turn and the first
    run that satisfies the syndrome is the output; if none does, the output is
    the alpha = 0 run, unconverged.  Brute force over the eleven runs."""
    (est, conv, iters), runs, _ = aewa_runs
    conv_k = np.stack([r[1] for r in runs])                     # (11, B)
    assert (conv == conv_k.any(axis=0)).all()
    first = np.where(conv_k.any(axis=0), conv_k.argmax(axis=0), 10)
    for b in range(est.shape[0]):
        e_k, _, it_k = runs[first[b]]
        assert (est[b] == e_k[b]).all() and iters[b] == it_k[b], b
    # the schedule is needed: some shots converge only at alpha < 1, and
    # at smaller alpha than EWAInit's usual 0.5 too
    assert (first > 0).any() and (first[conv] > 5).any()


def test_aewa_first_attempt_is_plain_bp(aewa_runs):
    """At alpha = 1, Pi^(t) = Pi^(0) (eq. (EWAInit)), i.e. LLR-BP4: where
    plain BP converges AEWA-BP returns its result exactly."""
    (est, conv, iters), _, (est_p, conv_p, iters_p) = aewa_runs
    assert conv[conv_p].all()
    assert (est[conv_p] == est_p[conv_p]).all() and (iters[conv_p] == iters_p[conv_p]).all()
    assert conv.mean() > conv_p.mean()
