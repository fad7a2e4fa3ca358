"""Pins of the oracle's prior LLR, lambda function and horizontal update
against closed forms and textbook identities (Sec. II-B1)."""
import numpy as np
import pytest

import oracle
from inputs import X, Y, Z, random_priors


def star_code(paulis):
    """One check on len(paulis) qubits with the given Pauli entries."""
    return np.array([paulis], dtype=np.uint8)


@pytest.mark.parametrize("p", [0.001, 0.01, 0.05, 0.1, 0.16, 0.3])
def test_initial_message_closed_form_depolarizing(p):
    """Depolarising prior: Pi_W = ln(3(1-p)/p) and lambda(Pi) =
    ln((1 - 2p/3) / (2p/3)), the log-odds of commuting with a check entry."""
    H = star_code([X, Y, Z])
    tr = oracle.trace(H, [0], oracle.depolarizing(p), T=1)
    want = np.log((1 - 2 * p / 3) / (2 * p / 3))
    assert np.allclose(tr["m_v2c"][0], want, rtol=0, atol=1e-12)
    # Plain BP records Pi^(0) as its auxiliary state
    assert np.allclose(tr["aux"][0], np.log(3 * (1 - p) / p), atol=1e-12)


def test_lambda_is_commutation_log_odds():
    """lambda_{H}(Pi) = ln P(E commutes with H) / P(E anticommutes with H)
    computed from the probabilities directly: (p^I + p^H) / (sum of the other two)."""
    pri = random_priors(3, seed=11)
    for h in (X, Y, Z):
        H = star_code([h, h, h])
        tr = oracle.trace(H, [0], pri, T=1)
        for j in range(3):
            pX, pY, pZ = pri[j]
            pI = 1 - pX - pY - pZ
            p = {X: pX, Y: pY, Z: pZ}
            anti = sum(v for k, v in p.items() if k != h)
            assert tr["m_v2c"][0][j] == pytest.approx(np.log((pI + p[h]) / anti), abs=1e-12)


@pytest.mark.parametrize("s", [0, 1])
def test_degree_two_check_forwards_the_other_message(s):
    """A weight-2 check passes (-1)^s times the other qubit's message."""
    pri = random_priors(2, seed=5)
    H = star_code([X, Z])
    tr = oracle.trace(H, [s], pri, T=1)
    m0, m1 = tr["m_v2c"][0]
    sign = -1.0 if s else 1.0
    assert tr["m_c2v"][0][0] == pytest.approx(sign * m1, abs=1e-12)
    assert tr["m_c2v"][0][1] == pytest.approx(sign * m0, abs=1e-12)


def boxplus(a, b):
    """Hagenauer's box-plus written with min and two log1p corrections."""
    return (np.sign(a) * np.sign(b) * min(abs(a), abs(b))
            + np.log1p(np.exp(-abs(a + b))) - np.log1p(np.exp(-abs(a - b))))


@pytest.mark.parametrize("seed", range(6))
def test_check_update_matches_boxplus(seed):
    """For a weight-4 check, 2 atanh(prod tanh(m/2)) over the other three
    edges equals the box-plus of those three messages."""
    pri = random_priors(4, seed=seed, lo=0.005, hi=0.3)
    H = star_code([X, Y, Z, X])
    for s in (0, 1):
        tr = oracle.trace(H, [s], pri, T=1)
        m = tr["m_v2c"][0]
        for e in range(4):
            others = [m[f] for f in range(4) if f != e]
            want = boxplus(boxplus(others[0], others[1]), others[2]) * (-1 if s else 1)
            assert tr["m_c2v"][0][e] == pytest.approx(want, abs=1e-10)


def test_clip_applies_to_messages():
    """A weight-1 check gives an infinite check message, clipped to the
    saturation value (msg_clip) on both message directions."""
    H = np.array([[X, 0], [Z, Z]], dtype=np.uint8)
    tr = oracle.trace(H, [1, 0], oracle.depolarizing(0.01), T=3, msg_clip=25.0)
    assert tr["m_c2v"][0][0] == -25.0
    assert np.abs(tr["m_v2c"]).max() <= 25.0
