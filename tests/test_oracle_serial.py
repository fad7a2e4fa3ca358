"""Pins of the oracle's serial schedule (Algorithm 1's serial update: the
qubits in order, each taking the c->v messages of its checks from the
v->c messages as they stand, then updating its posterior and sending new
v->c messages).  Table I's serial rows need the missing Fig. 2 and are not
pinned; see the design notes."""
import numpy as np
import pytest

import oracle
from inputs import random_priors, random_syndromes, random_tree_code
from oracle import codes
from test_oracle_tree import brute_force_posterior_llr


def boxplus(a, b):
    """Hagenauer's pairwise box-plus: 2 atanh(tanh(a/2) tanh(b/2)) written as
    sign(a) sign(b) min(|a|,|b|) + log1p(e^-|a+b|) - log1p(e^-|a-b|)."""
    return (np.sign(a) * np.sign(b) * np.minimum(abs(a), abs(b))
            + np.log1p(np.exp(-abs(a + b))) - np.log1p(np.exp(-abs(a - b))))


@pytest.mark.parametrize("seed", range(8))
def test_serial_plain_bp_is_exact_on_trees(seed):
    """BP is exact on a tree under any schedule that keeps sweeping."""
    n = 4 + seed % 5
    H = random_tree_code(n, seed=100 + seed)
    prior = random_priors(n, seed=200 + seed)
    for syn in random_syndromes(H.shape[0], 3, seed=300 + seed):
        tr = oracle.trace(H, syn, prior, variant="plain", T=2 * n, schedule="serial")
        want = brute_force_posterior_llr(H, prior, syn)
        assert np.allclose(tr["Q"][-1], want, rtol=0, atol=1e-9)


@pytest.mark.parametrize("variant,kw", [("plain", {}), ("ewainit", {"alpha": 0.5}),
                                        ("momentum", {"alpha": 0.6, "gamma": 0.3}), ("adagrad", {"alpha": 5.0})])
def test_serial_messages_follow_the_sweep_order(variant, kw):
    """At its turn in sweep t, qubit j reads, on each of its checks, the
    v->c message of sweep t from the qubits before it and that of sweep t-1
    from the qubits after it; the c->v message is the check update of those
    (recomputed here with pairwise box-plus), with the syndrome sign."""
    H, _ = codes.build_code("planar", 5)
    ch = oracle.depolarizing(0.08)
    _, syn = oracle.sample(H, *ch, seed=5, shot0=0, B=6)
    prior = np.tile(ch, (H.shape[1], 1))
    ii, jj, _ = oracle.edges(H)
    for s in syn:
        T = 4
        tr = oracle.trace(H, s, prior, variant=variant, T=T, schedule="serial", **kw)
        for t in range(1, T + 1):
            for e in range(ii.size):
                others = [f for f in np.nonzero(ii == ii[e])[0] if f != e]
                vals = [tr["m_v2c"][t][f] if jj[f] < jj[e] else tr["m_v2c"][t - 1][f] for f in others]
                acc = vals[0]
                for v in vals[1:]:
                    acc = boxplus(acc, v)
                want = np.clip(-acc if s[ii[e]] else acc, -30, 30)
                # the oracle's long double tanh product resolves 1 - tanh(|m|/2)
                # to 2^-63, i.e. |m| to about 2^-63 e^|m| near saturation
                tol = 1e-9 + 2.0 ** -63 * np.exp(abs(want))
                assert abs(tr["m_c2v"][t - 1][e] - want) < tol, (variant, t, e)


def test_serial_reductions_to_plain():
    """EWAInit-BP at alpha = 1 is plain BP bit for bit under the serial
    schedule too (eq. (EWAInit)); Momentum-BP at alpha = 1, gamma = 0 equals
    plain BP (Sec. III-A1)."""
    H, _ = codes.build_code("toric", 4)
    ch = oracle.depolarizing(0.1)
    _, syn = oracle.sample(H, *ch, seed=9, shot0=0, B=5)
    prior = np.tile(ch, (H.shape[1], 1))
    for s in syn:
        ref = oracle.trace(H, s, prior, variant="plain", T=8, schedule="serial")
        ewa = oracle.trace(H, s, prior, variant="ewainit", alpha=1.0, T=8, schedule="serial")
        for k in ("m_v2c", "m_c2v", "Q", "dec"):
            assert (ewa[k] == ref[k]).all()
        mom = oracle.trace(H, s, prior, variant="momentum", alpha=1.0, gamma=0.0, T=8, schedule="serial")
        assert np.allclose(mom["Q"], ref["Q"], atol=1e-8)


def test_serial_equals_parallel_where_no_earlier_neighbour():
    """In the first sweep, a c->v message into a qubit from a check whose
    other qubits all come later is built from the initial messages only,
    exactly as under the parallel schedule; qubit 0 sees only such checks,
    so its whole first posterior matches."""
    H, _ = codes.build_code("planar", 5)
    ch = oracle.depolarizing(0.06)
    _, syn = oracle.sample(H, *ch, seed=3, shot0=0, B=4)
    prior = np.tile(ch, (H.shape[1], 1))
    ii, jj, _ = oracle.edges(H)
    fresh = np.array([jj[ii == ii[e]].min() == jj[e] for e in range(ii.size)])
    assert fresh.sum() >= H.shape[0] and not fresh.all()
    for s in syn:
        ser = oracle.trace(H, s, prior, variant="plain", T=1, schedule="serial")
        par = oracle.trace(H, s, prior, variant="plain", T=1)
        assert (ser["m_c2v"][0][fresh] == par["m_c2v"][0][fresh]).all()
        assert not np.allclose(ser["m_c2v"][0][~fresh], par["m_c2v"][0][~fresh])
        assert np.allclose(ser["Q"][0][0], par["Q"][0][0], rtol=0, atol=1e-12)


def test_serial_converges_faster_than_parallel():
    """Sec. II-B: the serial schedule converges faster (and is slightly more
    accurate) than the parallel one; planar d = 7 at p = 0.05, plain BP."""
    H, _ = codes.build_code("planar", 7)
    ch = oracle.depolarizing(0.05)
    err, syn = oracle.sample(H, *ch, seed=11, shot0=0, B=600)
    prior = np.tile(ch, (H.shape[1], 1))
    e_p, c_p, it_p = oracle.decode(H, syn, prior, "plain", max_iter=50, nthreads=4)
    e_s, c_s, it_s = oracle.decode(H, syn, prior, "plain", max_iter=50, nthreads=4, schedule="serial")
    assert it_s[c_s & c_p].mean() < it_p[c_s & c_p].mean()
    f_p, _ = codes.logical_failure(H, err, e_p)
    f_s, _ = codes.logical_failure(H, err, e_s)
    assert f_s.mean() <= f_p.mean()
