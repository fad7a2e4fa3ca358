"""Differentiable unrolled EWAInit-BP on the GPU (bpq_train_forward /
bpq_train_backward behind a torch.autograd.Function) against the float64
oracle (oracle/unrolled.py): the loss, the gradients of the oracle
(autograd) and FP64 central finite differences of the oracle forward."""
import numpy as np
import pytest
import torch

import oracle
from oracle import unrolled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bpq():
    import paper_2407_11523_gb300 as bpq
    return bpq


def setup(bpq, B, p, seed, d=9):
    t = bpq.Tanner("planar", d)
    ch = oracle.depolarizing(p)
    err, syn = bpq.sample(t, *ch, seed=seed, shot0=0, B=B)
    prior = bpq.prior_tensor(t, *ch)
    return t, err, syn, prior, ch


def params(T, E, seed, spread=0.0):
    rng = np.random.default_rng(seed)
    a = 0.5 + spread * rng.standard_normal(T)
    b = spread * np.abs(rng.standard_normal(T))
    w = 1.0 + spread * rng.standard_normal(E)
    return a, b, w


def oracle_inputs(t, err, syn, ch):
    from inputs import unpack_bits
    H = t.dense()
    s = unpack_bits(syn.cpu().numpy().view(np.uint32), t.M)
    e = err.cpu().numpy()
    prior = np.tile(np.asarray(ch, dtype=np.float32).astype(np.float64), (t.N, 1))
    return H, s, e, prior


@pytest.mark.parametrize("T,K", [(8, 5), (25, 5), (25, 25)])
def test_loss_matches_oracle(bpq, T, K):
    t, err, syn, prior, ch = setup(bpq, 32, 0.05, 1)
    a, b, w = params(T, t.E, 2, spread=0.05)
    L = bpq.unrolled_loss(t, syn, err, prior, torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda"),
                          torch.tensor(w, device="cuda"), T=T, ckpt_every=K)
    H, s, e, pri = oracle_inputs(t, err, syn, ch)
    Lr = float(unrolled.loss(unrolled.forward(unrolled.Graph(H), s, pri, torch.tensor(a), torch.tensor(b),
                                              torch.tensor(w), T), e))
    assert L.item() == pytest.approx(Lr, rel=2e-4)


@pytest.mark.parametrize("T", [6, 12])
def test_gradients_match_oracle_and_finite_differences(bpq, T):
    t, err, syn, prior, ch = setup(bpq, 8, 0.06, 3)
    a, b, w = params(T, t.E, 4, spread=0.1)
    ta = torch.tensor(a, device="cuda", dtype=torch.float32, requires_grad=True)
    tb = torch.tensor(b, device="cuda", dtype=torch.float32, requires_grad=True)
    tw = torch.tensor(w, device="cuda", dtype=torch.float32, requires_grad=True)
    L = bpq.unrolled_loss(t, syn, err, prior, ta, tb, tw, T=T, ckpt_every=5)
    L.backward()
    ga, gb, gw = (x.grad.detach().cpu().numpy().astype(np.float64) for x in (ta, tb, tw))
    H, s, e, pri = oracle_inputs(t, err, syn, ch)
    Lr, ra, rb, rw = unrolled.loss_and_grads(H, s, e, pri, a, b, w, T)
    for g, r in ((ga, ra), (gb, rb), (gw, rw)):
        scale = np.abs(r).max()
        assert np.abs(g - r).max() <= 2e-3 * scale + 1e-7, (np.abs(g - r).max(), scale)
    # FP64 central differences of the oracle forward, for a few coordinates
    g = unrolled.Graph(H)

    def f(aa, bb, ww):
        return float(unrolled.loss(unrolled.forward(g, s, pri, torch.tensor(aa), torch.tensor(bb),
                                                    torch.tensor(ww), T), e))

    h = 1e-6
    for k in (1, T - 1):
        dv = np.zeros(T); dv[k] = h
        fd = (f(a + dv, b, w) - f(a - dv, b, w)) / (2 * h)
        assert ga[k] == pytest.approx(fd, rel=5e-3, abs=1e-6)
    for k in (3, 100, t.E - 1):
        dv = np.zeros(t.E); dv[k] = h
        fd = (f(a, b, w + dv) - f(a, b, w - dv)) / (2 * h)
        assert gw[k] == pytest.approx(fd, rel=5e-3, abs=1e-6)


def test_backward_is_deterministic_and_checkpoint_independent(bpq):
    t, err, syn, prior, ch = setup(bpq, 64, 0.07, 5)
    T = 25
    a, b, w = params(T, t.E, 6, spread=0.05)
    grads = []
    for K in (5, 5, 25, 7):
        ta = torch.tensor(a, device="cuda", dtype=torch.float32, requires_grad=True)
        tb = torch.tensor(b, device="cuda", dtype=torch.float32, requires_grad=True)
        tw = torch.tensor(w, device="cuda", dtype=torch.float32, requires_grad=True)
        bpq.unrolled_loss(t, syn, err, prior, ta, tb, tw, T=T, ckpt_every=K).backward()
        grads.append([x.grad.clone() for x in (ta, tb, tw)])
    for g0, g1 in zip(grads[0], grads[1]):
        assert torch.equal(g0, g1)
    for gk in grads[2:]:
        for g0, g1 in zip(grads[0], gk):
            assert torch.equal(g0, g1)  # recomputation reproduces the forward exactly


def test_training_lowers_the_loss(bpq):
    t, err, syn, prior, ch = setup(bpq, 1024, 0.06, 9)
    T = 25
    a = torch.full((T,), 0.5, device="cuda", requires_grad=True)
    b = torch.zeros(T, device="cuda", requires_grad=True)
    w = torch.ones(t.E, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([a, b, w], lr=0.02)
    losses = []
    for _ in range(15):
        opt.zero_grad()
        L = bpq.unrolled_loss(t, syn, err, prior, a, b, w, T=T)
        L.backward()
        opt.step()
        with torch.no_grad():
            a.clamp_(0.0, 1.0)
            b.clamp_(0.0, 0.95)
        losses.append(L.item())
    assert losses[-1] < losses[0]


def test_momentum_model_at_fixed_parameters_is_momentum_bp(bpq):
    """The Momentum model at constant alpha, gamma, beta = 0, w = 1 is
    Momentum-BP (eqs. (mombp1), (mombp2), (mombp5)): its final posterior
    matches the C oracle's Momentum-BP trace."""
    t, err, syn, prior, ch = setup(bpq, 16, 0.05, 11, d=7)
    T = 10
    Q, _ = bpq.unrolled_posterior(t, syn, err, prior, torch.full((T,), 0.6, device="cuda"),
                                  torch.zeros(T, device="cuda"), torch.ones(t.E, device="cuda"), T=T,
                                  model="momentum", gamma=torch.full((T,), 0.3, device="cuda"))
    H, s, e, pri = oracle_inputs(t, err, syn, ch)
    Q = Q.cpu().numpy()
    for b in range(s.shape[0]):
        tr = oracle.trace(H, s[b], pri, variant="momentum", alpha=0.6, gamma=0.3, T=T)
        assert np.abs(Q[b] - tr["Q"][-1]).max() <= 4e-4 + 1e-5 * np.abs(tr["Q"][-1]).max()


@pytest.mark.parametrize("T", [6, 12])
def test_momentum_gradients_match_oracle_and_finite_differences(bpq, T):
    t, err, syn, prior, ch = setup(bpq, 8, 0.06, 13)
    rng = np.random.default_rng(14)
    a = 0.6 + 0.1 * rng.standard_normal(T)
    gm = 0.3 + 0.1 * rng.standard_normal(T)
    b = 0.1 * np.abs(rng.standard_normal(T))
    w = 1.0 + 0.1 * rng.standard_normal(t.E)
    ts = [torch.tensor(x, device="cuda", dtype=torch.float32, requires_grad=True) for x in (a, b, w, gm)]
    L = bpq.unrolled_loss(t, syn, err, prior, ts[0], ts[1], ts[2], T=T, ckpt_every=5, model="momentum",
                          gamma=ts[3])
    L.backward()
    ga, gb, gw, gg = (x.grad.detach().cpu().numpy().astype(np.float64) for x in ts)
    H, s, e, pri = oracle_inputs(t, err, syn, ch)
    Lr, ra, rb, rw, rg = unrolled.loss_and_grads(H, s, e, pri, a, b, w, T, model="momentum", gamma=gm)
    assert L.item() == pytest.approx(Lr, rel=2e-4)
    for g, r in ((ga, ra), (gb, rb), (gw, rw), (gg, rg)):
        scale = np.abs(r).max()
        assert np.abs(g - r).max() <= 2e-3 * scale + 1e-7, (np.abs(g - r).max(), scale)
    g = unrolled.Graph(H)

    def f(aa, gg_):
        return float(unrolled.loss(unrolled.forward(g, s, pri, torch.tensor(aa), torch.tensor(b), torch.tensor(w), T,
                                                    model="momentum", gamma=torch.tensor(gg_)), e))

    h = 1e-6
    for k in (0, T - 1):
        dv = np.zeros(T); dv[k] = h
        assert ga[k] == pytest.approx((f(a + dv, gm) - f(a - dv, gm)) / (2 * h), rel=5e-3, abs=1e-6)
        assert gg[k] == pytest.approx((f(a, gm + dv) - f(a, gm - dv)) / (2 * h), rel=5e-3, abs=1e-6)


def test_momentum_backward_is_checkpoint_independent(bpq):
    t, err, syn, prior, ch = setup(bpq, 32, 0.07, 15)
    T = 20
    rng = np.random.default_rng(16)
    vals = (0.6 + 0.05 * rng.standard_normal(T), 0.05 * np.abs(rng.standard_normal(T)),
            1.0 + 0.05 * rng.standard_normal(t.E), 0.3 + 0.05 * rng.standard_normal(T))
    grads = []
    for K in (5, 20, 7):
        ts = [torch.tensor(x, device="cuda", dtype=torch.float32, requires_grad=True) for x in vals]
        bpq.unrolled_loss(t, syn, err, prior, ts[0], ts[1], ts[2], T=T, ckpt_every=K, model="momentum",
                          gamma=ts[3]).backward()
        grads.append([x.grad.clone() for x in ts])
    for gk in grads[1:]:
        for g0, g1 in zip(grads[0], gk):
            assert torch.equal(g0, g1)


# ---------------------------------------------------------------- coset loss


@pytest.mark.parametrize("model,T,K", [("ewainit", 8, 5), ("ewainit", 25, 5), ("momentum", 12, 5)])
def test_coset_loss_matches_oracle(bpq, model, T, K):
    """The coset loss (every iteration's checks and logicals) against the
    oracle's coset_loss, with the oracle's own logical operators passed to
    the kernel."""
    from oracle import codes
    t, err, syn, prior, ch = setup(bpq, 32, 0.05, 21)
    a, b, w = params(T, t.E, 22, spread=0.05)
    gm = np.full(T, 0.3)
    H, s, e, pri = oracle_inputs(t, err, syn, ch)
    Lg = codes.logical_operators(H)
    kw = dict(model=model, gamma=torch.tensor(gm, device="cuda", dtype=torch.float32) if model == "momentum" else None)
    L = bpq.unrolled_loss(t, syn, err, prior, torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda"),
                          torch.tensor(w, device="cuda"), T=T, ckpt_every=K, loss="coset", logicals=Lg, **kw)
    Qs = unrolled.forward(unrolled.Graph(H), s, pri, torch.tensor(a), torch.tensor(b), torch.tensor(w), T,
                          model=model, gamma=torch.tensor(gm) if model == "momentum" else None, every=True)
    Lr = float(unrolled.coset_loss(Qs, H, s, e, Lg))
    assert L.item() == pytest.approx(Lr, rel=2e-4)


@pytest.mark.parametrize("model", ["ewainit", "momentum"])
def test_coset_gradients_match_oracle_and_finite_differences(bpq, model):
    from oracle import codes
    T = 8
    t, err, syn, prior, ch = setup(bpq, 8, 0.06, 23)
    a, b, w = params(T, t.E, 24, spread=0.1)
    gm = 0.3 + 0.05 * np.random.default_rng(25).standard_normal(T)
    H, s, e, pri = oracle_inputs(t, err, syn, ch)
    Lg = codes.logical_operators(H)
    vals = (a, b, w) + ((gm,) if model == "momentum" else ())
    ts = [torch.tensor(x, device="cuda", dtype=torch.float32, requires_grad=True) for x in vals]
    L = bpq.unrolled_loss(t, syn, err, prior, ts[0], ts[1], ts[2], T=T, ckpt_every=5, model=model,
                          gamma=ts[3] if model == "momentum" else None, loss="coset", logicals=Lg)
    L.backward()
    got = [x.grad.detach().cpu().numpy().astype(np.float64) for x in ts]
    ref = unrolled.loss_and_grads(H, s, e, pri, a, b, w, T, model=model, gamma=gm if model == "momentum" else None,
                                  kind="coset", logicals=Lg)
    assert L.item() == pytest.approx(ref[0], rel=2e-4)
    for g, r in zip(got, ref[1:]):
        scale = np.abs(r).max()
        assert np.abs(g - r).max() <= 2e-3 * scale + 1e-7, (np.abs(g - r).max(), scale)
    g_ = unrolled.Graph(H)

    def f(aa, ww):
        Qs = unrolled.forward(g_, s, pri, torch.tensor(aa), torch.tensor(b), torch.tensor(ww), T, model=model,
                              gamma=torch.tensor(gm) if model == "momentum" else None, every=True)
        return float(unrolled.coset_loss(Qs, H, s, e, Lg))

    h = 1e-6
    for k in (1, T - 1):
        dv = np.zeros(T); dv[k] = h
        assert got[0][k] == pytest.approx((f(a + dv, w) - f(a - dv, w)) / (2 * h), rel=5e-3, abs=1e-6)
    for k in (3, 100, t.E - 1):
        dv = np.zeros(t.E); dv[k] = h
        assert got[2][k] == pytest.approx((f(a, w + dv) - f(a, w - dv)) / (2 * h), rel=5e-3, abs=1e-6)


def test_coset_backward_is_deterministic_and_checkpoint_independent(bpq):
    t, err, syn, prior, ch = setup(bpq, 64, 0.07, 27)
    T = 20
    a, b, w = params(T, t.E, 28, spread=0.05)
    grads = []
    for K in (5, 5, 20, 7):
        ts = [torch.tensor(x, device="cuda", dtype=torch.float32, requires_grad=True) for x in (a, b, w)]
        bpq.unrolled_loss(t, syn, err, prior, *ts, T=T, ckpt_every=K, loss="coset").backward()
        grads.append([x.grad.clone() for x in ts])
    for gk in grads[1:]:
        for g0, g1 in zip(grads[0], gk):
            assert torch.equal(g0, g1)


def test_coset_loss_refusals(bpq):
    t, err, syn, prior, ch = setup(bpq, 4, 0.05, 29, d=5)
    T = 4
    args = (torch.full((T,), 0.5, device="cuda"), torch.zeros(T, device="cuda"), torch.ones(t.E, device="cuda"))
    with pytest.raises(bpq.BPQError):
        bpq.unrolled_loss(t, syn, err, prior, *args, T=T, loss="coset", logicals=np.zeros((5, t.N), np.uint8))
    with pytest.raises(bpq.BPQError):
        bpq.unrolled_loss(t, syn, err, prior, *args, T=T, loss="coset", logicals=np.zeros((0, t.N), np.uint8))
