"""Oracle for the differentiable, unrolled EWAInit-BP decoder.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): plain float64 PyTorch CPU
code, differentiated by torch.autograd, used to check the CUDA forward and
backward kernels.

The model is EWAInit-BP (Sec. III-B, Algorithm 2) run for a fixed number T
of flooding iterations, without the stopping rule, with three sets of
trainable parameters added in the manner of neural BP (the paper's
conclusion points to neural BP as a way to strengthen the algorithm):

  * alpha_t, t = 1..T: the EWA weight of iteration t,
        Pi^(t) = alpha_t Pi^(0) + (1 - alpha_t) Q^(t-1)      (t > 1; eq. (EWAInit));
  * beta_t: damping of the variable-to-check messages,
        m_v->c^(t) = (1 - beta_t) lambda(...) + beta_t m_v->c^(t-1);
  * w_e: a weight on each check-to-variable message,
        m_c->v^(t) = w_e (-1)^{s_i} 2 atanh(prod tanh(m_v->c^(t-1)/2))  (eq. (h_update)).

With alpha_t = alpha, beta_t = 0 and w_e = 1 it is EWAInit-BP exactly.

The Momentum model replaces the EWA prior by Momentum-BP's posterior
recursion (Sec. III-A1, eqs. (mombp1), (mombp2) with the gradient of
(mombp3)), with a trainable step alpha_t and momentum rate gamma_t:

  g^(t) = gamma_t g^(t-1) + (1 - gamma_t) (Q^(t-1) - Pi^(0) - S^(t)),
  Q^(t) = Q^(t-1) - alpha_t g^(t),         Q^(0) = Pi^(0), g^(0) = 0,

and the same beta_t, w_e; alpha_t = alpha, gamma_t = gamma, beta_t = 0,
w_e = 1 is Momentum-BP.  In both models the v->c message is lambda of the
posterior minus the edge's own message (eq. (mombp5); for EWAInit this is
eq. (v_update), since Q = Pi^(t) + S).
Messages are clipped to [-clip, clip] as in the decoder.  Two losses: the
cross-entropy of the final posterior against the true error, averaged over
qubits and shots (per qubit the log-probabilities of (I, X, Y, Z) are
log softmax(0, -Q_X, -Q_Y, -Q_Z), since Q_W = ln P(I)/P(W)); and the coset
loss (coset_loss): for every iteration, -log of the probability, under the
product of the posterior marginals, that the estimate satisfies each check's
syndrome bit and has the true error's parity with each logical operator,
averaged over checks, logicals, iterations and shots.
"""
from __future__ import annotations

import numpy as np
import torch


def _anti(a, b):
    return (a != 0) & (b != 0) & (a != b)


class Graph:
    """Check-major edge list of a Pauli check matrix and the index arrays the
    vectorised forward needs."""

    def __init__(self, H: np.ndarray):
        H = np.asarray(H)
        self.M, self.N = H.shape
        ii, jj = np.nonzero(H)
        self.E = ii.size
        self.chk = torch.as_tensor(ii, dtype=torch.long)
        self.var = torch.as_tensor(jj, dtype=torch.long)
        self.pauli = torch.as_tensor(H[ii, jj].astype(np.int64))
        # the other edges of the same check (padded with -1)
        others = []
        for e in range(self.E):
            o = [f for f in np.nonzero(ii == ii[e])[0] if f != e]
            others.append(o + [-1] * (3 - len(o)))
        self.others = torch.as_tensor(np.array(others, dtype=np.int64))
        # anticommutation of each edge with W = X, Y, Z: (E, 3)
        self.anti = torch.as_tensor(np.stack([_anti(np.full(self.E, w), H[ii, jj]) for w in (1, 2, 3)], 1)
                                    .astype(np.float64))
        # one-hot of the commuting Pauli H of each edge: (E, 3)
        self.own = torch.as_tensor(np.stack([H[ii, jj] == w for w in (1, 2, 3)], 1).astype(np.float64))


def lam(q: torch.Tensor, own: torch.Tensor, anti: torch.Tensor) -> torch.Tensor:
    """lambda_H(q) = ln((1 + e^{-q_H}) / sum_{W != H} e^{-q_W}), eq. (lambda);
    q: (..., E, 3)."""
    num = 1.0 + (torch.exp(-q) * own).sum(-1)
    den = (torch.exp(-q) * anti).sum(-1)
    return torch.log(num / den)


def phi(x: torch.Tensor) -> torch.Tensor:
    """phi(x) = -ln tanh(x/2) for x >= 0 (its own inverse)."""
    return torch.log1p(2.0 / torch.expm1(x))


def forward(g: Graph, syn, prior, alpha, beta, w, T: int, clip: float = 30.0, model: str = "ewainit",
            gamma=None, every: bool = False):
    """Q^(T) (B, N, 3) of the unrolled decoder (every=True: the list of
    Q^(1) .. Q^(T)).  syn: (B, M) 0/1; prior: (N, 3) probabilities; alpha,
    beta (and gamma for model "momentum"): (T,); w: (E,)."""
    syn = torch.as_tensor(np.asarray(syn), dtype=torch.float64)
    prior = torch.as_tensor(np.asarray(prior), dtype=torch.float64)
    B = syn.shape[0]
    pI = 1.0 - prior.sum(-1, keepdim=True)
    Pi0 = torch.log(pI / prior)                                   # (N, 3)
    sign = 1.0 - 2.0 * syn[:, g.chk]                              # (B, E): (-1)^{s_i}
    v2c = lam(Pi0[g.var].expand(B, g.E, 3), g.own, g.anti).clamp(-clip, clip)   # eq. (init)
    Qprev = Pi0.expand(B, g.N, 3)
    Q = Qprev
    Qs = []
    gm = torch.zeros(B, g.N, 3, dtype=torch.float64)
    for t in range(T):
        Pit = Pi0 if t == 0 else alpha[t] * Pi0 + (1.0 - alpha[t]) * Qprev
        # eq. (h_update): 2 atanh(prod_f tanh(m_f/2)) written with Gallager's
        # identity  = prod_f sign(m_f) * phi(sum_f phi(|m_f|)),
        # phi(x) = -ln tanh(x/2) = log1p(2/expm1(x)), which keeps full double
        # accuracy near message saturation (the literal product loses ~1e-4
        # there) and gives the stable derivative sinh(m_out)/sinh(m_f)
        mag = phi(v2c.abs())
        sgn = torch.sign(v2c)
        mag_pad = torch.cat([mag, torch.zeros(B, 1, dtype=mag.dtype)], 1)         # index -1 -> phi = 0
        sgn_pad = torch.cat([sgn, torch.ones(B, 1, dtype=sgn.dtype)], 1)
        ext = mag_pad[:, g.others].sum(-1)                                         # (B, E)
        psign = sgn_pad[:, g.others].prod(-1)
        c2v = (w * sign * psign * phi(ext)).clamp(-clip, clip)
        S = torch.zeros(B, g.N, 3, dtype=torch.float64).index_add(1, g.var, c2v[..., None] * g.anti)
        if model == "momentum":
            gm = gamma[t] * gm + (1.0 - gamma[t]) * (Qprev - Pi0 - S)              # eqs. (mombp1), (mombp3)
            Q = Qprev - alpha[t] * gm                                              # eq. (mombp2)
        else:
            Q = Pit.expand(B, g.N, 3) + S                                          # eq. (p_update)
        q_own = Q[:, g.var, :] - c2v[..., None] * g.anti                           # Q minus own message
        new = lam(q_own, g.own, g.anti).clamp(-clip, clip)
        v2c = (1.0 - beta[t]) * new + beta[t] * v2c
        Qprev = Q
        Qs.append(Q)
    return Qs if every else Q


def loss(Q: torch.Tensor, err) -> torch.Tensor:
    """Mean over shots and qubits of -log P(E_j = true Pauli), with
    log P = log softmax(0, -Q_X, -Q_Y, -Q_Z)."""
    err = torch.as_tensor(np.asarray(err), dtype=torch.long)
    logits = torch.cat([torch.zeros_like(Q[..., :1]), -Q], -1)
    logp = torch.log_softmax(logits, -1)
    return -logp.gather(-1, err[..., None]).squeeze(-1).mean()


MIN_PROB = 1e-30  # -log P is taken of max(P, MIN_PROB)


def parity_distribution(ca: torch.Tensor) -> torch.Tensor:
    """(P(even), P(odd)) of the sum mod 2 of independent bits, from each
    bit's (P(0), P(1)) along dimension -2: the convolution over the bits in
    order, (e, o) <- (e c + o a, e a + o c)."""
    eo = torch.stack([torch.ones_like(ca[..., 0, 0]), torch.zeros_like(ca[..., 0, 0])], -1)
    for j in range(ca.shape[-2]):
        c, a = ca[..., j, 0], ca[..., j, 1]
        eo = torch.stack([eo[..., 0] * c + eo[..., 1] * a, eo[..., 0] * a + eo[..., 1] * c], -1)
    return eo


def coset_loss(Qs, H, syn, err, logicals) -> torch.Tensor:
    """Mean over shots and iterations of
        mean_i -log P(<E^, H_i> = s_i) + mean_L -log P(<E^, L> = <E, L>),
    E^ distributed as the product of the iteration's posterior marginals
    (P(W) proportional to e^{-Q_W}, Q_I = 0; Q_W = ln P(I)/P(W)) and E the
    true error: each operator's parity distribution is the convolution over
    its support of (P(E^_j commutes with R_j), P(it anticommutes)).
    Qs: list of (B, N, 3); H: (M, N) and logicals: (n, N) Pauli codes;
    syn: (B, M) 0/1; err: (B, N) Pauli codes."""
    H = np.asarray(H)
    Lg = np.asarray(logicals)
    err = np.asarray(err)
    target_l = np.stack([(_anti(err, Lg[l][None, :])).sum(-1) % 2 for l in range(Lg.shape[0])], -1)   # (B, n)
    groups = [(H, torch.as_tensor(np.asarray(syn), dtype=torch.long)),
              (Lg, torch.as_tensor(target_l, dtype=torch.long))]
    total = 0.0
    for Q in Qs:
        logits = torch.cat([torch.zeros_like(Q[..., :1]), -Q], -1)
        pi = torch.softmax(logits, -1)                                          # (B, N, 4): I, X, Y, Z
        term = 0.0
        for R, target in groups:
            rows = []
            for r in range(R.shape[0]):
                supp = np.nonzero(R[r])[0]
                an = torch.as_tensor(np.stack([_anti(np.full(supp.size, w), R[r, supp]) for w in (1, 2, 3)], -1)
                                     .astype(np.float64))                      # (w, 3): W anticommutes with R_j
                p = pi[:, supp, 1:]                                             # (B, w, 3)
                a = (p * an).sum(-1)
                c = pi[:, supp, 0] + (p * (1.0 - an)).sum(-1)
                rows.append(parity_distribution(torch.stack([c, a], -1)))      # (B, 2)
            eo = torch.stack(rows, 1)                                           # (B, rows, 2)
            P = eo.gather(-1, target[..., None]).squeeze(-1)
            term = term + (-torch.log(P.clamp_min(MIN_PROB))).mean(-1)
        total = total + term
    return (total / len(Qs)).mean()


def loss_and_grads(H, syn, err, prior, alpha, beta, w, T: int, clip: float = 30.0, model: str = "ewainit",
                   gamma=None, kind: str = "posterior", logicals=None):
    """(loss, d loss / d alpha, d beta, d w) in float64 by autograd; for
    model "momentum" also d loss / d gamma, as a fifth element.  kind
    "posterior" (loss) or "coset" (coset_loss with `logicals`)."""
    g = Graph(H)
    a = torch.tensor(np.asarray(alpha, dtype=np.float64), requires_grad=True)
    b = torch.tensor(np.asarray(beta, dtype=np.float64), requires_grad=True)
    ww = torch.tensor(np.asarray(w, dtype=np.float64), requires_grad=True)
    gm = None if gamma is None else torch.tensor(np.asarray(gamma, dtype=np.float64), requires_grad=True)
    if kind == "coset":
        L = coset_loss(forward(g, syn, prior, a, b, ww, T, clip, model=model, gamma=gm, every=True), H, syn, err,
                       logicals)
    else:
        L = loss(forward(g, syn, prior, a, b, ww, T, clip, model=model, gamma=gm), err)
    L.backward()
    out = (L.item(), a.grad.numpy(), b.grad.numpy(), ww.grad.numpy())
    if model == "momentum":
        out = out + (gm.grad.numpy(),)
    return out
