/*
 * Oracle for GF(4) log-likelihood belief propagation (LLR-BP4) decoding of
 * stabilizer-code syndromes, in the parallel (flooding) schedule, with the
 * three variants of "Improved Belief Propagation Decoding Algorithms for
 * Surface Codes" (Chen, Yi, Liang, Wang): Momentum-BP, AdaGrad-BP and
 * EWAInit-BP.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, double-precision CPU
 * restatement of the paper's update rules, written to check the CUDA decoder.
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load it.  It shares no code with the CUDA path.
 *
 * Every step follows the paper in its order and notation:
 *   prior LLR          Pi_{v_j,W} = ln(p^I / p^W)        Sec. II-B1, eq. before (init)
 *   lambda             lambda_{H_ij}(p^X,p^Y,p^Z)         Sec. II-B1, eq. (lambda)
 *   initial messages   m^(0)_{v->c} = lambda(Pi)           Sec. II-B1, eq. (init)
 *   horizontal update  w = 2 atanh(prod tanh(m/2)),        Sec. II-B1, eq. (h_update)
 *                      m_{c->v} = (-1)^{s_i} w             and the sign rule below it
 *   vertical update    lambda_{H_ij}(Pi + sum of other     Sec. II-B1, eq. (v_update)
 *                      anticommuting c->v messages)
 *   posterior          Q = Pi + sum of anticommuting       Sec. II-B1, eq. (p_update)
 *                      c->v messages
 *   hard decision      I if all Q_W > 0, else argmin_W     Sec. II-B1, text after (p_update)
 *   Momentum-BP        g, Q recursion; v->c from Q minus   Sec. III-A1, eqs. (mombp1),
 *                      the raw c->v message                (mombp2), (mombp5), (mombp3)
 *   AdaGrad-BP         Q = Q_prev - alpha g'/(sqrt(G)+eps) Sec. III-A2, eq. (boost) and the
 *                                                          g', G definitions below it
 *   EWAInit-BP         Pi^(t) = alpha Pi^(0) + (1-alpha)   Sec. III-B, Algorithm 2,
 *                      Q^(t-1)                             eq. (EWAInit)
 *   AEWA-BP            EWAInit-BP with alpha = 1.0, 0.9,   Appendix C
 *                      ..., 0.0 in turn until a run
 *                      converges
 *
 * Readings taken where the paper is silent or ambiguous (each one is listed
 * in the design notes of the repository):
 *   - Pi_W = ln(p^I/p^W) with p^I = 1 - p^X - p^Y - p^Z (the printed
 *     ln((1-p)/p) is the binary special case).
 *   - In (v_update) the anticommutation condition is taken on the summed
 *     check i', and the 3-vector form of (mombp5): the message is
 *     lambda_{H_ij} of {Q_W - [<W,H_ij>=1] m_{c_i->v_j}}_W.
 *   - Momentum-BP and AdaGrad-BP under flooding: all c->v messages of
 *     iteration t use the v->c messages of t-1; the gradient is
 *     Q^(t-1) - Pi - S^(t); Q^(0) = Pi, g^(0) = 0.
 *   - AdaGrad-BP: Q^(1) = Pi + S^(1); (boost) applies from t = 2; G
 *     accumulates from t = 1 (g'^(1) = -S^(1)) unless adagrad_g_from_iter1
 *     is 0, in which case it starts at t = 2.
 *   - Every c->v and v->c message is clipped to [-msg_clip, msg_clip]
 *     (the paper does not say how saturated messages are handled).
 *   - Hard decision ties: strict "all Q_W > 0" for I, else the first
 *     minimum in the order X, Y, Z.
 *   - The horizontal update is evaluated in long double so that the
 *     literal tanh/atanh form keeps its accuracy near the clip value.
 *
 * Working precision.  The default build computes in double (FP64).  Two
 * other builds of this same file serve one purpose: to show which results
 * the working precision decides.  -DORACLE_REAL="long double" computes every
 * quantity in long double (x87 80-bit on x86-64, IEEE binary128 on AArch64);
 * -DORACLE_STORE_F32 keeps double arithmetic but rounds every stored
 * message, posterior, prior and state value (and every partial sum) to
 * binary32, the precision in which a single-precision decoder keeps them.
 * The update rules are the same in all three builds.
 *
 * Pauli codes used throughout: 0 = I, 1 = X, 2 = Y, 3 = Z.  W indexes
 * {X, Y, Z} as 0, 1, 2 (code W+1).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <tgmath.h>

#ifndef ORACLE_REAL
#define ORACLE_REAL double
#endif
typedef ORACLE_REAL real;

/* A value as the decoder stores it: unchanged, or rounded to binary32 in the
 * ORACLE_STORE_F32 build. */
static real st(real x) {
#ifdef ORACLE_STORE_F32
    return (real)(float)x;
#else
    return x;
#endif
}

enum { OR_PLAIN = 0, OR_MOMENTUM = 1, OR_ADAGRAD = 2, OR_EWAINIT = 3, OR_AEWA = 4 };

/* Trace-product <A, B>: 1 when the single-qubit Paulis anticommute. */
static int anticommutes(int a, int b) { return a != 0 && b != 0 && a != b; }

static real clip(real x, real c) {
    if (x > c) return c;
    if (x < -c) return -c;
    return x;
}

/* lambda_{H}(q^X, q^Y, q^Z) = ln((1 + e^{-q^H}) / (e^{-q^X}+e^{-q^Y}+e^{-q^Z} - e^{-q^H})),
 * eq. (lambda).  The denominator is the sum over the two Paulis W != H, which
 * is what the printed difference equals; summing them directly avoids the
 * cancellation of the printed form. */
static real lambda_fn(int h, const real q[3]) {
    real num = 1.0 + exp(-q[h - 1]);
    real den = 0.0;
    for (int w = 0; w < 3; ++w)
        if (w != h - 1) den += exp(-q[w]);
    return log(num / den);
}

typedef struct {
    int N, M, E;
    const uint8_t *H;   /* M x N Pauli codes */
    int *chk_ptr;       /* M+1: edges of check i are chk_ptr[i]..chk_ptr[i+1]-1 */
    int *edge_var;      /* E: qubit of edge e */
    int *edge_chk;      /* E: check of edge e */
    uint8_t *edge_p;    /* E: H_ij of edge e */
    int *var_ptr;       /* N+1 */
    int *var_edges;     /* E: edges of qubit j, ordered by check */
} graph;

static int graph_build(graph *g, int N, int M, const uint8_t *H) {
    memset(g, 0, sizeof *g);
    g->N = N; g->M = M; g->H = H;
    int E = 0;
    for (long k = 0; k < (long)M * N; ++k) E += H[k] != 0;
    g->E = E;
    g->chk_ptr = malloc(sizeof(int) * (M + 1));
    g->edge_var = malloc(sizeof(int) * (E + 1));
    g->edge_chk = malloc(sizeof(int) * (E + 1));
    g->edge_p = malloc(E + 1);
    g->var_ptr = calloc(N + 1, sizeof(int));
    g->var_edges = malloc(sizeof(int) * (E + 1));
    if (!g->chk_ptr || !g->edge_var || !g->edge_chk || !g->edge_p || !g->var_ptr || !g->var_edges)
        return -1;
    int e = 0;
    for (int i = 0; i < M; ++i) {
        g->chk_ptr[i] = e;
        for (int j = 0; j < N; ++j) {
            uint8_t p = H[(long)i * N + j];
            if (p > 3) return -2;
            if (p) { g->edge_var[e] = j; g->edge_chk[e] = i; g->edge_p[e] = p; ++e; }
        }
    }
    g->chk_ptr[M] = e;
    for (e = 0; e < E; ++e) g->var_ptr[g->edge_var[e] + 1]++;
    for (int j = 0; j < N; ++j) g->var_ptr[j + 1] += g->var_ptr[j];
    int *fill = calloc(N + 1, sizeof(int));
    if (!fill) return -1;
    for (e = 0; e < E; ++e) {
        int j = g->edge_var[e];
        g->var_edges[g->var_ptr[j] + fill[j]++] = e;
    }
    free(fill);
    return 0;
}

static void graph_free(graph *g) {
    free(g->chk_ptr); free(g->edge_var); free(g->edge_chk); free(g->edge_p);
    free(g->var_ptr); free(g->var_edges);
}

typedef struct {
    real alpha, gamma, eps, msg_clip;
    int adagrad_g_from_iter1;
    int serial;  /* 0: parallel (flooding) schedule; 1: serial schedule of Algorithm 1 */
} params;

/* Optional per-iteration record of one shot (all arrays may be NULL). */
typedef struct {
    double *m_v2c;   /* (T+1) x E : v->c messages after iteration t (t = 0 is eq. (init)) */
    double *m_c2v;   /* T x E     : c->v messages of iteration t = 1..T */
    double *S;       /* T x N x 3 : sum of anticommuting c->v messages */
    double *Q;       /* T x N x 3 : posterior LLRs */
    double *aux;     /* T x N x 3 : g (Momentum), G (AdaGrad), Pi^(t) (EWAInit), Pi (Plain) */
    uint8_t *dec;    /* T x N     : hard decisions */
} trace;

/* Copy n working-precision values into a caller's double array. */
static void put(double *dst, const real *src, size_t n) {
    for (size_t k = 0; k < n; ++k) dst[k] = (double)src[k];
}

typedef struct {
    real *Pi0, *Pit, *Q, *Qprev, *S, *gstate;
    real *m_v2c, *m_c2v;
    uint8_t *est;
} workspace;

static int ws_alloc(workspace *w, int N, int E) {
    size_t n3 = (size_t)3 * N;
    w->Pi0 = malloc(sizeof(real) * n3);
    w->Pit = malloc(sizeof(real) * n3);
    w->Q = malloc(sizeof(real) * n3);
    w->Qprev = malloc(sizeof(real) * n3);
    w->S = malloc(sizeof(real) * n3);
    w->gstate = malloc(sizeof(real) * n3);
    w->m_v2c = malloc(sizeof(real) * (E + 1));
    w->m_c2v = malloc(sizeof(real) * (E + 1));
    w->est = malloc(N + 1);
    return (w->Pi0 && w->Pit && w->Q && w->Qprev && w->S && w->gstate && w->m_v2c &&
            w->m_c2v && w->est) ? 0 : -1;
}

static void ws_free(workspace *w) {
    free(w->Pi0); free(w->Pit); free(w->Q); free(w->Qprev); free(w->S); free(w->gstate);
    free(w->m_v2c); free(w->m_c2v); free(w->est);
}

/* Hard decision of Sec. II-B1: I if every Q_W > 0, else the W with the
 * smallest Q_W (first minimum in X, Y, Z order). Returns the Pauli code. */
static int hard_decision(const real q[3]) {
    if (q[0] > 0 && q[1] > 0 && q[2] > 0) return 0;
    int best = 0;
    for (int w = 1; w < 3; ++w)
        if (q[w] < q[best]) best = w;
    return best + 1;
}

/* <H, E^> = s, the stopping test of Algorithms 1 and 2. */
static int syndrome_matches(const graph *g, const uint8_t *est, const uint8_t *syn) {
    for (int i = 0; i < g->M; ++i) {
        int par = 0;
        for (int e = g->chk_ptr[i]; e < g->chk_ptr[i + 1]; ++e)
            par ^= anticommutes(est[g->edge_var[e]], g->edge_p[e]);
        if (par != (syn[i] & 1)) return 0;
    }
    return 1;
}

/* m_{c_i -> v_j} of edge e (check i) from the current v->c messages of the
 * other edges of check i, eq. (h_update) with the syndrome sign, clipped. */
static real c2v_edge(const graph *g, const workspace *w, const uint8_t *syn, int e, real c) {
    const int i = g->edge_chk[e];
    long double prod = 1.0L;
    for (int f = g->chk_ptr[i]; f < g->chk_ptr[i + 1]; ++f)
        if (f != e) prod *= tanhl((long double)w->m_v2c[f] / 2.0L);
    long double wv = 2.0L * atanhl(prod);
    real m = (syn[i] & 1) ? -(real)wv : (real)wv;
    return st(clip(m, c));
}

/* Posterior of one qubit-Pauli pair k = 3j + W for each variant, from the
 * sum S of its anticommuting c->v messages (the rules of Sec. II-B1 and
 * Sec. III, identical under both schedules). */
static int posterior(int variant, const params *pr, int t, workspace *w, int k, real S) {
    real Pi = w->Pi0[k], Qp = w->Qprev[k];
    switch (variant) {
    case OR_PLAIN: w->Q[k] = st(Pi + S); return 0;
    case OR_EWAINIT: w->Q[k] = st(w->Pit[k] + S); return 0;
    case OR_MOMENTUM: {
        real grad = st(Qp - Pi - S);
        w->gstate[k] = st(pr->gamma * w->gstate[k] + (1.0 - pr->gamma) * grad);
        w->Q[k] = st(Qp - pr->alpha * w->gstate[k]);
        return 0;
    }
    case OR_ADAGRAD: {
        real gp = st(Qp - Pi - S);
        if (t >= 2 || pr->adagrad_g_from_iter1) w->gstate[k] = st(w->gstate[k] + gp * gp);
        w->Q[k] = st(t == 1 ? Pi + S : Qp - pr->alpha * gp / (sqrt(w->gstate[k]) + pr->eps));
        return 0;
    }
    }
    return -1;
}

/* One iteration of the serial schedule (Algorithm 1's serial update): the
 * qubits are visited in order j = 1..N; at its turn qubit j takes the c->v
 * messages of its checks from the v->c messages as they stand (already
 * updated in this iteration for the qubits before j), updates its
 * posterior (EWAInit: with Pi^(t)_j = alpha Pi^(0)_j + (1 - alpha) Q^(t-1)_j
 * for t > 1), and sends its new v->c messages: eq. (v_update) for plain and
 * EWAInit BP, eq. (mombp5) for Momentum and AdaGrad BP. */
static int serial_sweep(const graph *g, const uint8_t *syn, int variant, const params *pr, int t, workspace *w) {
    const real c = pr->msg_clip;
    for (int j = 0; j < g->N; ++j) {
        if (variant == OR_EWAINIT && t > 1)
            for (int k = 0; k < 3; ++k)
                w->Pit[3 * j + k] = st(pr->alpha * w->Pi0[3 * j + k] + (1.0 - pr->alpha) * w->Qprev[3 * j + k]);
        for (int a = g->var_ptr[j]; a < g->var_ptr[j + 1]; ++a) {
            const int e = g->var_edges[a];
            w->m_c2v[e] = c2v_edge(g, w, syn, e, c);
        }
        for (int k = 0; k < 3; ++k) {
            real s = 0.0;
            for (int a = g->var_ptr[j]; a < g->var_ptr[j + 1]; ++a) {
                const int e = g->var_edges[a];
                if (anticommutes(k + 1, g->edge_p[e])) s = st(s + w->m_c2v[e]);
            }
            w->S[3 * j + k] = s;
            if (posterior(variant, pr, t, w, 3 * j + k, s)) return -1;
        }
        for (int a = g->var_ptr[j]; a < g->var_ptr[j + 1]; ++a) {
            const int e = g->var_edges[a], h = g->edge_p[e];
            real q[3];
            for (int k = 0; k < 3; ++k) {
                if (variant == OR_PLAIN || variant == OR_EWAINIT) {
                    const real *base = (variant == OR_EWAINIT) ? &w->Pit[3 * j] : &w->Pi0[3 * j];
                    real s = 0.0;
                    for (int b = g->var_ptr[j]; b < g->var_ptr[j + 1]; ++b) {
                        const int f = g->var_edges[b];
                        if (f != e && anticommutes(k + 1, g->edge_p[f])) s = st(s + w->m_c2v[f]);
                    }
                    q[k] = st(base[k] + s);
                } else {
                    q[k] = st(w->Q[3 * j + k] - (anticommutes(k + 1, h) ? w->m_c2v[e] : 0.0));
                }
            }
            w->m_v2c[e] = st(clip(lambda_fn(h, q), c));
        }
    }
    return 0;
}

/* Decode one shot.  stop_early = 1 applies the stopping rule; 0 runs exactly
 * max_iter iterations (used for recording traces).  Returns the number of
 * iterations run; *converged reports whether the last decision matched. */
static int decode_shot(const graph *g, const uint8_t *syn, const double *prior, int variant,
                       const params *pr, int max_iter, int stop_early, workspace *w,
                       uint8_t *est_out, int *converged, trace *tr) {
    const int N = g->N, E = g->E;
    const real c = pr->msg_clip;

    /* Prior LLRs Pi^(0)_{v_j,W} = ln(p^I / p^W). */
    for (int j = 0; j < N; ++j) {
        real pI = 1.0 - (real)prior[3 * j] - (real)prior[3 * j + 1] - (real)prior[3 * j + 2];
        for (int k = 0; k < 3; ++k) w->Pi0[3 * j + k] = st(log(pI / (real)prior[3 * j + k]));
    }
    /* Initial messages, eq. (init). */
    for (int e = 0; e < E; ++e)
        w->m_v2c[e] = st(clip(lambda_fn(g->edge_p[e], &w->Pi0[3 * g->edge_var[e]]), c));
    if (tr && tr->m_v2c) put(tr->m_v2c, w->m_v2c, E);

    /* Q^(0) = Pi^(0) and g^(0) = 0 (Algorithm 1 initialization); G^(0) = 0. */
    for (int k = 0; k < 3 * N; ++k) {
        w->Qprev[k] = w->Pi0[k];
        w->gstate[k] = 0.0;
        w->Pit[k] = w->Pi0[k];
    }

    int t = 0, conv = 0;
    for (t = 1; t <= max_iter; ++t) {
        if (pr->serial) {
            if (serial_sweep(g, syn, variant, pr, t, w)) return -1;
            goto decide;
        }
        /* EWAInit-BP: Pi^(t) = alpha Pi^(0) + (1 - alpha) Q^(t-1) when t > 1, eq. (EWAInit). */
        if (variant == OR_EWAINIT && t > 1)
            for (int k = 0; k < 3 * N; ++k)
                w->Pit[k] = st(pr->alpha * w->Pi0[k] + (1.0 - pr->alpha) * w->Qprev[k]);

        /* Horizontal update, eq. (h_update) and the syndrome sign. */
        for (int i = 0; i < g->M; ++i) {
            for (int e = g->chk_ptr[i]; e < g->chk_ptr[i + 1]; ++e) {
                long double prod = 1.0L;
                for (int f = g->chk_ptr[i]; f < g->chk_ptr[i + 1]; ++f)
                    if (f != e) prod *= tanhl((long double)w->m_v2c[f] / 2.0L);
                long double wv = 2.0L * atanhl(prod);
                real m = (syn[i] & 1) ? -(real)wv : (real)wv;
                w->m_c2v[e] = st(clip(m, c));
            }
        }

        /* Sum of the c->v messages from checks that anticommute with W. */
        for (int j = 0; j < N; ++j)
            for (int k = 0; k < 3; ++k) {
                real s = 0.0;
                for (int a = g->var_ptr[j]; a < g->var_ptr[j + 1]; ++a) {
                    int e = g->var_edges[a];
                    if (anticommutes(k + 1, g->edge_p[e])) s = st(s + w->m_c2v[e]);
                }
                w->S[3 * j + k] = s;
            }

        /* Posterior update of each variant. */
        for (int k = 0; k < 3 * N; ++k) {
            real Pi = w->Pi0[k], S = w->S[k], Qp = w->Qprev[k];
            switch (variant) {
            case OR_PLAIN: /* eq. (p_update) */
                w->Q[k] = st(Pi + S);
                break;
            case OR_EWAINIT: /* eq. (p_update) with Pi replaced by Pi^(t), Algorithm 2 */
                w->Q[k] = st(w->Pit[k] + S);
                break;
            case OR_MOMENTUM: { /* eqs. (mombp1), (mombp2); the gradient as expanded in (mombp3) */
                real grad = st(Qp - Pi - S);
                w->gstate[k] = st(pr->gamma * w->gstate[k] + (1.0 - pr->gamma) * grad);
                w->Q[k] = st(Qp - pr->alpha * w->gstate[k]);
                break;
            }
            case OR_ADAGRAD: { /* eq. (boost) with g' and G as defined below it */
                real gp = st(Qp - Pi - S);
                if (t >= 2 || pr->adagrad_g_from_iter1) w->gstate[k] = st(w->gstate[k] + gp * gp);
                if (t == 1)
                    w->Q[k] = st(Pi + S);
                else
                    w->Q[k] = st(Qp - pr->alpha * gp / (sqrt(w->gstate[k]) + pr->eps));
                break;
            }
            default:
                return -1;
            }
        }

        /* Vertical update. */
        for (int e = 0; e < E; ++e) {
            int j = g->edge_var[e], h = g->edge_p[e], i = g->edge_chk[e];
            real q[3];
            if (variant == OR_PLAIN || variant == OR_EWAINIT) {
                /* eq. (v_update): prior plus the anticommuting messages of the other checks */
                const real *base = (variant == OR_EWAINIT) ? &w->Pit[3 * j] : &w->Pi0[3 * j];
                for (int k = 0; k < 3; ++k) {
                    real s = 0.0;
                    for (int a = g->var_ptr[j]; a < g->var_ptr[j + 1]; ++a) {
                        int f = g->var_edges[a];
                        if (g->edge_chk[f] != i && anticommutes(k + 1, g->edge_p[f])) s = st(s + w->m_c2v[f]);
                    }
                    q[k] = st(base[k] + s);
                }
            } else {
                /* eq. (mombp5): posterior minus the raw message of this check */
                for (int k = 0; k < 3; ++k)
                    q[k] = st(w->Q[3 * j + k] - (anticommutes(k + 1, h) ? w->m_c2v[e] : 0.0));
            }
            w->m_v2c[e] = st(clip(lambda_fn(h, q), c));
        }

    decide:
        /* Hard decision and stopping test. */
        for (int j = 0; j < N; ++j) w->est[j] = (uint8_t)hard_decision(&w->Q[3 * j]);
        conv = syndrome_matches(g, w->est, syn);

        if (tr) {
            size_t o3 = (size_t)(t - 1) * 3 * N;
            if (tr->m_v2c) put(tr->m_v2c + (size_t)t * E, w->m_v2c, E);
            if (tr->m_c2v) put(tr->m_c2v + (size_t)(t - 1) * E, w->m_c2v, E);
            if (tr->S) put(tr->S + o3, w->S, 3 * N);
            if (tr->Q) put(tr->Q + o3, w->Q, 3 * N);
            if (tr->aux) {
                const real *src = (variant == OR_EWAINIT) ? w->Pit
                                : (variant == OR_PLAIN) ? w->Pi0 : w->gstate;
                put(tr->aux + o3, src, 3 * N);
            }
            if (tr->dec) memcpy(tr->dec + (size_t)(t - 1) * N, w->est, N);
        }

        for (int k = 0; k < 3 * N; ++k) w->Qprev[k] = w->Q[k];
        if (stop_early && conv) break;
    }
    if (t > max_iter) t = max_iter;
    memcpy(est_out, w->est, N);
    *converged = conv;
    return t;
}

/* ---------------------------------------------------------------- batch API */

typedef struct {
    const graph *g;
    const uint8_t *syn;
    const double *prior;
    int variant;
    const params *pr;
    int max_iter;
    int b0, b1;
    uint8_t *est, *conv;
    int32_t *iters;
    int status;
} job;

/* AEWA-BP (Appendix C): EWAInit-BP with the discount factor taken from
 * 1.0, 0.9, ..., 0.0 in turn (11 values, large to small) until a run
 * converges; the outputs are those of the last run. */
static int decode_shot_aewa(const graph *g, const uint8_t *syn, const double *prior, const params *pr,
                            int max_iter, workspace *w, uint8_t *est_out, int *converged) {
    int it = 0;
    for (int k = 0; k <= 10; ++k) {
        params p = *pr;
        p.alpha = 1.0 - 0.1 * k;
        it = decode_shot(g, syn, prior, OR_EWAINIT, &p, max_iter, 1, w, est_out, converged, NULL);
        if (it < 0 || *converged) break;
    }
    return it;
}

static void *run_job(void *arg) {
    job *jb = arg;
    workspace w;
    if (ws_alloc(&w, jb->g->N, jb->g->E)) { jb->status = -1; ws_free(&w); return NULL; }
    for (int b = jb->b0; b < jb->b1; ++b) {
        int cv = 0;
        int it = jb->variant == OR_AEWA
                     ? decode_shot_aewa(jb->g, jb->syn + (size_t)b * jb->g->M, jb->prior, jb->pr, jb->max_iter, &w,
                                        jb->est + (size_t)b * jb->g->N, &cv)
                     : decode_shot(jb->g, jb->syn + (size_t)b * jb->g->M, jb->prior, jb->variant, jb->pr,
                                   jb->max_iter, 1, &w, jb->est + (size_t)b * jb->g->N, &cv, NULL);
        if (it < 0) { jb->status = it; break; }
        jb->conv[b] = (uint8_t)cv;
        jb->iters[b] = it;
    }
    ws_free(&w);
    return NULL;
}

/* Decode B shots.  syn: B x M bytes (0/1).  prior: N x 3 probabilities
 * (p^X, p^Y, p^Z) per qubit.  est: B x N Pauli codes; conv: B flags;
 * iters: B iteration counts.  nthreads > 1 splits the shots over threads. */
int oracle_decode(int N, int M, const uint8_t *H, int B, const uint8_t *syn, const double *prior,
                  int variant, double alpha, double gamma, double eps, double msg_clip,
                  int adagrad_g_from_iter1, int serial, int max_iter, uint8_t *est, uint8_t *conv,
                  int32_t *iters, int nthreads) {
    if (N <= 0 || M < 0 || B < 0 || max_iter < 1 || variant < 0 || variant > 4) return -1;
    if (serial && variant == OR_AEWA) return -1;
    graph g;
    if (graph_build(&g, N, M, H)) { graph_free(&g); return -2; }
    params pr = {alpha, gamma, eps, msg_clip, adagrad_g_from_iter1, serial ? 1 : 0};
    if (nthreads < 1) nthreads = 1;
    if (nthreads > B) nthreads = B > 0 ? B : 1;
    job *jobs = calloc(nthreads, sizeof(job));
    pthread_t *th = calloc(nthreads, sizeof(pthread_t));
    int rc = 0;
    for (int k = 0; k < nthreads; ++k) {
        jobs[k] = (job){&g, syn, prior, variant, &pr, max_iter,
                        (int)((long)B * k / nthreads), (int)((long)B * (k + 1) / nthreads),
                        est, conv, iters, 0};
    }
    if (nthreads == 1) {
        run_job(&jobs[0]);
    } else {
        for (int k = 0; k < nthreads; ++k) pthread_create(&th[k], NULL, run_job, &jobs[k]);
        for (int k = 0; k < nthreads; ++k) pthread_join(th[k], NULL);
    }
    for (int k = 0; k < nthreads; ++k)
        if (jobs[k].status) rc = jobs[k].status;
    free(jobs); free(th);
    graph_free(&g);
    return rc;
}

/* Run exactly T iterations on one shot (no stopping) and record every
 * intermediate quantity in the caller's arrays (see struct trace). */
int oracle_trace(int N, int M, const uint8_t *H, const uint8_t *syn, const double *prior,
                 int variant, double alpha, double gamma, double eps, double msg_clip,
                 int adagrad_g_from_iter1, int serial, int T, double *m_v2c, double *m_c2v, double *S,
                 double *Q, double *aux, uint8_t *dec) {
    if (N <= 0 || M < 0 || T < 1 || variant < 0 || variant > 3) return -1;
    graph g;
    if (graph_build(&g, N, M, H)) { graph_free(&g); return -2; }
    params pr = {alpha, gamma, eps, msg_clip, adagrad_g_from_iter1, serial ? 1 : 0};
    workspace w;
    if (ws_alloc(&w, N, g.E)) { ws_free(&w); graph_free(&g); return -3; }
    trace tr = {m_v2c, m_c2v, S, Q, aux, dec};
    uint8_t *est = malloc(N);
    int cv = 0;
    int it = decode_shot(&g, syn, prior, variant, &pr, T, 0, &w, est, &cv, &tr);
    free(est);
    ws_free(&w);
    graph_free(&g);
    return it < 0 ? it : 0;
}

/* Number of nonzero entries of H (edges of the Tanner graph). */
int oracle_num_edges(int N, int M, const uint8_t *H) {
    int E = 0;
    for (long k = 0; k < (long)M * N; ++k) E += H[k] != 0;
    return E;
}

/* The hard decision of Sec. II-B1 on one posterior triple (exported so that
 * the rule can be tested over every sign and tie pattern). */
int oracle_hard_decision(const double *q) {
    const real r[3] = {q[0], q[1], q[2]};
    return hard_decision(r);
}
