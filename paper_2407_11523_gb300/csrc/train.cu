// Differentiable unrolled decoders (bpq_train_*): a fixed number T of
// flooding iterations without the stopping rule, with per-iteration
// trainable parameters, in two models:
//
//   EWAInit (Sec. III-B, Algorithm 2), EWA weight alpha_t:
//     Pi^(t)     = alpha_t Pi^(0) + (1 - alpha_t) Q^(t-1)              (t > 1)
//     Q^(t)      = Pi^(t) + S^(t)
//   Momentum (Sec. III-A1, eqs. (mombp1)-(mombp3)), step alpha_t, rate gamma_t:
//     g^(t)      = gamma_t g^(t-1) + (1 - gamma_t) (Q^(t-1) - Pi^(0) - S^(t))
//     Q^(t)      = Q^(t-1) - alpha_t g^(t),          Q^(0) = Pi^(0), g^(0) = 0
//
// and, in both, per-iteration damping beta_t of the variable-to-check
// messages and a weight w_e on every check-to-variable message (neural-BP
// style; the paper's conclusion names neural BP as a direction):
//
//   m_c->v^(t)  = clip(w_e (-1)^{s_i} r_e),  r_e = 2 atanh prod_{f != e} tanh(m_v->c^(t-1)_f / 2)
//   S^(t)       = sum of anticommuting m_c->v^(t)
//   m_v->c^(t)  = (1 - beta_t) clip(lambda_H(Q^(t) - own message)) + beta_t m_v->c^(t-1)
//
// Two losses:
//   posterior:  mean over shots and qubits of -log softmax(0, -Q_X, -Q_Y, -Q_Z)[true Pauli]
//               of the final posterior Q^(T);
//   coset:      mean over shots and iterations t = 1..T of
//                 mean over checks i of -log P_t(<E^, H_i> = s_i)
//               + mean over logical operators L of -log P_t(<E^, L> = <E, L>),
//               where E^ is drawn from the product of the posterior marginals
//               of iteration t (pi_W proportional to e^{-Q_W}, Q_I = 0) and E is
//               the true error: the probability that the soft decision of every
//               iteration satisfies the syndrome and lies in the true error's
//               coset (neural-BP decoders for quantum codes train on this kind
//               of loss).  The parity distribution of a check or logical is the
//               (P(even), P(odd)) convolution over its qubits of each qubit's
//               (commute, anticommute) probabilities, sums of positive terms, so
//               small probabilities keep their relative accuracy.
//
// At constant alpha (and gamma), beta_t = 0, w_e = 1 the forward pass is
// EWAInit-BP (Momentum-BP).  One CTA decodes one shot (thread x owns check
// x and qubit x).  The forward kernel stores a checkpoint (m_v->c, Q, and g
// for Momentum) every K iterations; the backward kernel recomputes each
// K-iteration segment from its checkpoint into shared memory and runs the
// adjoint through it in reverse.  The check-node derivative uses
// d r_e / d m_f = sinh(r_e) / sinh(m_f), which follows from
// 1 - tanh^2 = 1 / cosh^2 and avoids the 1 / (1 - P^2) of the product form.
// Per-shot gradient rows are reduced over shots by a separate kernel, so
// results are deterministic.  Arithmetic is fp32 with accurate library
// functions (this path is sized for training, not for the decode rate).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "bpq_internal.h"
#include "decode_launch.h"

using bpq::fail;

namespace bpq {
namespace tr {

constexpr int kEWAInit = BPQ_TRAIN_EWAINIT, kMomentum = BPQ_TRAIN_MOMENTUM;
constexpr int kCoset = BPQ_TRAIN_LOSS_COSET;
constexpr int kMaxLogicals = 4;
constexpr float kMinProb = 1e-30f;  // -log P is taken of max(P, kMinProb); no gradient below

struct TrainArgs {
    const uint8_t *table;
    uint32_t off_chk_pauli, off_var_pauli;
    const int32_t *var_canon, *chk_ptr;
    const uint32_t *syn;
    const uint8_t *err;
    const float *prior, *alpha, *beta, *w, *gamma;
    int N, M, E, W, B, T, K, nck, n_pad;
    int ck_floats;     // floats per checkpoint: 7 n_pad (EWAInit) or 10 n_pad (Momentum)
    int width;         // floats per gradient row: 2T + E (+ T for Momentum)
    float clip;
    int loss_kind;     // BPQ_TRAIN_LOSS_POSTERIOR or BPQ_TRAIN_LOSS_COSET
    const uint8_t *logicals;  // coset loss: [n_log][N] Pauli codes
    int n_log;
    float *ckpt;       // [B][nck][ck_floats]: m_v->c (4 n_pad slots), Q (3 n_pad), g (3 n_pad)
    float *loss_shot;  // [B] sum over qubits of the cross-entropy
    float *Q_out;      // optional [B][N][3]
    float *rows;       // [B][width] per-shot gradients: alpha | beta | w | gamma
};

__device__ __forceinline__ uint32_t anti(uint32_t a, uint32_t b) { return (a != 0u) & (b != 0u) & (a != b); }

// phi(x) = -ln tanh(x/2) = log1p(2 / expm1(x)), x >= 0
__device__ __forceinline__ float phi(float x) { return log1pf(2.0f / expm1f(x)); }

// lambda_H(q) = ln((1 + e^{-q_H}) / sum_{W != H} e^{-q_W}) with a common
// shift; also returns d lambda / d q_W in dl.
__device__ __forceinline__ float lambda_grad(uint32_t h, const float (&q)[3], float (&dl)[3]) {
    const float c0 = fminf(0.f, fminf(q[0], fminf(q[1], q[2])));
    const float e0 = expf(c0);
    float e[3];
#pragma unroll
    for (int w = 0; w < 3; ++w) e[w] = expf(c0 - q[w]);
    const float C = e0 + e[h - 1];
    float A = 0.f;
#pragma unroll
    for (int w = 0; w < 3; ++w)
        if (w != (int)h - 1) A += e[w];
#pragma unroll
    for (int w = 0; w < 3; ++w) dl[w] = (w == (int)h - 1) ? -e[w] / C : e[w] / A;
    return logf(C) - logf(A);
}

__device__ __forceinline__ float block_sum(float v, float *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    return s;  // valid on thread 0
}

// Sum of v over the CTA (two values), received by every thread.  red2:
// 32 float2 of shared memory.
__device__ __forceinline__ float2 block_sum2_all(float2 v, float2 *red2) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red2[threadIdx.x >> 5] = v;
    __syncthreads();
    float2 r = make_float2(0.f, 0.f);
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
        r.x += red2[k].x;
        r.y += red2[k].y;
    }
    return r;
}

// Parity distribution (P(even), P(odd)) of the sum of two independent bits
// with distributions x and y.
__device__ __forceinline__ float2 parity_combine(float2 x, float2 y) {
    return make_float2(x.x * y.x + x.y * y.y, x.x * y.y + x.y * y.x);
}

// Parity distribution of the bits of all threads of the CTA (each thread's
// (P(even), P(odd)); (1, 0) for none), received by every thread.
__device__ __forceinline__ float2 block_parity_all(float2 v, float2 *red2) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = parity_combine(v, make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red2[threadIdx.x >> 5] = v;
    __syncthreads();
    float2 r = make_float2(1.f, 0.f);
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r = parity_combine(r, red2[k]);
    return r;
}

// Posterior marginals (pi_I, pi_X, pi_Y, pi_Z) of a qubit: pi_W proportional
// to e^{-Q_W}, Q_I = 0.
__device__ __forceinline__ void marginals(const float (&Q)[3], float (&pi)[4]) {
    const float c0 = fminf(0.f, fminf(Q[0], fminf(Q[1], Q[2])));
    const float e[4] = {expf(c0), expf(c0 - Q[0]), expf(c0 - Q[1]), expf(c0 - Q[2])};
    const float z = e[0] + e[1] + e[2] + e[3];
#pragma unroll
    for (int k = 0; k < 4; ++k) pi[k] = e[k] / z;
}

// (P(the qubit's error commutes with P), P(it anticommutes)), P in 1..3.
__device__ __forceinline__ float2 comm_anti(const float (&pi)[4], uint32_t P) {
    float c = pi[0], an = 0.f;
#pragma unroll
    for (int w = 1; w <= 3; ++w) {
        if (anti((uint32_t)w, P))
            an += pi[w];
        else
            c += pi[w];
    }
    return make_float2(c, an);
}

struct Adj {
    uint32_t sl[4];   // slots of the owned check (zero slot for padding)
    uint32_t cp;      // check Paulis, 2 bits per edge
    uint32_t vp;      // qubit Paulis, 2 bits per edge
    int ce;           // canonical index of the check's first edge
    uint32_t sb;      // syndrome bit
};

__device__ __forceinline__ void load_adj(const TrainArgs &a, int x, int shot, Adj &d) {
    const uint32_t zero = 4u * (uint32_t)a.n_pad;
    d.cp = d.vp = 0;
    d.ce = 0;
    d.sb = 0;
    for (int n = 0; n < 4; ++n) d.sl[n] = zero;
    if (x < a.M) {
        const uint16_t *cs = reinterpret_cast<const uint16_t *>(a.table) + 4 * x;
        for (int n = 0; n < 4; ++n) d.sl[n] = cs[n] == kNoSlot ? zero : cs[n];
        d.cp = a.table[a.off_chk_pauli + x];
        d.ce = a.chk_ptr[x];
        d.sb = (a.syn[(size_t)shot * a.W + (x >> 5)] >> (x & 31)) & 1u;
    }
    if (x < a.N) d.vp = a.table[a.off_var_pauli + x];
}

// Check pass of iteration t: r_e and m_c->v for the owned check (reads v2c).
__device__ __forceinline__ void check_forward(const TrainArgs &a, const Adj &d, const float *v2c, float (&r)[4],
                                              float (&out)[4], int t) {
    float mag[4], sg[4];
    for (int n = 0; n < 4; ++n) {
        const float m = v2c[d.sl[n]];
        const bool valid = ((d.cp >> (2 * n)) & 3u) != 0u;
        mag[n] = valid ? phi(fabsf(m)) : 0.f;
        sg[n] = (valid && m < 0.f) ? -1.f : 1.f;
    }
    const float sigma = d.sb ? -1.f : 1.f;
    for (int n = 0; n < 4; ++n) {
        float ext = 0.f, ps = 1.f;
        for (int f = 0; f < 4; ++f)
            if (f != n) {
                ext += mag[f];
                ps *= sg[f];
            }
        r[n] = ps * phi(ext);  // 2 atanh prod_{f != n} tanh(m_f/2)
        const bool valid = ((d.cp >> (2 * n)) & 3u) != 0u;
        const float wv = valid ? a.w[d.ce + n] * sigma * r[n] : 0.f;  // padding has no weight
        out[n] = fminf(fmaxf(wv, -a.clip), a.clip);
    }
    (void)t;
}

// Forward: one CTA per shot.
// Parities <E, L> of the true error with the logical operators (bit l),
// the same on every thread.
__device__ __forceinline__ uint32_t true_logical_parities(const TrainArgs &a, int x, int shot, float2 *red2) {
    uint32_t tau = 0;
    for (int l = 0; l < a.n_log; ++l) {
        float v = 0.f;
        if (x < a.N) v = anti(a.err[(size_t)shot * a.N + x], a.logicals[(size_t)l * a.N + x]) ? 1.f : 0.f;
        const float n = block_sum2_all(make_float2(v, 0.f), red2).x;
        tau |= ((uint32_t)n & 1u) << l;
    }
    return tau;
}

// Coset loss of one iteration for one shot (the thread's part; the CTA's
// threads together hold mean_i -log P(<E^, H_i> = s_i) + mean_L -log P(<E^,
// L> = <E, L>)).  pi: the thread's qubit's marginals (x < N); ub2: [S4]
// float2 edge slots.
__device__ __forceinline__ float coset_loss_forward(const TrainArgs &a, const Adj &d, int x, const float (&pi)[4],
                                                    uint32_t tau, float2 *ub2, float2 *red2) {
    if (x < a.N)
        for (int k = 0; k < 4; ++k) {
            const uint32_t p = (d.vp >> (2 * k)) & 3u;
            ub2[4 * x + k] = p ? comm_anti(pi, p) : make_float2(1.f, 0.f);
        }
    __syncthreads();
    float part = 0.f;
    if (x < a.M) {
        float2 eo = make_float2(1.f, 0.f);
        for (int n = 0; n < 4; ++n)
            if ((d.cp >> (2 * n)) & 3u) eo = parity_combine(eo, ub2[d.sl[n]]);
        part += -logf(fmaxf(d.sb ? eo.y : eo.x, kMinProb)) / (float)a.M;
    }
    for (int l = 0; l < a.n_log; ++l) {
        const uint32_t P = x < a.N ? a.logicals[(size_t)l * a.N + x] : 0u;
        const float2 eo = block_parity_all(P ? comm_anti(pi, P) : make_float2(1.f, 0.f), red2);
        if (x == 0) part += -logf(fmaxf(((tau >> l) & 1u) ? eo.y : eo.x, kMinProb)) / (float)a.n_log;
    }
    return part;
}

template <int MODEL>
__global__ void train_forward_kernel(const TrainArgs a) {
    extern __shared__ __align__(16) float sm[];
    const int Np = a.n_pad, S4 = 4 * Np + 4;
    const bool coset = a.loss_kind == kCoset;
    float2 *ub2 = reinterpret_cast<float2 *>(sm);  // [S4] edge parity distributions (coset loss only)
    float *v2c = sm + (coset ? 2 * S4 : 0);       // [4Np + 4]
    float *c2v = v2c + S4;                         // [4Np + 4]
    float *Pi0 = c2v + S4;                         // [3Np]
    float *Qp = Pi0 + 3 * Np;                      // [3Np]
    float *Gp = Qp + 3 * Np;                       // [3Np] momentum g^(t-1) (Momentum only)
    float *red = Gp + (MODEL == kMomentum ? 3 * Np : 0);  // [64]
    float2 *red2 = reinterpret_cast<float2 *>(red);
    const int x = threadIdx.x, shot = blockIdx.x;
    Adj d;
    load_adj(a, x, shot, d);
    const uint32_t tau = coset ? true_logical_parities(a, x, shot, red2) : 0u;
    float coset_sum = 0.f;
    const uint32_t zero = 4u * (uint32_t)Np;
    if (x == 0) {
        v2c[zero] = 0.f;
        c2v[zero] = 0.f;
    }
    float Q[3] = {0.f, 0.f, 0.f};
    if (x < a.N) {
        const float px = a.prior[3 * x], py = a.prior[3 * x + 1], pz = a.prior[3 * x + 2];
        const float pI = 1.f - px - py - pz;
        Pi0[x] = logf(pI / px);
        Pi0[Np + x] = logf(pI / py);
        Pi0[2 * Np + x] = logf(pI / pz);
        for (int w = 0; w < 3; ++w) {
            Qp[w * Np + x] = Pi0[w * Np + x];
            if (MODEL == kMomentum) Gp[w * Np + x] = 0.f;
        }
        // eq. (init)
        const float q[3] = {Pi0[x], Pi0[Np + x], Pi0[2 * Np + x]};
        for (int k = 0; k < 4; ++k) {
            const uint32_t p = (d.vp >> (2 * k)) & 3u;
            float dl[3];
            v2c[4 * x + k] = p ? fminf(fmaxf(lambda_grad(p, q, dl), -a.clip), a.clip) : 0.f;
        }
    }
    __syncthreads();
    float *ck = a.ckpt + (size_t)shot * a.nck * a.ck_floats;
    for (int t = 1; t <= a.T; ++t) {
        if ((t - 1) % a.K == 0) {  // checkpoint (m_v->c^(t-1), Q^(t-1), g^(t-1))
            float *c = ck + (size_t)((t - 1) / a.K) * a.ck_floats;
            for (int k = x; k < 4 * Np; k += blockDim.x) c[k] = v2c[k];
            for (int k = x; k < 3 * Np; k += blockDim.x) c[4 * Np + k] = Qp[k];
            if (MODEL == kMomentum)
                for (int k = x; k < 3 * Np; k += blockDim.x) c[7 * Np + k] = Gp[k];
        }
        if (x < a.M) {
            float r[4], out[4];
            check_forward(a, d, v2c, r, out, t);
            for (int n = 0; n < 4; ++n)
                if ((d.cp >> (2 * n)) & 3u) c2v[d.sl[n]] = out[n];
        }
        __syncthreads();
        if (x < a.N) {
            const float al = a.alpha[t - 1], be = a.beta[t - 1];
            float S[3] = {0.f, 0.f, 0.f}, cin[4];
            for (int k = 0; k < 4; ++k) {
                const uint32_t p = (d.vp >> (2 * k)) & 3u;
                cin[k] = p ? c2v[4 * x + k] : 0.f;
                for (int w = 0; w < 3; ++w) S[w] += anti(w + 1, p) ? cin[k] : 0.f;
            }
            for (int w = 0; w < 3; ++w) {
                if (MODEL == kMomentum) {
                    const float gm = a.gamma[t - 1];
                    const float g = gm * Gp[w * Np + x] + (1.f - gm) * (Qp[w * Np + x] - Pi0[w * Np + x] - S[w]);
                    Q[w] = Qp[w * Np + x] - al * g;
                    Gp[w * Np + x] = g;
                } else {
                    const float pit = t > 1 ? al * Pi0[w * Np + x] + (1.f - al) * Qp[w * Np + x] : Pi0[w * Np + x];
                    Q[w] = pit + S[w];
                }
            }
            for (int k = 0; k < 4; ++k) {
                const uint32_t p = (d.vp >> (2 * k)) & 3u;
                if (!p) continue;
                float q[3], dl[3];
                for (int w = 0; w < 3; ++w) q[w] = Q[w] - (anti(w + 1, p) ? cin[k] : 0.f);
                const float L = fminf(fmaxf(lambda_grad(p, q, dl), -a.clip), a.clip);
                v2c[4 * x + k] = (1.f - be) * L + be * v2c[4 * x + k];
            }
            for (int w = 0; w < 3; ++w) Qp[w * Np + x] = Q[w];
        }
        __syncthreads();
        if (coset) {
            float pi[4] = {1.f, 0.f, 0.f, 0.f};
            if (x < a.N) marginals(Q, pi);
            coset_sum += coset_loss_forward(a, d, x, pi, tau, ub2, red2);
        }
    }
    // cross-entropy of the final posterior against the true error (posterior
    // loss), or the coset loss's mean over iterations
    float ce = coset ? coset_sum / (float)a.T : 0.f;
    if (x < a.N && !coset) {
        const float z[4] = {0.f, -Q[0], -Q[1], -Q[2]};
        const float zm = fmaxf(fmaxf(z[0], z[1]), fmaxf(z[2], z[3]));
        float se = 0.f;
        for (int k = 0; k < 4; ++k) se += expf(z[k] - zm);
        const int e = a.err[(size_t)shot * a.N + x];
        ce = zm + logf(se) - z[e];
    }
    if (x < a.N && a.Q_out)
        for (int w = 0; w < 3; ++w) a.Q_out[((size_t)shot * a.N + x) * 3 + w] = Q[w];
    const float tot = block_sum(ce, red);
    if (x == 0) a.loss_shot[shot] = tot;
}

// Backward: one CTA per shot; segments of K iterations recomputed from the
// checkpoints into shared memory, adjoint in reverse.
// Adds d (coset loss of iteration t) / d Q^(t) to Qbar (x < N): Qt = Q^(t)
// [3][Np] in shared memory; ub2 [S4] float2 scratch.  Every thread calls it.
// With P_match = (1 + sigma prod_j u_j) / 2 (u_j = c_j - a_j, sigma = +-1 the
// target parity), d (-log P_match) / d u_j = -sigma U'_j / (2 P_match), U'_j
// the product over the other qubits, and d u_j / d Q_W = 2 pi_W (c_j -
// [W commutes with the operator's Pauli on j]).
__device__ __forceinline__ void coset_loss_backward(const TrainArgs &a, const Adj &d, int x, const float *Qt,
                                                    uint32_t tau, float2 *ub2, float2 *red2, float (&Qbar)[3]) {
    const int Np = a.n_pad;
    float pi[4] = {1.f, 0.f, 0.f, 0.f};
    float2 ca[4];
    if (x < a.N) {
        const float Q[3] = {Qt[x], Qt[Np + x], Qt[2 * Np + x]};
        marginals(Q, pi);
        for (int k = 0; k < 4; ++k) {
            const uint32_t p = (d.vp >> (2 * k)) & 3u;
            ca[k] = p ? comm_anti(pi, p) : make_float2(1.f, 0.f);
            ub2[4 * x + k] = ca[k];
        }
    }
    __syncthreads();
    const float scale_c = 1.f / ((float)a.B * (float)a.T * (float)a.M);
    const float scale_l = 1.f / ((float)a.B * (float)a.T * (float)a.n_log);
    if (x < a.M) {
        float2 in[4];
        float2 eo = make_float2(1.f, 0.f);
        for (int n = 0; n < 4; ++n) {
            in[n] = ((d.cp >> (2 * n)) & 3u) ? ub2[d.sl[n]] : make_float2(1.f, 0.f);
            eo = parity_combine(eo, in[n]);
        }
        const float P = d.sb ? eo.y : eo.x, sigma = d.sb ? -1.f : 1.f;
        for (int n = 0; n < 4; ++n) {
            if (!((d.cp >> (2 * n)) & 3u)) continue;
            float U = 1.f;
            for (int m = 0; m < 4; ++m)
                if (m != n) U *= in[m].x - in[m].y;
            ub2[d.sl[n]].x = P > kMinProb ? -sigma * U / P * scale_c : 0.f;
        }
    }
    float gl[kMaxLogicals];
    float2 cl[kMaxLogicals];
    for (int l = 0; l < a.n_log; ++l) {
        const uint32_t P = x < a.N ? a.logicals[(size_t)l * a.N + x] : 0u;
        cl[l] = P ? comm_anti(pi, P) : make_float2(1.f, 0.f);
        const float2 eo = block_parity_all(cl[l], red2);
        const float u = cl[l].x - cl[l].y;
        const float lg = P ? logf(fmaxf(fabsf(u), 1e-30f)) : 0.f, ng = (P && u < 0.f) ? 1.f : 0.f;
        const float2 sums = block_sum2_all(make_float2(lg, ng), red2);
        const float Pm = ((tau >> l) & 1u) ? eo.y : eo.x, sigma = ((tau >> l) & 1u) ? -1.f : 1.f;
        gl[l] = 0.f;
        if (P && Pm > kMinProb) {
            const float U = ((int)(sums.y - ng) & 1 ? -1.f : 1.f) * expf(sums.x - lg);  // product over the others
            gl[l] = -sigma * U / Pm * scale_l;
        }
    }
    __syncthreads();
    if (x < a.N) {
        for (int k = 0; k < 4; ++k) {
            const uint32_t p = (d.vp >> (2 * k)) & 3u;
            if (!p) continue;
            const float g = ub2[4 * x + k].x;
            for (int w = 0; w < 3; ++w) Qbar[w] += g * pi[w + 1] * (ca[k].x - (anti(w + 1, p) ? 0.f : 1.f));
        }
        for (int l = 0; l < a.n_log; ++l) {
            const uint32_t P = a.logicals[(size_t)l * a.N + x];
            if (!P) continue;
            for (int w = 0; w < 3; ++w) Qbar[w] += gl[l] * pi[w + 1] * (cl[l].x - (anti(w + 1, P) ? 0.f : 1.f));
        }
    }
    __syncthreads();  // ub2 is rewritten by the next iteration
}

template <int MODEL>
__global__ void train_backward_kernel(const TrainArgs a) {
    extern __shared__ __align__(16) float sm[];
    const int Np = a.n_pad, K = a.K, S4 = 4 * Np + 4;
    const bool coset = a.loss_kind == kCoset;
    float *Pi0 = sm;                                 // [3Np]
    float *vh = Pi0 + 3 * Np;                        // [(K+1)][S4]   m_v->c^(t0 .. t0+K)
    float *cbar = vh + (size_t)(K + 1) * S4;         // [S4] adjoint of m_c->v^(t)
    // coset loss scratch, [S4] float2 over vh[K] and cbar: the adjoint never
    // reads m_v->c^(t0+K), and cbar is dead from the barrier that ends one
    // adjoint iteration's check step until step A of the next writes it
    float2 *ub2 = reinterpret_cast<float2 *>(vh + (size_t)K * S4);
    float *ch = cbar + S4;                           // [K][S4]       m_c->v^(t0+1 .. t0+K)
    float *Qh = ch + (size_t)K * S4;                 // [(K+1)][3Np]  Q^(t0 .. t0+K)
    float *gh = Qh + (size_t)(K + 1) * 3 * Np;       // [(K+1)][3Np]  g^(t0 .. t0+K) (Momentum only)
    float *vbar = gh + (MODEL == kMomentum ? (size_t)(K + 1) * 3 * Np : 0);  // [S4] adjoint of m_v->c^(t)
    float *red = vbar + S4;                          // [64]
    float2 *red2 = reinterpret_cast<float2 *>(red);
    const int x = threadIdx.x, shot = blockIdx.x;
    Adj d;
    load_adj(a, x, shot, d);
    const uint32_t tau = coset ? true_logical_parities(a, x, shot, red2) : 0u;
    const uint32_t zero = 4u * (uint32_t)Np;
    if (x < a.N) {
        const float px = a.prior[3 * x], py = a.prior[3 * x + 1], pz = a.prior[3 * x + 2];
        const float pI = 1.f - px - py - pz;
        Pi0[x] = logf(pI / px);
        Pi0[Np + x] = logf(pI / py);
        Pi0[2 * Np + x] = logf(pI / pz);
    }
    for (int k = x; k < S4; k += blockDim.x) vbar[k] = 0.f;
    if (x == 0) {
        for (int s = 0; s <= K; ++s) vh[(size_t)s * S4 + zero] = 0.f;
        for (int s = 0; s < K; ++s) ch[(size_t)s * S4 + zero] = 0.f;
    }
    float Qbar[3] = {0.f, 0.f, 0.f};  // adjoint of Q^(t) of the owned qubit
    float gbar[3] = {0.f, 0.f, 0.f};  // adjoint of g^(t) (Momentum)
    float wbar[4] = {0.f, 0.f, 0.f, 0.f};
    float *row = a.rows + (size_t)shot * a.width;
    const float sigma = d.sb ? -1.f : 1.f;
    __syncthreads();

    for (int c = a.nck - 1; c >= 0; --c) {
        const int t0 = c * K, t1 = min(a.T, t0 + K);
        // ---- recompute iterations t0+1 .. t1 from checkpoint c ----
        const float *ck = a.ckpt + ((size_t)shot * a.nck + c) * a.ck_floats;
        for (int k = x; k < 4 * Np; k += blockDim.x) vh[k] = ck[k];
        for (int k = x; k < 3 * Np; k += blockDim.x) Qh[k] = ck[4 * Np + k];
        if (MODEL == kMomentum)
            for (int k = x; k < 3 * Np; k += blockDim.x) gh[k] = ck[7 * Np + k];
        __syncthreads();
        for (int t = t0 + 1; t <= t1; ++t) {
            const int s = t - t0;
            const float *v_in = vh + (size_t)(s - 1) * S4;
            float *c_out = ch + (size_t)(s - 1) * S4;
            if (x < a.M) {
                float r[4], out[4];
                check_forward(a, d, v_in, r, out, t);
                for (int n = 0; n < 4; ++n)
                    if ((d.cp >> (2 * n)) & 3u) c_out[d.sl[n]] = out[n];
            }
            __syncthreads();
            if (x < a.N) {
                const float al = a.alpha[t - 1], be = a.beta[t - 1];
                const float *Qprev = Qh + (size_t)(s - 1) * 3 * Np;
                float *Qnew = Qh + (size_t)s * 3 * Np;
                float *v_out = vh + (size_t)s * S4;
                float Sm[3] = {0.f, 0.f, 0.f}, cin[4], Q[3];
                for (int k = 0; k < 4; ++k) {
                    const uint32_t p = (d.vp >> (2 * k)) & 3u;
                    cin[k] = p ? c_out[4 * x + k] : 0.f;
                    for (int w = 0; w < 3; ++w) Sm[w] += anti(w + 1, p) ? cin[k] : 0.f;
                }
                for (int w = 0; w < 3; ++w) {
                    if (MODEL == kMomentum) {
                        const float gm = a.gamma[t - 1];
                        const float *gprev = gh + (size_t)(s - 1) * 3 * Np;
                        const float g = gm * gprev[w * Np + x] +
                                        (1.f - gm) * (Qprev[w * Np + x] - Pi0[w * Np + x] - Sm[w]);
                        Q[w] = Qprev[w * Np + x] - al * g;
                        gh[(size_t)s * 3 * Np + w * Np + x] = g;
                    } else {
                        const float pit =
                            t > 1 ? al * Pi0[w * Np + x] + (1.f - al) * Qprev[w * Np + x] : Pi0[w * Np + x];
                        Q[w] = pit + Sm[w];
                    }
                    Qnew[w * Np + x] = Q[w];
                }
                for (int k = 0; k < 4; ++k) {
                    const uint32_t p = (d.vp >> (2 * k)) & 3u;
                    if (!p) {
                        v_out[4 * x + k] = 0.f;
                        continue;
                    }
                    float q[3], dl[3];
                    for (int w = 0; w < 3; ++w) q[w] = Q[w] - (anti(w + 1, p) ? cin[k] : 0.f);
                    const float L = fminf(fmaxf(lambda_grad(p, q, dl), -a.clip), a.clip);
                    v_out[4 * x + k] = (1.f - be) * L + be * v_in[4 * x + k];
                }
            }
            __syncthreads();
        }
        // ---- posterior loss: gradient at the last iteration ----
        if (!coset && t1 == a.T && x < a.N) {
            const float *Q = Qh + (size_t)(t1 - t0) * 3 * Np;
            const float z[4] = {0.f, -Q[x], -Q[Np + x], -Q[2 * Np + x]};
            const float zm = fmaxf(fmaxf(z[0], z[1]), fmaxf(z[2], z[3]));
            float se = 0.f;
            for (int k = 0; k < 4; ++k) se += expf(z[k] - zm);
            const int e = a.err[(size_t)shot * a.N + x];
            const float scale = 1.f / ((float)a.B * (float)a.N);
            for (int w = 0; w < 3; ++w) {
                const float pw = expf(z[w + 1] - zm) / se;
                Qbar[w] = -(pw - (e == w + 1 ? 1.f : 0.f)) * scale;  // d CE / d Q_W = -(p_W - [W = true])
            }
        }
        // ---- adjoint through iterations t1 .. t0+1 ----
        for (int t = t1; t > t0; --t) {
            const int s = t - t0;
            const float *v_prev = vh + (size_t)(s - 1) * S4;  // m_v->c^(t-1)
            const float *c_t = ch + (size_t)(s - 1) * S4;     // m_c->v^(t)
            const float *Qt = Qh + (size_t)s * 3 * Np;        // Q^(t)
            const float *Qprev = Qh + (size_t)(s - 1) * 3 * Np;
            const float al = a.alpha[t - 1], be = a.beta[t - 1];
            float bb = 0.f, ab = 0.f, gb = 0.f;
            // coset loss: the gradient of iteration t's term joins Q^(t)'s adjoint
            if (coset) coset_loss_backward(a, d, x, Qt, tau, ub2, red2, Qbar);
            // step A (qubit role): damping, lambda, posterior, EWA prior
            if (x < a.N) {
                float Qacc[3] = {0.f, 0.f, 0.f}, cb_part[4] = {0.f, 0.f, 0.f, 0.f};
                for (int k = 0; k < 4; ++k) {
                    const uint32_t p = (d.vp >> (2 * k)) & 3u;
                    if (!p) continue;
                    const float cin = c_t[4 * x + k];
                    float q[3], dl[3];
                    for (int w = 0; w < 3; ++w) q[w] = Qt[w * Np + x] - (anti(w + 1, p) ? cin : 0.f);
                    const float lam = lambda_grad(p, q, dl);
                    const float L = fminf(fmaxf(lam, -a.clip), a.clip);
                    const float vb = vbar[4 * x + k];
                    bb += vb * (v_prev[4 * x + k] - L);
                    // a clipped lambda passes no gradient (and its dl may be
                    // inf / nan where C or A underflowed)
                    const float Lb = (fabsf(lam) <= a.clip) ? (1.f - be) * vb : 0.f;
                    if (Lb != 0.f) {
                        for (int w = 0; w < 3; ++w) {
                            Qacc[w] += Lb * dl[w];
                            if (anti(w + 1, p)) cb_part[k] -= Lb * dl[w];
                        }
                    }
                }
                float Qtot[3], Sbar[3];
                for (int w = 0; w < 3; ++w) Qtot[w] = Qbar[w] + Qacc[w];
                if (MODEL == kMomentum) {
                    // Q^(t) = Q^(t-1) - alpha g^(t);  g^(t) = gamma g^(t-1) + (1 - gamma) D,
                    // D = Q^(t-1) - Pi^(0) - S^(t)
                    const float gm = a.gamma[t - 1];
                    const float *gt = gh + (size_t)s * 3 * Np, *gprev = gh + (size_t)(s - 1) * 3 * Np;
                    float Sm[3] = {0.f, 0.f, 0.f};
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t p = (d.vp >> (2 * k)) & 3u;
                        for (int w = 0; w < 3; ++w)
                            if (p && anti(w + 1, p)) Sm[w] += c_t[4 * x + k];
                    }
                    for (int w = 0; w < 3; ++w) {
                        const float gtot = gbar[w] - al * Qtot[w];  // adjoint of g^(t)
                        const float D = Qprev[w * Np + x] - Pi0[w * Np + x] - Sm[w];
                        ab -= Qtot[w] * gt[w * Np + x];
                        gb += gtot * (gprev[w * Np + x] - D);
                        Sbar[w] = -(1.f - gm) * gtot;
                        Qbar[w] = Qtot[w] + (1.f - gm) * gtot;  // adjoint of Q^(t-1)
                        gbar[w] = gm * gtot;                    // adjoint of g^(t-1)
                    }
                } else {
                    for (int w = 0; w < 3; ++w) Sbar[w] = Qtot[w];
                    if (t > 1) {
                        for (int w = 0; w < 3; ++w) {
                            ab += Qtot[w] * (Pi0[w * Np + x] - Qprev[w * Np + x]);
                            Qbar[w] = (1.f - al) * Qtot[w];
                        }
                    } else {
                        Qbar[0] = Qbar[1] = Qbar[2] = 0.f;
                    }
                }
                for (int k = 0; k < 4; ++k) {
                    const uint32_t p = (d.vp >> (2 * k)) & 3u;
                    float cb = cb_part[k];
                    for (int w = 0; w < 3; ++w)
                        if (anti(w + 1, p)) cb += Sbar[w];
                    cbar[4 * x + k] = p ? cb : 0.f;
                    vbar[4 * x + k] = p ? be * vbar[4 * x + k] : 0.f;  // damping path to m_v->c^(t-1)
                }
            }
            const float sum_b = block_sum(bb, red);
            const float sum_a = block_sum(ab, red);
            const float sum_g = MODEL == kMomentum ? block_sum(gb, red) : 0.f;
            if (x == 0) {
                row[t - 1] = (MODEL == kMomentum || t > 1) ? sum_a : 0.f;
                row[a.T + t - 1] = sum_b;
                if (MODEL == kMomentum) row[2 * a.T + a.E + t - 1] = sum_g;
            }
            __syncthreads();
            // step B (check role): message weights and the check-node derivative
            if (x < a.M) {
                float mag[4], sg[4], r[4], rb[4];
                for (int n = 0; n < 4; ++n) {
                    const float m = v_prev[d.sl[n]];
                    const bool valid = ((d.cp >> (2 * n)) & 3u) != 0u;
                    mag[n] = valid ? phi(fabsf(m)) : 0.f;
                    sg[n] = (valid && m < 0.f) ? -1.f : 1.f;
                }
                for (int n = 0; n < 4; ++n) {
                    rb[n] = 0.f;
                    if (!((d.cp >> (2 * n)) & 3u)) continue;
                    float ext = 0.f, ps = 1.f;
                    for (int f = 0; f < 4; ++f)
                        if (f != n) {
                            ext += mag[f];
                            ps *= sg[f];
                        }
                    r[n] = ps * phi(ext);
                    const float we = a.w[d.ce + n];
                    const float cb = cbar[d.sl[n]];
                    if (fabsf(we * sigma * r[n]) <= a.clip) {
                        wbar[n] += cb * sigma * r[n];
                        rb[n] = cb * we * sigma;
                    }
                }
                for (int f = 0; f < 4; ++f) {
                    if (!((d.cp >> (2 * f)) & 3u)) continue;
                    const float mf = v_prev[d.sl[f]];
                    const float smf = sinhf(copysignf(fmaxf(fabsf(mf), 1e-30f), mf));
                    float acc = 0.f;
                    for (int n = 0; n < 4; ++n)
                        if (n != f && rb[n] != 0.f) acc += rb[n] * sinhf(r[n]) / smf;  // d r_n / d m_f
                    vbar[d.sl[f]] += acc;
                }
            }
            __syncthreads();
        }
    }
    if (x < a.M)
        for (int n = 0; n < 4; ++n)
            if ((d.cp >> (2 * n)) & 3u) row[2 * a.T + d.ce + n] = wbar[n];
}

// out[k] = scale * sum_b rows[b][offset + k] for k < count (fixed order, so
// deterministic).
__global__ void reduce_rows_kernel(const float *rows, int B, int width, int offset, int count, float *out,
                                   float scale) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += rows[(size_t)b * width + offset + k];
    out[k] = s * scale;
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

int fill(const bpq_tanner *t, int model, const uint32_t *syn, const uint8_t *err, const float *prior, int B, int T,
         int K, const float *alpha, const float *beta, const float *gamma, const float *w, float clip,
         const bpq_train_loss *loss, void *work, size_t work_bytes, TrainArgs &a) {
    int rc = need_uploaded(t);
    if (rc) return rc;
    if (model != kEWAInit && model != kMomentum) return fail(BPQ_EINVAL, "unknown training model");
    if (B < 1 || T < 1 || T > 255 || K < 1) return fail(BPQ_EINVAL, "bad B, T or checkpoint interval");
    if (!syn || !err || !prior || !alpha || !beta || !w || !work) return fail(BPQ_EINVAL, "NULL argument");
    if (misaligned(work, kBufferAlign)) return fail(BPQ_EINVAL, "workspace not 16-byte aligned");
    if (misaligned(syn, kWordAlign) || misaligned(prior, kWordAlign) || misaligned(alpha, kWordAlign) ||
        misaligned(beta, kWordAlign) || misaligned(w, kWordAlign) || (gamma && misaligned(gamma, kWordAlign)))
        return fail(BPQ_EINVAL, "an input array not 4-byte aligned");
    if (model == kMomentum && !gamma) return fail(BPQ_EINVAL, "the Momentum model needs gamma");
    if (!(clip > 0.f)) return fail(BPQ_EINVAL, "msg_clip must be positive");
    const int kind = loss ? loss->kind : BPQ_TRAIN_LOSS_POSTERIOR;
    if (kind != BPQ_TRAIN_LOSS_POSTERIOR && kind != BPQ_TRAIN_LOSS_COSET) return fail(BPQ_EINVAL, "unknown loss");
    if (kind == BPQ_TRAIN_LOSS_COSET && (!loss->logicals_dev || loss->n_logicals < 1 ||
                                         loss->n_logicals > kMaxLogicals))
        return fail(BPQ_EINVAL, "the coset loss needs 1 to 4 logical operators");
    if (std::max(t->N, t->M) > 1024) return fail(BPQ_EINVAL, "training kernels take codes of up to 1024 nodes");
    if (work_bytes < bpq_train_workspace_bytes(t, model, B, T, K))
        return fail(BPQ_EINVAL, "training workspace too small");
    a = TrainArgs{};
    a.table = t->d_table;
    a.off_chk_pauli = t->off_chk_pauli;
    a.off_var_pauli = t->off_var_pauli;
    a.var_canon = t->d_var_canon;
    a.chk_ptr = t->d_chk_ptr;
    a.syn = syn;
    a.err = err;
    a.prior = prior;
    a.alpha = alpha;
    a.beta = beta;
    a.w = w;
    a.gamma = gamma;
    a.N = t->N;
    a.M = t->M;
    a.E = t->E;
    a.W = (t->M + 31) / 32;
    a.B = B;
    a.T = T;
    a.K = K;
    a.nck = (T + K - 1) / K;
    a.n_pad = (t->N + 3) & ~3;
    a.ck_floats = (model == kMomentum ? 10 : 7) * a.n_pad;
    a.width = (model == kMomentum ? 3 : 2) * T + t->E;
    a.clip = clip;
    a.loss_kind = kind;
    a.logicals = kind == BPQ_TRAIN_LOSS_COSET ? loss->logicals_dev : nullptr;
    a.n_log = kind == BPQ_TRAIN_LOSS_COSET ? loss->n_logicals : 0;
    uint8_t *p = static_cast<uint8_t *>(work);
    a.ckpt = reinterpret_cast<float *>(p);
    p += a256(sizeof(float) * (size_t)B * a.nck * a.ck_floats);
    a.loss_shot = reinterpret_cast<float *>(p);
    p += a256(sizeof(float) * B);
    a.rows = reinterpret_cast<float *>(p);
    return BPQ_OK;
}

int threads_for(const bpq_tanner *t) { return ((std::max(t->N, t->M) + 31) / 32) * 32; }

}  // namespace tr
}  // namespace bpq

extern "C" {

size_t bpq_train_workspace_bytes(const bpq_tanner *t, int model, int B, int T, int ckpt_every) {
    if (!t || B < 1 || T < 1 || ckpt_every < 1) return 0;
    if (model != BPQ_TRAIN_EWAINIT && model != BPQ_TRAIN_MOMENTUM) return 0;
    const size_t np = (size_t)((t->N + 3) & ~3);
    const size_t nck = (size_t)((T + ckpt_every - 1) / ckpt_every);
    const size_t per_ck = (model == BPQ_TRAIN_MOMENTUM ? 10 : 7) * np;
    const size_t width = (size_t)(model == BPQ_TRAIN_MOMENTUM ? 3 : 2) * T + t->E;
    return bpq::tr::a256(sizeof(float) * (size_t)B * nck * per_ck) + bpq::tr::a256(sizeof(float) * B) +
           bpq::tr::a256(sizeof(float) * (size_t)B * width);
}

int bpq_train_forward(const bpq_tanner *t, int model, const uint32_t *syn_dev, const uint8_t *err_dev,
                      const float *prior_dev, int B, int T, int ckpt_every, const float *alpha_dev,
                      const float *beta_dev, const float *gamma_dev, const float *w_dev, float msg_clip,
                      const bpq_train_loss *loss, float *loss_dev, float *Q_dev, void *work_dev, size_t work_bytes,
                      void *stream) {
    bpq::tr::TrainArgs a;
    int rc = bpq::tr::fill(t, model, syn_dev, err_dev, prior_dev, B, T, ckpt_every, alpha_dev, beta_dev, gamma_dev,
                           w_dev, msg_clip, loss, work_dev, work_bytes, a);
    if (rc) return rc;
    if (!loss_dev) return fail(BPQ_EINVAL, "NULL loss output");
    a.Q_out = Q_dev;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool mom = model == BPQ_TRAIN_MOMENTUM;
    const bool coset = a.loss_kind == BPQ_TRAIN_LOSS_COSET;
    const size_t S4 = 4 * (size_t)a.n_pad + 4;
    const size_t smem = sizeof(float) * ((coset ? 4 : 2) * S4 + (mom ? 9 : 6) * (size_t)a.n_pad + 64);
    if (smem > 227 * 1024) return fail(BPQ_EINVAL, "code too large for the training kernels' shared memory");
    void (*fn)(const bpq::tr::TrainArgs) = mom ? bpq::tr::train_forward_kernel<bpq::tr::kMomentum>
                                               : bpq::tr::train_forward_kernel<bpq::tr::kEWAInit>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail(BPQ_ECUDA, std::string("train forward attribute: ") + cudaGetErrorString(e));
    fn<<<B, bpq::tr::threads_for(t), smem, st>>>(a);
    // per-shot sums: over qubits (posterior loss) or already normalised (coset loss)
    bpq::tr::reduce_rows_kernel<<<1, 32, 0, st>>>(a.loss_shot, B, 1, 0, 1, loss_dev,
                                                  coset ? 1.f / (float)B : 1.f / ((float)B * (float)t->N));
    return bpq::cuda_check(cudaGetLastError(), "train forward launch");
}

int bpq_train_backward(const bpq_tanner *t, int model, const uint32_t *syn_dev, const uint8_t *err_dev,
                       const float *prior_dev, int B, int T, int ckpt_every, const float *alpha_dev,
                       const float *beta_dev, const float *gamma_dev, const float *w_dev, float msg_clip,
                       const bpq_train_loss *loss, float *grad_alpha_dev, float *grad_beta_dev,
                       float *grad_gamma_dev, float *grad_w_dev, void *work_dev, size_t work_bytes, void *stream) {
    bpq::tr::TrainArgs a;
    int rc = bpq::tr::fill(t, model, syn_dev, err_dev, prior_dev, B, T, ckpt_every, alpha_dev, beta_dev, gamma_dev,
                           w_dev, msg_clip, loss, work_dev, work_bytes, a);
    if (rc) return rc;
    const bool mom = model == BPQ_TRAIN_MOMENTUM;
    if (!grad_alpha_dev || !grad_beta_dev || !grad_w_dev || (mom && !grad_gamma_dev))
        return fail(BPQ_EINVAL, "NULL gradient output");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int K = a.K, Np = a.n_pad, S4 = 4 * Np + 4;
    const size_t hist = (size_t)(K + 1) * 3 * Np * (mom ? 2 : 1);
    // the coset loss's scratch lives in dead parts of the history (no extra bytes)
    const size_t smem = sizeof(float) * (3 * Np + (size_t)(K + 1) * S4 + (size_t)K * S4 + hist + 2 * S4 + 64);
    if (smem > 227 * 1024) return fail(BPQ_EINVAL, "checkpoint interval too long for shared memory");
    void (*fn)(const bpq::tr::TrainArgs) = mom ? bpq::tr::train_backward_kernel<bpq::tr::kMomentum>
                                               : bpq::tr::train_backward_kernel<bpq::tr::kEWAInit>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail(BPQ_ECUDA, std::string("train backward attribute: ") + cudaGetErrorString(e));
    fn<<<B, bpq::tr::threads_for(t), smem, st>>>(a);
    // per-shot rows hold [alpha | beta | w | gamma]
    const int width = a.width;
    bpq::tr::reduce_rows_kernel<<<(T + 127) / 128, 128, 0, st>>>(a.rows, B, width, 0, T, grad_alpha_dev, 1.f);
    bpq::tr::reduce_rows_kernel<<<(T + 127) / 128, 128, 0, st>>>(a.rows, B, width, T, T, grad_beta_dev, 1.f);
    bpq::tr::reduce_rows_kernel<<<(t->E + 127) / 128, 128, 0, st>>>(a.rows, B, width, 2 * T, t->E, grad_w_dev,
                                                                     1.f);
    if (mom)
        bpq::tr::reduce_rows_kernel<<<(T + 127) / 128, 128, 0, st>>>(a.rows, B, width, 2 * T + t->E, T,
                                                                     grad_gamma_dev, 1.f);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(BPQ_ECUDA, std::string("train backward launch: ") + cudaGetErrorString(e));
    return BPQ_OK;
}

}  // extern "C"
