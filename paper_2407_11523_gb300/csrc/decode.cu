// Flooding-schedule GF(4) belief propagation on sm_103a: one group of G warps
// decodes one shot at a time; each thread owns up to NPT checks and NPT qubits
// (node j belongs to thread j mod 32G).  The shot's edge messages live in
// shared memory, one float per edge, updated in place: the check pass turns
// variable-to-check messages into check-to-variable messages and the variable
// pass turns them back.  Groups synchronise on their own named barrier, so
// every shot stops as soon as its hard decision satisfies the syndrome, and
// the group then takes the next shot from a global work queue (a persistent
// kernel, grid = SMs x resident CTAs).  The Tanner-graph adjacency is staged
// once per CTA into shared memory by a bulk TMA copy.
//
// Arithmetic (Sec. II-B1 and Sec. III of the paper, fp32):
//  * check-to-variable, eq. (h_update): with phi(x) = -ln tanh(x/2) (its own
//    inverse), 2 atanh(prod_k tanh(m_k/2)) = sign * phi(sum_k phi(|m_k|)),
//    sign = (-1)^{s_i} prod_k sign(m_k).  Variable-to-check messages are
//    stored as sign(m) * phi(|m|), so the check pass only sums magnitudes
//    and XORs sign bits; phi(S) = log1p(2 / expm1(S)) keeps full relative
//    accuracy for large and small S.
//  * variable-to-check, eqs. (lambda), (v_update), (mombp5): the message is
//    lambda_H(Q - own anticommuting message) = ln(C / A) with
//    C = 1 + e^{-Q_H} and A = (e^{-Q_a} + e^{-Q_b}) e^{m_c->v}, a, b the two
//    Paulis other than H.  All four exponentials share the shift
//    c0 = min(0, Q_X, Q_Y, Q_Z), so nothing overflows, and the stored value
//    phi(|lambda|) = ln((C+A)/|C-A|) = log1p(2 min(C,A) / |C-A|) comes out
//    of C and A without forming lambda.
//  * message saturation: |m| <= msg_clip on both directions, i.e.
//    phi(|m_v->c|) >= phi(msg_clip) and |m_c->v| <= msg_clip.
#include <cuda_runtime.h>

#include "bpq_internal.h"
#include "decode_launch.h"

namespace bpq {

namespace {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared (TMA), completion signalled on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after `limit` polls (each poll may itself suspend
// for a short hardware-defined time).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit) {
    for (uint32_t n = 0; n < limit; ++n)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void group_sync(int G, int bar_id) {
    if (G == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(G * 32) : "memory");
    }
}

// Barrier over the group that also returns whether any thread's pred is set.
__device__ __forceinline__ int group_any(int G, int bar_id, int pred) {
    if (G == 1) {
        __syncwarp();
        return __any_sync(0xffffffffu, pred);
    }
    int r;
    asm volatile(
        "{ .reg .pred p, q; setp.ne.s32 p, %1, 0; bar.red.or.pred q, %2, %3, p; selp.s32 %0, 1, 0, q; }"
        : "=r"(r)
        : "r"(pred), "r"(bar_id), "r"(G * 32)
        : "memory");
    return r;
}

// <A, B> for single-qubit Pauli codes (0 = I, 1 = X, 2 = Y, 3 = Z).
__device__ __forceinline__ uint32_t anti(uint32_t a, uint32_t b) {
    return (a != 0u) & (b != 0u) & (a != b);
}

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// Hardware approximations (PTX .approx, flush-to-zero): relative error about
// 2^-22 for ex2 and rcp, absolute error about 2^-22 for lg2 near 1.
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Check-to-variable magnitude w = phi(S) = ln(1 + 2 / (e^S - 1)), S >= 0,
// needed to an absolute accuracy.  e^S - 1 keeps its relative accuracy:
// below S = 1/4 from its Taylor series to S^6/720 (truncation < 5e-8
// relative), above from 2^(S log2 e) - 1 (the ex2 error is amplified at most
// e^S/(e^S-1) < 4.6 times).  Then w = ln2 * lg2(1 + 2/(e^S-1)); S = 0 gives
// w = inf (clipped by the caller), S -> inf gives w -> 0.
__device__ __forceinline__ float phi_check(float S) {
    S = fminf(S, 80.0f);
    const float poly =
        S * fmaf(S, fmaf(S, fmaf(S, fmaf(S, fmaf(S, 1.0f / 720.0f, 1.0f / 120.0f), 1.0f / 24.0f), 1.0f / 6.0f), 0.5f), 1.0f);
    const float em1 = S < 0.25f ? poly : ex2(S * kLog2e) - 1.0f;
    return kLn2 * lg2(fmaf(2.0f, rcp(em1), 1.0f));
}

// phi(|lambda|) = ln(1 + r), r = 2 min(C,A) / |C - A|, needed to a relative
// accuracy (small values are summed by the check pass): below r = 1/16 from
// the series r - r^2/2 + r^3/3 - r^4/4 + r^5/5 (truncation < 2e-7 relative),
// above from ln2 * lg2(1 + r).
__device__ __forceinline__ float log1p_rel(float r) {
    const float poly = r * fmaf(r, fmaf(r, fmaf(r, fmaf(r, 0.2f, -0.25f), 1.0f / 3.0f), -0.5f), 1.0f);
    return r < 0.0625f ? poly : kLn2 * lg2(1.0f + r);
}

}  // namespace

template <int VARIANT, int NPT, bool TRACE>
__global__ void __launch_bounds__(512) decode_kernel(const DecodeArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);
    int *grp_shot = reinterpret_cast<int *>(smem + 16);
    uint8_t *tab = smem + kSmemHeader;

    const int tid = threadIdx.x;
    const int G = a.G;
    const int T = G * 32;
    const int group = tid / T;
    const int tg = tid - group * T;
    const int bar_id = 1 + group;
    const int N = a.N, M = a.M;
    const int npt = a.npt;
    float *slots = reinterpret_cast<float *>(smem + kSmemHeader + a.table_bytes + (size_t)group * a.group_bytes);
    uint8_t *decs = reinterpret_cast<uint8_t *>(slots + a.slots_floats);

    // ---- stage the adjacency table once per CTA (bulk TMA copy) ----
    if (tid == 0) {
        mbar_init(mbar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(mbar, a.table_bytes);
        bulk_g2s(tab, a.table, a.table_bytes, mbar);
    }
    const bool staged = mbar_wait_bounded(mbar, 0, 1u << 22);
    if (__syncthreads_or(!staged)) {
        if (tid == 0) atomicExch(a.work + 1, 1u);
        mbar_wait_bounded(mbar, 0, 1u << 22);  // let an in-flight copy land before exiting
        return;
    }

    // ---- per-thread adjacency and prior LLRs, kept in registers ----
    uint32_t cs_lo[NPT], cs_hi[NPT], cinfo[NPT], vinfo[NPT];
    float Pi[NPT][3];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        cs_lo[k] = cs_hi[k] = 0xFFFFFFFFu;
        cinfo[k] = vinfo[k] = 0u;
        Pi[k][0] = Pi[k][1] = Pi[k][2] = 0.f;
        if (k < npt) {
            const int i = k * T + tg;
            if (i < M) {
                const uint2 s = *reinterpret_cast<const uint2 *>(tab + 8 * i);
                cs_lo[k] = s.x;
                cs_hi[k] = s.y;
                cinfo[k] = tab[a.off_chk_pauli + i];
            }
            const int j = k * T + tg;
            if (j < N) {
                vinfo[k] = tab[a.off_var_pauli + j];
                const float px = a.prior[3 * j], py = a.prior[3 * j + 1], pz = a.prior[3 * j + 2];
                const float pI = 1.0f - px - py - pz;
                // Pi_{v_j,W} = ln(p^I / p^W)
                Pi[k][0] = logf(pI / px);
                Pi[k][1] = logf(pI / py);
                Pi[k][2] = logf(pI / pz);
            }
        }
    }

    const float clip = a.clip, phi_clip = a.phi_clip;

    for (;;) {
        if (tg == 0) grp_shot[group] = (int)atomicAdd(a.work, 1u);
        group_sync(G, bar_id);
        const int shot = grp_shot[group];
        if (shot >= a.B) break;

        // syndrome bits of the owned checks (bit k <-> check k*T + tg)
        uint32_t sbits = 0;
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int i = k * T + tg;
            if (k < npt && i < M) {
                const uint32_t w = __ldg(a.syn + (size_t)shot * a.W + (i >> 5));
                sbits |= ((w >> (i & 31)) & 1u) << k;
            }
        }

        // per-qubit state: Q^(0) = Pi^(0), g^(0) = G^(0) = 0
        float Qp[NPT][3], gs[NPT][3];
        uint32_t dk[NPT];
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            dk[k] = 0;
#pragma unroll
            for (int w = 0; w < 3; ++w) {
                Qp[k][w] = Pi[k][w];
                gs[k][w] = 0.f;
            }
        }

        // variable-to-check messages of eq. (init): lambda(Pi^(0)), written as
        // the variable pass with Q = Pi^(0) and no incoming messages
        auto variable_pass = [&](int t, const float (&Qk)[3], int k, int j, const float (&win)[4]) {
            const uint32_t vp = vinfo[k];
            const float c0 = fminf(0.f, fminf(Qk[0], fminf(Qk[1], Qk[2])));
            const float e0 = ex2(c0 * kLog2e);
            const float eX = ex2((c0 - Qk[0]) * kLog2e), eY = ex2((c0 - Qk[1]) * kLog2e),
                        eZ = ex2((c0 - Qk[2]) * kLog2e);
            float out[4];
#pragma unroll
            for (int n = 0; n < 4; ++n) {
                const uint32_t p = (vp >> (2 * n)) & 3u;
                out[n] = 0.f;
                if (p) {
                    const float C = e0 + (p == 1u ? eX : p == 2u ? eY : eZ);
                    const float Ab = p == 1u ? eY + eZ : p == 2u ? eX + eZ : eX + eY;
                    const float A = Ab * ex2(win[n] * kLog2e);
                    const float mx = fmaxf(C, A), mn = fminf(C, A);
                    float ph = log1p_rel(2.0f * mn * rcp(mx - mn));
                    ph = fmaxf(ph, phi_clip);  // |lambda| <= msg_clip
                    out[n] = (A > C) ? -ph : ph;
                    if (TRACE && a.tr_v2c) {
                        const float lam = fminf(fmaxf(kLn2 * (lg2(C) - lg2(A)), -clip), clip);
                        a.tr_v2c[((size_t)shot * (a.max_iter + 1) + t) * a.E + a.var_canon[4 * j + n]] = lam;
                    }
                }
            }
            *reinterpret_cast<float4 *>(slots + 4 * j) = make_float4(out[0], out[1], out[2], out[3]);
        };

#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int j = k * T + tg;
            if (k < npt && j < N) {
                const float z4[4] = {0.f, 0.f, 0.f, 0.f};
                variable_pass(0, Pi[k], k, j, z4);
            }
        }
        group_sync(G, bar_id);

        int conv = 0, iters = 0;
        for (int t = 1;; ++t) {
            const bool do_check = t > 1 && (!TRACE || t > a.max_iter);
            const bool do_msgs = t <= a.max_iter;
            int mismatch = 0;

            // ---- check pass: syndrome test of the previous decision, then eq. (h_update) ----
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int i = k * T + tg;
                if (k < npt && i < M) {
                    const uint32_t sl[4] = {cs_lo[k] & 0xFFFFu, cs_lo[k] >> 16, cs_hi[k] & 0xFFFFu, cs_hi[k] >> 16};
                    const uint32_t cp = cinfo[k];
                    const uint32_t sb = (sbits >> k) & 1u;
                    float mag[4];
                    uint32_t sg[4];
#pragma unroll
                    for (int n = 0; n < 4; ++n) {
                        const bool valid = sl[n] != kNoSlot;
                        const float v = valid ? slots[sl[n]] : 0.f;
                        mag[n] = fabsf(v);
                        sg[n] = valid ? (__float_as_uint(v) >> 31) : 0u;
                    }
                    if (do_check) {
                        uint32_t par = sb;
#pragma unroll
                        for (int n = 0; n < 4; ++n)
                            if (sl[n] != kNoSlot) par ^= anti(decs[sl[n] >> 2], (cp >> (2 * n)) & 3u);
                        mismatch |= (int)par;
                    }
                    if (do_msgs) {
                        const uint32_t par_all = sb ^ sg[0] ^ sg[1] ^ sg[2] ^ sg[3];
                        const float e01 = mag[0] + mag[1], e23 = mag[2] + mag[3];
                        const float ext[4] = {mag[1] + e23, mag[0] + e23, e01 + mag[3], e01 + mag[2]};
#pragma unroll
                        for (int n = 0; n < 4; ++n) {
                            if (sl[n] != kNoSlot) {
                                const float wv = fminf(phi_check(ext[n]), clip);
                                const float m = (par_all ^ sg[n]) ? -wv : wv;
                                slots[sl[n]] = m;
                                if (TRACE && a.tr_c2v)
                                    a.tr_c2v[((size_t)shot * a.max_iter + (t - 1)) * a.E + a.chk_ptr[i] + n] = m;
                            }
                        }
                    }
                }
            }
            const int any = group_any(G, bar_id, mismatch);
            if (do_check && !any) {
                conv = 1;
                iters = t - 1;
                break;
            }
            if (!do_msgs) {
                conv = 0;
                iters = a.max_iter;
                break;
            }

            // ---- variable pass: posterior of the variant, decision, eq. (v_update)/(mombp5) ----
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int j = k * T + tg;
                if (k < npt && j < N) {
                    const float4 w4 = *reinterpret_cast<const float4 *>(slots + 4 * j);
                    const float win[4] = {w4.x, w4.y, w4.z, w4.w};
                    const uint32_t vp = vinfo[k];
                    float S[3] = {0.f, 0.f, 0.f};
#pragma unroll
                    for (int n = 0; n < 4; ++n) {
                        const uint32_t p = (vp >> (2 * n)) & 3u;
                        if (p) {
                            if (p != 1u) S[0] += win[n];
                            if (p != 2u) S[1] += win[n];
                            if (p != 3u) S[2] += win[n];
                        }
                    }
                    float Q[3];
#pragma unroll
                    for (int w = 0; w < 3; ++w) {
                        if (VARIANT == BPQ_PLAIN) {
                            Q[w] = Pi[k][w] + S[w];  // eq. (p_update)
                        } else if (VARIANT == BPQ_EWAINIT) {
                            // eq. (EWAInit): Pi^(t) = alpha Pi^(0) + (1-alpha) Q^(t-1), t > 1
                            const float pit = t > 1 ? a.alpha * Pi[k][w] + (1.f - a.alpha) * Qp[k][w] : Pi[k][w];
                            Q[w] = pit + S[w];
                        } else if (VARIANT == BPQ_MOMENTUM) {
                            // eqs. (mombp1), (mombp2) with the gradient of (mombp3)
                            const float grad = Qp[k][w] - Pi[k][w] - S[w];
                            gs[k][w] = a.gamma * gs[k][w] + (1.f - a.gamma) * grad;
                            Q[w] = Qp[k][w] - a.alpha * gs[k][w];
                        } else {
                            // eq. (boost) from t = 2; G accumulates g'^2
                            const float gp = Qp[k][w] - Pi[k][w] - S[w];
                            if (t >= 2 || a.ada_from1) gs[k][w] += gp * gp;
                            Q[w] = t == 1 ? Pi[k][w] + S[w] : Qp[k][w] - a.alpha * gp * rcp(sqrt_approx(gs[k][w]) + a.eps);
                        }
                        Qp[k][w] = Q[w];
                    }
                    // hard decision: I if all Q_W > 0, else the first minimum of X, Y, Z
                    uint32_t d;
                    if (Q[0] > 0.f && Q[1] > 0.f && Q[2] > 0.f) {
                        d = 0;
                    } else {
                        d = 1;
                        float mq = Q[0];
                        if (Q[1] < mq) { d = 2; mq = Q[1]; }
                        if (Q[2] < mq) d = 3;
                    }
                    dk[k] = d;
                    decs[j] = (uint8_t)d;
                    if (TRACE) {
                        const size_t o = (size_t)shot * a.max_iter + (t - 1);
                        if (a.tr_Q) {
                            a.tr_Q[(o * N + j) * 3 + 0] = Q[0];
                            a.tr_Q[(o * N + j) * 3 + 1] = Q[1];
                            a.tr_Q[(o * N + j) * 3 + 2] = Q[2];
                        }
                        if (a.tr_dec) a.tr_dec[o * N + j] = (uint8_t)d;
                    }
                    variable_pass(t, Q, k, j, win);
                }
            }
            group_sync(G, bar_id);
        }

        // ---- outputs ----
        if (!TRACE || a.est) {
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int j = k * T + tg;
                if (k < npt && j < N) a.est[(size_t)shot * N + j] = (uint8_t)dk[k];
            }
        }
        if (tg == 0 && (!TRACE || a.conv)) {
            a.conv[shot] = (uint8_t)conv;
            a.iters[shot] = (uint8_t)iters;
        }
    }
}

namespace {

using KernelFn = void (*)(const DecodeArgs);

template <bool TRACE>
KernelFn pick(int variant, int NPT) {
#define BPQ_CASE(V)                                              \
    case V:                                                      \
        if (NPT == 1) return decode_kernel<V, 1, TRACE>;         \
        if (NPT == 2) return decode_kernel<V, 2, TRACE>;         \
        return decode_kernel<V, 4, TRACE>;
    switch (variant) {
        BPQ_CASE(BPQ_PLAIN)
        BPQ_CASE(BPQ_MOMENTUM)
        BPQ_CASE(BPQ_ADAGRAD)
        BPQ_CASE(BPQ_EWAINIT)
    }
#undef BPQ_CASE
    return nullptr;
}

}  // namespace

int decode_launch_shape(const bpq_tanner *t, LaunchShape *s) {
    const int nodes = t->N > t->M ? t->N : t->M;
    int T = t->threads_per_shot;
    if (T <= 0) {
        const int need = (nodes + kMaxNodesPerThread - 1) / kMaxNodesPerThread;
        T = ((need + 31) / 32) * 32;
    }
    if (T % 32 || T < 32 || T > 512) return fail(BPQ_EINVAL, "threads per shot must be a multiple of 32 in [32, 512]");
    const int npt = (nodes + T - 1) / T;
    if (npt > kMaxNodesPerThread) return fail(BPQ_EINVAL, "too few threads per shot for this code");
    int gpc = t->shots_per_cta;
    if (gpc <= 0) gpc = 512 / T > 0 ? 512 / T : 1;
    if (gpc > 15) gpc = 15;
    while (gpc > 1 && gpc * T > 512) --gpc;
    s->T = T;
    s->G = T / 32;
    s->npt = npt;
    s->NPT = npt <= 1 ? 1 : npt <= 2 ? 2 : 4;
    s->groups_per_cta = gpc;
    s->slots_floats = (uint32_t)((4 * t->N + 3) & ~3);
    s->group_bytes = (uint32_t)(s->slots_floats * 4 + ((t->N + 15) & ~15));
    s->smem = kSmemHeader + (uint32_t)t->table.size() + (size_t)gpc * s->group_bytes;
    if (s->smem > 227 * 1024) return fail(BPQ_EINVAL, "shared memory of the launch shape exceeds 227 KB");
    return BPQ_OK;
}

int decode_launch(const bpq_tanner *t, DecodeArgs &a, int variant, bool trace, cudaStream_t st, int *ctas_out) {
    LaunchShape s;
    int rc = decode_launch_shape(t, &s);
    if (rc) return rc;
    KernelFn fn = trace ? pick<true>(variant, s.NPT) : pick<false>(variant, s.NPT);
    if (!fn) return fail(BPQ_EINVAL, "bad variant");
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
    if (e != cudaSuccess) return fail(BPQ_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    const int threads = s.T * s.groups_per_cta;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, s.smem);
    if (e != cudaSuccess || per_sm < 1)
        return fail(BPQ_ECUDA, "launch shape does not fit on an SM");
    long ctas = (long)per_sm * t->num_sms;
    const long need = (a.B + s.groups_per_cta - 1) / s.groups_per_cta;
    if (ctas > need) ctas = need;
    if (ctas < 1) ctas = 1;
    a.G = s.G;
    a.npt = s.npt;
    a.slots_floats = s.slots_floats;
    a.group_bytes = s.group_bytes;
    if (ctas_out) *ctas_out = (int)ctas;
    fn<<<(unsigned)ctas, threads, s.smem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(BPQ_ECUDA, std::string("decode launch: ") + cudaGetErrorString(e));
    return BPQ_OK;
}

}  // namespace bpq
