// Flooding-schedule GF(4) belief propagation on sm_103a: one group of G warps
// decodes one shot at a time; each thread owns NPT checks and NPT qubits
// (node j belongs to thread j mod 32G).  The shot's edge messages live in
// shared memory, one float per edge, updated in place: the check pass turns
// variable-to-check messages into check-to-variable messages and the variable
// pass turns them back.  Groups synchronise on their own named barrier, so
// every shot stops as soon as its hard decision satisfies the syndrome, and
// the group then takes the next shot from a global work queue (a persistent
// kernel, grid = SMs x resident CTAs).  The Tanner-graph adjacency is staged
// once per CTA into shared memory by a bulk TMA copy; the per-qubit prior
// LLRs sit in shared memory (shared by the CTA's groups) and the per-qubit
// variant state in the group's shared memory, so that registers hold only
// adjacency and temporaries.
//
// Arithmetic (Sec. II-B1 and Sec. III of the paper, fp32):
//  * check-to-variable, eq. (h_update): 2 atanh(prod_k tanh(m_k/2)) with
//    sign (-1)^{s_i} prod_k sign(m_k).  Variable-to-check messages are
//    stored as sign(m) * delta, delta = 1 - tanh(|m|/2) in (0, 1]; the check
//    pass XORs sign bits and forms D = 1 - prod_k (1 - delta_k) with
//    a (+) b = a + b - ab (no relative accuracy is lost for small deltas,
//    i.e. confident messages), then |m_c->v| = 2 atanh(1 - D) =
//    ln(2/D - 1): one reciprocal, one fma and one logarithm per edge.  AdaGrad-BP
//    keeps Gallager's sign/phi form (see PhiForm) for its conditioning.
//  * variable-to-check, eqs. (lambda), (v_update), (mombp5): the message is
//    lambda_H(Q - own anticommuting message) = ln(C / A) with
//    C = 1 + e^{-Q_H} and A = (e^{-Q_a} + e^{-Q_b}) e^{m_c->v}, a, b the two
//    Paulis other than H.  All four exponentials share the shift
//    c0 = min(0, Q_X, Q_Y, Q_Z), so nothing overflows, and the stored value
//    delta = 1 - tanh(|lambda|/2) = 2 min(C, A) / (C + A) comes out of C
//    and A without forming lambda (one reciprocal per edge, no logarithm).
//  * message saturation: |m| <= msg_clip on both directions, i.e.
//    delta(m_v->c) >= 2 / (e^msg_clip + 1) and |m_c->v| <= msg_clip.
//  * units: every log-likelihood the kernel keeps (Pi, Q, S, the variant
//    state and the c->v messages) is in bits, i.e. the paper's natural-log
//    value times log2 e, so that ex2 and lg2 take and give them without a
//    scale factor.  The decisions are unchanged (a positive scale), the EWA
//    and momentum recursions are linear, AdaGrad's alpha and eps are scaled
//    by log2 e on the host, and the trace reports natural-log values.
//  * pairs: independent fp32 adds, multiplies and fmas of two edges (or two
//    sums) go through one packed f32x2 instruction (__fadd2_rn, __fmul2_rn,
//    __ffma2_rn), each lane rounded as the scalar operation.
//
// Specialisations: SPLIT (tables whose qubits have at most two X and two Z
// edges: the edge type is fixed by its position, so no per-edge Pauli
// selects) and FULL (split tables without padding, e.g. the toric codes: no
// zero/trash slot choice, no unused positions, no check-side clip).
//
// Bounds-checked build: with BPQ_DEBUG defined (decode_debug_*.cu compile
// these headers a second time, into namespace dk_debug), every CTA checks its
// launch's shared-memory layout against the dynamic shared memory it got,
// every thread checks the slot indices and table offsets of the nodes it
// loads, and every output write checks its index.  A failed check sets the
// device error word (work[1] = 5) and substitutes a safe index (the zero slot,
// or no write); a CTA whose layout does not fit returns before its first
// barrier.  Nothing traps.
#pragma once

#include <cuda_runtime.h>

#include "bpq_internal.h"
#include "decode_launch.h"

namespace bpq {
namespace dk {

// Error word value of a failed bounds check (BPQ_DEBUG builds).
constexpr uint32_t kBoundsError = 5u;

#ifdef BPQ_DEBUG
__device__ __forceinline__ uint32_t dynamic_smem_bytes() {
    uint32_t v;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
    return v;
}
// true when idx < limit; else records the failure in the error word
__device__ __forceinline__ bool bpq_in_bounds(size_t idx, size_t limit, uint32_t *err) {
    if (idx < limit) return true;
    atomicExch(err, kBoundsError);
    return false;
}
#define BPQ_IN_BOUNDS(idx, limit, err) ::bpq::dk::bpq_in_bounds((size_t)(idx), (size_t)(limit), (err))
#else
#define BPQ_IN_BOUNDS(idx, limit, err) true
#endif

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy accesses to shared memory before
// later async-proxy (TMA) accesses; with a CTA barrier after it, a bulk copy
// issued by one thread cannot be overtaken by other threads' earlier stores.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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
// The same, but always executed: used where the result only feeds a select,
// so that the compiler keeps the code straight-line instead of branching
// around the special-function unit.
__device__ __forceinline__ float ex2_always(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_always(float x) {
    float y;
    asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
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

// Messages on the check side are carried as delta = 1 - tanh(|m|/2) in
// (0, 1] (sign kept in the float's sign bit), so that eq. (h_update)
// becomes a product: with tanh(|w|/2) = prod_f (1 - delta_f), the
// complement D = 1 - prod_f (1 - delta_f) is accumulated with
// a (+) b = a + b - ab = 1 - (1-a)(1-b), which loses no relative accuracy
// when every delta is small (confident messages), and
// |w| = 2 atanh(1 - D) = ln((2 - D) / D).
__device__ __forceinline__ float oplus(float a, float b) { return fmaf(-a, b, a + b); }
// Two (+) at once with packed f32x2 instructions, each lane rounded as oplus.
__device__ __forceinline__ float2 oplus2(float2 a, float2 b) {
    return __ffma2_rn(make_float2(-a.x, -a.y), b, __fadd2_rn(a, b));
}

// |m_{c->v}| = log2((2 - D) / D) = log2(2/D - 1) in bits (see the unit note
// at the top), D in [0, 1]: the rcp error (2^-22 relative) gives an absolute
// error below 2^-21 in 2/D - 1 near D = 1 and a relative one for small D.
// D = 0 (only certain incoming messages, e.g. a degree-1 check) gives +inf,
// clipped by the caller.
__device__ __forceinline__ float c2v_magnitude(float D) { return lg2(fmaf(2.0f, rcp(D), -1.0f)); }

// AdaGrad-BP keeps Gallager's form instead: v->c messages stored as
// sign * phi(|m|), phi(x) = -ln tanh(x/2) (its own inverse), summed by the
// check pass, 2 atanh(prod tanh(m/2)) = sign * phi(sum phi(|m|)).  phi keeps
// relative accuracy at both ends (small and large |m|), which AdaGrad's
// scale-invariant step g'/(sqrt(G)+eps) needs; delta = 1 - tanh(|m|/2) holds
// only absolute accuracy for uncertain (small) messages.
template <int VARIANT>
struct PhiForm {
    static constexpr bool value = VARIANT == BPQ_ADAGRAD;
};

// Check-to-variable magnitude w = phi(S) = ln(1 + 2 / (e^S - 1)), S >= 0,
// returned in bits (w log2 e), needed to an absolute accuracy.  e^S - 1
// keeps its relative accuracy: below S = 1/4 from its Taylor series to
// S^6/720 (truncation < 5e-8 relative), above from 2^(S log2 e) - 1 (the ex2
// error is amplified at most e^S/(e^S-1) < 4.6 times).  Then
// w log2 e = lg2(1 + 2/(e^S-1)); S = 0 gives inf (clipped by the caller),
// S -> inf gives 0.
__device__ __forceinline__ float phi_check(float S) {
    // (for S > 88, 2^(S log2 e) overflows to inf, 2/inf = 0 and w = 0)
    const float poly =
        S * fmaf(S, fmaf(S, fmaf(S, fmaf(S, fmaf(S, 1.0f / 720.0f, 1.0f / 120.0f), 1.0f / 24.0f), 1.0f / 6.0f), 0.5f), 1.0f);
    const float big = ex2_always(S * kLog2e) - 1.0f;
    const float em1 = S < 0.25f ? poly : big;
    return lg2(fmaf(2.0f, rcp(em1), 1.0f));
}

// phi(|lambda|) = ln(1 + r), r = 2 min(C,A) / |C - A|, needed to a relative
// accuracy (small values are summed by the check pass): below r = 1/16 from
// the series r - r^2/2 + r^3/3 - r^4/4 + r^5/5 (truncation < 2e-7 relative),
// above from ln2 * lg2(1 + r).
__device__ __forceinline__ float log1p_rel(float r) {
    const float poly = r * fmaf(r, fmaf(r, fmaf(r, fmaf(r, 0.2f, -0.25f), 1.0f / 3.0f), -0.5f), 1.0f);
    const float big = kLn2 * lg2_always(1.0f + r);
    return r < 0.0625f ? poly : big;
}

// Number of per-qubit state arrays a variant keeps in shared memory
// (decode_state_arrays).
template <int VARIANT>
struct StateArrays {
    static constexpr int n = decode_state_arrays(VARIANT);
};

// Sum of the c->v messages from checks that anticommute with X, Y, Z
// (S_W of eq. (p_update)) in the generic layout: position n of the qubit
// holds an edge with Pauli (vp >> 2n) & 3 (0 = unused slot).
__device__ __forceinline__ void anticommuting_sums(uint32_t vp, const float (&w)[4], float &SX, float &SY,
                                                   float &SZ) {
    SX = SY = SZ = 0.f;
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        const uint32_t p = (vp >> (2 * n)) & 3u;
        SX += (p != 0u && p != 1u) ? w[n] : 0.f;
        SY += (p != 0u && p != 2u) ? w[n] : 0.f;
        SZ += (p != 0u && p != 3u) ? w[n] : 0.f;
    }
}

// Bytes 0..3: 1 where the decision d anticommutes with the qubit's edge at
// position n (pp holds the edge Paulis one per byte; unused bytes are 0).
__device__ __forceinline__ uint32_t anti_bytes(uint32_t d, uint32_t pp) {
    const uint32_t x = (d * 0x01010101u) ^ pp;                       // 0 where d == p
    const uint32_t ne = (x | (x >> 1)) & 0x01010101u;                // 1 where d != p
    const uint32_t nz = (pp | (pp >> 1)) & 0x01010101u;              // 1 where p != I
    return d ? (ne & nz) : 0u;
}

// The same for the split layout, where positions 0, 1 hold X edges and 2, 3
// Z edges: X anticommutes with Y, Z (d >= 2) and Z with X, Y (d in {1, 2}).
// Bit 0: the X positions' bit; bit 1: the Z positions'.
__device__ __forceinline__ uint32_t anti_bits_split(uint32_t d) {
    return (d >= 2u ? 1u : 0u) | (d - 1u < 2u ? 2u : 0u);
}

// The scalars the iteration loop reads, copied once per shot into locals.
// The one-code kernel reads its DecodeArgs from the constant bank; the
// batched kernel keeps the descriptor in shared memory, where every slot
// store could alias it and force a reload on each use.
struct ShotParams {
    int N, M, Np, max_iter, ada_from1;
    float clip2, vclip, alpha, gamma, eps;  // vclip: delta_clip, or phi_clip in the phi form
};

template <bool PHI>
__device__ __forceinline__ ShotParams shot_params(const DecodeArgs &a, float alpha) {
    ShotParams p;
    p.N = a.N;
    p.M = a.M;
    p.Np = a.n_pad;
    p.max_iter = a.max_iter;
    p.ada_from1 = a.ada_from1;
    p.clip2 = a.clip2;
    p.vclip = PHI ? a.phi_clip : a.delta_clip;
    p.alpha = alpha;
    p.gamma = a.gamma;
    p.eps = a.eps;
    return p;
}

// Variable-to-check messages of one qubit (position n of the layout), from
// its posterior Q and the incoming check-to-variable messages win: stored
// as sign * delta(|lambda|) (sign * phi(|lambda|) with PHI), the least
// significant bit replaced by whether this iteration's decision
// anticommutes with the edge (byte n of ab in the generic layout; bit 0 of
// ab for positions 0, 1 and bit 1 for positions 2, 3 in the split one),
// which the next check pass reads for the syndrome test.  Generic layout: slots 4j .. 4j+3, one float4 store.
// Split layout: slots n * n_pad + j; unused positions are written (as 0)
// only at t = 0, when ALL is set.  FULL: every position is used.
template <bool TRACE, bool SPLIT, bool PHI, bool ALL, bool FULL>
__device__ __forceinline__ void emit_v2c(const DecodeArgs &a, const ShotParams &sp, float *slots, int j, int t,
                                         int shot, uint32_t vp, float QX, float QY, float QZ, const float (&win)[4],
                                         uint32_t ab) {
    const float c0 = fminf(0.f, fminf(QX, fminf(QY, QZ)));
    const float e0 = ex2(c0);
    const float eX = ex2(c0 - QX), eY = ex2(c0 - QY), eZ = ex2(c0 - QZ);
    // C = 1 + e^{-Q_H} and the two anticommuting terms, for H = X, Y, Z
    float CX, CY, CZ, AX, AY, AZ;
    if (FULL) {
        // (C_X, A_X) and (C_Z, A_Z) in two f32x2 sums; C_Y, A_Y are unused in
        // the split layout (in the other kernels the pairs cost registers)
        const float2 cax = __fadd2_rn(make_float2(e0, eY), make_float2(eX, eZ));
        const float2 caz = __fadd2_rn(make_float2(e0, eX), make_float2(eZ, eY));
        CX = cax.x;
        AX = cax.y;
        CZ = caz.x;
        AZ = caz.y;
        CY = AY = 0.f;
    } else {
        CX = e0 + eX;
        CY = e0 + eY;
        CZ = e0 + eZ;
        AX = eY + eZ;
        AY = eX + eZ;
        AZ = eX + eY;
    }
    float C[4], Ab[4], x[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        const uint32_t p = (vp >> (2 * n)) & 3u;
        if (SPLIT) {
            C[n] = n < 2 ? CX : CZ;
            Ab[n] = n < 2 ? AX : AZ;
        } else {
            C[n] = p == 1u ? CX : p == 2u ? CY : CZ;
            Ab[n] = p == 1u ? AX : p == 2u ? AY : AZ;
        }
        x[n] = ex2(win[n]);
    }
    // lambda = ln(C / A), A = Ab e^{m_in}; delta = 1 - tanh(|lambda|/2) =
    // 2 min(C, A) / (C + A), at least delta_clip; or phi(|lambda|) =
    // log1p(2 min(C, A) / |C - A|), at least phi_clip (|lambda| <= msg_clip).
    // Edges n, n+1 share packed two-lane fp32 instructions (f32x2): each lane
    // rounds as the scalar operation would.
    float A[4], dl[4];
    uint32_t neg[4];  // sign bit of C - A: set iff A > C, i.e. lambda < 0 (C = A gives +0)
#pragma unroll
    for (int n = 0; n < 4; n += 2) {
        const float2 A2 = __fmul2_rn(make_float2(Ab[n], Ab[n + 1]), make_float2(x[n], x[n + 1]));
        A[n] = A2.x;
        A[n + 1] = A2.y;
        const float2 cma = __fadd2_rn(make_float2(C[n], C[n + 1]), make_float2(-A2.x, -A2.y));
        neg[n] = __float_as_uint(cma.x) & 0x80000000u;
        neg[n + 1] = __float_as_uint(cma.y) & 0x80000000u;
        if (PHI) {
#pragma unroll
            for (int h = n; h < n + 2; ++h) {
                const float mx = fmaxf(C[h], A[h]), mn = fminf(C[h], A[h]);
                dl[h] = fmaxf(log1p_rel(2.0f * mn * rcp(mx - mn)), sp.vclip);
            }
        } else {
            const float2 s2 = __fadd2_rn(make_float2(C[n], C[n + 1]), A2);
            const float m0 = fminf(C[n], A2.x), m1 = fminf(C[n + 1], A2.y);
            const float2 d2 = __fmul2_rn(__fadd2_rn(make_float2(m0, m1), make_float2(m0, m1)),
                                         make_float2(rcp(s2.x), rcp(s2.y)));
            dl[n] = fmaxf(d2.x, sp.vclip);
            dl[n + 1] = fmaxf(d2.y, sp.vclip);
        }
    }
    float out[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        const uint32_t p = (vp >> (2 * n)) & 3u;
        const uint32_t abit = SPLIT ? (n < 2 ? ab & 1u : ab >> 1) : (ab >> (8 * n)) & 1u;
        const uint32_t bits = (__float_as_uint(dl[n]) & ~1u) | abit | neg[n];
        out[n] = (FULL || p) ? __uint_as_float(bits) : 0.f;
        if (TRACE && a.tr_v2c && p) {
            const float lam = fminf(fmaxf(kLn2 * (lg2(C[n]) - lg2(A[n])), -a.clip), a.clip);
            const int s = SPLIT ? n * sp.Np + j : 4 * j + n;
            a.tr_v2c[((size_t)shot * (sp.max_iter + 1) + t) * a.E + a.var_canon[s]] = lam;
        }
    }
    if (SPLIT) {
#pragma unroll
        for (int n = 0; n < 4; ++n)
            if (ALL || FULL || ((vp >> (2 * n)) & 3u)) slots[n * sp.Np + j] = out[n];
    } else {
        *reinterpret_cast<float4 *>(slots + 4 * j) = make_float4(out[0], out[1], out[2], out[3]);
    }
}

// The posterior rules of Momentum-BP and AdaGrad-BP, written with explicit
// round-to-nearest intrinsics so that every kernel that uses them (one shot
// per thread, or two shots per thread in f32x2 lanes) rounds alike.
//  eqs. (mombp1)-(mombp3): g = gamma g_prev + (1 - gamma)(Q_prev - Pi - S),
//                           Q = Q_prev - alpha g
__device__ __forceinline__ float momentum_g(const ShotParams &sp, float qp, float Pi, float S, float g_prev) {
    const float grad = __fsub_rn(__fsub_rn(qp, Pi), S);
    return __fmaf_rn(sp.gamma, g_prev, __fmul_rn(1.f - sp.gamma, grad));
}
__device__ __forceinline__ float momentum_q(const ShotParams &sp, float qp, float g) {
    return __fmaf_rn(-sp.alpha, g, qp);
}
//  eq. (boost): g' = Q_prev - Pi - S, G += g'^2 (from t = 2, or from t = 1),
//               Q = Q_prev - alpha g' / (sqrt(G) + eps)
__device__ __forceinline__ float adagrad_gp(float qp, float Pi, float S) { return __fsub_rn(__fsub_rn(qp, Pi), S); }
__device__ __forceinline__ float adagrad_G(float G, float gp, bool accumulate) {
    return accumulate ? __fmaf_rn(gp, gp, G) : G;
}
__device__ __forceinline__ float adagrad_q(const ShotParams &sp, float qp, float gp, float G) {
    return __fmaf_rn(-__fmul_rn(sp.alpha, gp), rcp(__fadd_rn(sqrt_approx(G), sp.eps)), qp);
}

// Per-thread adjacency of the owned checks and qubits of one code:
// cs: the four message slots of each owned check (padding -> zero slot);
// info: check Paulis (bits 0-7) | qubit Paulis (bits 8-15); pp: qubit
// Paulis one per byte.
template <int NPT>
struct ThreadAdj {
    uint32_t cs_lo[NPT], cs_hi[NPT], info[NPT], pp[NPT];
};

template <int NPT>
__device__ __forceinline__ void load_adjacency(const DecodeArgs &a, const uint8_t *tab, int T, int tg, int npt,
                                               ThreadAdj<NPT> &adj) {
    const uint32_t kZero = 4u * (uint32_t)a.n_pad;
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        adj.cs_lo[k] = adj.cs_hi[k] = kZero | (kZero << 16);
        adj.info[k] = 0u;
        adj.pp[k] = 0u;
        const int i = k * T + tg;
        if (k < npt && i < a.M && BPQ_IN_BOUNDS(8 * i + 7, a.table_bytes, a.work + 1) &&
            BPQ_IN_BOUNDS(a.off_chk_pauli + i, a.table_bytes, a.work + 1)) {
            const uint2 s = *reinterpret_cast<const uint2 *>(tab + 8 * i);
            uint32_t s0 = s.x & 0xFFFFu, s1 = s.x >> 16, s2 = s.y & 0xFFFFu, s3 = s.y >> 16;
#ifdef BPQ_DEBUG
            // a slot index is an edge slot (< 4 n_pad) or no slot
            uint32_t *sv[4] = {&s0, &s1, &s2, &s3};
            for (int n = 0; n < 4; ++n)
                if (*sv[n] != kNoSlot && !BPQ_IN_BOUNDS(*sv[n], kZero, a.work + 1)) *sv[n] = kNoSlot;
#endif
            adj.cs_lo[k] = (s0 == kNoSlot ? kZero : s0) | ((s1 == kNoSlot ? kZero : s1) << 16);
            adj.cs_hi[k] = (s2 == kNoSlot ? kZero : s2) | ((s3 == kNoSlot ? kZero : s3) << 16);
            adj.info[k] = tab[a.off_chk_pauli + i];
        }
        if (k < npt && i < a.N && BPQ_IN_BOUNDS(a.off_var_pauli + i, a.table_bytes, a.work + 1)) {
            const uint32_t vp = tab[a.off_var_pauli + i];
            adj.info[k] |= vp << 8;
            adj.pp[k] = (vp & 3u) | (((vp >> 2) & 3u) << 8) | (((vp >> 4) & 3u) << 16) | (((vp >> 6) & 3u) << 24);
        }
    }
}

// Prior LLRs Pi_{v_j,W} = ln(p^I / p^W) of a code into shared memory
// ([3][n_pad], computed by all threads of the CTA).
__device__ __forceinline__ void load_prior(const DecodeArgs &a, float *PiS) {
    const int Np = a.n_pad;
    for (int j = threadIdx.x; j < a.N; j += blockDim.x) {
        const float px = a.prior[3 * j], py = a.prior[3 * j + 1], pz = a.prior[3 * j + 2];
        const float pI = 1.0f - px - py - pz;
        PiS[j] = log2f(pI / px);
        PiS[Np + j] = log2f(pI / py);
        PiS[2 * Np + j] = log2f(pI / pz);
    }
}

// Shared-memory regions of shot group `group` of a code laid out from `base`
// (base = the staged table): table | Pi [3][Np] | groups.
struct GroupMem {
    float *PiS, *slots, *state;
};

__device__ __forceinline__ GroupMem group_mem(const DecodeArgs &a, uint8_t *base, int group) {
    GroupMem m;
    m.PiS = reinterpret_cast<float *>(base + a.table_bytes);
    uint8_t *g = base + a.table_bytes + (size_t)12 * a.n_pad + (size_t)group * a.group_bytes;
    m.slots = reinterpret_cast<float *>(g);
    m.state = m.slots + a.slots_floats;
    return m;
}

// Decode one shot with a group of G warps (thread tg of 32G): eq. (init),
// then iterations of the check pass and the variable pass until the hard
// decision satisfies the syndrome or max_iter is reached; writes the shot's
// outputs.  npt <= NPT is the number of nodes each thread owns.  FULL
// (split layout only): every check has four edges and every qubit two X and
// two Z edges, so no edge is padding.  STAGED: a.syn, a.est, a.conv and
// a.iters may point into shared memory (the serving kernel stages each
// request's syndrome and outputs there), so the syndrome words are read with
// a generic load instead of the read-only global path.
template <int VARIANT, int NPT, bool TRACE, bool SPLIT, bool FULL, bool STAGED = false>
__device__ __forceinline__ int decode_shot(const DecodeArgs &a, const ThreadAdj<NPT> &adj, const GroupMem &m,
                                           int npt, int T, int tg, int G, int bar_id, int shot, float alpha) {
    const ShotParams sp = shot_params<PhiForm<VARIANT>::value>(a, alpha);
    const int N = sp.N, M = sp.M, Np = sp.Np;
    const uint32_t kZero = 4u * (uint32_t)Np, kTrash = kZero + 1u;
    float *slots = m.slots, *state = m.state;
    const float *PiS = m.PiS;

    // syndrome bits of the owned checks (bit k <-> check k*T + tg)
    uint32_t sbits = 0;
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int i = k * T + tg;
        if (k < npt && i < M) {
            const uint32_t *src = a.syn + (size_t)shot * a.W + (i >> 5);
            const uint32_t w = STAGED ? *reinterpret_cast<const volatile uint32_t *>(src) : __ldg(src);
            sbits |= ((w >> (i & 31)) & 1u) << k;
        }
    }

    // eq. (init): lambda(Pi^(0)), i.e. the variable pass with Q = Pi^(0)
    // and no incoming messages; Q^(0) = Pi^(0), g^(0) = G^(0) = 0; EWAInit
    // starts from Pi^(1) = Pi^(0) and keeps alpha Pi^(0)
    uint32_t dk[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        dk[k] = 0;
        const int j = k * T + tg;
        if (k < npt && j < N) {
            const float PX = PiS[j], PY = PiS[Np + j], PZ = PiS[2 * Np + j];
            if (StateArrays<VARIANT>::n >= 3) {
                state[j] = PX;
                state[Np + j] = PY;
                state[2 * Np + j] = PZ;
            }
            if (VARIANT == BPQ_EWAINIT) {
                state[3 * Np + j] = alpha * PX;
                state[4 * Np + j] = alpha * PY;
                state[5 * Np + j] = alpha * PZ;
            } else if (StateArrays<VARIANT>::n == 6) {
                state[3 * Np + j] = 0.f;
                state[4 * Np + j] = 0.f;
                state[5 * Np + j] = 0.f;
            }
            const float z4[4] = {0.f, 0.f, 0.f, 0.f};
            emit_v2c<TRACE, SPLIT, PhiForm<VARIANT>::value, true, FULL>(a, sp, slots, j, 0, shot, adj.info[k] >> 8,
                                                                        PX, PY, PZ, z4, 0u);
        }
    }
    group_sync(G, bar_id);

    int conv = 0, iters = 0;
    for (int t = 1;; ++t) {
        const bool do_check = t > 1 && (!TRACE || t > sp.max_iter);
        const bool do_msgs = t <= sp.max_iter;
        uint32_t mismatch = 0;

        // ---- check pass: syndrome test of the previous decision, then eq. (h_update) ----
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int i = k * T + tg;
            if (k < npt && i < M) {
                const uint32_t sl[4] = {adj.cs_lo[k] & 0xFFFFu, adj.cs_lo[k] >> 16, adj.cs_hi[k] & 0xFFFFu,
                                        adj.cs_hi[k] >> 16};
                const uint32_t sb = (sbits >> k) & 1u;
                uint32_t u[4];
#pragma unroll
                for (int n = 0; n < 4; ++n) u[n] = __float_as_uint(slots[sl[n]]);
                // bit 31: the product of the incoming signs; bit 0: the parity
                // of the previous decision on this check's edges
                const uint32_t ux = u[0] ^ u[1] ^ u[2] ^ u[3];
                if (do_check) mismatch |= (ux ^ sb) & 1u;
                if (do_msgs) {
                    float mag[4];
#pragma unroll
                    for (int n = 0; n < 4; ++n) mag[n] = __uint_as_float(u[n] & 0x7FFFFFFEu);
                    // (-1)^{s_i} times the product of the incoming signs
                    const uint32_t sgn = (ux ^ (sb << 31)) & 0x80000000u;
                    float ext[4];
                    if (PhiForm<VARIANT>::value) {
                        // extrinsic sums of phi(|m|) over the other three edges
                        const float e01 = mag[0] + mag[1], e23 = mag[2] + mag[3];
                        ext[0] = mag[1] + e23;
                        ext[1] = mag[0] + e23;
                        ext[2] = e01 + mag[3];
                        ext[3] = e01 + mag[2];
                    } else {
                        // extrinsic D of each edge: the (+) of the other three deltas,
                        // two (+) per packed f32x2 instruction pair (each lane equals
                        // the scalar oplus; a (+) b and b (+) a round alike)
                        const float2 d = oplus2(make_float2(mag[0], mag[2]), make_float2(mag[1], mag[3]));
                        const float2 e01 = oplus2(make_float2(mag[1], mag[0]), make_float2(d.y, d.y));
                        const float2 e23 = oplus2(make_float2(mag[3], mag[2]), make_float2(d.x, d.x));
                        ext[0] = e01.x;
                        ext[1] = e01.y;
                        ext[2] = e23.x;
                        ext[3] = e23.y;
                    }
#pragma unroll
                    for (int n = 0; n < 4; ++n) {
                        // every incoming delta is at least delta_clip, so without
                        // padding (FULL) the delta-form magnitude is at most
                        // msg_clip already (up to rounding); padded edges read
                        // delta = 0 and need the clip
                        const float w0 = PhiForm<VARIANT>::value ? phi_check(ext[n]) : c2v_magnitude(ext[n]);
                        const float wv = FULL && !PhiForm<VARIANT>::value ? w0 : fminf(w0, sp.clip2);
                        const float mm = __uint_as_float(__float_as_uint(wv) ^ ((sgn ^ u[n]) & 0x80000000u));
                        slots[FULL ? sl[n] : sl[n] == kZero ? kTrash : sl[n]] = mm;
                        if (TRACE && a.tr_c2v && sl[n] != kZero)
                            a.tr_c2v[((size_t)shot * sp.max_iter + (t - 1)) * a.E + a.chk_ptr[i] + n] = kLn2 * mm;
                    }
                }
            }
        }
        const int any = group_any(G, bar_id, (int)mismatch);
        if (do_check && !any) {
            conv = 1;
            iters = t - 1;
            break;
        }
        if (!do_msgs) {
            conv = 0;
            iters = sp.max_iter;
            break;
        }

        // ---- variable pass: posterior of the variant, decision, eq. (v_update)/(mombp5) ----
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int j = k * T + tg;
            if (k < npt && j < N) {
                const uint32_t vp = adj.info[k] >> 8;
                float win[4], S[3];
                if (SPLIT) {
                    // positions 0, 1: X-type edges (anticommute with Z and Y);
                    // 2, 3: Z-type edges (with X and Y); unused slots hold 0
#pragma unroll
                    for (int n = 0; n < 4; ++n) win[n] = slots[n * Np + j];
                    const float2 s20 = __fadd2_rn(make_float2(win[0], win[2]), make_float2(win[1], win[3]));
                    S[2] = s20.x;
                    S[0] = s20.y;
                    S[1] = S[0] + S[2];
                } else {
                    const float4 w4 = *reinterpret_cast<const float4 *>(slots + 4 * j);
                    win[0] = w4.x;
                    win[1] = w4.y;
                    win[2] = w4.z;
                    win[3] = w4.w;
                    anticommuting_sums(vp, win, S[0], S[1], S[2]);
                }
                const float Pi[3] = {PiS[j], PiS[Np + j], PiS[2 * Np + j]};
                float Q[3];
                if (VARIANT == BPQ_EWAINIT) {
                    // eq. (EWAInit): the state holds Pi^(t) (Pi^(0) at t = 1), so
                    // Q^(t) = Pi^(t) + S and Pi^(t+1) = alpha Pi^(0) + (1-alpha) Q^(t);
                    // Paulis X and Y share one f32x2 pair
                    const float oma = 1.f - alpha;
                    const float2 q01 = __fadd2_rn(make_float2(state[j], state[Np + j]), make_float2(S[0], S[1]));
                    const float2 n01 = __ffma2_rn(make_float2(oma, oma), q01,
                                                  make_float2(state[3 * Np + j], state[4 * Np + j]));
                    Q[0] = q01.x;
                    Q[1] = q01.y;
                    Q[2] = state[2 * Np + j] + S[2];
                    state[j] = n01.x;
                    state[Np + j] = n01.y;
                    state[2 * Np + j] = fmaf(oma, Q[2], state[5 * Np + j]);
                } else {
#pragma unroll
                    for (int w = 0; w < 3; ++w) {
                        if (VARIANT == BPQ_PLAIN) {
                            Q[w] = Pi[w] + S[w];  // eq. (p_update)
                        } else if (VARIANT == BPQ_MOMENTUM) {
                            // eqs. (mombp1), (mombp2) with the gradient of (mombp3)
                            const float qp = state[w * Np + j];
                            const float g = momentum_g(sp, qp, Pi[w], S[w], state[(3 + w) * Np + j]);
                            Q[w] = momentum_q(sp, qp, g);
                            state[w * Np + j] = Q[w];
                            state[(3 + w) * Np + j] = g;
                        } else {
                            // eq. (boost) from t = 2; G accumulates g'^2
                            const float qp = state[w * Np + j];
                            const float gp = adagrad_gp(qp, Pi[w], S[w]);
                            const float Gs = adagrad_G(state[(3 + w) * Np + j], gp, t >= 2 || sp.ada_from1);
                            Q[w] = t == 1 ? Pi[w] + S[w] : adagrad_q(sp, qp, gp, Gs);
                            state[w * Np + j] = Q[w];
                            state[(3 + w) * Np + j] = Gs;
                        }
                    }
                }
                // hard decision: I if all Q_W > 0, else the first minimum of X, Y, Z
                // (the minimum is shared with emit_v2c's c0)
                const float mq = fminf(Q[0], fminf(Q[1], Q[2]));
                const uint32_t d = mq > 0.f ? 0u : Q[0] == mq ? 1u : Q[1] == mq ? 2u : 3u;
                dk[k] = d;
                // per-edge <E^_j, H_ij> for the next syndrome test (carried in the
                // messages' least significant bits)
                const uint32_t ab = SPLIT ? anti_bits_split(d) : anti_bytes(d, adj.pp[k]);
                if (TRACE) {
                    const size_t o = (size_t)shot * sp.max_iter + (t - 1);
                    if (a.tr_Q) {
                        a.tr_Q[(o * N + j) * 3 + 0] = kLn2 * Q[0];
                        a.tr_Q[(o * N + j) * 3 + 1] = kLn2 * Q[1];
                        a.tr_Q[(o * N + j) * 3 + 2] = kLn2 * Q[2];
                    }
                    if (a.tr_dec) a.tr_dec[o * N + j] = (uint8_t)d;
                }
                emit_v2c<TRACE, SPLIT, PhiForm<VARIANT>::value, false, FULL>(a, sp, slots, j, t, shot, vp, Q[0], Q[1],
                                                                             Q[2], win, ab);
            }
        }
        group_sync(G, bar_id);
    }

    // ---- outputs ----
    if (!TRACE || a.est) {
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int j = k * T + tg;
            if (k < npt && j < N && BPQ_IN_BOUNDS((size_t)shot * N + j, (size_t)a.B * N, a.work + 1))
                a.est[(size_t)shot * N + j] = (uint8_t)dk[k];
        }
    }
    if (tg == 0 && (!TRACE || a.conv) && BPQ_IN_BOUNDS(shot, a.B, a.work + 1)) {
        a.conv[shot] = (uint8_t)conv;
        a.iters[shot] = (uint8_t)iters;
    }
    return conv;
}

// One code per launch: a persistent grid; every shot group takes shots from
// the global queue until the batch is exhausted.
template <int VARIANT, int NPT, bool TRACE, bool SPLIT, bool FULL = false>
__global__ void __launch_bounds__(NPT <= 2 ? 1024 : 512, 1) decode_kernel(const DecodeArgs a) {
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
    const GroupMem m = group_mem(a, tab, group);
#ifdef BPQ_DEBUG
    // the launch's layout fits the dynamic shared memory (uniform across the
    // CTA, so an early return happens before any barrier)
    {
        const size_t need = kSmemHeader + (size_t)a.table_bytes + (size_t)12 * a.n_pad +
                            (size_t)(blockDim.x / T) * a.group_bytes;
        const bool ok = need <= dynamic_smem_bytes() && a.n_pad >= a.N && a.slots_floats >= 4u * a.n_pad + 2u &&
                        a.group_bytes >= 4u * (a.slots_floats + (uint32_t)StateArrays<VARIANT>::n * a.n_pad) &&
                        (a.off_var_pauli + (uint32_t)a.N <= a.table_bytes);
        if (!ok) {
            if (tid == 0) atomicExch(a.work + 1, kBoundsError);
            return;
        }
    }
#endif

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
    load_prior(a, m.PiS);
    if (tg == 0) m.slots[4 * a.n_pad] = 0.f;  // the zero slot
    const bool staged = mbar_wait_bounded(mbar, 0, 1u << 22);
    if (__syncthreads_or(!staged)) {
        if (tid == 0) atomicExch(a.work + 1, 1u);
        mbar_wait_bounded(mbar, 0, 1u << 22);  // let an in-flight copy land before exiting
        return;
    }

    ThreadAdj<NPT> adj;
    load_adjacency<NPT>(a, tab, T, tg, NPT, adj);

    for (;;) {
        if (tg == 0) grp_shot[group] = (int)atomicAdd(a.work, 1u);
        group_sync(G, bar_id);
        const int shot = grp_shot[group];
        if (shot >= a.B) break;
        if (VARIANT == BPQ_AEWA) {
            // Appendix C: EWAInit-BP with alpha = 1.0, 0.9, ..., 0.0 in turn until
            // a run converges (the outputs are those of the last run); alpha_k =
            // (10 - k) / 10 by IEEE division, the float nearest to it
            for (int k = 0; k <= 10; ++k)
                if (decode_shot<BPQ_EWAINIT, NPT, TRACE, SPLIT, FULL>(a, adj, m, NPT, T, tg, G, bar_id, shot,
                                                                    (float)(10 - k) / 10.0f))
                    break;
        } else {
            decode_shot<VARIANT, NPT, TRACE, SPLIT, FULL>(a, adj, m, NPT, T, tg, G, bar_id, shot, a.alpha);
        }
    }
}

// The shots of the current item taken by one shot group of the batched
// kernel: the group takes the item's shots one by one from the item's
// counter until none are left.  NPT, SPLIT and FULL are the item's nodes
// per thread and table layout, so each item runs the decode_shot
// specialisation that the one-code kernel runs for it.
template <int VARIANT, int NPT, bool SPLIT, bool FULL>
__device__ __forceinline__ void batch_item_shots(const DecodeArgs &a, const ThreadAdj<2> &adj2, const GroupMem &m,
                                                 uint32_t *next, int *slot, int T, int tg, int G, int bar_id) {
    ThreadAdj<NPT> adj;
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        adj.cs_lo[k] = adj2.cs_lo[k];
        adj.cs_hi[k] = adj2.cs_hi[k];
        adj.info[k] = adj2.info[k];
        adj.pp[k] = adj2.pp[k];
    }
    for (;;) {
        if (tg == 0) *slot = (int)atomicAdd(next, 1u);
        group_sync(G, bar_id);
        const int shot = *slot;
        if (shot >= a.B) break;
        decode_shot<VARIANT, NPT, false, SPLIT, FULL>(a, adj, m, NPT, T, tg, G, bar_id, shot, a.alpha);
    }
}

// Many codes in one launch.  A CTA of kBatchThreads works on one item (a
// code's batch) at a time: it splits into that code's shot groups (T_g
// threads each, one or two nodes per thread), which take the item's shots
// until none are left; only then does the CTA synchronise, pick the next
// item with shots left (scanning from its starting item) and re-stage that
// code's adjacency (bulk TMA) and prior.  Every shot is decoded by the
// decode_shot specialisation of decode_kernel for its code (nodes per
// thread and layout), so results equal those of decode_kernel bit for bit.
// GENERIC: items may use the generic table layout; without it every item
// has the split layout, and the kernel holds only the split paths.
template <int VARIANT, bool GENERIC>
__global__ void __launch_bounds__(kBatchThreads, 1) decode_batch_kernel(const BatchArgs b) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);
    int *code_slot = reinterpret_cast<int *>(smem + 8);    // the item being decoded
    int *grp_shot = reinterpret_cast<int *>(smem + 16);    // [kMaxGroupsPerCta]
    DecodeArgs *desc = reinterpret_cast<DecodeArgs *>(smem + kSmemHeader);
    uint8_t *tab = smem + kSmemHeader + kDescBytes;
    const int tid = threadIdx.x;

    if (tid == 0) {
        mbar_init(mbar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    int cur = -1;
    int from = b.start[blockIdx.x < (unsigned)kMaxBatchCtas ? blockIdx.x : 0];
    uint32_t phase = 0;
    ThreadAdj<2> adj;
    for (;;) {
        if (tid == 0) {
            int pick = -1;
            for (int k = 0; k < b.ncodes && pick < 0; ++k) {
                const int g = (from + k) % b.ncodes;
                const uint32_t taken = *reinterpret_cast<volatile const uint32_t *>(b.work + 2 + g);
                if (taken < (uint32_t)b.codes[g].B) pick = g;
            }
            *code_slot = pick;
        }
        __syncthreads();
        const int g = *code_slot;
        if (g < 0) break;
        from = g;
        if (g != cur) {
            // switch item: descriptor, adjacency (bulk TMA), prior, zero
            // slots.  The new table may cover the previous item's prior,
            // message slots and state, written with ordinary stores: every
            // thread fences them against the async proxy before the barrier
            // that precedes the copy.
            const uint32_t *src = reinterpret_cast<const uint32_t *>(b.codes + g);
            for (int w = tid; w < (int)(sizeof(DecodeArgs) / 4); w += blockDim.x)
                reinterpret_cast<uint32_t *>(desc)[w] = src[w];
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
                mbar_expect_tx(mbar, desc->table_bytes);
                bulk_g2s(tab, desc->table, desc->table_bytes, mbar);
            }
            load_prior(*desc, reinterpret_cast<float *>(tab + desc->table_bytes));
            const bool staged = mbar_wait_bounded(mbar, phase, 1u << 22);
            phase ^= 1u;
            if (__syncthreads_or(!staged)) {
                if (tid == 0) atomicExch(b.work + 1, 1u);
                mbar_wait_bounded(mbar, phase ^ 1u, 1u << 22);
                return;
            }
            const int T = desc->G * 32;
            const int group = tid / T;
            if (group < desc->groups_per_cta && tid - group * T == 0) {
                const GroupMem m = group_mem(*desc, tab, group);
                m.slots[4 * desc->n_pad] = 0.f;
            }
            load_adjacency<2>(*desc, tab, T, tid - group * T, desc->npt, adj);
            __syncthreads();
            cur = g;
        }
        const DecodeArgs &a = *desc;
        const int G = a.G, T = G * 32;
        const int group = tid / T, tg = tid - group * T;
        if (group < a.groups_per_cta) {
            const GroupMem m = group_mem(a, tab, group);
            const int bar_id = 1 + group;
            uint32_t *next = b.work + 2 + g;
            int *slot = grp_shot + group;
            const bool one = a.npt == 1;
            if (a.split == 2) {
                if (one)
                    batch_item_shots<VARIANT, 1, true, true>(a, adj, m, next, slot, T, tg, G, bar_id);
                else
                    batch_item_shots<VARIANT, 2, true, true>(a, adj, m, next, slot, T, tg, G, bar_id);
            } else if (a.split == 1 || !GENERIC) {
                if (one)
                    batch_item_shots<VARIANT, 1, true, false>(a, adj, m, next, slot, T, tg, G, bar_id);
                else
                    batch_item_shots<VARIANT, 2, true, false>(a, adj, m, next, slot, T, tg, G, bar_id);
            } else if (GENERIC) {
                if (one)
                    batch_item_shots<VARIANT, 1, false, false>(a, adj, m, next, slot, T, tg, G, bar_id);
                else
                    batch_item_shots<VARIANT, 2, false, false>(a, adj, m, next, slot, T, tg, G, bar_id);
            }
        }
        __syncthreads();
    }
}

}  // namespace dk

// AEWA-BP: single-code, non-trace kernels only.
#define BPQ_DEFINE_PICK_AEWA(NAME)                                                       \
    DecodeKernelFn NAME(int npt, bool trace, bool split) {                               \
        if (trace) return nullptr;                                                       \
        switch (npt) {                                                                   \
            case 1: return split ? dk::decode_kernel<BPQ_AEWA, 1, false, true>             \
                               : dk::decode_kernel<BPQ_AEWA, 1, false, false>;           \
            case 2: return split ? dk::decode_kernel<BPQ_AEWA, 2, false, true>             \
                               : dk::decode_kernel<BPQ_AEWA, 2, false, false>;           \
            case 3: return split ? dk::decode_kernel<BPQ_AEWA, 3, false, true>             \
                               : dk::decode_kernel<BPQ_AEWA, 3, false, false>;           \
            case 4: return split ? dk::decode_kernel<BPQ_AEWA, 4, false, true>             \
                               : dk::decode_kernel<BPQ_AEWA, 4, false, false>;           \
        }                                                                                \
        return nullptr;                                                                  \
    }

// Instantiate the kernels of one variant and return the one for (NPT,
// trace, split layout).
#define BPQ_PICK_NPT(V, NPT, TR)                                                         \
    (split ? dk::decode_kernel<V, NPT, TR, true> : dk::decode_kernel<V, NPT, TR, false>)
#define BPQ_DEFINE_PICK(NAME, V)                                                         \
    DecodeKernelFn NAME(int npt, bool trace, bool split) {                               \
        switch (npt * 2 + (trace ? 1 : 0)) {                                             \
            case 2: return BPQ_PICK_NPT(V, 1, false);                                    \
            case 3: return BPQ_PICK_NPT(V, 1, true);                                     \
            case 4: return BPQ_PICK_NPT(V, 2, false);                                    \
            case 5: return BPQ_PICK_NPT(V, 2, true);                                     \
            case 6: return BPQ_PICK_NPT(V, 3, false);                                    \
            case 7: return BPQ_PICK_NPT(V, 3, true);                                     \
            case 8: return BPQ_PICK_NPT(V, 4, false);                                    \
            case 9: return BPQ_PICK_NPT(V, 4, true);                                     \
        }                                                                                \
        return nullptr;                                                                  \
    }

// The batched kernel of one variant (instantiated in a translation unit of
// its own): generic = items may use the generic table layout.
#define BPQ_DEFINE_PICK_BATCH(NAME, V)                                                   \
    BatchKernelFn NAME(bool generic) {                                                   \
        return generic ? dk::decode_batch_kernel<V, true> : dk::decode_batch_kernel<V, false>; \
    }

// The non-trace kernels of one variant for split tables without padding
// (bpq_tanner::full), instantiated in translation units of their own so
// that they compile in parallel with the others.
#define BPQ_DEFINE_PICK_FULL(NAME, V)                                                    \
    DecodeKernelFn NAME(int npt) {                                                       \
        switch (npt) {                                                                   \
            case 1: return dk::decode_kernel<V, 1, false, true, true>;                   \
            case 2: return dk::decode_kernel<V, 2, false, true, true>;                   \
            case 3: return dk::decode_kernel<V, 3, false, true, true>;                   \
            case 4: return dk::decode_kernel<V, 4, false, true, true>;                   \
        }                                                                                \
        return nullptr;                                                                  \
    }

}  // namespace bpq
