// Two shots per thread: the flooding-schedule decoder of decode_kernel.cuh
// for codes in the split table layout, with every thread working on the
// same nodes of two shots at once ("lanes" 0 and 1).  Each message slot is a
// float2 holding the edge's message in both shots, so one 64-bit shared-
// memory access and one address serve two shots, and every floating-point
// step of the update rules runs as one packed f32x2 instruction over the two
// lanes.  Each lane rounds exactly as the one-shot kernel's scalar operation,
// so per-shot results are bit-identical to decode_kernel's.
//
// The lanes are independent shots with their own iteration counts: when a
// lane's decision satisfies its syndrome (or it reaches max_iter) the group
// writes that shot's outputs and the lane takes the next shot from the work
// queue at once, restarting from the initial messages of eq. (init) (which
// do not depend on the shot, since the prior is shared) while the other lane
// carries on.  The group synchronises on its named barrier twice per
// iteration: after the check pass, which also publishes the lanes' syndrome-
// test votes (warp votes gathered in a shared flag word), and after the
// variable pass.
#pragma once

#include "decode_kernel.cuh"

namespace bpq {
namespace dk {

__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 min2(float2 a, float2 b) { return make_float2(fminf(a.x, b.x), fminf(a.y, b.y)); }
__device__ __forceinline__ float2 max2(float2 a, float2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(rcp(a.x), rcp(a.y)); }
__device__ __forceinline__ float2 ex22(float2 a) { return make_float2(ex2(a.x), ex2(a.y)); }

// Shared memory of one shot pair: two vote words (16 bytes), the float2
// message slots (4 n_pad + the zero slot + the trash slot, padded to
// 4 n_pad + 4) and the variant state (float2 [arrays][n_pad]).  The CTA also
// holds the staged table, the prior LLRs and the initial messages
// (float [4 n_pad]) of eq. (init).
struct PairMem {
    const float *PiS, *init;
    uint32_t *votes;
    float2 *slots, *state;
};

constexpr uint32_t kPairVoteBytes = 16;

__device__ __forceinline__ PairMem pair_mem(const DecodeArgs &a, uint8_t *base, int group) {
    PairMem m;
    m.PiS = reinterpret_cast<const float *>(base + a.table_bytes);
    m.init = m.PiS + 3 * a.n_pad;
    uint8_t *g = base + a.table_bytes + (size_t)28 * a.n_pad + (size_t)group * a.group_bytes;
    m.votes = reinterpret_cast<uint32_t *>(g);
    m.slots = reinterpret_cast<float2 *>(g + kPairVoteBytes);
    m.state = m.slots + a.slots_floats;
    return m;
}

// Barrier over the group that returns, per lane, whether any thread's vote
// is set: bit k of the result for bit k of `votes`.  Each warp ORs its two
// warp-wide votes into the shared word votes_smem[parity] before the
// barrier; the word of the other parity, read in the previous iteration, is
// cleared before the next barrier so that the next iteration finds it zero.
__device__ __forceinline__ uint32_t group_any2(int G, int bar_id, uint32_t votes, uint32_t *votes_smem, int tg,
                                               uint32_t parity) {
    const uint32_t w = (__any_sync(0xffffffffu, votes & 1u) ? 1u : 0u) | (__any_sync(0xffffffffu, votes & 2u) ? 2u : 0u);
    if (G == 1) {
        __syncwarp();
        return w;
    }
    if ((tg & 31) == 0 && w) atomicOr(votes_smem + parity, w);
    group_sync(G, bar_id);
    const uint32_t any = *reinterpret_cast<volatile uint32_t *>(votes_smem + parity);
    if (tg == 0) votes_smem[parity ^ 1u] = 0u;
    return any;
}

// Variable-to-check messages of one qubit for both lanes (split layout):
// emit_v2c's arithmetic, each step one f32x2 instruction over the lanes.
// ab: lane 0's anticommutation bits in bits 0-1, lane 1's in bits 8-9.
template <bool PHI, bool FULL>
__device__ __forceinline__ void emit_v2c_pair(const ShotParams &sp, float2 *slots, int j, uint32_t vp, float2 QX,
                                              float2 QY, float2 QZ, const float2 (&win)[4], uint32_t ab) {
    const float2 c0 = min2(f2(0.f), min2(QX, min2(QY, QZ)));
    const float2 e0 = ex22(c0);
    const float2 eX = ex22(add2(c0, neg2(QX))), eY = ex22(add2(c0, neg2(QY))), eZ = ex22(add2(c0, neg2(QZ)));
    // C = 1 + e^{-Q_H} and the two anticommuting terms for H = X (positions
    // 0, 1) and H = Z (positions 2, 3)
    const float2 CX = add2(e0, eX), AX = add2(eY, eZ), CZ = add2(e0, eZ), AZ = add2(eX, eY);
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        const float2 C = n < 2 ? CX : CZ;
        const float2 A = mul2(n < 2 ? AX : AZ, ex22(win[n]));
        const float2 cma = add2(C, neg2(A));
        const uint32_t neg0 = __float_as_uint(cma.x) & 0x80000000u, neg1 = __float_as_uint(cma.y) & 0x80000000u;
        float2 dl;
        if (PHI) {
            const float mx0 = fmaxf(C.x, A.x), mn0 = fminf(C.x, A.x);
            const float mx1 = fmaxf(C.y, A.y), mn1 = fminf(C.y, A.y);
            dl.x = fmaxf(log1p_rel(2.0f * mn0 * rcp(mx0 - mn0)), sp.vclip);
            dl.y = fmaxf(log1p_rel(2.0f * mn1 * rcp(mx1 - mn1)), sp.vclip);
        } else {
            const float2 m = min2(C, A);
            dl = max2(mul2(add2(m, m), rcp2(add2(C, A))), f2(sp.vclip));
        }
        const uint32_t sh = n < 2 ? 0u : 1u;
        const uint32_t b0 = (__float_as_uint(dl.x) & ~1u) | ((ab >> sh) & 1u) | neg0;
        const uint32_t b1 = (__float_as_uint(dl.y) & ~1u) | ((ab >> (8 + sh)) & 1u) | neg1;
        if (FULL || ((vp >> (2 * n)) & 3u)) slots[n * sp.Np + j] = make_float2(__uint_as_float(b0), __uint_as_float(b1));
    }
}

// Decode shots two at a time with a group of G warps (thread tg of 32G)
// until the queue is empty.
template <int VARIANT, int NPT, bool FULL>
__device__ __forceinline__ void decode_pairs(const DecodeArgs &a, const ThreadAdj<NPT> &adj, const PairMem &m, int T,
                                             int tg, int G, int bar_id, int *grp_shot) {
    constexpr bool PHI = PhiForm<VARIANT>::value;
    constexpr int NS = StateArrays<VARIANT>::n;
    const ShotParams sp = shot_params<PHI>(a, a.alpha);
    const int N = sp.N, M = sp.M, Np = sp.Np;
    const uint32_t kZero = 4u * (uint32_t)Np, kTrash = kZero + 1u;
    float2 *slots = m.slots, *state = m.state;
    const float *PiS = m.PiS, *init = m.init;
    uint32_t parity = 0;

    // start both lanes
    if (tg == 0) {
        grp_shot[0] = (int)atomicAdd(a.work, 1u);
        grp_shot[1] = (int)atomicAdd(a.work, 1u);
        m.votes[0] = m.votes[1] = 0u;
    }
    group_sync(G, bar_id);
    int shot[2] = {grp_shot[0], grp_shot[1]};
    int t[2] = {1, 1};
    uint32_t sbits = 0;  // bit 2k + lane: the syndrome bit of owned check k
    uint32_t dk[NPT];     // decisions: lane 0 in bits 0-7, lane 1 in bits 8-15
    auto load_syndrome = [&](int lane) {
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int i = k * T + tg;
            sbits &= ~(1u << (2 * k + lane));
            if (i < M && shot[lane] < a.B) {
                const uint32_t w = __ldg(a.syn + (size_t)shot[lane] * a.W + (i >> 5));
                sbits |= ((w >> (i & 31)) & 1u) << (2 * k + lane);
            }
        }
    };
    // eq. (init) for `lanes` (bit k = lane k): the shot-independent initial
    // messages, Q^(0) = Pi^(0), g^(0) = G^(0) = 0, EWAInit's Pi^(1) = Pi^(0)
    auto restart = [&](uint32_t lanes) {
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int j = k * T + tg;
            if (j < N) {
#pragma unroll
                for (int n = 0; n < 4; ++n) {
                    float *s = reinterpret_cast<float *>(slots + n * Np + j);
                    if (lanes & 1u) s[0] = init[n * Np + j];
                    if (lanes & 2u) s[1] = init[n * Np + j];
                }
                if (NS >= 3) {
#pragma unroll
                    for (int w = 0; w < 3; ++w) {
                        const float pw = PiS[w * Np + j];
                        float *s = reinterpret_cast<float *>(state + w * Np + j);
                        float *s3 = reinterpret_cast<float *>(state + (3 + w) * Np + j);
                        const float v3 = VARIANT == BPQ_EWAINIT ? a.alpha * pw : 0.f;
                        if (lanes & 1u) { s[0] = pw; s3[0] = v3; }
                        if (lanes & 2u) { s[1] = pw; s3[1] = v3; }
                    }
                }
            }
        }
    };
    if (shot[0] >= a.B && shot[1] >= a.B) return;
    load_syndrome(0);
    load_syndrome(1);
#pragma unroll
    for (int k = 0; k < NPT; ++k) dk[k] = 0;
    restart(3u);
    group_sync(G, bar_id);

    for (;;) {
        uint32_t mismatch = 0;
        // ---- check pass: syndrome tests of the lanes' previous decisions, then eq. (h_update) ----
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int i = k * T + tg;
            if (i < M) {
                const uint32_t sl[4] = {adj.cs_lo[k] & 0xFFFFu, adj.cs_lo[k] >> 16, adj.cs_hi[k] & 0xFFFFu,
                                        adj.cs_hi[k] >> 16};
                const uint32_t sb0 = (sbits >> (2 * k)) & 1u, sb1 = (sbits >> (2 * k + 1)) & 1u;
                float2 v[4];
#pragma unroll
                for (int n = 0; n < 4; ++n) v[n] = slots[sl[n]];
                uint32_t u0[4], u1[4];
#pragma unroll
                for (int n = 0; n < 4; ++n) {
                    u0[n] = __float_as_uint(v[n].x);
                    u1[n] = __float_as_uint(v[n].y);
                }
                const uint32_t ux0 = u0[0] ^ u0[1] ^ u0[2] ^ u0[3], ux1 = u1[0] ^ u1[1] ^ u1[2] ^ u1[3];
                mismatch |= ((ux0 ^ sb0) & 1u) | (((ux1 ^ sb1) & 1u) << 1);
                float2 mag[4];
#pragma unroll
                for (int n = 0; n < 4; ++n)
                    mag[n] = make_float2(__uint_as_float(u0[n] & 0x7FFFFFFEu), __uint_as_float(u1[n] & 0x7FFFFFFEu));
                const uint32_t sgn0 = (ux0 ^ (sb0 << 31)) & 0x80000000u, sgn1 = (ux1 ^ (sb1 << 31)) & 0x80000000u;
                float2 ext[4];
                if (PHI) {
                    const float2 e01 = add2(mag[0], mag[1]), e23 = add2(mag[2], mag[3]);
                    ext[0] = add2(mag[1], e23);
                    ext[1] = add2(mag[0], e23);
                    ext[2] = add2(e01, mag[3]);
                    ext[3] = add2(e01, mag[2]);
                } else {
                    // a (+) b = a + b - ab, as oplus
                    const float2 d01 = fma2(neg2(mag[0]), mag[1], add2(mag[0], mag[1]));
                    const float2 d23 = fma2(neg2(mag[2]), mag[3], add2(mag[2], mag[3]));
                    ext[0] = fma2(neg2(mag[1]), d23, add2(mag[1], d23));
                    ext[1] = fma2(neg2(mag[0]), d23, add2(mag[0], d23));
                    ext[2] = fma2(neg2(mag[3]), d01, add2(mag[3], d01));
                    ext[3] = fma2(neg2(mag[2]), d01, add2(mag[2], d01));
                }
#pragma unroll
                for (int n = 0; n < 4; ++n) {
                    float2 w;
                    if (PHI) {
                        w = make_float2(phi_check(ext[n].x), phi_check(ext[n].y));
                    } else {
                        // c2v_magnitude on both lanes
                        const float2 q = fma2(f2(2.0f), rcp2(ext[n]), f2(-1.0f));
                        w = make_float2(lg2(q.x), lg2(q.y));
                    }
                    if (!(FULL && !PHI)) w = min2(w, f2(sp.clip2));
                    const uint32_t b0 = __float_as_uint(w.x) ^ ((sgn0 ^ u0[n]) & 0x80000000u);
                    const uint32_t b1 = __float_as_uint(w.y) ^ ((sgn1 ^ u1[n]) & 0x80000000u);
                    slots[FULL ? sl[n] : sl[n] == kZero ? kTrash : sl[n]] =
                        make_float2(__uint_as_float(b0), __uint_as_float(b1));
                }
            }
        }
        // a lane's first check pass has no previous decision to test
        const uint32_t tested = (t[0] > 1 ? 1u : 0u) | (t[1] > 1 ? 2u : 0u);
        const uint32_t any = group_any2(G, bar_id, mismatch & tested, m.votes, tg, parity);
        parity ^= 1u;
        uint32_t fin = 0;
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            if (shot[l] >= a.B) continue;
            const bool conv = t[l] > 1 && !((any >> l) & 1u);
            if (conv || t[l] > sp.max_iter) {
                fin |= 1u << l;
                // outputs: the decision of the lane's last iteration
#pragma unroll
                for (int k = 0; k < NPT; ++k) {
                    const int j = k * T + tg;
                    if (j < N && BPQ_IN_BOUNDS((size_t)shot[l] * N + j, (size_t)a.B * N, a.work + 1))
                        a.est[(size_t)shot[l] * N + j] = (uint8_t)((dk[k] >> (8 * l)) & 0xFFu);
                }
                if (tg == 0 && BPQ_IN_BOUNDS(shot[l], a.B, a.work + 1)) {
                    a.conv[shot[l]] = conv ? 1 : 0;
                    a.iters[shot[l]] = (uint8_t)(conv ? t[l] - 1 : sp.max_iter);
                    grp_shot[l] = (int)atomicAdd(a.work, 1u);
                }
            }
        }

        // ---- variable pass: posterior of the variant, decision, eq. (v_update)/(mombp5) ----
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int j = k * T + tg;
            if (j < N) {
                const uint32_t vp = adj.info[k] >> 8;
                float2 win[4];
#pragma unroll
                for (int n = 0; n < 4; ++n) win[n] = slots[n * Np + j];
                // positions 0, 1: X-type edges (anticommute with Z and Y); 2, 3:
                // Z-type edges (with X and Y); unused slots hold 0
                const float2 SZ = add2(win[0], win[1]), SX = add2(win[2], win[3]);
                const float2 SY = add2(SX, SZ);
                float2 Q[3];
                if (VARIANT == BPQ_EWAINIT) {
                    // eq. (EWAInit): Q^(t) = Pi^(t) + S, Pi^(t+1) = alpha Pi^(0) + (1-alpha) Q^(t)
                    const float2 oma = f2(1.f - sp.alpha);
                    Q[0] = add2(state[j], SX);
                    Q[1] = add2(state[Np + j], SY);
                    Q[2] = add2(state[2 * Np + j], SZ);
                    state[j] = fma2(oma, Q[0], state[3 * Np + j]);
                    state[Np + j] = fma2(oma, Q[1], state[4 * Np + j]);
                    state[2 * Np + j] = fma2(oma, Q[2], state[5 * Np + j]);
                } else {
                    const float2 S[3] = {SX, SY, SZ};
#pragma unroll
                    for (int w = 0; w < 3; ++w) {
                        const float Pi = PiS[w * Np + j];
                        if (VARIANT == BPQ_PLAIN) {
                            Q[w] = add2(f2(Pi), S[w]);  // eq. (p_update)
                        } else if (VARIANT == BPQ_MOMENTUM) {
                            const float2 qp = state[w * Np + j], gprev = state[(3 + w) * Np + j];
                            const float2 g = make_float2(momentum_g(sp, qp.x, Pi, S[w].x, gprev.x),
                                                         momentum_g(sp, qp.y, Pi, S[w].y, gprev.y));
                            Q[w] = make_float2(momentum_q(sp, qp.x, g.x), momentum_q(sp, qp.y, g.y));
                            state[w * Np + j] = Q[w];
                            state[(3 + w) * Np + j] = g;
                        } else {
                            const float2 qp = state[w * Np + j], G2 = state[(3 + w) * Np + j];
                            const float gp0 = adagrad_gp(qp.x, Pi, S[w].x), gp1 = adagrad_gp(qp.y, Pi, S[w].y);
                            const float Gs0 = adagrad_G(G2.x, gp0, t[0] >= 2 || sp.ada_from1);
                            const float Gs1 = adagrad_G(G2.y, gp1, t[1] >= 2 || sp.ada_from1);
                            Q[w].x = t[0] == 1 ? Pi + S[w].x : adagrad_q(sp, qp.x, gp0, Gs0);
                            Q[w].y = t[1] == 1 ? Pi + S[w].y : adagrad_q(sp, qp.y, gp1, Gs1);
                            state[w * Np + j] = Q[w];
                            state[(3 + w) * Np + j] = make_float2(Gs0, Gs1);
                        }
                    }
                }
                // hard decision per lane: I if all Q_W > 0, else the first minimum of X, Y, Z
                const float mq0 = fminf(Q[0].x, fminf(Q[1].x, Q[2].x));
                const float mq1 = fminf(Q[0].y, fminf(Q[1].y, Q[2].y));
                const uint32_t d0 = mq0 > 0.f ? 0u : Q[0].x == mq0 ? 1u : Q[1].x == mq0 ? 2u : 3u;
                const uint32_t d1 = mq1 > 0.f ? 0u : Q[0].y == mq1 ? 1u : Q[1].y == mq1 ? 2u : 3u;
                dk[k] = d0 | (d1 << 8);
                const uint32_t ab = anti_bits_split(d0) | (anti_bits_split(d1) << 8);
                emit_v2c_pair<PHI, FULL>(sp, slots, j, vp, Q[0], Q[1], Q[2], win, ab);
            }
        }
        if (fin) restart(fin);  // finished lanes start their next shot from eq. (init)
        group_sync(G, bar_id);
        if (fin) {
#pragma unroll
            for (int l = 0; l < 2; ++l)
                if ((fin >> l) & 1u) {
                    shot[l] = grp_shot[l];
                    t[l] = 0;
                    load_syndrome(l);
                }
            if (shot[0] >= a.B && shot[1] >= a.B) break;
        }
        ++t[0];
        ++t[1];
    }
}

// One code per launch, two shots per thread: a persistent grid whose shot
// groups take shots from the global queue until the batch is exhausted.
template <int VARIANT, int NPT, bool FULL>
__global__ void __launch_bounds__(1024, 1) decode_pair_kernel(const DecodeArgs a) {
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
    const PairMem m = pair_mem(a, tab, group);
#ifdef BPQ_DEBUG
    {
        const size_t need = kSmemHeader + (size_t)a.table_bytes + (size_t)28 * a.n_pad +
                            (size_t)(blockDim.x / T) * a.group_bytes;
        const bool ok = need <= dynamic_smem_bytes() && a.n_pad >= a.N && a.slots_floats >= 4u * a.n_pad + 2u &&
                        a.group_bytes >= kPairVoteBytes + 8u * (a.slots_floats +
                                                               (uint32_t)StateArrays<VARIANT>::n * a.n_pad) &&
                        (a.off_var_pauli + (uint32_t)a.N <= a.table_bytes) && blockDim.x / T <= kMaxPairGroupsPerCta;
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
    float *PiS = reinterpret_cast<float *>(tab + a.table_bytes);
    load_prior(a, PiS);
    if (tg == 0) m.slots[4 * a.n_pad] = make_float2(0.f, 0.f);  // the zero slot
    const bool staged = mbar_wait_bounded(mbar, 0, 1u << 22);
    if (__syncthreads_or(!staged)) {
        if (tid == 0) atomicExch(a.work + 1, 1u);
        mbar_wait_bounded(mbar, 0, 1u << 22);  // let an in-flight copy land before exiting
        return;
    }
    // the initial messages of eq. (init), lambda(Pi^(0)) on every edge: the
    // one-shot kernel's variable pass with no incoming messages, into a
    // shared per-CTA table (unused positions of padded qubits hold 0)
    {
        const ShotParams sp = shot_params<PhiForm<VARIANT>::value>(a, a.alpha);
        float *init = PiS + 3 * a.n_pad;
        const float z4[4] = {0.f, 0.f, 0.f, 0.f};
        for (int j = tid; j < a.N; j += blockDim.x) {
            const uint32_t vp = tab[a.off_var_pauli + j];
            emit_v2c<false, true, PhiForm<VARIANT>::value, true, FULL>(a, sp, init, j, 0, 0, vp, PiS[j],
                                                                      PiS[a.n_pad + j], PiS[2 * a.n_pad + j], z4, 0u);
        }
        // unused positions (padded qubits) read 0 in both lanes
        if (!FULL)
            for (int s = tg; s < 4 * a.n_pad; s += T) m.slots[s] = make_float2(0.f, 0.f);
    }
    __syncthreads();

    ThreadAdj<NPT> adj;
    load_adjacency<NPT>(a, tab, T, tg, NPT, adj);
    decode_pairs<VARIANT, NPT, FULL>(a, adj, m, T, tg, G, bar_id, grp_shot + 2 * group);
}

}  // namespace dk

// The two-shots-per-thread kernels of one variant (split tables; FULL for
// tables without padding), for nodes per thread npt in {1, 2}.
#define BPQ_DEFINE_PICK_PAIR(NAME, V, FULLV)                                             \
    DecodeKernelFn NAME(int npt) {                                                       \
        switch (npt) {                                                                   \
            case 1: return dk::decode_pair_kernel<V, 1, FULLV>;                          \
            case 2: return dk::decode_pair_kernel<V, 2, FULLV>;                          \
        }                                                                                \
        return nullptr;                                                                  \
    }

}  // namespace bpq
