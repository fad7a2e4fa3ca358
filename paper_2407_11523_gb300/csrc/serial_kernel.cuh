// Serial-schedule decoding kernels (bpq_decode_serial, bpq_decode_serial_trace):
// Algorithm 1's serial update, where the qubits are visited in index order
// and qubit j, at its turn, takes the c->v messages of its checks from the
// v->c messages as they stand (this sweep's for the qubits before j, the
// previous sweep's for those after it), updates its posterior and sends its
// new v->c messages.
//
// GB300 mapping.  Qubit j depends, within a sweep, only on the earlier
// qubits that share a check with it.  Levels level(j) = 1 + max level of
// those qubits (0 if none) split the sweep into sets of mutually independent
// qubits whose inputs all come from lower levels, so visiting the levels in
// order, all qubits of a level at once, gives exactly the serial order's
// result.  Surface codes in index order have about 2L levels of up to about
// 2L qubits each.  A warp decodes one shot (serial_kernel) or two
// (serial_pair_kernel): its lanes take the qubits of a level, then
// __syncwarp, level after level.  The shot's edge messages, its variant
// state and one byte per qubit (the syndrome bits of its checks and its
// decision) sit in the warp's shared memory; the per-qubit tables are staged
// once per CTA by a bulk TMA copy.  Persistent CTAs; warps take shots from
// an atomic queue.
//
// Two shots per warp: each lane works on the same qubit of both shots, whose
// messages and state share 64-bit slots, so the table reads, the slot
// addresses and the loop are shared, the simple floating-point steps run as
// packed f32x2 instructions, and the two independent chains overlap.  Each
// shot stops on its own; the warp then takes the next shot for that half at
// the end of the sweep.  Every step rounds as in serial_kernel, so results
// are the same bit for bit.
//
// Layout.  Per-qubit arrays (prior, state, the qubit byte) are indexed by
// the qubit's position v in the sweep's level order, so the lanes of a level
// touch consecutive words; message slots are assigned by the host
// (bpq::build_serial_table) so that the lanes of one access fall in distinct
// banks.  Every qubit runs four edges: padding edges read the zero slot
// (delta 0, the identity of the check rule), enter no posterior sum and
// write the trash slot, so the per-edge work is straight code with no branch
// on the degree.  SPLIT (split-layout codes, bpq_tanner::split): edges 0, 1
// of a qubit have Pauli X and edges 2, 3 Pauli Z (or are padding), so the
// sums and the per-edge Pauli choices are fixed by the position.
//
// Stopping rule.  The syndrome test of a check needs the decisions of all
// its qubits in this sweep; the last of them in the sweep order sees the
// others' new messages (their least significant bits carry the
// anticommutation of each decision with the edge's Pauli) when it updates,
// so it tests the check at its turn and the warp ORs the mismatches at the
// end of the sweep: the same test as a separate pass over the checks after
// the sweep.
//
// Arithmetic is that of the parallel kernel (decode_kernel.cuh): v->c
// messages stored as sign * delta (AdaGrad-BP: sign * phi) with the
// decision's anticommutation bit in the least significant bit, and
// log-likelihoods in bits; every step is an explicit intrinsic, so no
// contraction choice of the compiler can make the two kernels differ.
#pragma once

#include <cuda_runtime.h>

#include "bpq_internal.h"
#include "decode_kernel.cuh"
#include "decode_launch.h"

namespace bpq {

struct SerialArgs {
    const uint8_t *table;  // SerialVar[N] | level_ptr u16[L+1] | canon u16[N][4] (bpq_tanner::serial)
    uint32_t table_bytes;  // bytes staged in shared memory: SerialVar[N] | level_ptr
    uint32_t off_levels, off_canon;
    int nlevels;
    const uint32_t *syn;   // [B][W]
    const float *prior;    // [N][3]
    uint8_t *est, *conv, *iters;
    uint32_t *work;        // [0] next shot, [1] device error word
    float *tr_v2c, *tr_c2v, *tr_Q;
    uint8_t *tr_dec;
    int N, M, E, W, B, max_iter;
    int n_pad;             // N rounded up to 4 (per-qubit array stride)
    uint32_t zero_slot;    // message slots: [0, zero_slot) edges, zero_slot, zero_slot + 1 trash
    uint32_t msg_floats;   // zero_slot + 2 rounded up to 4
    uint32_t warp_bytes;   // shared memory of one warp: messages | state | syndrome | qubit bytes
    uint32_t off_syn, off_qb;  // byte offsets inside a warp's region
    uint32_t syn_stride;   // words between the two shots' syndromes (two shots per warp)
    float alpha, gamma, eps, clip, clip2, delta_clip, phi_clip;
    int ada_from1;
};

namespace sk {

using namespace dk;

// Per-qubit state arrays (each n_pad floats, or float2 with two shots per
// warp) of the serial kernels: EWAInit Q^(t-1); Momentum Q^(t-1), g; AdaGrad
// Q^(t-1), G.  The kernels and serial_launch's sizing both read this.
__host__ __device__ constexpr int serial_state_arrays(int variant) {
    return variant == BPQ_PLAIN ? 0 : variant == BPQ_EWAINIT ? 3 : 6;
}

// The four edge Paulis of a qubit one per byte (anti_bytes' format).
__device__ __forceinline__ uint32_t pauli_bytes(uint32_t pauli) {
    return (pauli & 3u) | (((pauli >> 2) & 3u) << 8) | (((pauli >> 4) & 3u) << 16) | (((pauli >> 6) & 3u) << 24);
}

// Bit k: whether decision d anticommutes with the qubit's edge k.
template <bool SPLIT>
__device__ __forceinline__ uint32_t anti_bits4(uint32_t d, uint32_t pauli) {
    if (SPLIT) {
        // X edges (0, 1) anticommute with Y, Z; Z edges (2, 3) with X, Y
        return (d >= 2u ? 3u : 0u) | (d - 1u < 2u ? 12u : 0u);
    } else {
        const uint32_t ab = anti_bytes(d, pauli_bytes(pauli));
        return (ab | (ab >> 7) | (ab >> 14) | (ab >> 21)) & 15u;
    }
}

// |m_{c->v}| in bits of one edge from the magnitudes of its check's other
// three v->c messages (eq. (h_update)), clipped.
template <bool PHI>
__device__ __forceinline__ float c2v_mag(const SerialArgs &a, float m0, float m1, float m2) {
    if (PHI) return fminf(phi_check(__fadd_rn(__fadd_rn(m0, m1), m2)), a.clip2);
    return fminf(lg2(__fmaf_rn(2.0f, rcp(oplus(oplus(m0, m1), m2)), -1.0f)), a.clip2);
}
template <bool PHI>
__device__ __forceinline__ float2 c2v_mag2(const SerialArgs &a, float2 m0, float2 m1, float2 m2) {
    if (PHI) {
        const float2 s = __fadd2_rn(__fadd2_rn(m0, m1), m2);
        return make_float2(fminf(phi_check(s.x), a.clip2), fminf(phi_check(s.y), a.clip2));
    }
    const float2 D = oplus2(oplus2(m0, m1), m2);
    const float2 r = __ffma2_rn(make_float2(2.0f, 2.0f), make_float2(rcp(D.x), rcp(D.y)), make_float2(-1.0f, -1.0f));
    return make_float2(fminf(lg2(r.x), a.clip2), fminf(lg2(r.y), a.clip2));
}

// S_X, S_Y, S_Z (eq. (p_update)) from the c->v messages of the four edges.
template <bool SPLIT>
__device__ __forceinline__ void posterior_sums(uint32_t pauli, const float (&w)[4], float (&S)[3]) {
    if (SPLIT) {
        S[2] = __fadd_rn(w[0], w[1]);
        S[0] = __fadd_rn(w[2], w[3]);
        S[1] = __fadd_rn(S[0], S[2]);
    } else {
        anticommuting_sums(pauli, w, S[0], S[1], S[2]);
    }
}

// Q_W of the variant for one qubit of one shot at sweep t from Pi_W, S_W and
// the state (qp = Q^(t-1), s2 = g or G); updates the state.
template <int VARIANT>
__device__ __forceinline__ float posterior(const SerialArgs &a, float Pi, float S, float &qp, float &s2, int t,
                                           float alpha) {
    if (VARIANT == BPQ_PLAIN) return __fadd_rn(Pi, S);  // eq. (p_update)
    if (VARIANT == BPQ_EWAINIT) {
        // eq. (EWAInit) for the qubit at its turn
        const float base = t > 1 ? __fmaf_rn(alpha, Pi, __fmul_rn(1.f - alpha, qp)) : Pi;
        qp = __fadd_rn(base, S);
        return qp;
    }
    if (VARIANT == BPQ_MOMENTUM) {
        // eqs. (mombp1), (mombp2)
        s2 = __fmaf_rn(a.gamma, s2, __fmul_rn(1.f - a.gamma, __fsub_rn(__fsub_rn(qp, Pi), S)));
        qp = __fmaf_rn(-a.alpha, s2, qp);
        return qp;
    }
    // eq. (boost) from t = 2; G accumulates g'^2
    const float gp = __fsub_rn(__fsub_rn(qp, Pi), S);
    if (t >= 2 || a.ada_from1) s2 = __fmaf_rn(gp, gp, s2);
    qp = t == 1 ? __fadd_rn(Pi, S) : __fmaf_rn(-__fmul_rn(a.alpha, gp), rcp(__fadd_rn(sqrt_approx(s2), a.eps)), qp);
    return qp;
}

// Hard decision: I if all Q_W > 0, else the first minimum of X, Y, Z.
__device__ __forceinline__ uint32_t decide(float QX, float QY, float QZ) {
    if (QX > 0.f && QY > 0.f && QZ > 0.f) return 0u;
    uint32_t d = 1;
    float mq = QX;
    if (QY < mq) {
        d = 2;
        mq = QY;
    }
    if (QZ < mq) d = 3;
    return d;
}

// Message bits of one edge: sign * delta (sign * phi with PHI) from C and A
// (eq. (v_update) as C / A ratios), least significant bit = abit.
template <bool PHI>
__device__ __forceinline__ uint32_t v2c_bits(const SerialArgs &a, float C, float A, uint32_t abit) {
    float dl;
    if (PHI) {
        const float mx = fmaxf(C, A), mn = fminf(C, A);
        dl = fmaxf(log1p_rel(__fmul_rn(__fmul_rn(2.0f, mn), rcp(__fsub_rn(mx, mn)))), a.phi_clip);
    } else {
        dl = fmaxf(__fmul_rn(__fmul_rn(2.0f, fminf(C, A)), rcp(__fadd_rn(C, A))), a.delta_clip);
    }
    return (__float_as_uint(dl) & ~1u) | abit | (A > C ? 0x80000000u : 0u);
}

// v->c messages of one qubit of one shot from its posterior (bits) and its
// incoming c->v messages win (bits), written to msg[STRIDE * slot] for the
// qubit's four edge slots; bit k of abits becomes edge k's least significant
// bit.  With TRACE, the natural-log message lambda of each real edge goes to
// tr_v2c at sweep t (canonical edge index ce[k]).
template <bool TRACE, bool PHI, bool SPLIT, int STRIDE>
__device__ __forceinline__ void send_v2c(const SerialArgs &a, float *msg, const SerialVar &sv, const uint16_t *ce,
                                         int t, int shot, float QX, float QY, float QZ, const float (&win)[4],
                                         uint32_t abits) {
    const float c0 = fminf(0.f, fminf(QX, fminf(QY, QZ)));
    const float e0 = ex2(c0);
    const float eX = ex2(__fsub_rn(c0, QX)), eY = ex2(__fsub_rn(c0, QY)), eZ = ex2(__fsub_rn(c0, QZ));
    const float CX = __fadd_rn(e0, eX), CY = __fadd_rn(e0, eY), CZ = __fadd_rn(e0, eZ);
    const float AX = __fadd_rn(eY, eZ), AY = __fadd_rn(eX, eZ), AZ = __fadd_rn(eX, eY);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t p = SPLIT ? (k < 2 ? 1u : 3u) : (sv.pauli >> (2 * k)) & 3u;
        const float C = p == 1u ? CX : p == 2u ? CY : CZ;
        const float Ab = p == 1u ? AX : p == 2u ? AY : AZ;
        const float A = __fmul_rn(Ab, ex2(win[k]));
        msg[STRIDE * sv.own[k]] = __uint_as_float(v2c_bits<PHI>(a, C, A, (abits >> k) & 1u));
        if (TRACE && a.tr_v2c && ((sv.real >> k) & 1u)) {
            const float lam = fminf(fmaxf(kLn2 * (lg2(C) - lg2(A)), -a.clip), a.clip);
            a.tr_v2c[((size_t)shot * (a.max_iter + 1) + t) * a.E + ce[k]] = lam;
        }
    }
}

// Syndrome bits of a qubit's four edges' checks (bit k), from the shot's
// syndrome words in shared memory.
__device__ __forceinline__ uint32_t qubit_syndrome(const SerialVar &sv, const uint32_t *syn) {
    uint32_t q = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t i = sv.chk[k];
        q |= (((sv.real >> k) & 1u) ? (syn[i >> 5] >> (i & 31)) & 1u : 0u) << k;
    }
    return q;
}

// ---------------------------------------------------------------- one shot per warp

// Shared memory of one warp: messages | state | syndrome words | one byte per
// qubit (bits 0-3: syndrome bits of its edges' checks; bits 4-5: decision).
struct WarpMem {
    float *msg, *state;
    uint32_t *syn;
    uint8_t *qb;
};

__device__ __forceinline__ WarpMem warp_mem(const SerialArgs &a, uint8_t *base, int warp) {
    WarpMem m;
    uint8_t *p = base + (size_t)warp * a.warp_bytes;
    m.msg = reinterpret_cast<float *>(p);
    m.state = m.msg + a.msg_floats;
    m.syn = reinterpret_cast<uint32_t *>(p + a.off_syn);
    m.qb = p + a.off_qb;
    return m;
}

// The update of the qubit at sweep position v in sweep t (t >= 1): c->v
// messages of its checks (eq. (h_update), from the messages as they stand),
// posterior of the variant, decision, new v->c messages.  Returns the
// syndrome mismatch of the checks this qubit is the last of (bit 0).
template <int VARIANT, bool TRACE, bool SPLIT>
__device__ __forceinline__ uint32_t update_qubit(const SerialArgs &a, const WarpMem &m, const float *PiS,
                                                 const SerialVar &sv, const uint16_t *ce, int v, int t, int shot,
                                                 float alpha) {
    constexpr bool PHI = PhiForm<VARIANT>::value;
    constexpr int NS = serial_state_arrays(VARIANT);
    const int Np = a.n_pad;
    const uint32_t qb = m.qb[v];
    float win[4];
    uint32_t par[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t u0 = __float_as_uint(m.msg[sv.oth[k][0]]), u1 = __float_as_uint(m.msg[sv.oth[k][1]]),
                       u2 = __float_as_uint(m.msg[sv.oth[k][2]]);
        const uint32_t ux = u0 ^ u1 ^ u2 ^ ((qb >> k) & 1u);  // bit 0: the check's parity without this edge
        par[k] = ux;
        const uint32_t sgn = (ux ^ (qb << (31 - k))) & 0x80000000u;
        const float w = c2v_mag<PHI>(a, __uint_as_float(u0 & 0x7FFFFFFEu), __uint_as_float(u1 & 0x7FFFFFFEu),
                                     __uint_as_float(u2 & 0x7FFFFFFEu));
        win[k] = SPLIT && !((sv.real >> k) & 1u) ? 0.f : __uint_as_float(__float_as_uint(w) ^ sgn);
        if (TRACE && a.tr_c2v && ((sv.real >> k) & 1u))
            a.tr_c2v[((size_t)shot * a.max_iter + (t - 1)) * a.E + ce[k]] = kLn2 * win[k];
    }
    float S[3];
    posterior_sums<SPLIT>(sv.pauli, win, S);
    float Q[3];
#pragma unroll
    for (int w = 0; w < 3; ++w) {
        float qp = NS >= 3 ? m.state[w * Np + v] : 0.f;
        float s2 = NS == 6 ? m.state[(3 + w) * Np + v] : 0.f;
        Q[w] = posterior<VARIANT>(a, PiS[w * Np + v], S[w], qp, s2, t, alpha);
        if (NS >= 3) m.state[w * Np + v] = qp;
        if (NS == 6) m.state[(3 + w) * Np + v] = s2;
    }
    const uint32_t d = decide(Q[0], Q[1], Q[2]);
    m.qb[v] = (uint8_t)((qb & 15u) | (d << 4));
    if (TRACE) {
        const size_t o = (size_t)shot * a.max_iter + (t - 1);
        const int j = sv.j;
        if (a.tr_Q) {
            a.tr_Q[(o * a.N + j) * 3 + 0] = kLn2 * Q[0];
            a.tr_Q[(o * a.N + j) * 3 + 1] = kLn2 * Q[1];
            a.tr_Q[(o * a.N + j) * 3 + 2] = kLn2 * Q[2];
        }
        if (a.tr_dec) a.tr_dec[o * a.N + j] = (uint8_t)d;
    }
    const uint32_t ab = anti_bits4<SPLIT>(d, sv.pauli);
    uint32_t mismatch = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) mismatch |= (par[k] ^ (ab >> k)) & (sv.last >> k) & 1u;
    send_v2c<TRACE, PHI, SPLIT, 1>(a, m.msg, sv, ce, t, shot, Q[0], Q[1], Q[2], win, ab);
    return mismatch;
}

// Eq. (init) for one shot of a warp at the qubits of this lane: the qubit
// bytes take the syndrome bits of each qubit's checks; Q^(0) = Pi^(0),
// g^(0) = G^(0) = 0; lambda(Pi^(0)) on every edge.  STRIDE/x: the shot's
// component of two-shot slots (1/0 with one shot per warp).
template <int VARIANT, bool TRACE, bool SPLIT, int STRIDE>
__device__ __forceinline__ void init_shot(const SerialArgs &a, float *msg, float *state, const uint32_t *syn,
                                          uint8_t *qb, const float *PiS, const SerialVar *vars,
                                          const uint16_t *canon, int lane, int shot) {
    constexpr bool PHI = PhiForm<VARIANT>::value;
    constexpr int NS = serial_state_arrays(VARIANT);
    const int Np = a.n_pad;
    for (int v = lane; v < a.N; v += 32) {
        const SerialVar sv = vars[v];
        qb[STRIDE * v] = (uint8_t)qubit_syndrome(sv, syn);
        const float PX = PiS[v], PY = PiS[Np + v], PZ = PiS[2 * Np + v];
        if (NS >= 3) {
            state[STRIDE * v] = PX;
            state[STRIDE * (Np + v)] = PY;
            state[STRIDE * (2 * Np + v)] = PZ;
        }
        if (NS == 6) {
            state[STRIDE * (3 * Np + v)] = 0.f;
            state[STRIDE * (4 * Np + v)] = 0.f;
            state[STRIDE * (5 * Np + v)] = 0.f;
        }
        const float z4[4] = {0.f, 0.f, 0.f, 0.f};
        send_v2c<TRACE, PHI, SPLIT, STRIDE>(a, msg, sv, canon + 4 * v, 0, shot, PX, PY, PZ, z4, 0u);
    }
}

// Decode one shot with one warp: eq. (init), then sweeps level by level
// until the decisions satisfy the syndrome (tested during every sweep) or
// max_iter sweeps have run (TRACE: always max_iter sweeps).
template <int VARIANT, bool TRACE, bool SPLIT>
__device__ __forceinline__ void decode_serial_shot(const SerialArgs &a, const WarpMem &m, const float *PiS,
                                                   const SerialVar *vars, const uint16_t *lp, const uint16_t *canon,
                                                   int lane, int shot) {
    const int N = a.N;
    for (int w = lane; w < a.W; w += 32) m.syn[w] = __ldg(a.syn + (size_t)shot * a.W + w);
    __syncwarp();
    init_shot<VARIANT, TRACE, SPLIT, 1>(a, m.msg, m.state, m.syn, m.qb, PiS, vars, canon, lane, shot);
    __syncwarp();
    int conv = 0, iters = a.max_iter;
    for (int t = 1; t <= a.max_iter; ++t) {
        uint32_t mismatch = 0;
        for (int l = 0; l < a.nlevels; ++l) {
            for (int v = lp[l] + lane; v < lp[l + 1]; v += 32)
                mismatch |= update_qubit<VARIANT, TRACE, SPLIT>(a, m, PiS, vars[v], canon + 4 * v, v, t, shot,
                                                                a.alpha);
            __syncwarp();
        }
        if (TRACE) continue;
        if (!__any_sync(0xffffffffu, mismatch)) {
            conv = 1;
            iters = t;
            break;
        }
    }
    if (!TRACE || a.est)
        for (int v = lane; v < N; v += 32) a.est[(size_t)shot * N + vars[v].j] = (uint8_t)(m.qb[v] >> 4);
    if (lane == 0 && (!TRACE || a.conv)) {
        a.conv[shot] = (uint8_t)conv;
        a.iters[shot] = (uint8_t)iters;
    }
    __syncwarp();
}

// Stage the serial table (bulk TMA) and the prior LLRs Pi_{v,W} = log2(p^I /
// p^W) in sweep order; zero slot of every warp's messages (at zero_off floats
// from the warp's region).  Returns false (after setting the error word) if
// the copy did not complete.
__device__ __forceinline__ bool stage_serial(const SerialArgs &a, uint8_t *smem, uint32_t zero_off, float **PiS_out,
                                             uint8_t **wbase_out) {
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);
    uint8_t *tab = smem + 128;
    float *PiS = reinterpret_cast<float *>(tab + a.table_bytes);
    uint8_t *wbase = reinterpret_cast<uint8_t *>(PiS + 3 * a.n_pad);
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(mbar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(mbar, a.table_bytes);
        bulk_g2s(tab, a.table, a.table_bytes, mbar);
    }
    if ((tid & 31) == 0) reinterpret_cast<float *>(wbase + (size_t)(tid >> 5) * a.warp_bytes)[zero_off] = 0.f;
    const bool staged = mbar_wait_bounded(mbar, 0, 1u << 22);
    if (__syncthreads_or(!staged)) {
        if (tid == 0) atomicExch(a.work + 1, 1u);
        mbar_wait_bounded(mbar, 0, 1u << 22);
        return false;
    }
    const SerialVar *vars = reinterpret_cast<const SerialVar *>(tab);
    const int Np = a.n_pad;
    for (int v = tid; v < a.N; v += blockDim.x) {
        const int j = vars[v].j;
        const float px = a.prior[3 * j], py = a.prior[3 * j + 1], pz = a.prior[3 * j + 2];
        const float pI = 1.0f - px - py - pz;
        PiS[v] = log2f(pI / px);
        PiS[Np + v] = log2f(pI / py);
        PiS[2 * Np + v] = log2f(pI / pz);
    }
    __syncthreads();
    *PiS_out = PiS;
    *wbase_out = wbase;
    return true;
}

// Persistent kernel, one shot per warp.
template <int VARIANT, bool TRACE, bool SPLIT>
__global__ void __launch_bounds__(1024, 1) serial_kernel(const SerialArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    float *PiS;
    uint8_t *wbase;
    if (!stage_serial(a, smem, a.zero_slot, &PiS, &wbase)) return;
    const int lane = threadIdx.x & 31;
    const WarpMem m = warp_mem(a, wbase, threadIdx.x >> 5);
    const SerialVar *vars = reinterpret_cast<const SerialVar *>(smem + 128);
    const uint16_t *lp = reinterpret_cast<const uint16_t *>(smem + 128 + a.off_levels);
    const uint16_t *canon = reinterpret_cast<const uint16_t *>(a.table + a.off_canon);  // traces only
    for (;;) {
        int shot = 0;
        if (lane == 0) shot = (int)atomicAdd(a.work, 1u);
        shot = __shfl_sync(0xffffffffu, shot, 0);
        if (shot >= a.B) break;
        decode_serial_shot<VARIANT, TRACE, SPLIT>(a, m, PiS, vars, lp, canon, lane, shot);
    }
}

// ---------------------------------------------------------------- two shots per warp

// Shared memory of one warp: float2 messages | float2 state | the two shots'
// syndrome words (syn_stride apart) | two bytes per qubit (one per shot, in
// WarpMem's format).
struct PairMem {
    float2 *msg, *state;
    uint32_t *syn;
    uint8_t *qb;
};

__device__ __forceinline__ PairMem pair_mem(const SerialArgs &a, uint8_t *base, int warp) {
    PairMem m;
    uint8_t *p = base + (size_t)warp * a.warp_bytes;
    m.msg = reinterpret_cast<float2 *>(p);
    m.state = m.msg + a.msg_floats;
    m.syn = reinterpret_cast<uint32_t *>(p + a.off_syn);
    m.qb = p + a.off_qb;
    return m;
}

// update_qubit for both shots of a warp (sweeps tA and tB); bit x of the
// result: the mismatch of shot x.
template <int VARIANT, bool SPLIT, bool FULL>
__device__ __forceinline__ uint32_t update_pair(const SerialArgs &a, const PairMem &m, const float *PiS,
                                                const SerialVar &sv, int v, int tA, int tB, float alpha) {
    constexpr bool PHI = PhiForm<VARIANT>::value;
    constexpr int NS = serial_state_arrays(VARIANT);
    const int Np = a.n_pad;
    const uint32_t q2 = *reinterpret_cast<const uint16_t *>(m.qb + 2 * v);
    const uint32_t qa = q2 & 0xFFu, qb = q2 >> 8;
    float wa[4], wb[4];
    uint32_t pa[4], pb[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 f0 = m.msg[sv.oth[k][0]], f1 = m.msg[sv.oth[k][1]], f2 = m.msg[sv.oth[k][2]];
        const uint32_t a0 = __float_as_uint(f0.x), a1 = __float_as_uint(f1.x), a2 = __float_as_uint(f2.x);
        const uint32_t b0 = __float_as_uint(f0.y), b1 = __float_as_uint(f1.y), b2 = __float_as_uint(f2.y);
        const uint32_t uxa = a0 ^ a1 ^ a2 ^ ((qa >> k) & 1u), uxb = b0 ^ b1 ^ b2 ^ ((qb >> k) & 1u);
        pa[k] = uxa;
        pb[k] = uxb;
        const uint32_t sa = (uxa ^ (qa << (31 - k))) & 0x80000000u, sb = (uxb ^ (qb << (31 - k))) & 0x80000000u;
        const float2 w = c2v_mag2<PHI>(
            a, make_float2(__uint_as_float(a0 & 0x7FFFFFFEu), __uint_as_float(b0 & 0x7FFFFFFEu)),
            make_float2(__uint_as_float(a1 & 0x7FFFFFFEu), __uint_as_float(b1 & 0x7FFFFFFEu)),
            make_float2(__uint_as_float(a2 & 0x7FFFFFFEu), __uint_as_float(b2 & 0x7FFFFFFEu)));
        const bool pad = SPLIT && !FULL && !((sv.real >> k) & 1u);
        wa[k] = pad ? 0.f : __uint_as_float(__float_as_uint(w.x) ^ sa);
        wb[k] = pad ? 0.f : __uint_as_float(__float_as_uint(w.y) ^ sb);
    }
    float SA[3], SB[3];
    if (SPLIT) {
        const float2 sz = __fadd2_rn(make_float2(wa[0], wb[0]), make_float2(wa[1], wb[1]));
        const float2 sx = __fadd2_rn(make_float2(wa[2], wb[2]), make_float2(wa[3], wb[3]));
        const float2 sy = __fadd2_rn(sx, sz);
        SA[0] = sx.x, SA[1] = sy.x, SA[2] = sz.x;
        SB[0] = sx.y, SB[1] = sy.y, SB[2] = sz.y;
    } else {
        posterior_sums<false>(sv.pauli, wa, SA);
        posterior_sums<false>(sv.pauli, wb, SB);
    }
    float QA[3], QB[3];
#pragma unroll
    for (int w = 0; w < 3; ++w) {
        const float Pi = PiS[w * Np + v];
        float2 qp = NS >= 3 ? m.state[w * Np + v] : make_float2(0.f, 0.f);
        float2 s2 = NS == 6 ? m.state[(3 + w) * Np + v] : make_float2(0.f, 0.f);
        if (VARIANT == BPQ_EWAINIT) {
            // packed form of posterior<EWAINIT>
            const float oma = 1.f - alpha;
            const float2 mix = __ffma2_rn(make_float2(alpha, alpha), make_float2(Pi, Pi),
                                          __fmul2_rn(make_float2(oma, oma), qp));
            qp = __fadd2_rn(make_float2(tA > 1 ? mix.x : Pi, tB > 1 ? mix.y : Pi), make_float2(SA[w], SB[w]));
            QA[w] = qp.x;
            QB[w] = qp.y;
        } else {
            QA[w] = posterior<VARIANT>(a, Pi, SA[w], qp.x, s2.x, tA, alpha);
            QB[w] = posterior<VARIANT>(a, Pi, SB[w], qp.y, s2.y, tB, alpha);
        }
        if (NS >= 3) m.state[w * Np + v] = qp;
        if (NS == 6) m.state[(3 + w) * Np + v] = s2;
    }
    const uint32_t da = decide(QA[0], QA[1], QA[2]), db = decide(QB[0], QB[1], QB[2]);
    *reinterpret_cast<uint16_t *>(m.qb + 2 * v) = (uint16_t)((qa & 15u) | (da << 4) | (((qb & 15u) | (db << 4)) << 8));
    const uint32_t aba = anti_bits4<SPLIT>(da, sv.pauli), abb = anti_bits4<SPLIT>(db, sv.pauli);
    uint32_t mismatch = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        mismatch |= (((pa[k] ^ (aba >> k)) & 1u) | (((pb[k] ^ (abb >> k)) & 1u) << 1)) & (((sv.last >> k) & 1u) * 3u);
    // eq. (v_update) for both shots (send_v2c's steps, packed where they round alike)
    const float ca = fminf(0.f, fminf(QA[0], fminf(QA[1], QA[2]))), cb = fminf(0.f, fminf(QB[0], fminf(QB[1], QB[2])));
    const float2 e0 = make_float2(ex2(ca), ex2(cb));
    const float2 eX = make_float2(ex2(__fsub_rn(ca, QA[0])), ex2(__fsub_rn(cb, QB[0])));
    const float2 eY = make_float2(ex2(__fsub_rn(ca, QA[1])), ex2(__fsub_rn(cb, QB[1])));
    const float2 eZ = make_float2(ex2(__fsub_rn(ca, QA[2])), ex2(__fsub_rn(cb, QB[2])));
    const float2 CX = __fadd2_rn(e0, eX), CY = __fadd2_rn(e0, eY), CZ = __fadd2_rn(e0, eZ);
    const float2 AX = __fadd2_rn(eY, eZ), AY = __fadd2_rn(eX, eZ), AZ = __fadd2_rn(eX, eY);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t p = SPLIT ? (k < 2 ? 1u : 3u) : (sv.pauli >> (2 * k)) & 3u;
        const float2 C = p == 1u ? CX : p == 2u ? CY : CZ;
        const float2 Ab = p == 1u ? AX : p == 2u ? AY : AZ;
        const float2 A = __fmul2_rn(Ab, make_float2(ex2(wa[k]), ex2(wb[k])));
        float2 out;
        if (PHI) {
            out.x = __uint_as_float(v2c_bits<true>(a, C.x, A.x, (aba >> k) & 1u));
            out.y = __uint_as_float(v2c_bits<true>(a, C.y, A.y, (abb >> k) & 1u));
        } else {
            const float2 mn = __fmul2_rn(make_float2(2.0f, 2.0f), make_float2(fminf(C.x, A.x), fminf(C.y, A.y)));
            const float2 sm = __fadd2_rn(C, A);
            const float2 r = __fmul2_rn(mn, make_float2(rcp(sm.x), rcp(sm.y)));
            const float dla = fmaxf(r.x, a.delta_clip), dlb = fmaxf(r.y, a.delta_clip);
            out.x = __uint_as_float((__float_as_uint(dla) & ~1u) | ((aba >> k) & 1u) | (A.x > C.x ? 0x80000000u : 0u));
            out.y = __uint_as_float((__float_as_uint(dlb) & ~1u) | ((abb >> k) & 1u) | (A.y > C.y ? 0x80000000u : 0u));
        }
        m.msg[sv.own[k]] = out;
    }
    return mismatch;
}

// Start shot `shot` in component x of a warp's two-shot slots.
template <int VARIANT, bool SPLIT>
__device__ __forceinline__ void start_pair_shot(const SerialArgs &a, const PairMem &m, const float *PiS,
                                                const SerialVar *vars, int lane, int x, int shot) {
    uint32_t *syn = m.syn + x * a.syn_stride;
    for (int w = lane; w < a.W; w += 32) syn[w] = __ldg(a.syn + (size_t)shot * a.W + w);
    __syncwarp();
    init_shot<VARIANT, false, SPLIT, 2>(a, reinterpret_cast<float *>(m.msg) + x, reinterpret_cast<float *>(m.state) + x,
                                        syn, m.qb + x, PiS, vars, nullptr, lane, shot);
}

// Persistent kernel, two shots per warp (at most kSerialPairWarps warps, so
// that a thread may hold 128 registers); each half takes the next shot from
// the queue when its shot stops (at the end of a sweep).  FULL: split layout
// without padding edges (bpq_tanner::full).
constexpr int kSerialPairWarps = 16;
template <int VARIANT, bool SPLIT, bool FULL>
__global__ void __launch_bounds__(32 * kSerialPairWarps, 1) serial_pair_kernel(const SerialArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    float *PiS;
    uint8_t *wbase;
    if (!stage_serial(a, smem, 2 * a.zero_slot, &PiS, &wbase)) return;
    if ((threadIdx.x & 31) == 0)
        reinterpret_cast<float *>(wbase + (size_t)(threadIdx.x >> 5) * a.warp_bytes)[2 * a.zero_slot + 1] = 0.f;
    const int lane = threadIdx.x & 31;
    const PairMem m = pair_mem(a, wbase, threadIdx.x >> 5);
    const SerialVar *vars = reinterpret_cast<const SerialVar *>(smem + 128);
    const uint16_t *lp = reinterpret_cast<const uint16_t *>(smem + 128 + a.off_levels);
    int shot[2], t[2];
    bool live[2];
#pragma unroll
    for (int x = 0; x < 2; ++x) {
        int s = 0;
        if (lane == 0) s = (int)atomicAdd(a.work, 1u);
        shot[x] = __shfl_sync(0xffffffffu, s, 0);
        live[x] = shot[x] < a.B;
        t[x] = 1;
        if (live[x]) start_pair_shot<VARIANT, SPLIT>(a, m, PiS, vars, lane, x, shot[x]);
    }
    __syncwarp();
    while (live[0] || live[1]) {
        uint32_t mismatch = 0;
        for (int l = 0; l < a.nlevels; ++l) {
            for (int v = lp[l] + lane; v < lp[l + 1]; v += 32)
                mismatch |= update_pair<VARIANT, SPLIT, FULL>(a, m, PiS, vars[v], v, t[0], t[1], a.alpha);
            __syncwarp();
        }
        const bool bad[2] = {__any_sync(0xffffffffu, mismatch & 1u) != 0, __any_sync(0xffffffffu, mismatch & 2u) != 0};
#pragma unroll
        for (int x = 0; x < 2; ++x) {
            if (!live[x]) continue;
            if (bad[x] && t[x] < a.max_iter) {
                ++t[x];
                continue;
            }
            // the shot stops: converged at sweep t, or max_iter sweeps without
            for (int v = lane; v < a.N; v += 32)
                a.est[(size_t)shot[x] * a.N + vars[v].j] = (uint8_t)(m.qb[2 * v + x] >> 4);
            if (lane == 0) {
                a.conv[shot[x]] = (uint8_t)(bad[x] ? 0 : 1);
                a.iters[shot[x]] = (uint8_t)t[x];
            }
            int s = 0;
            if (lane == 0) s = (int)atomicAdd(a.work, 1u);
            shot[x] = __shfl_sync(0xffffffffu, s, 0);
            live[x] = shot[x] < a.B;
            t[x] = 1;
            __syncwarp();
            if (live[x]) start_pair_shot<VARIANT, SPLIT>(a, m, PiS, vars, lane, x, shot[x]);
            __syncwarp();
        }
    }
}

using SerialKernelFn = void (*)(const SerialArgs);
// The one-shot-per-warp kernels (serial.cu) and the two-shot ones
// (serial_pair.cu) of a variant; split: the code has the split layout.
SerialKernelFn pick_serial(int variant, bool trace, bool split);
SerialKernelFn pick_serial_pair(int variant, int layout);  // layout: 0 generic, 1 split, 2 split without padding

}  // namespace sk

// Two shots per warp are chosen automatically from this many shots per
// resident one-shot warp (where shared memory holds kSerialPairWarps
// two-shot warps per SM; planar d = 7 on GB300: 1.14e8 one-shot against
// 1.23e8 two-shot EWAInit-BP shots/s at 1e6 shots, 7.0e7 against 6.3e7 at 1e5).
constexpr long kSerialPairShots = 128;

}  // namespace bpq
