// Serial-schedule decoding (bpq_decode_serial, bpq_decode_serial_trace):
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
// 2L qubits each.  One warp decodes one shot: its lanes take the qubits of a
// level, then __syncwarp, level after level; the shot's edge messages (one
// float per check-major edge, plus a zero slot), variant state, decisions
// and syndrome sit in the warp's shared memory, and the per-qubit tables
// (edges, their checks and the checks' other edges, ordered by level) are
// staged once per CTA by a bulk TMA copy.  Persistent CTAs; warps take shots
// from an atomic queue.
//
// Arithmetic is that of the parallel kernel (decode_kernel.cuh): v->c
// messages stored as sign * delta (AdaGrad-BP: sign * phi) with the
// decision's anticommutation bit in the least significant bit,
// log-likelihoods in bits, and the syndrome test after each sweep reads the
// parity of each check from those bits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "bpq_internal.h"
#include "decode_kernel.cuh"
#include "decode_launch.h"

namespace bpq {

struct SerialArgs {
    const uint8_t *table;  // SerialVar[N] | level_ptr u16[L+1] | chk_ptr u16[M+1] (bpq_tanner::serial)
    uint32_t table_bytes, off_levels, off_chkptr;
    int nlevels;
    const uint32_t *syn;   // [B][W]
    const float *prior;    // [N][3]
    uint8_t *est, *conv, *iters;
    uint32_t *work;        // [0] next shot, [1] device error word
    float *tr_v2c, *tr_c2v, *tr_Q;
    uint8_t *tr_dec;
    int N, M, E, W, B, max_iter;
    int n_pad;             // N rounded up to 4 (state array stride)
    uint32_t msg_floats;   // E + 1 rounded up to 4
    uint32_t warp_bytes;   // shared memory of one warp: messages | state | syndrome | decisions
    uint32_t off_syn, off_est;  // byte offsets inside a warp's region
    float alpha, gamma, eps, clip, clip2, delta_clip, phi_clip;
    int ada_from1;
};

namespace sk {

using namespace dk;

// Per-qubit state arrays (each n_pad floats) of the serial kernel in a warp's
// shared memory: EWAInit Q^(t-1); Momentum Q^(t-1), g; AdaGrad Q^(t-1), G.
// The kernel and serial_launch's sizing both read this.
__host__ __device__ constexpr int serial_state_arrays(int variant) {
    return variant == BPQ_PLAIN ? 0 : variant == BPQ_EWAINIT ? 3 : 6;
}

// Shared memory of one warp: messages | state | syndrome words | decisions.
struct WarpMem {
    float *msg, *state;
    uint32_t *syn;
    uint8_t *est;
};

__device__ __forceinline__ WarpMem warp_mem(const SerialArgs &a, uint8_t *base, int warp) {
    WarpMem m;
    uint8_t *p = base + (size_t)warp * a.warp_bytes;
    m.msg = reinterpret_cast<float *>(p);
    m.state = m.msg + a.msg_floats;
    m.syn = reinterpret_cast<uint32_t *>(p + a.off_syn);
    m.est = p + a.off_est;
    return m;
}

// The four edge Paulis of a qubit one per byte (anti_bytes' format).
__device__ __forceinline__ uint32_t pauli_bytes(uint32_t pauli) {
    return (pauli & 3u) | (((pauli >> 2) & 3u) << 8) | (((pauli >> 4) & 3u) << 16) | (((pauli >> 6) & 3u) << 24);
}

// v->c messages of one qubit from its posterior (bits) and its incoming
// c->v messages win (bits), written to the qubit's edges: sign * delta
// (sign * phi with PHI), the least significant bit replaced by byte k of ab.
// With TRACE, the natural-log message lambda goes to tr_v2c at sweep t.
template <bool TRACE, bool PHI>
__device__ __forceinline__ void send_v2c(const SerialArgs &a, float *msg, const SerialVar &sv, int t, int shot,
                                         float QX, float QY, float QZ, const float (&win)[4], uint32_t ab) {
    const float c0 = fminf(0.f, fminf(QX, fminf(QY, QZ)));
    const float e0 = ex2(c0);
    const float eX = ex2(c0 - QX), eY = ex2(c0 - QY), eZ = ex2(c0 - QZ);
    const float CX = e0 + eX, CY = e0 + eY, CZ = e0 + eZ;
    const float AX = eY + eZ, AY = eX + eZ, AZ = eX + eY;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k >= sv.deg) break;
        const uint32_t p = (sv.pauli >> (2 * k)) & 3u;
        const float C = p == 1u ? CX : p == 2u ? CY : CZ;
        const float Ab = p == 1u ? AX : p == 2u ? AY : AZ;
        const float A = Ab * ex2(win[k]);
        float dl;
        if (PHI) {
            const float mx = fmaxf(C, A), mn = fminf(C, A);
            dl = fmaxf(log1p_rel(2.0f * mn * rcp(mx - mn)), a.phi_clip);
        } else {
            dl = fmaxf(2.0f * fminf(C, A) * rcp(C + A), a.delta_clip);
        }
        const uint32_t bits = (__float_as_uint(dl) & ~1u) | ((ab >> (8 * k)) & 1u) | (A > C ? 0x80000000u : 0u);
        msg[sv.own[k]] = __uint_as_float(bits);
        if (TRACE && a.tr_v2c) {
            const float lam = fminf(fmaxf(kLn2 * (lg2(C) - lg2(A)), -a.clip), a.clip);
            a.tr_v2c[((size_t)shot * (a.max_iter + 1) + t) * a.E + sv.own[k]] = lam;
        }
    }
}

// The update of one qubit at its turn in sweep t (t >= 1): c->v messages of
// its checks (eq. (h_update), from the messages as they stand), posterior
// of the variant, decision, new v->c messages.
template <int VARIANT, bool TRACE>
__device__ __forceinline__ void update_qubit(const SerialArgs &a, const WarpMem &m, const float *PiS,
                                             const SerialVar &sv, int t, int shot, float alpha) {
    constexpr bool PHI = PhiForm<VARIANT>::value;
    const int j = sv.j, Np = a.n_pad;
    float win[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k >= sv.deg) break;
        const uint32_t u0 = __float_as_uint(m.msg[sv.oth[k][0]]), u1 = __float_as_uint(m.msg[sv.oth[k][1]]),
                       u2 = __float_as_uint(m.msg[sv.oth[k][2]]);
        const uint32_t i = sv.chk[k];
        const uint32_t sb = (m.syn[i >> 5] >> (i & 31)) & 1u;
        const uint32_t sgn = (u0 ^ u1 ^ u2 ^ (sb << 31)) & 0x80000000u;
        const float m0 = __uint_as_float(u0 & 0x7FFFFFFEu), m1 = __uint_as_float(u1 & 0x7FFFFFFEu),
                    m2 = __uint_as_float(u2 & 0x7FFFFFFEu);
        const float w = fminf(PHI ? phi_check(m0 + m1 + m2) : c2v_magnitude(oplus(oplus(m0, m1), m2)), a.clip2);
        win[k] = __uint_as_float(__float_as_uint(w) ^ sgn);
        if (TRACE && a.tr_c2v) a.tr_c2v[((size_t)shot * a.max_iter + (t - 1)) * a.E + sv.own[k]] = kLn2 * win[k];
    }
    float S[3];
    anticommuting_sums(sv.pauli, win, S[0], S[1], S[2]);
    const float Pi[3] = {PiS[j], PiS[Np + j], PiS[2 * Np + j]};
    float *state = m.state;
    float Q[3];
#pragma unroll
    for (int w = 0; w < 3; ++w) {
        if (VARIANT == BPQ_PLAIN) {
            Q[w] = Pi[w] + S[w];  // eq. (p_update)
        } else if (VARIANT == BPQ_EWAINIT) {
            // eq. (EWAInit) for qubit j at its turn
            const float qp = state[w * Np + j];
            Q[w] = (t > 1 ? alpha * Pi[w] + (1.f - alpha) * qp : Pi[w]) + S[w];
            state[w * Np + j] = Q[w];
        } else if (VARIANT == BPQ_MOMENTUM) {
            // eqs. (mombp1), (mombp2)
            const float qp = state[w * Np + j];
            const float g = a.gamma * state[(3 + w) * Np + j] + (1.f - a.gamma) * (qp - Pi[w] - S[w]);
            Q[w] = qp - a.alpha * g;
            state[w * Np + j] = Q[w];
            state[(3 + w) * Np + j] = g;
        } else {
            // eq. (boost) from t = 2; G accumulates g'^2
            const float qp = state[w * Np + j];
            const float gp = qp - Pi[w] - S[w];
            float Gs = state[(3 + w) * Np + j];
            if (t >= 2 || a.ada_from1) Gs += gp * gp;
            Q[w] = t == 1 ? Pi[w] + S[w] : qp - a.alpha * gp * rcp(sqrt_approx(Gs) + a.eps);
            state[w * Np + j] = Q[w];
            state[(3 + w) * Np + j] = Gs;
        }
    }
    uint32_t d;
    if (Q[0] > 0.f && Q[1] > 0.f && Q[2] > 0.f) {
        d = 0;
    } else {
        d = 1;
        float mq = Q[0];
        if (Q[1] < mq) { d = 2; mq = Q[1]; }
        if (Q[2] < mq) d = 3;
    }
    m.est[j] = (uint8_t)d;
    if (TRACE) {
        const size_t o = (size_t)shot * a.max_iter + (t - 1);
        if (a.tr_Q) {
            a.tr_Q[(o * a.N + j) * 3 + 0] = kLn2 * Q[0];
            a.tr_Q[(o * a.N + j) * 3 + 1] = kLn2 * Q[1];
            a.tr_Q[(o * a.N + j) * 3 + 2] = kLn2 * Q[2];
        }
        if (a.tr_dec) a.tr_dec[o * a.N + j] = (uint8_t)d;
    }
    send_v2c<TRACE, PHI>(a, m.msg, sv, t, shot, Q[0], Q[1], Q[2], win, anti_bytes(d, pauli_bytes(sv.pauli)));
}

// Decode one shot with one warp: eq. (init), then sweeps level by level
// until the decisions satisfy the syndrome (tested after every sweep) or
// max_iter sweeps have run (TRACE: always max_iter sweeps).
template <int VARIANT, bool TRACE>
__device__ __forceinline__ void decode_serial_shot(const SerialArgs &a, const WarpMem &m, const float *PiS,
                                                   const SerialVar *vars, const uint16_t *lp, const uint16_t *cp,
                                                   int lane, int shot) {
    constexpr bool PHI = PhiForm<VARIANT>::value;
    const int N = a.N, M = a.M, Np = a.n_pad;
    for (int w = lane; w < a.W; w += 32) m.syn[w] = __ldg(a.syn + (size_t)shot * a.W + w);
    // eq. (init): lambda(Pi^(0)) on every edge; Q^(0) = Pi^(0), g^(0) = G^(0) = 0
    for (int v = lane; v < N; v += 32) {
        const SerialVar sv = vars[v];
        const int j = sv.j;
        const float PX = PiS[j], PY = PiS[Np + j], PZ = PiS[2 * Np + j];
        if (serial_state_arrays(VARIANT) >= 3) {
            m.state[j] = PX;
            m.state[Np + j] = PY;
            m.state[2 * Np + j] = PZ;
        }
        if (serial_state_arrays(VARIANT) == 6) {
            m.state[3 * Np + j] = 0.f;
            m.state[4 * Np + j] = 0.f;
            m.state[5 * Np + j] = 0.f;
        }
        const float z4[4] = {0.f, 0.f, 0.f, 0.f};
        send_v2c<TRACE, PHI>(a, m.msg, sv, 0, shot, PX, PY, PZ, z4, 0u);
    }
    __syncwarp();
    int conv = 0, iters = a.max_iter;
    for (int t = 1; t <= a.max_iter; ++t) {
        for (int l = 0; l < a.nlevels; ++l) {
            for (int v = lp[l] + lane; v < lp[l + 1]; v += 32)
                update_qubit<VARIANT, TRACE>(a, m, PiS, vars[v], t, shot, a.alpha);
            __syncwarp();
        }
        if (TRACE) continue;
        // <H, E^> = s from the decision bits carried by the messages
        uint32_t mismatch = 0;
        for (int i = lane; i < M; i += 32) {
            uint32_t par = (m.syn[i >> 5] >> (i & 31)) & 1u;
            for (int e = cp[i]; e < cp[i + 1]; ++e) par ^= __float_as_uint(m.msg[e]) & 1u;
            mismatch |= par;
        }
        if (!__any_sync(0xffffffffu, mismatch)) {
            conv = 1;
            iters = t;
            break;
        }
    }
    if (!TRACE || a.est)
        for (int j = lane; j < N; j += 32) a.est[(size_t)shot * N + j] = m.est[j];
    if (lane == 0 && (!TRACE || a.conv)) {
        a.conv[shot] = (uint8_t)conv;
        a.iters[shot] = (uint8_t)iters;
    }
    __syncwarp();
}

// Persistent kernel: the CTA stages the serial table (bulk TMA) and the
// prior LLRs (bits) once; each warp then decodes shots from the queue.
template <int VARIANT, bool TRACE>
__global__ void __launch_bounds__(1024, 1) serial_kernel(const SerialArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);
    uint8_t *tab = smem + 128;
    float *PiS = reinterpret_cast<float *>(tab + a.table_bytes);
    uint8_t *wbase = reinterpret_cast<uint8_t *>(PiS + 3 * a.n_pad);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const WarpMem m = warp_mem(a, wbase, warp);

    if (tid == 0) {
        mbar_init(mbar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(mbar, a.table_bytes);
        bulk_g2s(tab, a.table, a.table_bytes, mbar);
    }
    const int Np = a.n_pad;
    for (int j = tid; j < a.N; j += blockDim.x) {
        const float px = a.prior[3 * j], py = a.prior[3 * j + 1], pz = a.prior[3 * j + 2];
        const float pI = 1.0f - px - py - pz;
        PiS[j] = log2f(pI / px);
        PiS[Np + j] = log2f(pI / py);
        PiS[2 * Np + j] = log2f(pI / pz);
    }
    if (lane == 0) m.msg[a.E] = 0.f;  // the zero slot
    const bool staged = mbar_wait_bounded(mbar, 0, 1u << 22);
    if (__syncthreads_or(!staged)) {
        if (tid == 0) atomicExch(a.work + 1, 1u);
        mbar_wait_bounded(mbar, 0, 1u << 22);
        return;
    }
    const SerialVar *vars = reinterpret_cast<const SerialVar *>(tab);
    const uint16_t *lp = reinterpret_cast<const uint16_t *>(tab + a.off_levels);
    const uint16_t *cp = reinterpret_cast<const uint16_t *>(tab + a.off_chkptr);
    for (;;) {
        int shot = 0;
        if (lane == 0) shot = (int)atomicAdd(a.work, 1u);
        shot = __shfl_sync(0xffffffffu, shot, 0);
        if (shot >= a.B) break;
        decode_serial_shot<VARIANT, TRACE>(a, m, PiS, vars, lp, cp, lane, shot);
    }
}

using SerialKernelFn = void (*)(const SerialArgs);

SerialKernelFn pick_serial(int variant, bool trace) {
    switch (variant * 2 + (trace ? 1 : 0)) {
        case 0: return serial_kernel<BPQ_PLAIN, false>;
        case 1: return serial_kernel<BPQ_PLAIN, true>;
        case 2: return serial_kernel<BPQ_MOMENTUM, false>;
        case 3: return serial_kernel<BPQ_MOMENTUM, true>;
        case 4: return serial_kernel<BPQ_ADAGRAD, false>;
        case 5: return serial_kernel<BPQ_ADAGRAD, true>;
        case 6: return serial_kernel<BPQ_EWAINIT, false>;
        case 7: return serial_kernel<BPQ_EWAINIT, true>;
    }
    return nullptr;
}

}  // namespace sk

namespace {

// Validate, fill the arguments from the parallel decoder's (parameters in
// the kernel's units) and launch.
int serial_launch(const bpq_tanner *t, const uint32_t *syn, const float *prior, int variant, const bpq_params *params,
                  int max_iter, int B, void *work, bool trace, uint8_t *est, uint8_t *conv, uint8_t *iters,
                  float *tr_v2c, float *tr_c2v, float *tr_Q, uint8_t *tr_dec, cudaStream_t st) {
    int rc = need_uploaded(t);
    if (rc) return rc;
    if (variant < BPQ_PLAIN || variant > BPQ_EWAINIT)
        return fail(BPQ_EINVAL, "the serial schedule takes plain, Momentum, AdaGrad or EWAInit BP");
    DecodeArgs d;
    rc = fill_decode_args(t, syn, prior, variant, params, max_iter, B, work, d);
    if (rc) return rc;
    if (B == 0) return BPQ_OK;
    if (!trace && (!est || !conv || !iters)) return fail(BPQ_EINVAL, "NULL output");
    SerialArgs a;
    std::memset(&a, 0, sizeof a);
    a.table = t->d_serial;
    a.table_bytes = (uint32_t)t->serial.size();
    a.off_levels = t->serial_off_levels;
    a.off_chkptr = t->serial_off_chkptr;
    a.nlevels = t->serial_levels;
    a.syn = syn;
    a.prior = prior;
    a.est = est;
    a.conv = conv;
    a.iters = iters;
    a.work = static_cast<uint32_t *>(work);
    a.tr_v2c = tr_v2c;
    a.tr_c2v = tr_c2v;
    a.tr_Q = tr_Q;
    a.tr_dec = tr_dec;
    a.N = t->N;
    a.M = t->M;
    a.E = t->E;
    a.W = (t->M + 31) / 32;
    a.B = B;
    a.max_iter = max_iter;
    a.n_pad = (t->N + 3) & ~3;
    a.msg_floats = (uint32_t)((t->E + 1 + 3) & ~3);
    const uint32_t state_bytes = 4u * (uint32_t)(sk::serial_state_arrays(variant) * a.n_pad);
    a.off_syn = 4u * a.msg_floats + state_bytes;
    a.off_est = a.off_syn + 4u * (uint32_t)((a.W + 3) & ~3);
    a.warp_bytes = (a.off_est + (uint32_t)t->N + 15u) & ~15u;
    a.alpha = d.alpha;
    a.gamma = d.gamma;
    a.eps = d.eps;
    a.clip = d.clip;
    a.clip2 = d.clip2;
    a.delta_clip = d.delta_clip;
    a.phi_clip = d.phi_clip;
    a.ada_from1 = d.ada_from1;

    const size_t fixed = 128 + a.table_bytes + (size_t)12 * a.n_pad;
    const size_t limit = 227 * 1024;
    if (fixed + a.warp_bytes > limit) return fail(BPQ_EINVAL, "code too large for the serial kernel's shared memory");
    int warps = (int)std::min<size_t>(32, (limit - fixed) / a.warp_bytes);
    const size_t smem = fixed + (size_t)warps * a.warp_bytes;
    sk::SerialKernelFn fn = sk::pick_serial(variant, trace);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail(BPQ_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, warps * 32, smem);
    if (e != cudaSuccess || per_sm < 1) return fail(BPQ_ECUDA, "serial kernel does not fit on an SM");
    long ctas = (long)per_sm * t->num_sms;
    const long need = (B + warps - 1) / warps;
    if (ctas > need) ctas = need;
    rc = cuda_check(cudaMemsetAsync(work, 0, 8, st), "workspace reset");
    if (rc) return rc;
    fn<<<(unsigned)std::max(1L, ctas), warps * 32, smem, st>>>(a);
    return cuda_check(cudaGetLastError(), "serial decode launch");
}

}  // namespace
}  // namespace bpq

extern "C" {

int bpq_decode_serial(const bpq_tanner *t, const uint32_t *syn_dev, const float *prior_dev, int variant,
                      const bpq_params *params, int max_iter, int B, uint8_t *est_dev, uint8_t *conv_dev,
                      uint8_t *iters_dev, void *work_dev, void *stream) {
    return bpq::serial_launch(t, syn_dev, prior_dev, variant, params, max_iter, B, work_dev, false, est_dev, conv_dev,
                              iters_dev, nullptr, nullptr, nullptr, nullptr, static_cast<cudaStream_t>(stream));
}

int bpq_decode_serial_trace(const bpq_tanner *t, const uint32_t *syn_dev, const float *prior_dev, int variant,
                            const bpq_params *params, int T, int B, float *m_v2c_dev, float *m_c2v_dev, float *Q_dev,
                            uint8_t *dec_dev, void *work_dev, void *stream) {
    return bpq::serial_launch(t, syn_dev, prior_dev, variant, params, T, B, work_dev, true, nullptr, nullptr, nullptr,
                              m_v2c_dev, m_c2v_dev, Q_dev, dec_dev, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
