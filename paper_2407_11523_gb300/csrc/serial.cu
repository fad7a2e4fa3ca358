// Host side of the serial-schedule decoders (serial_kernel.cuh) and the
// one-shot-per-warp kernels; the two-shots-per-warp kernels are instantiated
// in serial_pair.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "serial_kernel.cuh"

namespace bpq {
namespace sk {

SerialKernelFn pick_serial(int variant, bool trace, bool split) {
#define BPQ_SERIAL_CASE(V)                                                                   \
    case V:                                                                                  \
        return trace ? (split ? serial_kernel<V, true, true> : serial_kernel<V, true, false>) \
                     : (split ? serial_kernel<V, false, true> : serial_kernel<V, false, false>);
    switch (variant) {
        BPQ_SERIAL_CASE(BPQ_PLAIN)
        BPQ_SERIAL_CASE(BPQ_MOMENTUM)
        BPQ_SERIAL_CASE(BPQ_ADAGRAD)
        BPQ_SERIAL_CASE(BPQ_EWAINIT)
    }
#undef BPQ_SERIAL_CASE
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
    a.table_bytes = t->serial_off_canon;
    a.off_levels = t->serial_off_levels;
    a.off_canon = t->serial_off_canon;
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
    a.zero_slot = (uint32_t)t->serial_slots;
    a.msg_floats = (a.zero_slot + 2u + 3u) & ~3u;
    // one shot per warp: messages | state | syndrome words | qubit bytes;
    // two: the same with float2 slots, two syndromes and two bytes per qubit
    const uint32_t state_floats = (uint32_t)(sk::serial_state_arrays(variant) * a.n_pad);
    const uint32_t W4 = (uint32_t)((a.W + 3) & ~3);
    auto layout = [&](uint32_t k) {
        a.off_syn = 4u * k * (a.msg_floats + state_floats);
        a.syn_stride = W4;
        a.off_qb = a.off_syn + 4u * k * W4;
        a.warp_bytes = (a.off_qb + k * (uint32_t)a.n_pad + 15u) & ~15u;
    };
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
    layout(1);
    if (fixed + a.warp_bytes > limit) return fail(BPQ_EINVAL, "code too large for the serial kernel's shared memory");
    const long warps1 = (long)std::min<size_t>(32, (limit - fixed) / a.warp_bytes);
    // two shots per warp (not for traces): on request, or automatically where
    // shared memory still holds kSerialPairWarps two-shot warps per SM and the
    // batch gives every resident one-shot warp kSerialPairShots shots.  The
    // kernel is latency-bound: with fewer warps the two-shot kernel's shorter
    // instruction stream per shot does not make up for the lost warps (toric
    // d = 15 on GB300: 7 two-shot warps, 2.26e7 against 2.53e7 shots/s at
    // 1e5 shots, 3.2e7 against 3.3e7 at 1e6), and small batches, whose time
    // is set by their slowest shots, finish sooner with one shot per warp.
    bool pairs = false;
    if (!trace) {
        layout(2);
        const bool fits = fixed + a.warp_bytes <= limit;
        const int k = t->serial_shots_per_warp;
        if (k == 2 && !fits) return fail(BPQ_EINVAL, "two shots per warp do not fit in shared memory for this code");
        const bool full_occupancy = fits && (limit - fixed) / a.warp_bytes >= (size_t)sk::kSerialPairWarps;
        pairs = fits && (k == 2 || (k == 0 && full_occupancy && (long)B >= kSerialPairShots * warps1 * t->num_sms));
        if (!pairs) layout(1);
    }
    int warps = (int)std::min<size_t>(pairs ? sk::kSerialPairWarps : 32, (limit - fixed) / a.warp_bytes);
    const size_t smem = fixed + (size_t)warps * a.warp_bytes;
    sk::SerialKernelFn fn = pairs ? sk::pick_serial_pair(variant, t->full ? 2 : t->split ? 1 : 0)
                                  : sk::pick_serial(variant, trace, t->split);
    if (!fn) return fail(BPQ_EINVAL, "no serial kernel for this variant");
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail(BPQ_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, warps * 32, smem);
    if (e != cudaSuccess || per_sm < 1) return fail(BPQ_ECUDA, "serial kernel does not fit on an SM");
    long ctas = (long)per_sm * t->num_sms;
    const long per_cta = (long)warps * (pairs ? 2 : 1);
    const long need = (B + per_cta - 1) / per_cta;
    if (ctas > need) ctas = need;
    rc = cuda_check(cudaMemsetAsync(work, 0, 8, st), "workspace reset");
    if (rc) return rc;
    fn<<<(unsigned)std::max(1L, ctas), warps * 32, smem, st>>>(a);
    return cuda_check(cudaGetLastError(), "serial decode launch");
}

}  // namespace
}  // namespace bpq

using bpq::fail;

extern "C" {

int bpq_decode_serial(const bpq_tanner *t, const uint32_t *syn_dev, const float *prior_dev, int variant,
                      const bpq_params *params, int max_iter, int B, uint8_t *est_dev, uint8_t *conv_dev,
                      uint8_t *iters_dev, void *work_dev, void *stream) {
    return bpq::serial_launch(t, syn_dev, prior_dev, variant, params, max_iter, B, work_dev, false, est_dev, conv_dev,
                              iters_dev, nullptr, nullptr, nullptr, nullptr, static_cast<cudaStream_t>(stream));
}

int bpq_set_serial_shots_per_warp(bpq_tanner *t, int shots_per_warp) {
    if (!t) return fail(BPQ_EINVAL, "tanner is NULL");
    if (shots_per_warp < 0 || shots_per_warp > 2) return fail(BPQ_EINVAL, "shots per warp must be 0, 1 or 2");
    t->serial_shots_per_warp = shots_per_warp;
    return BPQ_OK;
}

int bpq_decode_serial_trace(const bpq_tanner *t, const uint32_t *syn_dev, const float *prior_dev, int variant,
                            const bpq_params *params, int T, int B, float *m_v2c_dev, float *m_c2v_dev, float *Q_dev,
                            uint8_t *dec_dev, void *work_dev, void *stream) {
    return bpq::serial_launch(t, syn_dev, prior_dev, variant, params, T, B, work_dev, true, nullptr, nullptr, nullptr,
                              m_v2c_dev, m_c2v_dev, Q_dev, dec_dev, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
