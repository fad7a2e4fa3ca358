// Launch-shape selection and launch of the decode kernel (the kernel itself
// is in decode_kernel.cuh, instantiated per variant in decode_<variant>.cu).
#include <cuda_runtime.h>

#include "bpq_internal.h"
#include "decode_launch.h"

namespace bpq {

namespace {

int state_arrays(int variant) { return decode_state_arrays(variant); }

DecodeKernelFn pick(int variant, int npt, bool trace, int layout) {
    const bool split = layout != 0, full = layout == 2 && !trace;
    switch (variant) {
        case BPQ_PLAIN: return full ? pick_plain_full(npt) : pick_plain(npt, trace, split);
        case BPQ_MOMENTUM: return full ? pick_momentum_full(npt) : pick_momentum(npt, trace, split);
        case BPQ_ADAGRAD: return full ? pick_adagrad_full(npt) : pick_adagrad(npt, trace, split);
        case BPQ_EWAINIT: return full ? pick_ewainit_full(npt) : pick_ewainit(npt, trace, split);
        case BPQ_AEWA: return full ? pick_aewa_full(npt) : pick_aewa(npt, trace, split);
    }
    return nullptr;
}

DecodeKernelFn pick_pair(int variant, int npt, int layout) {
    const bool full = layout == 2;
    switch (variant) {
        case BPQ_PLAIN: return full ? pick_plain_pair_full(npt) : pick_plain_pair(npt);
        case BPQ_MOMENTUM: return full ? pick_momentum_pair_full(npt) : pick_momentum_pair(npt);
        case BPQ_ADAGRAD: return full ? pick_adagrad_pair_full(npt) : pick_adagrad_pair(npt);
        case BPQ_EWAINIT: return full ? pick_ewainit_pair_full(npt) : pick_ewainit_pair(npt);
    }
    return nullptr;
}

}  // namespace

bool decode_uses_pairs(const bpq_tanner *t, int variant, bool trace) {
    if (trace || !t->split || variant < BPQ_PLAIN || variant > BPQ_EWAINIT) return false;
    if (t->shots_per_thread == 1) return false;
    if (t->shots_per_thread == 2) return true;
    // automatic: where the stored launch shape fits two shots per thread
    LaunchShape s;
    const std::string keep = bpq_last_error();
    const bool fits = decode_pair_shape(t, variant, &s) == BPQ_OK;
    set_error(keep);
    return fits;
}

int decode_pair_shape(const bpq_tanner *t, int variant, LaunchShape *s) {
    const int nodes = t->N > t->M ? t->N : t->M;
    int T = t->threads_per_shot;
    if (T <= 0) T = (((nodes + 1) / 2 + 31) / 32) * 32;  // two nodes per thread
    if (T % 32 || T < 32 || T > kMaxThreadsPerShot)
        return fail(BPQ_EINVAL, "threads per shot group must be a multiple of 32 in [32, 1024]");
    const int npt = (nodes + T - 1) / T;
    if (npt > 2) return fail(BPQ_EINVAL, "two shots per thread take at most two nodes per thread");
    const int max_groups = T == 32 ? kMaxPairGroupsPerCta : 15;
    int gpc = t->shots_per_cta;
    if (gpc <= 0) gpc = 256 / T > 0 ? 256 / T : 1;  // about 256 threads per CTA
    if (gpc > max_groups) gpc = max_groups;
    while (gpc > 1 && gpc * T > 1024) --gpc;
    s->T = T;
    s->G = T / 32;
    s->npt = npt;
    s->groups_per_cta = gpc;
    s->n_pad = (t->N + 3) & ~3;
    s->slots_floats = (uint32_t)(4 * s->n_pad + 4);  // float2 slots
    const int nstate = state_arrays(variant);
    // per group: two vote words (16 bytes) | float2 slots | float2 state
    s->group_bytes = (uint32_t)(16 + 8 * s->slots_floats + 8 * nstate * s->n_pad);
    // table | Pi [3][n_pad] | initial messages [4 n_pad] | groups
    s->smem = kSmemHeader + t->table.size() + (size_t)28 * s->n_pad + (size_t)gpc * s->group_bytes;
    if (s->smem > 227 * 1024) return fail(BPQ_EINVAL, "shared memory of the launch shape exceeds 227 KB");
    return BPQ_OK;
}

int decode_launch_shape(const bpq_tanner *t, int variant, LaunchShape *s) {
    const int nodes = t->N > t->M ? t->N : t->M;
    int T = t->threads_per_shot;
    if (T <= 0) T = (((nodes + 1) / 2 + 31) / 32) * 32;  // two nodes per thread
    if (T % 32 || T < 32 || T > kMaxThreadsPerShot)
        return fail(BPQ_EINVAL, "threads per shot must be a multiple of 32 in [32, 1024]");
    const int npt = (nodes + T - 1) / T;
    if (npt > kMaxNodesPerThread) return fail(BPQ_EINVAL, "too few threads per shot for this code");
    if (npt > 2 && T > 512) return fail(BPQ_EINVAL, "more than two nodes per thread needs at most 512 threads");
    // one-warp groups synchronise with __syncwarp; larger groups take one of
    // the 15 named barriers
    const int max_groups = T == 32 ? kMaxGroupsPerCta : 15;
    const int max_threads = npt <= 2 ? 1024 : 512;
    int gpc = t->shots_per_cta;
    if (gpc <= 0) gpc = 256 / T > 0 ? 256 / T : 1;  // about 256 threads per CTA
    if (gpc > max_groups) gpc = max_groups;
    while (gpc > 1 && gpc * T > max_threads) --gpc;
    s->T = T;
    s->G = T / 32;
    s->npt = npt;
    s->groups_per_cta = gpc;
    s->n_pad = (t->N + 3) & ~3;
    // message slots (+ zero and trash slots), state
    s->slots_floats = (uint32_t)(4 * s->n_pad + 4);
    const int nstate = state_arrays(variant < 0 ? BPQ_MOMENTUM : variant);
    s->group_bytes = (uint32_t)(4 * s->slots_floats + 4 * nstate * s->n_pad);
    s->smem = kSmemHeader + t->table.size() + (size_t)12 * s->n_pad + (size_t)gpc * s->group_bytes;
    if (s->smem > 227 * 1024) return fail(BPQ_EINVAL, "shared memory of the launch shape exceeds 227 KB");
    return BPQ_OK;
}

namespace {
// Shape of a code in the batched kernel with npt (1 or 2) nodes per thread:
// the fewest threads per shot group that cover max(N, M), and as many shot
// groups as fit in kBatchThreads threads and 227 KB of shared memory.
int batch_shape_npt(const bpq_tanner *t, int variant, int npt, LaunchShape *s) {
    const int nodes = t->N > t->M ? t->N : t->M;
    const int T = (((nodes + npt - 1) / npt + 31) / 32) * 32;
    if (T > kBatchThreads) return fail(BPQ_EINVAL, "code too large for the batched kernel");
    const int max_groups = T == 32 ? kMaxGroupsPerCta : 15;
    int gpc = kBatchThreads / T;
    if (gpc > max_groups) gpc = max_groups;
    s->T = T;
    s->G = T / 32;
    s->npt = npt;
    s->n_pad = (t->N + 3) & ~3;
    s->slots_floats = (uint32_t)(4 * s->n_pad + 4);
    const int nstate = state_arrays(variant);
    s->group_bytes = (uint32_t)(4 * s->slots_floats + 4 * nstate * s->n_pad);
    const size_t fixed = kSmemHeader + kDescBytes + t->table.size() + (size_t)12 * s->n_pad;
    while (gpc > 1 && fixed + (size_t)gpc * s->group_bytes > 227 * 1024) --gpc;
    s->groups_per_cta = gpc;
    s->smem = fixed + (size_t)gpc * s->group_bytes;
    if (s->smem > 227 * 1024) return fail(BPQ_EINVAL, "a code of the batch needs more than 227 KB of shared memory");
    return BPQ_OK;
}
}  // namespace

int decode_batch_shape(const bpq_tanner *t, int variant, LaunchShape *s) {
    if (t->batch_nodes_per_thread > 0) return batch_shape_npt(t, variant, t->batch_nodes_per_thread, s);
    // automatic: the node count per thread that keeps the most node slots of
    // a CTA busy (groups x nodes / (npt x kBatchThreads)); on a tie two nodes
    // per thread, whose twice as many groups balance the item's shots better
    LaunchShape one, two;
    const std::string keep = bpq_last_error();
    const int rc1 = batch_shape_npt(t, variant, 1, &one);
    const int rc2 = batch_shape_npt(t, variant, 2, &two);
    if (rc2) {
        if (rc1) return rc2;
        *s = one;
    } else {
        *s = !rc1 && 2 * one.groups_per_cta > two.groups_per_cta ? one : two;
    }
    set_error(keep);
    return BPQ_OK;
}

int decode_launch(const bpq_tanner *t, DecodeArgs &a, int variant, bool trace, cudaStream_t st, int *ctas_out) {
    LaunchShape s;
    bool pairs = decode_uses_pairs(t, variant, trace);
    if (pairs && t->shots_per_thread == 0) {
        // automatic choice: a pair's iteration does two shots' work, so a
        // batch's tail (its slowest shots) runs longer; pairing pays only
        // once each resident one-shot group would decode many shots.
        // Measured on GB300 (EWAInit-BP): toric d = 15 pairs win from 65536
        // shots, planar d = 25 from 16384, both about 100 shots per resident
        // one-shot group; planar d = 9 breaks even at 262144 (172 per group)
        LaunchShape one;
        int per_sm = 0;
        DecodeKernelFn f1 = nullptr;
        if (decode_launch_shape(t, variant, &one) == BPQ_OK && (f1 = pick(variant, one.npt, false, a.split)) &&
            cudaFuncSetAttribute(f1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)one.smem) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f1, one.T * one.groups_per_cta, one.smem) ==
                cudaSuccess &&
            (long)a.B < kPairShotsPerGroup * (long)per_sm * t->num_sms * one.groups_per_cta)
            pairs = false;
    }
    int rc = pairs ? decode_pair_shape(t, variant, &s) : decode_launch_shape(t, variant, &s);
    if (rc) return rc;
    DecodeKernelFn fn = nullptr;
    if (t->debug_checks) {
        fn = trace ? nullptr : pick_debug(variant, s.npt, pairs, a.split);
        if (!fn)
            return fail(BPQ_EINVAL, "no bounds-checked kernel for this launch (plain, Momentum, AdaGrad or EWAInit BP, "
                                    "at most two nodes per thread, not a trace)");
    } else {
        fn = pairs ? pick_pair(variant, s.npt, a.split) : pick(variant, s.npt, trace, a.split);
    }
    if (!fn) return fail(BPQ_EINVAL, "no kernel for this variant (AEWA-BP has no trace mode)");
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
    if (e != cudaSuccess) return fail(BPQ_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    const int threads = s.T * s.groups_per_cta;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, s.smem);
    if (e != cudaSuccess || per_sm < 1) return fail(BPQ_ECUDA, "launch shape does not fit on an SM");
    long ctas = (long)per_sm * t->num_sms;
    const long per_cta = (long)s.groups_per_cta * (pairs ? 2 : 1);
    const long need = (a.B + per_cta - 1) / per_cta;
    if (ctas > need) ctas = need;
    if (ctas < 1) ctas = 1;
    a.G = s.G;
    a.n_pad = s.n_pad;
    a.slots_floats = s.slots_floats;
    a.group_bytes = s.group_bytes;
    if (ctas_out) *ctas_out = (int)ctas;
    fn<<<(unsigned)ctas, threads, s.smem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(BPQ_ECUDA, std::string("decode launch: ") + cudaGetErrorString(e));
    return BPQ_OK;
}

}  // namespace bpq
