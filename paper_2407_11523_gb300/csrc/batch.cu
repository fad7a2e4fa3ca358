// Batched decoding of many codes in one persistent launch (bpq_batch_*).
// The plan (per-item descriptors and each CTA's starting item) is built on
// the host and copied once into the caller's device workspace;
// bpq_batch_launch then only enqueues a counter reset and the kernel, so it
// can be captured in a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "bpq_internal.h"
#include "decode_launch.h"

using bpq::fail;

struct bpq_batch {
    int device = -1;
    void *work = nullptr;
    bpq::BatchKernelFn fn = nullptr;
    bpq::BatchArgs args{};
    size_t smem = 0;
    int ctas = 0, npt_max = 0;
    long shots = 0;
};

namespace bpq {

BatchKernelFn pick_batch_kernel(int variant, bool generic) {
    switch (variant) {
        case BPQ_PLAIN: return pick_plain_batch(generic);
        case BPQ_MOMENTUM: return pick_momentum_batch(generic);
        case BPQ_ADAGRAD: return pick_adagrad_batch(generic);
        case BPQ_EWAINIT: return pick_ewainit_batch(generic);
    }
    return nullptr;
}

void batch_start_items(const std::vector<double> &weight, int ctas, int *start) {
    const int n = (int)weight.size();
    double total = 0;
    for (double w : weight) total += w;
    int g = 0;
    double below = 0;  // total weight of the items before g
    for (int c = 0; c < ctas; ++c) {
        // CTA c starts at the item holding weight position (c + 1/2) / ctas
        const double pos = total > 0 ? (c + 0.5) / ctas * total : 0.0;
        while (g < n - 1 && (weight[g] == 0 || below + weight[g] <= pos)) below += weight[g++];
        start[c] = g;
    }
}

namespace {
size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
}  // namespace
}  // namespace bpq

extern "C" {

size_t bpq_batch_workspace_bytes(int n_items) {
    if (n_items < 1) return 0;
    return bpq::batch_counter_bytes(n_items) + bpq::align256(sizeof(bpq::DecodeArgs) * n_items) +
           bpq::align256(sizeof(int) * bpq::kMaxBatchCtas);
}

int bpq_batch_plan(const bpq_batch_item *items, int n_items, int variant, const bpq_params *params, int max_iter,
                   void *work_dev, size_t work_bytes, void *stream, bpq_batch **out) {
    if (!out) return fail(BPQ_EINVAL, "out is NULL");
    *out = nullptr;
    if (!items || n_items < 1) return fail(BPQ_EINVAL, "no batch items");
    if (max_iter < 1 || max_iter > 255) return fail(BPQ_EINVAL, "max_iter must be in [1, 255]");
    if (variant < BPQ_PLAIN || variant > BPQ_EWAINIT)
        return fail(BPQ_EINVAL, "the batched kernel takes plain, Momentum, AdaGrad or EWAInit BP");
    if (!work_dev) return fail(BPQ_EINVAL, "NULL workspace");
    if (bpq::misaligned(work_dev, bpq::kBufferAlign)) return fail(BPQ_EINVAL, "workspace not 16-byte aligned");
    const int device = items[0].tanner ? items[0].tanner->device : -1;
    long total = 0;
    for (int g = 0; g < n_items; ++g) {
        const bpq_tanner *t = items[g].tanner;
        if (!t || !t->dev_blob) return fail(BPQ_ESTATE, "batch item without an uploaded tanner");
        if (t->device != device) return fail(BPQ_ESTATE, "batch items on different devices");
        if (items[g].B < 0) return fail(BPQ_EINVAL, "negative shot count");
        if (items[g].B > 0 && (!items[g].syn_dev || !items[g].prior_dev || !items[g].est_dev ||
                               !items[g].conv_dev || !items[g].iters_dev))
            return fail(BPQ_EINVAL, "NULL input or output in a batch item");
        if (bpq::misaligned(items[g].syn_dev, bpq::kWordAlign) || bpq::misaligned(items[g].prior_dev, bpq::kWordAlign))
            return fail(BPQ_EINVAL, "a batch item's syndromes or prior not 4-byte aligned");
        total += items[g].B;
    }
    if (work_bytes < bpq_batch_workspace_bytes(n_items)) return fail(BPQ_EINVAL, "batch workspace too small");
    int rc = bpq::cuda_set_device(device);
    if (rc) return rc;

    std::vector<bpq::DecodeArgs> desc(n_items);
    std::vector<double> weight(n_items);
    size_t smem = 0;
    int npt_max = 1;
    bool generic = false;  // some item uses the generic table layout
    long useful_ctas = 0;  // CTAs that the items can keep busy at once
    for (int g = 0; g < n_items; ++g) {
        const bpq_tanner *t = items[g].tanner;
        bpq::DecodeArgs &a = desc[g];
        rc = bpq::fill_decode_args(t, items[g].syn_dev, items[g].prior_dev, variant, params, max_iter,
                                   items[g].B, work_dev, a);
        if (rc) return rc;
        bpq::LaunchShape s;
        rc = bpq::decode_batch_shape(t, variant, &s);
        if (rc) return rc;
        a.est = items[g].est_dev;
        a.conv = items[g].conv_dev;
        a.iters = items[g].iters_dev;
        a.G = s.G;
        a.n_pad = s.n_pad;
        a.slots_floats = s.slots_floats;
        a.group_bytes = s.group_bytes;
        a.npt = s.npt;
        a.groups_per_cta = s.groups_per_cta;
        npt_max = std::max(npt_max, s.npt);
        generic = generic || a.split == 0;
        smem = std::max(smem, s.smem);
        weight[g] = (double)items[g].B * t->E;
        useful_ctas += (items[g].B + s.groups_per_cta - 1) / s.groups_per_cta;
    }
    if (smem > 227 * 1024) return fail(BPQ_EINVAL, "a code of the batch needs more than 227 KB of shared memory");

    bpq::BatchKernelFn fn = bpq::pick_batch_kernel(variant, generic);
    if (!fn) return fail(BPQ_EINVAL, "no batched kernel for this shape");
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail(BPQ_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, bpq::kBatchThreads, smem);
    if (e != cudaSuccess || per_sm < 1) return fail(BPQ_ECUDA, "batched kernel does not fit on an SM");
    long ctas = (long)per_sm * items[0].tanner->num_sms;
    ctas = std::min<long>({ctas, std::max(1L, useful_ctas), (long)bpq::kMaxBatchCtas});
    std::vector<int> start(ctas);
    bpq::batch_start_items(weight, (int)ctas, start.data());

    // device layout of the workspace: counters | descriptors | starting items
    uint8_t *w = static_cast<uint8_t *>(work_dev);
    bpq::DecodeArgs *d_desc = reinterpret_cast<bpq::DecodeArgs *>(w + bpq::batch_counter_bytes(n_items));
    int *d_start = reinterpret_cast<int *>(reinterpret_cast<uint8_t *>(d_desc) +
                                           bpq::align256(sizeof(bpq::DecodeArgs) * n_items));
    for (auto &a : desc) a.work = static_cast<uint32_t *>(work_dev);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rc = bpq::cuda_check(cudaMemcpyAsync(d_desc, desc.data(), sizeof(bpq::DecodeArgs) * n_items,
                                         cudaMemcpyHostToDevice, st), "descriptor copy");
    if (!rc)
        rc = bpq::cuda_check(cudaMemcpyAsync(d_start, start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice,
                                             st), "start copy");
    if (!rc) rc = bpq::cuda_check(cudaStreamSynchronize(st), "plan sync");
    if (rc) return rc;

    bpq_batch *b = new (std::nothrow) bpq_batch();
    if (!b) return fail(BPQ_ENOMEM, "allocation failed");
    b->device = device;
    b->work = work_dev;
    b->fn = fn;
    b->args.codes = d_desc;
    b->args.start = d_start;
    b->args.ncodes = n_items;
    b->args.work = static_cast<uint32_t *>(work_dev);
    b->smem = smem;
    b->npt_max = npt_max;
    b->shots = total;
    b->ctas = (int)ctas;
    *out = b;
    return BPQ_OK;
}

int bpq_batch_launch(const bpq_batch *b, void *stream) {
    if (!b) return fail(BPQ_EINVAL, "batch is NULL");
    int rc = bpq::cuda_set_device(b->device);
    if (rc) return rc;
    if (b->shots == 0) return BPQ_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rc = bpq::cuda_check(cudaMemsetAsync(b->work, 0, bpq::batch_counter_bytes(b->args.ncodes), st),
                         "batch counter reset");
    if (rc) return rc;
    b->fn<<<(unsigned)b->ctas, bpq::kBatchThreads, b->smem, st>>>(b->args);
    return bpq::cuda_check(cudaGetLastError(), "batched decode launch");
}

int bpq_batch_info(const bpq_batch *b, int *ctas, int *items, int *npt_max, long *shots) {
    if (!b) return fail(BPQ_EINVAL, "batch is NULL");
    if (ctas) *ctas = b->ctas;
    if (items) *items = b->args.ncodes;
    if (npt_max) *npt_max = b->npt_max;
    if (shots) *shots = b->shots;
    return BPQ_OK;
}

void bpq_batch_free(bpq_batch *b) { delete b; }

int bpq_set_batch_launch(bpq_tanner *t, int nodes_per_thread) {
    if (!t) return fail(BPQ_EINVAL, "tanner is NULL");
    if (nodes_per_thread < 0 || nodes_per_thread > 2) return fail(BPQ_EINVAL, "nodes per thread must be 0, 1 or 2");
    const int old = t->batch_nodes_per_thread;
    t->batch_nodes_per_thread = nodes_per_thread;
    bpq::LaunchShape s;
    int rc = bpq::decode_batch_shape(t, BPQ_MOMENTUM, &s);
    if (rc) t->batch_nodes_per_thread = old;
    return rc;
}

int bpq_get_batch_launch(const bpq_tanner *t, int variant, int *threads_per_shot, int *shots_per_cta,
                         int *nodes_per_thread) {
    if (!t) return fail(BPQ_EINVAL, "tanner is NULL");
    if (variant < BPQ_PLAIN || variant > BPQ_EWAINIT)
        return fail(BPQ_EINVAL, "the batched kernel takes plain, Momentum, AdaGrad or EWAInit BP");
    bpq::LaunchShape s;
    int rc = bpq::decode_batch_shape(t, variant, &s);
    if (rc) return rc;
    if (threads_per_shot) *threads_per_shot = s.T;
    if (shots_per_cta) *shots_per_cta = s.groups_per_cta;
    if (nodes_per_thread) *nodes_per_thread = s.npt;
    return BPQ_OK;
}

int bpq_autotune_batch(bpq_tanner *t, const uint32_t *syn_dev, const float *prior_dev, int variant,
                       const bpq_params *params, int max_iter, int B, uint8_t *est_dev, uint8_t *conv_dev,
                       uint8_t *iters_dev, void *work_dev, size_t work_bytes, void *stream, int *nodes_per_thread,
                       float *best_ms) {
    int rc = bpq::need_uploaded(t);
    if (rc) return rc;
    if (B < 1) return fail(BPQ_EINVAL, "autotune needs a non-empty sample");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int old = t->batch_nodes_per_thread;
    int best_npt = 0;
    float best = 1e30f;
    cudaEvent_t e0, e1;
    rc = bpq::cuda_check(cudaEventCreate(&e0), "cudaEventCreate");
    if (rc) return rc;
    rc = bpq::cuda_check(cudaEventCreate(&e1), "cudaEventCreate");
    if (rc) {
        cudaEventDestroy(e0);
        return rc;
    }
    const bpq_batch_item item{t, syn_dev, prior_dev, B, est_dev, conv_dev, iters_dev};
    for (int npt = 1; npt <= 2 && !rc; ++npt) {
        t->batch_nodes_per_thread = npt;
        bpq::LaunchShape shape;
        if (bpq::decode_batch_shape(t, variant, &shape)) continue;
        bpq_batch *plan = nullptr;
        rc = bpq_batch_plan(&item, 1, variant, params, max_iter, work_dev, work_bytes, stream, &plan);
        float ms = 0.f;
        for (int rep = 0; rep < 3 && !rc; ++rep) {  // one warm-up, two timed
            if (rep == 1) rc = bpq::cuda_check(cudaEventRecord(e0, st), "cudaEventRecord");
            if (!rc) rc = bpq_batch_launch(plan, stream);
        }
        if (!rc) rc = bpq::cuda_check(cudaEventRecord(e1, st), "cudaEventRecord");
        if (!rc) rc = bpq::cuda_check(cudaEventSynchronize(e1), "cudaEventSynchronize");
        if (!rc) rc = bpq::cuda_check(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
        bpq_batch_free(plan);
        if (!rc && ms / 2 < best) {
            best = ms / 2;
            best_npt = npt;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc || best_npt == 0) {
        t->batch_nodes_per_thread = old;
        return rc ? rc : fail(BPQ_EINVAL, "no batched shape fits this code");
    }
    t->batch_nodes_per_thread = best_npt;
    if (nodes_per_thread) *nodes_per_thread = best_npt;
    if (best_ms) *best_ms = best;
    return BPQ_OK;
}

}  // extern "C"
