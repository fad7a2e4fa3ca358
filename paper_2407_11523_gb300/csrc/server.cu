// Continuous-batching decoding server (bpq_server_*).
//
// A fixed set of CUDA streams ("lanes"), each owning a slice of the caller's
// device memory sized for max_batch shots, decodes micro-batches of requests
// with the batched multi-code kernel.  The host loop replays a request trace
// in real time: requests whose arrival time has passed wait in a FIFO; as
// soon as a lane is free, all waiting requests (up to max_batch) are grouped
// by code and sent to it (pinned-host -> device copy, one batched launch,
// device -> pinned-host copy, completion event).  Requests that arrive while
// other lanes are busy therefore run on the device concurrently with them.
// Each request's result is the one bpq_decode gives for it alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <new>
#include <vector>

#include "bpq_internal.h"
#include "decode_launch.h"

using bpq::fail;

namespace bpq {
BatchKernelFn pick_batch_kernel(int variant, int npt);
}

namespace {

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct Lane {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    // device slice
    uint32_t *work = nullptr;
    bpq::DecodeArgs *desc = nullptr;
    int *start = nullptr;
    uint32_t *syn = nullptr;
    uint8_t *est = nullptr, *conv = nullptr, *iters = nullptr;
    // pinned host staging
    bpq::DecodeArgs *desc_h = nullptr;
    int *start_h = nullptr;
    uint32_t *syn_h = nullptr;
    uint8_t *est_h = nullptr, *conv_h = nullptr, *iters_h = nullptr;
    // requests in flight: (request, code, offset of its estimate in est_h)
    std::vector<int> req;
    std::vector<long> est_off;
    std::vector<int> shot_of;  // index in the lane's conv/iters arrays
    bool busy = false;
};

}  // namespace

struct bpq_server {
    int device = -1;
    int variant = 0, max_iter = 0, max_batch = 0;
    std::vector<const bpq_tanner *> codes;
    std::vector<bpq::DecodeArgs> tmpl;  // per-code descriptor templates
    int Wmax = 0, Nmax = 0;
    bpq::BatchKernelFn fn = nullptr;
    size_t smem = 0;
    int ctas = 0;
    long launches = 0;  // batched kernel launches since creation
    std::vector<Lane> lanes;
};

namespace {

size_t lane_device_bytes(int n_codes, int max_batch, int Wmax, int Nmax) {
    return bpq::batch_counter_bytes(n_codes) + a256(sizeof(bpq::DecodeArgs) * n_codes) +
           a256(sizeof(int) * bpq::kMaxBatchCtas) + a256(sizeof(uint32_t) * (size_t)Wmax * max_batch) +
           a256((size_t)Nmax * max_batch) + 2 * a256(max_batch);
}

void free_server(bpq_server *s) {
    if (!s) return;
    if (s->device >= 0) cudaSetDevice(s->device);
    for (Lane &l : s->lanes) {
        if (l.st) cudaStreamSynchronize(l.st);
        if (l.done) cudaEventDestroy(l.done);
        if (l.st) cudaStreamDestroy(l.st);
        cudaFreeHost(l.desc_h);
        cudaFreeHost(l.start_h);
        cudaFreeHost(l.syn_h);
        cudaFreeHost(l.est_h);
        cudaFreeHost(l.conv_h);
        cudaFreeHost(l.iters_h);
    }
    delete s;
}

}  // namespace

extern "C" {

size_t bpq_server_device_bytes(const bpq_tanner *const *codes, int n_codes, int n_lanes, int max_batch) {
    if (!codes || n_codes < 1 || n_lanes < 1 || max_batch < 1) return 0;
    int Wmax = 0, Nmax = 0;
    for (int c = 0; c < n_codes; ++c) {
        if (!codes[c]) return 0;
        Wmax = std::max(Wmax, (codes[c]->M + 31) / 32);
        Nmax = std::max(Nmax, codes[c]->N);
    }
    return (size_t)n_lanes * lane_device_bytes(n_codes, max_batch, Wmax, Nmax);
}

int bpq_server_create(const bpq_tanner *const *codes, const float *const *priors_dev, int n_codes, int variant,
                      const bpq_params *params, int max_iter, int n_lanes, int max_batch, void *dev_mem,
                      size_t dev_bytes, bpq_server **out) {
    if (!out) return fail(BPQ_EINVAL, "out is NULL");
    *out = nullptr;
    if (!codes || !priors_dev || n_codes < 1) return fail(BPQ_EINVAL, "no codes");
    if (n_lanes < 1 || n_lanes > 64 || max_batch < 1) return fail(BPQ_EINVAL, "bad lane count or batch size");
    if (dev_bytes < bpq_server_device_bytes(codes, n_codes, n_lanes, max_batch) || !dev_mem)
        return fail(BPQ_EINVAL, "device memory budget too small");
    const int device = codes[0] ? codes[0]->device : -1;
    bpq_server *s = new (std::nothrow) bpq_server();
    if (!s) return fail(BPQ_ENOMEM, "allocation failed");
    s->device = device;
    s->variant = variant;
    s->max_iter = max_iter;
    s->max_batch = max_batch;
    int rc = BPQ_OK;
    int npt_max = 1;
    for (int c = 0; c < n_codes && !rc; ++c) {
        const bpq_tanner *t = codes[c];
        if (!t || !t->dev_blob || t->device != device) {
            rc = fail(BPQ_ESTATE, "server codes must be uploaded to one device");
            break;
        }
        if (!priors_dev[c]) {
            rc = fail(BPQ_EINVAL, "NULL prior");
            break;
        }
        bpq::DecodeArgs a;
        uint32_t dummy = 0;
        rc = bpq::fill_decode_args(t, &dummy, priors_dev[c], variant, params, max_iter, 1, dev_mem, a);
        if (rc) break;
        bpq::LaunchShape sh;
        rc = bpq::decode_batch_shape(t, variant, &sh);
        if (rc) break;
        const int gpc = sh.groups_per_cta;
        a.G = sh.G;
        a.n_pad = sh.n_pad;
        a.slots_floats = sh.slots_floats;
        a.group_bytes = sh.group_bytes;
        a.npt = sh.npt;
        a.groups_per_cta = gpc;
        npt_max = std::max(npt_max, sh.npt);
        s->smem = std::max(s->smem, sh.smem);
        s->codes.push_back(t);
        s->tmpl.push_back(a);
        s->Wmax = std::max(s->Wmax, (t->M + 31) / 32);
        s->Nmax = std::max(s->Nmax, t->N);
    }
    if (!rc && s->smem > 227 * 1024) rc = fail(BPQ_EINVAL, "a code needs more than 227 KB of shared memory");
    if (!rc) rc = bpq::cuda_set_device(device);
    if (!rc) {
        s->fn = bpq::pick_batch_kernel(variant, npt_max);
        if (!s->fn) {
            free_server(s);
            return fail(BPQ_EINVAL, "no batched kernel for these codes");
        }
        cudaError_t e = cudaFuncSetAttribute(s->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem);
        int per_sm = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, s->fn, bpq::kBatchThreads, s->smem);
        if (e != cudaSuccess || per_sm < 1) rc = fail(BPQ_ECUDA, "batched kernel does not fit on an SM");
        s->ctas = per_sm * s->codes[0]->num_sms;
    }
    const size_t lane_bytes = lane_device_bytes(n_codes, max_batch, s->Wmax, s->Nmax);
    uint8_t *base = static_cast<uint8_t *>(dev_mem);
    for (int l = 0; l < n_lanes && !rc; ++l) {
        s->lanes.emplace_back();
        Lane &L = s->lanes.back();
        uint8_t *p = base + (size_t)l * lane_bytes;
        L.work = reinterpret_cast<uint32_t *>(p);
        p += bpq::batch_counter_bytes(n_codes);
        L.desc = reinterpret_cast<bpq::DecodeArgs *>(p);
        p += a256(sizeof(bpq::DecodeArgs) * n_codes);
        L.start = reinterpret_cast<int *>(p);
        p += a256(sizeof(int) * bpq::kMaxBatchCtas);
        L.syn = reinterpret_cast<uint32_t *>(p);
        p += a256(sizeof(uint32_t) * (size_t)s->Wmax * max_batch);
        L.est = p;
        p += a256((size_t)s->Nmax * max_batch);
        L.conv = p;
        p += a256(max_batch);
        L.iters = p;
        cudaError_t e = cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&L.desc_h, sizeof(bpq::DecodeArgs) * n_codes, 0);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&L.start_h, sizeof(int) * bpq::kMaxBatchCtas, 0);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&L.syn_h, sizeof(uint32_t) * (size_t)s->Wmax * max_batch, 0);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&L.est_h, (size_t)s->Nmax * max_batch, 0);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&L.conv_h, max_batch, 0);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&L.iters_h, max_batch, 0);
        if (e != cudaSuccess) rc = fail(BPQ_ECUDA, std::string("server lane setup: ") + cudaGetErrorString(e));
    }
    if (rc) {
        free_server(s);
        return rc;
    }
    *out = s;
    return BPQ_OK;
}

int bpq_server_replay(bpq_server *s, int n_req, const int *code, const double *arrival_s, const uint32_t *syn_host,
                      const int64_t *syn_off, uint8_t *est_host, const int64_t *est_off, uint8_t *conv_host,
                      uint8_t *iters_host, double *done_s, int *lanes_used) {
    if (!s) return fail(BPQ_EINVAL, "server is NULL");
    if (n_req < 0 || (n_req > 0 && (!code || !arrival_s || !syn_host || !syn_off || !est_host || !est_off ||
                                    !conv_host || !iters_host || !done_s)))
        return fail(BPQ_EINVAL, "NULL request arrays");
    const int n_codes = (int)s->codes.size();
    for (int r = 0; r < n_req; ++r) {
        if (code[r] < 0 || code[r] >= n_codes) return fail(BPQ_EINVAL, "request code index out of range");
        if (r > 0 && arrival_s[r] < arrival_s[r - 1]) return fail(BPQ_EINVAL, "arrival times must not decrease");
    }
    int rc = bpq::cuda_set_device(s->device);
    if (rc) return rc;
    using clock = std::chrono::steady_clock;
    const auto t0 = clock::now();
    auto now = [&]() { return std::chrono::duration<double>(clock::now() - t0).count(); };
    std::deque<int> pending;
    int next = 0, completed = 0, max_busy = 0;
    std::vector<int> by_code_count(n_codes);
    while (completed < n_req) {
        // retire finished lanes
        for (Lane &L : s->lanes) {
            if (!L.busy) continue;
            cudaError_t q = cudaEventQuery(L.done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) return fail(BPQ_ECUDA, std::string("server lane: ") + cudaGetErrorString(q));
            const double tnow = now();
            for (size_t k = 0; k < L.req.size(); ++k) {
                const int r = L.req[k];
                const int N = s->codes[code[r]]->N;
                std::memcpy(est_host + est_off[r], L.est_h + L.est_off[k], N);
                conv_host[r] = L.conv_h[L.shot_of[k]];
                iters_host[r] = L.iters_h[L.shot_of[k]];
                done_s[r] = tnow;
            }
            completed += (int)L.req.size();
            L.req.clear();
            L.busy = false;
        }
        // admit arrivals
        const double tnow = now();
        while (next < n_req && arrival_s[next] <= tnow) pending.push_back(next++);
        // dispatch waiting requests to free lanes
        for (Lane &L : s->lanes) {
            if (L.busy || pending.empty()) continue;
            const int take = std::min<int>((int)pending.size(), s->max_batch);
            std::vector<int> batch(pending.begin(), pending.begin() + take);
            pending.erase(pending.begin(), pending.begin() + take);
            // group by code: count, then place
            std::fill(by_code_count.begin(), by_code_count.end(), 0);
            for (int r : batch) ++by_code_count[code[r]];
            std::vector<int> first(n_codes, 0);
            std::vector<long> syn_base(n_codes, 0), est_base(n_codes, 0);
            int shot = 0;
            long wsum = 0, nsum = 0;
            for (int c = 0; c < n_codes; ++c) {
                first[c] = shot;
                syn_base[c] = wsum;
                est_base[c] = nsum;
                shot += by_code_count[c];
                wsum += (long)by_code_count[c] * ((s->codes[c]->M + 31) / 32);
                nsum += (long)by_code_count[c] * s->codes[c]->N;
            }
            std::vector<int> fill(n_codes, 0);
            L.req.clear();
            L.est_off.clear();
            L.shot_of.clear();
            for (int r : batch) {
                const int c = code[r];
                const int W = (s->codes[c]->M + 31) / 32, N = s->codes[c]->N;
                const int k = fill[c]++;
                std::memcpy(L.syn_h + syn_base[c] + (long)k * W, syn_host + syn_off[r], sizeof(uint32_t) * W);
                L.req.push_back(r);
                L.est_off.push_back(est_base[c] + (long)k * N);
                L.shot_of.push_back(first[c] + k);
            }
            std::vector<double> weight(n_codes);
            long useful_ctas = 0;
            for (int c = 0; c < n_codes; ++c) {
                bpq::DecodeArgs a = s->tmpl[c];
                a.syn = L.syn + syn_base[c];
                a.est = L.est + est_base[c];
                a.conv = L.conv + first[c];
                a.iters = L.iters + first[c];
                a.B = by_code_count[c];
                a.work = L.work;
                L.desc_h[c] = a;
                weight[c] = (double)by_code_count[c] * s->codes[c]->E;
                useful_ctas += (by_code_count[c] + a.groups_per_cta - 1) / a.groups_per_cta;
            }
            const int ctas = (int)std::min<long>({(long)s->ctas, std::max(1L, useful_ctas), (long)bpq::kMaxBatchCtas});
            bpq::batch_start_items(weight, ctas, L.start_h);
            bpq::BatchArgs args;
            args.codes = L.desc;
            args.start = L.start;
            args.ncodes = n_codes;
            args.work = L.work;
            cudaError_t e = cudaMemcpyAsync(L.syn, L.syn_h, sizeof(uint32_t) * wsum, cudaMemcpyHostToDevice, L.st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(L.desc, L.desc_h, sizeof(bpq::DecodeArgs) * n_codes, cudaMemcpyHostToDevice,
                                    L.st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(L.start, L.start_h, sizeof(int) * ctas, cudaMemcpyHostToDevice, L.st);
            if (e == cudaSuccess) e = cudaMemsetAsync(L.work, 0, bpq::batch_counter_bytes(n_codes), L.st);
            if (e == cudaSuccess) {
                s->fn<<<(unsigned)ctas, bpq::kBatchThreads, s->smem, L.st>>>(args);
                e = cudaGetLastError();
                ++s->launches;
            }
            if (e == cudaSuccess) e = cudaMemcpyAsync(L.est_h, L.est, nsum, cudaMemcpyDeviceToHost, L.st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(L.conv_h, L.conv, shot, cudaMemcpyDeviceToHost, L.st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(L.iters_h, L.iters, shot, cudaMemcpyDeviceToHost, L.st);
            if (e == cudaSuccess) e = cudaEventRecord(L.done, L.st);
            if (e != cudaSuccess) return fail(BPQ_ECUDA, std::string("server dispatch: ") + cudaGetErrorString(e));
            L.busy = true;
        }
        int busy = 0;
        for (const Lane &L : s->lanes) busy += L.busy;
        max_busy = std::max(max_busy, busy);
    }
    if (lanes_used) *lanes_used = max_busy;
    return BPQ_OK;
}

int bpq_server_stats(const bpq_server *s, long *launches) {
    if (!s) return fail(BPQ_EINVAL, "server is NULL");
    if (launches) *launches = s->launches;
    return BPQ_OK;
}

void bpq_server_free(bpq_server *s) { free_server(s); }

}  // extern "C"
