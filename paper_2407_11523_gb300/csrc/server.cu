// Decoding servers (bpq_server_*).
//
// Slot-granular server (bpq_server_create_slots): a persistent kernel
// (serve_kernel.cuh) whose shot groups take the next request as soon as they
// finish a shot.  Each code has a ring of request slots in mapped pinned host
// memory: the host loop admits a request that has arrived into the next free
// slot of its code's ring (writing its syndrome there) and publishes the
// code's request count; it reads completions from a queue the kernel writes
// in mapped memory, copies the outputs out and frees the slot.  A request is
// therefore on the device from the moment a slot frees up, whatever else is
// running.  Every device-side wait is bounded: the kernel returns after an
// idle period with a status the host reads, and the host relaunches it (a
// captured CUDA graph) while requests remain.
//
// Lane server (bpq_server_create): a fixed set of CUDA streams ("lanes"), each owning a slice of the caller's
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

#include <atomic>

#include "bpq_internal.h"
#include "decode_launch.h"
#include "serve_kernel.cuh"

using bpq::fail;

namespace bpq {
BatchKernelFn pick_batch_kernel(int variant, bool generic);
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

// Slot-server state: rings and queues in mapped pinned host memory, claim
// counters and status in the caller's device memory.
struct SlotRings {
    int cap = 0;                       // slots per code
    uint32_t cq_len = 0;
    uint8_t *host = nullptr;           // one mapped pinned allocation
    uint32_t *tail = nullptr, *closed = nullptr;
    uint4 *cq = nullptr;
    uint4 *dst = nullptr;              // [n_codes][cap]: each slot's output offset and request (direct mode)
    uint32_t *consumed = nullptr;      // [n_codes][cap]: request number + 1 staged from the slot (direct mode)
    bpq::ServeOut *out_dev = nullptr;  // device: the output buffers of the current stream
    std::vector<uint32_t *> syn;       // per code [cap][W]
    std::vector<uint8_t *> est, conv, iters;  // per code [cap][N], [cap], [cap]
    // device
    uint32_t *head = nullptr, *cq_count = nullptr, *status = nullptr, *cap_dev = nullptr;
    bpq::DecodeArgs *desc = nullptr;
    bpq::ServeKernelFn fn = nullptr;
    uint32_t idle_limit = 0;
    int grid = 0;                      // resident CTAs of the serving kernel
    cudaStream_t st = nullptr;
    cudaEvent_t exited = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t stage_offset = 0, stage_bytes = 0;  // staging area in the kernel's shared memory
    // host loop of the last replay: turns with work, seconds spent admitting
    // requests and reading completions
    long turns = 0;
    double admit_s = 0.0, complete_s = 0.0;
};

struct bpq_server {
    int device = -1;
    bool slots = false;  // slot-granular server (else the lane server)
    SlotRings ring;
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
    SlotRings &R = s->ring;
    if (R.st) {
        if (R.closed) __atomic_store_n(R.closed, 1u, __ATOMIC_RELEASE);  // a running kernel exits
        cudaStreamSynchronize(R.st);
    }
    if (R.exec) cudaGraphExecDestroy(R.exec);
    if (R.graph) cudaGraphDestroy(R.graph);
    if (R.exited) cudaEventDestroy(R.exited);
    if (R.st) cudaStreamDestroy(R.st);
    if (R.host) cudaFreeHost(R.host);
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


namespace {

size_t slot_device_bytes(int n_codes) {
    return a256(sizeof(bpq::DecodeArgs) * (size_t)n_codes) + 2 * a256(sizeof(uint32_t) * (size_t)n_codes) + 512;
}

// Device pointer of a host buffer of `bytes` bytes if both its ends lie in
// page-locked (pinned or registered) host memory, else nullptr.
uint8_t *pinned_device_pointer(const void *p, size_t bytes) {
    if (!p || bytes == 0) return nullptr;
    cudaPointerAttributes a0{}, a1{};
    if (cudaPointerGetAttributes(&a0, p) != cudaSuccess ||
        cudaPointerGetAttributes(&a1, static_cast<const uint8_t *>(p) + bytes - 1) != cudaSuccess) {
        cudaGetLastError();  // pageable memory may report an error on older drivers
        return nullptr;
    }
    if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer) return nullptr;
    return static_cast<uint8_t *>(a0.devicePointer);
}

using steady = std::chrono::steady_clock;

int slot_status(bpq_server *s, uint32_t *st3) {
    SlotRings &R = s->ring;
    int rc = bpq::cuda_check(cudaMemcpyAsync(st3, R.status, 3 * sizeof(uint32_t), cudaMemcpyDeviceToHost, R.st),
                             "server status");
    if (!rc) rc = bpq::cuda_check(cudaStreamSynchronize(R.st), "server status");
    return rc;
}

int slot_launch(bpq_server *s) {
    SlotRings &R = s->ring;
    int rc = bpq::cuda_check(cudaGraphLaunch(R.exec, R.st), "server launch");
    if (!rc) rc = bpq::cuda_check(cudaEventRecord(R.exited, R.st), "server launch");
    if (!rc) ++s->launches;
    return rc;
}

int slot_replay(bpq_server *s, int n_req, const int *code, const double *arrival_s, const uint32_t *syn_host,
                const int64_t *syn_off, uint8_t *est_host, const int64_t *est_off, size_t est_bytes,
                uint8_t *conv_host, uint8_t *iters_host, double *done_s, int *lanes_used) {
    SlotRings &R = s->ring;
    const int n_codes = (int)s->codes.size(), cap = R.cap;
    // direct mode: with page-locked outputs and 16-byte aligned estimates
    // (the buffer's start, host and device address, and every offset; the
    // kernel stores them in 16-byte chunks) the kernel writes every result
    // where it belongs, and the host only reads the completion queue;
    // otherwise results go through the rings
    bpq::ServeOut out{nullptr, nullptr, nullptr};
    bool aligned = n_req > 0 && (reinterpret_cast<uintptr_t>(est_host) & 15u) == 0;
    for (int r = 0; r < n_req && aligned; ++r) aligned = (est_off[r] & 15) == 0;
    if (aligned) {
        out.est = pinned_device_pointer(est_host, est_bytes);
        out.conv = pinned_device_pointer(conv_host, (size_t)n_req);
        out.iters = pinned_device_pointer(iters_host, (size_t)n_req);
        if (!out.est || !out.conv || !out.iters || (reinterpret_cast<uintptr_t>(out.est) & 15u) != 0)
            out = bpq::ServeOut{nullptr, nullptr, nullptr};
    }
    const bool direct = out.est != nullptr;
    // a fresh stream of requests: claim counters, completion count, counters,
    // tails and queue
    int rc = bpq::cuda_check(cudaMemsetAsync(R.head, 0, sizeof(uint32_t) * n_codes, R.st), "server reset");
    if (!rc) rc = bpq::cuda_check(cudaMemsetAsync(R.status, 0, 6 * sizeof(uint32_t), R.st), "server reset");
    if (!rc) rc = bpq::cuda_check(cudaMemsetAsync(R.cq_count, 0, sizeof(uint32_t), R.st), "server reset");
    if (!rc)
        rc = bpq::cuda_check(cudaMemcpyAsync(R.out_dev, &out, sizeof out, cudaMemcpyHostToDevice, R.st),
                             "server outputs");
    if (!rc) rc = bpq::cuda_check(cudaStreamSynchronize(R.st), "server reset");
    if (rc) return rc;
    for (int c = 0; c < n_codes; ++c) __atomic_store_n(R.tail + c, 0u, __ATOMIC_RELAXED);
    std::memset(R.cq, 0, sizeof(uint4) * R.cq_len);
    std::memset(R.consumed, 0, sizeof(uint32_t) * (size_t)n_codes * cap);
    __atomic_store_n(R.closed, 0u, __ATOMIC_RELEASE);
    if (lanes_used) *lanes_used = 0;
    if (n_req == 0) return BPQ_OK;
    rc = slot_launch(s);
    if (rc) return rc;

    const auto t0 = steady::now();
    auto now = [&]() { return std::chrono::duration<double>(steady::now() - t0).count(); };
    // an error inside the loop first closes the stream and waits for the
    // kernel, so that it writes nothing to the caller's buffers afterwards
    auto stop = [&](int code_) {
        __atomic_store_n(R.closed, 1u, __ATOMIC_RELEASE);
        cudaStreamSynchronize(R.st);
        return code_;
    };
    // host bookkeeping in flat arrays: request in each slot (-1 free)
    std::vector<uint32_t> admitted(n_codes, 0);
    std::vector<int> req_of((size_t)n_codes * cap, -1);
    std::vector<int> W(n_codes), N(n_codes), N16(n_codes);
    for (int c = 0; c < n_codes; ++c) {
        W[c] = (s->codes[c]->M + 31) / 32;
        N[c] = s->codes[c]->N;
        N16[c] = (N[c] + 15) & ~15;
    }
    // arrived requests wait in a FIFO per code, so that a code whose ring is
    // full holds back only its own requests; a worklist holds the codes with
    // waiting requests that may have a free slot (new arrivals, or a slot
    // freed by a completion), so each turn of the loop costs only its work
    std::vector<std::vector<int>> pend(n_codes);
    std::vector<size_t> pend_head(n_codes, 0);
    std::vector<int> work, blocked;
    std::vector<char> queued(n_codes, 0);
    work.reserve(n_codes);
    blocked.reserve(n_codes);
    uint32_t admitted_total = 0;
    constexpr int kCompletionsPerTurn = 256, kArrivalsPerTurn = 1024;
    int next = 0, completed = 0;
    uint32_t cq_read = 0;
    R.turns = 0;
    R.admit_s = R.complete_s = 0.0;
    while (completed < n_req) {
        const int next0 = next, completed0 = completed;
        bool admitted_any = false;
        // requests that have arrived join their code's FIFO, a bounded number
        // per turn, so that a burst does not hold back the first admissions
        const double tnow = now();
        for (int n = 0; n < kArrivalsPerTurn && next < n_req && arrival_s[next] <= tnow; ++n) {
            const int c = code[next];
            pend[c].push_back(next);
            if (!queued[c]) {
                queued[c] = 1;
                work.push_back(c);
            }
            ++next;
        }
        // each listed code admits from its FIFO while the next slot of its
        // ring is free, then publishes its new count
        for (int c : work) {
            queued[c] = 0;
            std::vector<int> &P = pend[c];
            size_t &h = pend_head[c];
            bool any = false;
            while (h < P.size()) {
                // every admitted request that has not completed may still
                // write a completion, so at most cq_len - 1 of them: the queue
                // never overwrites an entry the host has not read.  (Ring mode
                // keeps this by itself: a slot is refilled only after its
                // completion has been read, and cq_len = codes x slots + 1.)
                if (admitted_total - (uint32_t)completed >= R.cq_len - 1u) {
                    if (!queued[c]) {
                        queued[c] = 1;
                        blocked.push_back(c);
                    }
                    break;
                }
                const uint32_t k = admitted[c];
                const int slot = (int)(k % (uint32_t)cap);
                int &occ = req_of[(size_t)c * cap + slot];
                if (direct) {
                    // the slot is free once the kernel has staged the request
                    // that used it (number k - cap), even while that request
                    // still decodes
                    if (k >= (uint32_t)cap &&
                        __atomic_load_n(R.consumed + (size_t)c * cap + slot, __ATOMIC_ACQUIRE) != k - cap + 1u)
                        break;  // a completion relists the code
                } else if (occ >= 0) {
                    break;  // ring full: a completion relists the code
                }
                const int r = P[h++];
                std::memcpy(R.syn[c] + (size_t)slot * W[c], syn_host + syn_off[r], sizeof(uint32_t) * W[c]);
                if (direct)
                    R.dst[(size_t)c * cap + slot] = make_uint4((uint32_t)est_off[r], (uint32_t)(est_off[r] >> 32),
                                                               (uint32_t)r, 0u);
                occ = r;
                ++admitted[c];
                ++admitted_total;
                any = true;
            }
            if (any) {
                __atomic_store_n(R.tail + c, admitted[c], __ATOMIC_RELEASE);
                admitted_any = true;
            }
        }
        work.clear();
        // codes held back by the completion queue's bound try again next turn
        work.swap(blocked);
        const double tadm = now();
        // completions, in the order the kernel wrote them, a bounded number per
        // turn so that freed slots are refilled promptly; one clock read per turn
        double tdone = -1.0;
        for (int n = 0; n < kCompletionsPerTurn; ++n) {
            uint4 *q = R.cq + (cq_read % R.cq_len);
            if (__atomic_load_n(&q->x, __ATOMIC_ACQUIRE) != cq_read + 1u) break;
            __builtin_prefetch(R.cq + ((cq_read + 4) % R.cq_len));
            if (tdone < 0) tdone = now();
            const int c = (int)q->y;
            const uint32_t k = q->z, cw = q->w;
            if (c < 0 || c >= n_codes) return stop(fail(BPQ_ECUDA, "server: completion of an unknown code"));
            int r;
            if (direct) {
                // the entry names the request; its outputs are in place
                r = (int)k;
                if (r < 0 || r >= n_req) return stop(fail(BPQ_ECUDA, "server: completion of an unknown request"));
            } else {
                const int slot = (int)(k % (uint32_t)cap);
                int &occ = req_of[(size_t)c * cap + slot];
                r = occ;
                if (r < 0) return stop(fail(BPQ_ECUDA, "server: completion of a request that is not in flight"));
                std::memcpy(est_host + est_off[r], R.est[c] + (size_t)slot * N16[c], N[c]);
                conv_host[r] = (uint8_t)(cw & 0xFFu);
                iters_host[r] = (uint8_t)((cw >> 8) & 0xFFu);
                occ = -1;
            }
            done_s[r] = tdone;
            if (!queued[c] && pend_head[c] < pend[c].size()) {
                queued[c] = 1;
                work.push_back(c);
            }
            ++completed;
            ++cq_read;
        }
        if (next != next0 || completed != completed0 || admitted_any) {
            const double tend = now();
            ++R.turns;
            R.admit_s += tadm - tnow;
            R.complete_s += tend - tadm;
            continue;
        }
        // the kernel returns after an idle period (or a device error): read its
        // status and relaunch it while requests remain (checked on the host
        // loop's idle turns only; the query is a driver call)
        const cudaError_t q = cudaEventQuery(R.exited);
        if (q == cudaSuccess && completed < n_req) {
            uint32_t st3[3];
            rc = slot_status(s, st3);
            if (rc) return stop(rc);
            if (st3[1]) return stop(fail(BPQ_ECUDA, "server: a bounded wait inside the kernel gave up"));
            // completions written just before the kernel returned are read first
            uint4 *qq = R.cq + (cq_read % R.cq_len);
            if (__atomic_load_n(&qq->x, __ATOMIC_ACQUIRE) == cq_read + 1u) continue;
            rc = slot_launch(s);
            if (rc) return stop(rc);
        } else if (q != cudaSuccess && q != cudaErrorNotReady) {
            return stop(fail(BPQ_ECUDA, std::string("server kernel: ") + cudaGetErrorString(q)));
        }
    }
    // every request is done: close the stream; the kernel's CTAs return
    __atomic_store_n(R.closed, 1u, __ATOMIC_RELEASE);
    rc = bpq::cuda_check(cudaStreamSynchronize(R.st), "server close");
    if (lanes_used) *lanes_used = R.grid;
    return rc;
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
    if (bpq::misaligned(dev_mem, bpq::kBufferAlign)) return fail(BPQ_EINVAL, "device memory not 16-byte aligned");
    const int device = codes[0] ? codes[0]->device : -1;
    bpq_server *s = new (std::nothrow) bpq_server();
    if (!s) return fail(BPQ_ENOMEM, "allocation failed");
    s->device = device;
    s->variant = variant;
    s->max_iter = max_iter;
    s->max_batch = max_batch;
    int rc = BPQ_OK;
    int npt_max = 1;
    bool generic = false;  // some code uses the generic table layout
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
        generic = generic || a.split == 0;
        s->smem = std::max(s->smem, sh.smem);
        s->codes.push_back(t);
        s->tmpl.push_back(a);
        s->Wmax = std::max(s->Wmax, (t->M + 31) / 32);
        s->Nmax = std::max(s->Nmax, t->N);
    }
    if (!rc && s->smem > 227 * 1024) rc = fail(BPQ_EINVAL, "a code needs more than 227 KB of shared memory");
    if (!rc) rc = bpq::cuda_set_device(device);
    if (!rc) {
        s->fn = bpq::pick_batch_kernel(variant, generic);
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
                      const int64_t *syn_off, uint8_t *est_host, const int64_t *est_off, size_t est_bytes,
                      uint8_t *conv_host, uint8_t *iters_host, double *done_s, int *lanes_used) {
    if (!s) return fail(BPQ_EINVAL, "server is NULL");
    if (n_req < 0 || (n_req > 0 && (!code || !arrival_s || !syn_host || !syn_off || !est_host || !est_off ||
                                    !conv_host || !iters_host || !done_s)))
        return fail(BPQ_EINVAL, "NULL request arrays");
    const int n_codes = (int)s->codes.size();
    for (int r = 0; r < n_req; ++r) {
        if (code[r] < 0 || code[r] >= n_codes) return fail(BPQ_EINVAL, "request code index out of range");
        if (r > 0 && arrival_s[r] < arrival_s[r - 1]) return fail(BPQ_EINVAL, "arrival times must not decrease");
        if (est_off[r] < 0 || (size_t)est_off[r] + (size_t)s->codes[code[r]]->N > est_bytes)
            return fail(BPQ_EINVAL, "a request's estimate lies outside est_host");
    }
    int rc = bpq::cuda_set_device(s->device);
    if (rc) return rc;
    if (s->slots)
        return slot_replay(s, n_req, code, arrival_s, syn_host, syn_off, est_host, est_off, est_bytes, conv_host,
                           iters_host, done_s, lanes_used);
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


size_t bpq_server_slot_device_bytes(int n_codes) { return n_codes < 1 ? 0 : slot_device_bytes(n_codes); }

int bpq_server_host_stats(const bpq_server *s, long *turns, double *admit_s, double *complete_s) {
    if (!s || !s->slots) return fail(BPQ_EINVAL, "not a slot server");
    if (turns) *turns = s->ring.turns;
    if (admit_s) *admit_s = s->ring.admit_s;
    if (complete_s) *complete_s = s->ring.complete_s;
    return BPQ_OK;
}

int bpq_server_create_slots(const bpq_tanner *const *codes, const float *const *priors_dev, int n_codes, int variant,
                            const bpq_params *params, int max_iter, int slots_per_code, int idle_timeout_us,
                            void *dev_mem, size_t dev_bytes, bpq_server **out) {
    if (!out) return fail(BPQ_EINVAL, "out is NULL");
    *out = nullptr;
    if (!codes || !priors_dev || n_codes < 1 || n_codes > 4096) return fail(BPQ_EINVAL, "bad code list");
    if (variant < BPQ_PLAIN || variant > BPQ_EWAINIT)
        return fail(BPQ_EINVAL, "the slot server decodes plain, Momentum, AdaGrad or EWAInit BP");
    if (slots_per_code < 1 || slots_per_code > (1 << 20)) return fail(BPQ_EINVAL, "slots per code must be in [1, 2^20]");
    if (idle_timeout_us < 1) return fail(BPQ_EINVAL, "idle timeout must be at least 1 us");
    if (!dev_mem || dev_bytes < slot_device_bytes(n_codes)) return fail(BPQ_EINVAL, "device memory budget too small");
    if (bpq::misaligned(dev_mem, bpq::kBufferAlign)) return fail(BPQ_EINVAL, "device memory not 16-byte aligned");
    const int device = codes[0] ? codes[0]->device : -1;
    bpq_server *s = new (std::nothrow) bpq_server();
    if (!s) return fail(BPQ_ENOMEM, "allocation failed");
    s->device = device;
    s->slots = true;
    s->variant = variant;
    s->max_iter = max_iter;
    SlotRings &R = s->ring;
    R.cap = slots_per_code;
    R.idle_limit = (uint32_t)idle_timeout_us;
    int rc = BPQ_OK;
    for (int c = 0; c < n_codes && !rc; ++c) {
        const bpq_tanner *t = codes[c];
        if (!t || !t->dev_blob || t->device != device) rc = fail(BPQ_ESTATE, "server codes must be uploaded to one device");
        else if (!priors_dev[c]) rc = fail(BPQ_EINVAL, "NULL prior");
        if (rc) break;
        bpq::DecodeArgs a;
        uint32_t dummy = 0;
        rc = bpq::fill_decode_args(t, &dummy, priors_dev[c], variant, params, max_iter, 1, dev_mem, a);
        if (rc) break;
        bpq::LaunchShape sh;
        rc = bpq::decode_batch_shape(t, variant, &sh);
        if (rc) break;
        a.G = sh.G;
        a.n_pad = sh.n_pad;
        a.slots_floats = sh.slots_floats;
        a.group_bytes = sh.group_bytes;
        a.npt = sh.npt;
        a.groups_per_cta = sh.groups_per_cta;
        a.B = slots_per_code;
        s->smem = std::max(s->smem, sh.smem);
        R.stage_bytes = std::max(R.stage_bytes, bpq::serve_stage_bytes(sh.groups_per_cta, t->N, (t->M + 31) / 32));
        s->codes.push_back(t);
        s->tmpl.push_back(a);
        s->Wmax = std::max(s->Wmax, (t->M + 31) / 32);
        s->Nmax = std::max(s->Nmax, t->N);
    }
    // the staging area follows the largest code's group memory
    R.stage_offset = (s->smem + 15) & ~size_t(15);
    s->smem = R.stage_offset + R.stage_bytes;
    if (!rc && s->smem > 227 * 1024) rc = fail(BPQ_EINVAL, "a code needs more than 227 KB of shared memory");
    if (!rc) rc = bpq::cuda_set_device(device);
    // mapped pinned host memory: tails, closed flag, completion queue, per-code
    // rings (estimate slots padded to 16 bytes)
    size_t total = 0;
    std::vector<size_t> o_syn(n_codes), o_est(n_codes), o_conv(n_codes), o_iters(n_codes);
    const size_t o_tail = total;
    total += a256(sizeof(uint32_t) * n_codes);
    const size_t o_closed = total;
    total += 256;
    R.cq_len = (uint32_t)std::min<size_t>((size_t)n_codes * slots_per_code + 1, size_t(1) << 31);
    const size_t o_cq = total;
    total += a256(sizeof(uint4) * R.cq_len);
    const size_t o_dst = total;
    total += a256(sizeof(uint4) * (size_t)n_codes * slots_per_code);
    const size_t o_consumed = total;
    total += a256(sizeof(uint32_t) * (size_t)n_codes * slots_per_code);
    for (int c = 0; c < (int)s->codes.size(); ++c) {
        const size_t W = (s->codes[c]->M + 31) / 32, N16 = ((size_t)s->codes[c]->N + 15) & ~size_t(15);
        o_syn[c] = total;
        total += a256(sizeof(uint32_t) * W * slots_per_code);
        o_est[c] = total;
        total += a256(N16 * slots_per_code);
        o_conv[c] = total;
        total += a256(slots_per_code);
        o_iters[c] = total;
        total += a256(slots_per_code);
    }
    if (!rc)
        rc = bpq::cuda_check(cudaHostAlloc((void **)&R.host, total, cudaHostAllocMapped | cudaHostAllocPortable),
                             "server rings (cudaHostAlloc)");
    uint8_t *dev_host = nullptr;
    if (!rc) rc = bpq::cuda_check(cudaHostGetDevicePointer((void **)&dev_host, R.host, 0), "cudaHostGetDevicePointer");
    if (!rc) {
        std::memset(R.host, 0, total);
        R.tail = reinterpret_cast<uint32_t *>(R.host + o_tail);
        R.closed = reinterpret_cast<uint32_t *>(R.host + o_closed);
        R.cq = reinterpret_cast<uint4 *>(R.host + o_cq);
        R.dst = reinterpret_cast<uint4 *>(R.host + o_dst);
        R.consumed = reinterpret_cast<uint32_t *>(R.host + o_consumed);
        for (int c = 0; c < n_codes; ++c) {
            R.syn.push_back(reinterpret_cast<uint32_t *>(R.host + o_syn[c]));
            R.est.push_back(R.host + o_est[c]);
            R.conv.push_back(R.host + o_conv[c]);
            R.iters.push_back(R.host + o_iters[c]);
            bpq::DecodeArgs &a = s->tmpl[c];
            a.syn = reinterpret_cast<const uint32_t *>(dev_host + o_syn[c]);
            a.est = dev_host + o_est[c];
            a.conv = dev_host + o_conv[c];
            a.iters = dev_host + o_iters[c];
        }
        // device memory: descriptors | head [n] | cap [n] | cq_count, status [3]
        uint8_t *p = static_cast<uint8_t *>(dev_mem);
        R.desc = reinterpret_cast<bpq::DecodeArgs *>(p);
        p += a256(sizeof(bpq::DecodeArgs) * n_codes);
        R.head = reinterpret_cast<uint32_t *>(p);
        p += a256(sizeof(uint32_t) * n_codes);
        R.cap_dev = reinterpret_cast<uint32_t *>(p);
        p += a256(sizeof(uint32_t) * n_codes);
        R.cq_count = reinterpret_cast<uint32_t *>(p);
        R.status = R.cq_count + 4;
        p += 256;
        R.out_dev = reinterpret_cast<bpq::ServeOut *>(p);
        std::vector<uint32_t> caps(n_codes, (uint32_t)slots_per_code);
        rc = bpq::cuda_check(cudaMemcpy(R.desc, s->tmpl.data(), sizeof(bpq::DecodeArgs) * n_codes,
                                        cudaMemcpyHostToDevice), "server descriptors");
        if (!rc)
            rc = bpq::cuda_check(cudaMemcpy(R.cap_dev, caps.data(), sizeof(uint32_t) * n_codes, cudaMemcpyHostToDevice),
                                 "server descriptors");
        if (!rc) rc = bpq::cuda_check(cudaMemset(R.cq_count, 0, 512), "server descriptors");  // and out_dev
    }
    if (!rc) {
        R.fn = bpq::pick_serve_kernel(variant);
        cudaError_t e = cudaFuncSetAttribute(R.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem);
        int per_sm = 0;
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, R.fn, bpq::kBatchThreads, s->smem);
        if (e != cudaSuccess || per_sm < 1) rc = fail(BPQ_ECUDA, "serving kernel does not fit on an SM");
        R.grid = per_sm * s->codes[0]->num_sms;
    }
    if (!rc) rc = bpq::cuda_check(cudaStreamCreateWithFlags(&R.st, cudaStreamNonBlocking), "server stream");
    if (!rc) rc = bpq::cuda_check(cudaEventCreateWithFlags(&R.exited, cudaEventDisableTiming), "server event");
    if (!rc) {
        // the launch path, captured once: clear the status words, start the grid
        bpq::ServeArgs args;
        args.codes = R.desc;
        args.cap = R.cap_dev;
        args.tail = reinterpret_cast<const uint32_t *>(dev_host + o_tail);
        args.head = R.head;
        args.closed = reinterpret_cast<const uint32_t *>(dev_host + o_closed);
        args.cq_count = R.cq_count;
        args.cq = reinterpret_cast<uint4 *>(dev_host + o_cq);
        args.cq_len = R.cq_len;
        args.status = R.status;
        args.idle_limit = R.idle_limit;
        args.stage_offset = (uint32_t)R.stage_offset;
        args.ncodes = n_codes;
        args.out = R.out_dev;
        args.dst = reinterpret_cast<const uint4 *>(dev_host + o_dst);
        args.consumed = reinterpret_cast<uint32_t *>(dev_host + o_consumed);
        cudaError_t e = cudaStreamBeginCapture(R.st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaMemsetAsync(R.status, 0, 3 * sizeof(uint32_t), R.st);  // error word and exit reason
            R.fn<<<(unsigned)R.grid, bpq::kBatchThreads, s->smem, R.st>>>(args);
            cudaError_t e2 = cudaStreamEndCapture(R.st, &R.graph);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&R.exec, R.graph, 0);
        if (e != cudaSuccess) rc = fail(BPQ_ECUDA, std::string("server launch graph: ") + cudaGetErrorString(e));
    }
    if (rc) {
        free_server(s);
        return rc;
    }
    *out = s;
    return BPQ_OK;
}

int bpq_server_slot_stats(bpq_server *s, long *code_switches, long *empty_scans, long *empty_claims) {
    if (!s || !s->slots) return fail(BPQ_EINVAL, "not a slot server");
    uint32_t st[6] = {0, 0, 0, 0, 0, 0};
    int rc = bpq::cuda_set_device(s->device);
    if (!rc) rc = bpq::cuda_check(cudaMemcpy(st, s->ring.status, sizeof st, cudaMemcpyDeviceToHost), "server stats");
    if (rc) return rc;
    if (code_switches) *code_switches = st[3];
    if (empty_scans) *empty_scans = st[4];
    if (empty_claims) *empty_claims = st[5];
    return BPQ_OK;
}

int bpq_server_stats(const bpq_server *s, long *launches) {
    if (!s) return fail(BPQ_EINVAL, "server is NULL");
    if (launches) *launches = s->launches;
    return BPQ_OK;
}

void bpq_server_free(bpq_server *s) { free_server(s); }

}  // extern "C"
