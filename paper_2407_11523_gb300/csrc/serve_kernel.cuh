// Slot-granular serving kernel (bpq_server_create_slots): a persistent grid
// that decodes single-shot requests as they arrive.  Each code has a ring of
// request slots in host-mapped memory; the host writes a request's syndrome
// into the next slot and publishes the code's request count (tail, a
// release store).  A shot group that finishes a shot takes the next
// published request of its CTA's current code at once: from the CTA's batch
// of claimed requests, which one group at a time refills (a shared-memory
// lock) by claiming up to one request per group of the CTA with a single
// compare-and-swap on the code's claim counter, so that a code's counter sees
// one claimer per CTA, not one per group.  It decodes it with decode_shot (the per-shot
// arithmetic of bpq_decode, so a served result equals the result of
// decoding that syndrome alone) and publishes its completion in a queue in
// host-mapped memory.  When the CTA's code has nothing left to claim, the
// CTA moves to another code with published requests, re-staging that code's
// adjacency (bulk TMA) and prior, as the batched kernel does.
//
// Waits are bounded: a CTA with nothing to claim sleeps about a microsecond
// and rescans; it exits when the host has closed the stream, or after
// idle_limit empty scans in a row (status word 2, the host relaunches the
// kernel if requests remain).  Nothing polls forever.
#pragma once

#include "decode_kernel.cuh"

namespace bpq {

// Output buffers of a request stream that the kernel writes directly: the
// caller's device-accessible (pinned) host buffers; est == nullptr: results
// go to the rings and the host copies them out.
struct ServeOut {
    uint8_t *est, *conv, *iters;
};

struct ServeArgs {
    const DecodeArgs *codes;   // per code: syn/est point at the code's rings (est slots padded to 16
                               // bytes), B = ring slots
    const uint32_t *cap;       // [ncodes] ring slots per code
    const uint32_t *tail;      // [ncodes] published requests (host-mapped, written by the host)
    uint32_t *head;            // [ncodes] claimed requests (device)
    const uint32_t *closed;    // host-mapped: 1 once every request has been published
    uint32_t *cq_count;        // device: completions so far
    uint4 *cq;                 // host-mapped completion queue [cq_len]: {e + 1, code, request number
                               //  (direct mode: the caller's request index), converged | iterations << 8}
    uint32_t cq_len;
    uint32_t *status;          // device: [1] error word (as bpq_decode's), [2] exit reason,
                               // [3] code switches, [4] empty scans, [5] claims that found nothing
    uint32_t idle_limit;       // empty scans before the kernel returns
    uint32_t stage_offset;     // byte offset of the staging area in dynamic shared memory
    int ncodes;
    const ServeOut *out;       // device: the caller's output buffers of this stream (est null: the rings)
    const uint4 *dst;          // host-mapped [ncodes][cap]: per slot {estimate offset (lo, hi), request, 0}
    uint32_t *consumed;        // host-mapped [ncodes][cap] (direct mode): request number + 1 whose syndrome
                               // the kernel has staged from the slot, which the host may then reuse
};

// Per-CTA staging of the requests in flight, after the code's group memory:
// estimates [groups][N] (decode_shot's layout) in an area of groups x N
// rounded up to 16 bytes per group, syndromes [groups][W], then the
// converged flags and iteration counts [groups].
__host__ __device__ inline size_t serve_stage_bytes(int groups, int N, int W) {
    return (size_t)groups * (((size_t)N + 15) & ~size_t(15)) + (size_t)groups * 4 * W + 2 * (size_t)groups + 16;
}

using ServeKernelFn = void (*)(const ServeArgs);
ServeKernelFn pick_serve_kernel(int variant);

namespace dk {

__device__ __forceinline__ uint32_t ld_acquire_sys(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(uint32_t *p, uint32_t v) {
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int VARIANT, int NPT>
__global__ void __launch_bounds__(kBatchThreads, 1) decode_serve_kernel(const ServeArgs s) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);
    int *ctl = reinterpret_cast<int *>(smem + 8);        // [0] the picked code, [1] stop reason
    int *grp_shot = reinterpret_cast<int *>(smem + 16);  // [kMaxGroupsPerCta]
    DecodeArgs *desc = reinterpret_cast<DecodeArgs *>(smem + kSmemHeader);
    uint8_t *tab = smem + kSmemHeader + kDescBytes;
    const int tid = threadIdx.x;

    if (tid == 0) {
        mbar_init(mbar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    __shared__ const uint32_t *ring_syn;
    __shared__ uint8_t *ring_est;
    // the CTA's batch of claimed requests of its current code: [cl_base,
    // cl_base + cl_cnt), refilled under cl_lock
    __shared__ int cl_lock, cl_base, cl_cnt;
    // each group's output offset and request number (direct mode), fetched
    // from host memory with the syndrome
    __shared__ uint4 grp_dst[kMaxGroupsPerCta];
    if (tid == 0) cl_lock = cl_base = cl_cnt = 0;
    int cur = -1;
    // the CTA's home code: every scan for a code with requests starts there,
    // so that the CTAs spread over the codes with requests instead of all
    // taking the first one published and then moving through the codes in
    // the same order
    const int from = (int)(blockIdx.x % (unsigned)s.ncodes);
    uint32_t phase = 0, idle = 0;
    ThreadAdj<NPT> adj;
    for (;;) {
        // ---- pick a code with published, unclaimed requests: warp 0 reads
        // the codes' counts in parallel (one code per lane, from `from` on) ----
        if (tid < 32) {
            int pick = -1;
            for (int base = 0; base < s.ncodes && pick < 0; base += 32) {
                const int k = base + tid;
                const int g = (from + k) % s.ncodes;
                const bool has = k < s.ncodes &&
                                 ld_acquire_sys(s.tail + g) > *reinterpret_cast<volatile const uint32_t *>(s.head + g);
                const uint32_t b = __ballot_sync(0xffffffffu, has);
                if (b) pick = (from + base + __ffs(b) - 1) % s.ncodes;
            }
            if (tid == 0) {
                int stop = 0;
                if (pick >= 0) {
                    idle = 0;
                } else {
                    atomicAdd(s.status + 4, 1u);
                    if (ld_acquire_sys(s.closed))
                        stop = 1;
                    else if (++idle > s.idle_limit)
                        stop = 2;
                    else
                        __nanosleep(1000);
                }
                ctl[0] = pick;
                ctl[1] = stop;
            }
        }
        __syncthreads();
        const int g = ctl[0], stop = ctl[1];
        if (g < 0) {
            __syncthreads();  // everyone has read ctl before thread 0 rewrites it
            if (stop) {
                if (tid == 0 && stop == 2) atomicMax(s.status + 2, 2u);
                return;
            }
            continue;
        }
        if (g != cur) {
            if (tid == 0) atomicAdd(s.status + 3, 1u);
            // switch code: descriptor, adjacency (bulk TMA), prior, zero slots; the
            // new table may cover the previous code's slots and state, written
            // with ordinary stores, so every thread fences them first
            const uint32_t *src = reinterpret_cast<const uint32_t *>(s.codes + g);
            for (int w = tid; w < (int)(sizeof(DecodeArgs) / 4); w += blockDim.x)
                reinterpret_cast<uint32_t *>(desc)[w] = src[w];
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
                // the kernel's ring pointers, kept aside; decode_shot reads and
                // writes the staging area (generic addresses into shared memory)
                ring_syn = desc->syn;
                ring_est = desc->est;
                uint8_t *st = smem + s.stage_offset;
                const size_t n16 = ((size_t)desc->N + 15) & ~size_t(15);
                desc->est = st;
                desc->syn = reinterpret_cast<const uint32_t *>(st + (size_t)desc->groups_per_cta * n16);
                desc->conv = st + (size_t)desc->groups_per_cta * (n16 + 4 * (size_t)desc->W);
                desc->iters = desc->conv + desc->groups_per_cta;
            }
            __syncthreads();
            if (tid == 0) {
                mbar_expect_tx(mbar, desc->table_bytes);
                bulk_g2s(tab, desc->table, desc->table_bytes, mbar);
            }
            load_prior(*desc, reinterpret_cast<float *>(tab + desc->table_bytes));
            const bool staged = mbar_wait_bounded(mbar, phase, 1u << 22);
            phase ^= 1u;
            if (__syncthreads_or(!staged)) {
                if (tid == 0) atomicExch(s.status + 1, 1u);
                mbar_wait_bounded(mbar, phase ^ 1u, 1u << 22);
                return;
            }
            const int T = desc->G * 32;
            const int group = tid / T;
            if (group < desc->groups_per_cta && tid - group * T == 0) {
                const GroupMem m = group_mem(*desc, tab, group);
                m.slots[4 * desc->n_pad] = 0.f;
            }
            load_adjacency<NPT>(*desc, tab, T, tid - group * T, desc->npt, adj);
            __syncthreads();
            cur = g;
        }
        const DecodeArgs &a = *desc;
        const int G = a.G, T = G * 32;
        const int group = tid / T, tg = tid - group * T;
        if (group < a.groups_per_cta) {
            const GroupMem m = group_mem(a, tab, group);
            const int bar_id = 1 + group;
            const uint32_t cap = s.cap[g];
            uint32_t t_seen = 0;  // (thread tg == 0) the code's count as last read, with acquire
            for (;;) {
                if (tg == 0) {
                    // take the next request of the CTA's batch; the group that
                    // finds the batch empty refills it from the code's counter
                    // (host memory is read again only when the requests seen so
                    // far are all claimed).  The lock is held only for that
                    // bounded refill; waiting for it is bounded too.
                    int claimed = -1;
                    uint32_t spins = 0;
                    while (atomicCAS(&cl_lock, 0, 1) != 0) {
                        if (++spins > (1u << 22)) {
                            atomicExch(s.status + 1, 3u);
                            break;
                        }
                        __nanosleep(32);
                    }
                    if (spins <= (1u << 22)) {
                        __threadfence_block();
                        volatile int *vb = &cl_base, *vc = &cl_cnt;
                        if (*vc == 0) {
                            const uint32_t want = (uint32_t)a.groups_per_cta;
                            uint32_t h = *reinterpret_cast<volatile const uint32_t *>(s.head + g);
                            if (h >= t_seen) t_seen = ld_acquire_sys(s.tail + g);
                            uint32_t backoff = 32;
                            // a deep backlog (at least 4 x grid x want published,
                            // unclaimed requests: more than every CTA could claim
                            // meanwhile) is claimed with one fetch-and-add and no
                            // retries; a shallow one with compare-and-swap, which
                            // never claims past the published count
                            if (h < t_seen && t_seen - h >= 4u * gridDim.x * want) {
                                *vb = (int)atomicAdd(s.head + g, want);
                                *vc = (int)want;
                            }
                            for (; *vc == 0;) {
                                if (h >= t_seen) {
                                    t_seen = ld_acquire_sys(s.tail + g);
                                    if (h >= t_seen) break;
                                }
                                const uint32_t n = min(t_seen - h, want);
                                const uint32_t o = atomicCAS(s.head + g, h, h + n);
                                if (o == h) {
                                    *vb = (int)h;
                                    *vc = (int)n;
                                    break;
                                }
                                h = o;
                                __nanosleep(backoff);
                                backoff = min(backoff * 2u, 1024u);
                            }
                        }
                        if (*vc > 0) {
                            claimed = *vb;
                            *vb = claimed + 1;
                            *vc = *vc - 1;
                        }
                        __threadfence_block();
                        atomicExch(&cl_lock, 0);
                    }
                    if (claimed >= 0 && (uint32_t)claimed >= t_seen) {
                        // (fetch-and-add path only, if the backlog test was
                        // outrun) wait for the request to be published, or for
                        // the stream to close without it; bounded
                        uint32_t n = 0;
                        for (;;) {
                            t_seen = ld_acquire_sys(s.tail + g);
                            if ((uint32_t)claimed < t_seen) break;
                            if (ld_acquire_sys(s.closed) || ++n > (1u << 24)) {
                                if (n > (1u << 24)) atomicExch(s.status + 1, 4u);
                                claimed = -1;
                                break;
                            }
                            __nanosleep(256);
                        }
                    }
                    grp_shot[group] = claimed;
                }
                group_sync(G, bar_id);
                const int k = grp_shot[group];
                if (k < 0) {
                    if (tg == 0) atomicAdd(s.status + 5, 1u);
                    break;
                }
                const int slot = (int)((uint32_t)k % cap);
                // stage the request's syndrome: coalesced loads from host memory
                // (ld.global.cv: the slot is rewritten by the host between uses)
                uint32_t *ssyn = const_cast<uint32_t *>(a.syn) + (size_t)group * a.W;
                for (int w = tg; w < a.W; w += T) ssyn[w] = __ldcv(ring_syn + (size_t)slot * a.W + w);
                if (tg == T - 1 && s.out->est) grp_dst[group] = __ldcv(s.dst + (size_t)g * cap + slot);
                group_sync(G, bar_id);
                // direct mode: the slot's syndrome and destination are in shared
                // memory now (read before the barrier), so the slot is free for
                // the next request even while this one decodes
                if (tg == 0 && s.out->est) st_release_sys(s.consumed + (size_t)g * cap + slot, (uint32_t)k + 1u);
                if (a.split)
                    decode_shot<VARIANT, NPT, false, true, false, true>(a, adj, m, a.npt, T, tg, G, bar_id, group,
                                                                         a.alpha);
                else
                    decode_shot<VARIANT, NPT, false, false, false, true>(a, adj, m, a.npt, T, tg, G, bar_id, group,
                                                                          a.alpha);
                group_sync(G, bar_id);
                // warp 0 alone writes to host memory: the estimate (decode_shot
                // wrote it at est + group * N) in 16-byte stores, to the request's
                // own output (direct mode: the offset the host left in the slot,
                // 16-byte aligned; the last partial chunk byte by byte) or to the
                // ring slot (stride N rounded up to 16), then the completion, which
                // carries the converged flag and iteration count
                if (tg < 32) {
                    const size_t n16 = ((size_t)a.N + 15) & ~size_t(15);
                    const uint8_t *se = a.est + (size_t)group * a.N;
                    uint8_t *const out_est = s.out->est;
                    uint8_t *dbase = ring_est + (size_t)slot * n16;
                    int full = (int)(n16 / 16);
                    if (out_est) {
                        const uint4 dm = grp_dst[group];
                        dbase = out_est + ((uint64_t)dm.x | ((uint64_t)dm.y << 32));
                        full = a.N / 16;
                        if (tg == 0) {
                            s.out->conv[dm.z] = a.conv[group];
                            s.out->iters[dm.z] = a.iters[group];
                        }
                        for (int j = 16 * full + tg; j < a.N; j += 32) dbase[j] = se[j];
                    }
                    uint4 *de = reinterpret_cast<uint4 *>(dbase);
                    for (int v = tg; v < full; v += 32) {
                        uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                        for (int b = 0; b < 16; ++b) {
                            const int j = 16 * v + b;
                            if (j < a.N) w[b >> 2] |= (uint32_t)se[j] << (8 * (b & 3));
                        }
                        de[v] = make_uint4(w[0], w[1], w[2], w[3]);
                    }
                    // the warp barrier orders the lanes' estimate stores before
                    // lane 0's fence, which orders them and the entry's fields
                    // before its release store
                    __syncwarp();
                    if (tg == 0) {
                        const uint32_t e = atomicAdd(s.cq_count, 1u);
                        uint4 *q = s.cq + (e % s.cq_len);
                        q->y = (uint32_t)g;
                        q->z = out_est ? grp_dst[group].z : (uint32_t)k;  // direct: the request itself
                        q->w = (uint32_t)a.conv[group] | ((uint32_t)a.iters[group] << 8);
                        __threadfence_system();
                        st_release_sys(&q->x, e + 1u);
                    }
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace dk
}  // namespace bpq
