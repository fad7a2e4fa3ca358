// Kernel arguments, launch-shape selection and per-variant kernel lookup of
// the decode kernel.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "bpq_internal.h"

namespace bpq {

// Per-qubit state arrays (each n_pad floats) a shot group of the flooding
// kernels keeps in shared memory: EWAInit the next prior Pi^(t+1) and
// alpha Pi^(0); Momentum Q^(t-1), g; AdaGrad Q^(t-1), G.  The kernels and the
// host's shared-memory sizing both read this.
__host__ __device__ constexpr int decode_state_arrays(int variant) { return variant == BPQ_PLAIN ? 0 : 6; }

constexpr uint32_t kSmemHeader = 256;  // mbarrier, current item, per-group shot indices
constexpr int kMaxGroupsPerCta = 32;   // named barriers limit multi-warp groups to 15

struct DecodeArgs {
    const uint8_t *table;      // staged adjacency (bpq_tanner::table on the device)
    uint32_t table_bytes;      // multiple of 16
    uint32_t off_chk_pauli, off_var_pauli;
    const uint32_t *syn;       // [B][W]
    const float *prior;        // [N][3]
    uint8_t *est, *conv, *iters;
    uint32_t *work;            // [0] next shot, [1] device error word
    float *tr_v2c, *tr_c2v, *tr_Q;
    uint8_t *tr_dec;
    const int32_t *var_canon, *chk_ptr;
    int N, M, E, W, B, max_iter;
    int G;                     // warps per shot group
    int n_pad;                 // N rounded up to a multiple of 4 (shared-memory array stride)
    uint32_t slots_floats, group_bytes;
    float alpha, gamma, eps, clip, delta_clip, phi_clip;
    float clip2;               // msg_clip in bits (msg_clip log2 e)
    int ada_from1;
    int split;                 // 0: generic layout; 1: split layout (bpq_tanner::split);
                               // 2: split layout with every slot used (bpq_tanner::full)
    // used by the batched kernel only
    int npt, groups_per_cta;
};

constexpr uint32_t kDescBytes = (sizeof(DecodeArgs) + 15) & ~15u;  // descriptor copy in shared memory
constexpr int kBatchThreads = 1024;  // CTA size of the batched kernel

constexpr int kMaxBatchCtas = 1024;  // entries of the starting-item array

// Arguments of the batched kernel, all in device memory: per-item
// descriptors (B = the item's shots), each CTA's starting item, and the
// counters work[1] (device error word) and work[2 + g] (next shot of item g).
struct BatchArgs {
    const DecodeArgs *codes;
    const int *start;
    int ncodes;
    uint32_t *work;
};

// Bytes of the counter block of a batch of n items (zeroed before each run).
inline size_t batch_counter_bytes(int n) { return ((size_t)4 * (2 + n) + 255) & ~size_t(255); }

struct LaunchShape {
    int T, G, npt, groups_per_cta;
    int n_pad;
    uint32_t slots_floats, group_bytes;
    size_t smem;
};

using DecodeKernelFn = void (*)(const DecodeArgs);
using BatchKernelFn = void (*)(const BatchArgs);

// Kernels of one variant, for nodes per thread npt in [1, 4]; split selects the
// specialisation for tables in the split layout, and the _full functions the
// non-trace kernels for split tables without padding.
DecodeKernelFn pick_plain(int npt, bool trace, bool split);
DecodeKernelFn pick_plain_full(int npt);
DecodeKernelFn pick_momentum(int npt, bool trace, bool split);
DecodeKernelFn pick_momentum_full(int npt);
DecodeKernelFn pick_adagrad(int npt, bool trace, bool split);
DecodeKernelFn pick_adagrad_full(int npt);
DecodeKernelFn pick_ewainit(int npt, bool trace, bool split);
DecodeKernelFn pick_ewainit_full(int npt);
DecodeKernelFn pick_aewa(int npt, bool trace, bool split);
DecodeKernelFn pick_aewa_full(int npt);
// Batched kernels (decode_*_batch.cu): generic = some item uses the generic
// table layout (else every item has the split layout).
BatchKernelFn pick_plain_batch(bool generic);
BatchKernelFn pick_momentum_batch(bool generic);
BatchKernelFn pick_adagrad_batch(bool generic);
BatchKernelFn pick_ewainit_batch(bool generic);
// Two shots per thread (decode_pair.cuh), split tables, npt in {1, 2}; the
// _full functions for split tables without padding.
DecodeKernelFn pick_plain_pair(int npt);
DecodeKernelFn pick_plain_pair_full(int npt);
DecodeKernelFn pick_momentum_pair(int npt);
DecodeKernelFn pick_momentum_pair_full(int npt);
DecodeKernelFn pick_adagrad_pair(int npt);
DecodeKernelFn pick_adagrad_pair_full(int npt);
DecodeKernelFn pick_ewainit_pair(int npt);
DecodeKernelFn pick_ewainit_pair_full(int npt);

// Bounds-checked kernels (decode_debug.cu; bpq_set_debug_checks): npt in
// {1, 2}, pairs on split layouts; nullptr where none is compiled.
DecodeKernelFn pick_debug(int variant, int npt, bool pairs, int layout);

int decode_launch_shape(const bpq_tanner *t, int variant, LaunchShape *s);
// Whether bpq_decode runs the two-shots-per-thread kernel for this graph and
// variant (split table layout, not AEWA-BP, not a trace), and its shape: a
// shot group of s->T threads decodes two shots at a time.
bool decode_uses_pairs(const bpq_tanner *t, int variant, bool trace);
int decode_pair_shape(const bpq_tanner *t, int variant, LaunchShape *s);
constexpr int kMaxPairGroupsPerCta = 28;  // two shot indices per group in the 256-byte header
// Automatic choice of two shots per thread: from this many shots per
// resident one-shot group of the batch.
constexpr long kPairShotsPerGroup = 128;
// Shape of a code inside the batched kernel (CTAs of kBatchThreads threads).
int decode_batch_shape(const bpq_tanner *t, int variant, LaunchShape *s);

// Starting item of each of `ctas` CTAs, spread over the items in proportion
// to weight[g] (shots x edges; items of weight 0 get none).
void batch_start_items(const std::vector<double> &weight, int ctas, int *start);

// Shared host helpers (api.cu).
int need_uploaded(const bpq_tanner *t);
int cuda_check(cudaError_t e, const char *what);
int cuda_set_device(int device);
int fill_decode_args(const bpq_tanner *t, const uint32_t *syn, const float *prior, int variant,
                     const bpq_params *params, int max_iter, int B, void *work, DecodeArgs &a);
int decode_launch(const bpq_tanner *t, DecodeArgs &a, int variant, bool trace, cudaStream_t st, int *ctas_out);

}  // namespace bpq
