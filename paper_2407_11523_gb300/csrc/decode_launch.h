// Kernel arguments and launch-shape selection of the decode kernel.
#pragma once

#include <cuda_runtime.h>

#include "bpq_internal.h"

namespace bpq {

constexpr uint32_t kSmemHeader = 128;  // mbarrier + per-group shot indices

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
    int G, npt;                // warps per shot group, nodes per thread
    uint32_t slots_floats, group_bytes;
    float alpha, gamma, eps, clip, phi_clip;
    int ada_from1;
};

struct LaunchShape {
    int T, G, npt, NPT, groups_per_cta;
    uint32_t slots_floats, group_bytes;
    size_t smem;
};

int decode_launch_shape(const bpq_tanner *t, LaunchShape *s);
int decode_launch(const bpq_tanner *t, DecodeArgs &a, int variant, bool trace, cudaStream_t st, int *ctas_out);

}  // namespace bpq
