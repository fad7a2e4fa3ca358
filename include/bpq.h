/*
 * bpq.h - C ABI of the GB300 (sm_103a) GF(4) belief-propagation decoder for
 * surface codes: plain LLR-BP4, Momentum-BP, AdaGrad-BP and EWAInit-BP under
 * the parallel (flooding) schedule, after "Improved Belief Propagation
 * Decoding Algorithms for Surface Codes" (Chen, Yi, Liang, Wang).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Return value: BPQ_OK (0) on success, a negative bpq_status otherwise.
 *    bpq_last_error() then returns a message for the calling thread.
 *  - Pointers named *_dev are device pointers owned by the caller (for
 *    example torch tensors' data_ptr()); pointers named *_host are host
 *    pointers owned by the caller.  The library never frees them.
 *  - Alignment: device buffers passed as void * (workspaces, dev_buf,
 *    dev_mem) start on a 16-byte boundary (cudaMalloc and torch give 256),
 *    and uint32 / float arrays on a 4-byte one; an entry point refuses a
 *    misaligned base with BPQ_EINVAL before any device access.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  GPU entry
 *    points only enqueue work on it and return; they do not synchronize,
 *    except where a function says otherwise.
 *  - Pauli codes: 0 = I, 1 = X, 2 = Y, 3 = Z.  Per-qubit probability and
 *    LLR triples are ordered (X, Y, Z).
 *  - Syndromes are bit-packed: shot b, check i is bit (i % 32) of the uint32
 *    word syn[b * W + i / 32], W = ceil(M / 32).
 *  - A non-converged shot is a normal result (converged = 0), not an error.
 */
#ifndef BPQ_H
#define BPQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bpq_tanner bpq_tanner; /* opaque Tanner graph, library-owned */

enum bpq_code { BPQ_PLANAR = 0, BPQ_TORIC = 1, BPQ_XZZX = 2 };

/* Decoder variants: LLR-BP4 (Sec. II-B1), Momentum-BP (Sec. III-A1,
 * Algorithm 1), AdaGrad-BP (Sec. III-A2), EWAInit-BP (Sec. III-B,
 * Algorithm 2), and AEWA-BP (Appendix C): EWAInit-BP run with
 * alpha = 1.0, 0.9, ..., 0.0 in turn until a run converges; its outputs are
 * those of the last run (iters counts that run only).  AEWA-BP is offered by
 * bpq_decode and bpq_decode_host (not by the trace, batch or server paths). */
enum bpq_variant { BPQ_PLAIN = 0, BPQ_MOMENTUM = 1, BPQ_ADAGRAD = 2, BPQ_EWAINIT = 3, BPQ_AEWA = 4 };

enum bpq_status {
    BPQ_OK = 0,
    BPQ_EINVAL = -1,  /* bad argument (size, probability, null pointer, ...) */
    BPQ_ENOMEM = -2,  /* host or device allocation failed */
    BPQ_ECUDA = -3,   /* a CUDA runtime call failed */
    BPQ_ESTATE = -4   /* handle not in the required state (e.g. not uploaded) */
};

/* Decoder parameters.
 *   alpha: Momentum-BP learning rate (eq. (mombp2)); AdaGrad-BP boost rate
 *          (eq. (boost)); EWAInit-BP discount factor (eq. (EWAInit)).
 *          Unused by plain BP.
 *   gamma: Momentum-BP decay (eq. (mombp1)); unused otherwise.
 *   eps:   AdaGrad-BP epsilon of eq. (boost).
 *   msg_clip: every check-to-variable and variable-to-check LLR message is
 *          clipped to [-msg_clip, msg_clip] (the paper is silent on message
 *          saturation; 30 by default).
 *   adagrad_g_from_iter1: 1 = the squared-gradient sum G starts at t = 1
 *          (g'(1) = -S(1)); 0 = G starts at t = 2.  Eq. (boost) applies from
 *          t = 2 either way ("takes effect after the first iteration"). */
typedef struct {
    float alpha;
    float gamma;
    float eps;
    float msg_clip;
    int32_t adagrad_g_from_iter1;
} bpq_params;

/* Paper defaults for a variant (Sec. III-A2: AdaGrad alpha = 5; Sec. IV-A /
 * Table I: Momentum gamma = 0, alpha = 0.5; EWAInit alpha = 0.5). */
void bpq_default_params(int variant, bpq_params *out);

/* ------------------------------------------------------------ Tanner graph */

/* Build the check matrix of a surface code of distance d (2 <= d <= 32) on
 * the host.  Planar: [[2d^2-2d+1, 1, d]]; toric: [[2d^2, 2, d]] (d >= 3);
 * XZZX: the planar code with a Hadamard on the second hypergraph-product
 * block (Sec. II-A; Sec. IV-B builds the codes as hypergraph products of
 * repetition codes).  Qubit order: hypergraph-product block 1 (row-major
 * d x d, toric) or (d x d, planar), then block 2; checks: X-type rows, then
 * Z-type rows.  Does not touch the GPU.  *out must be released with
 * bpq_free_tanner.  Errors: EINVAL for a bad code or d, ENOMEM. */
int bpq_build_tanner(int code, int d, bpq_tanner **out);

/* Build a Tanner graph from a dense M x N matrix of Pauli codes (row-major,
 * host).  Every check and every qubit may have at most 4 non-identity
 * entries (the decoder's padded degree); K is reported as -1 and no logical
 * operators are known unless set with bpq_tanner_set_logicals.
 * Errors: EINVAL (sizes, entries > 3, degree > 4, max(N, M) > 2048), ENOMEM. */
int bpq_tanner_from_paulis(int M, int N, const uint8_t *H_host, bpq_tanner **out);

/* Give a custom Tanner graph 2K logical operators (2K x N Pauli codes,
 * host) for bpq_check_logical.  Must precede bpq_tanner_upload. */
int bpq_tanner_set_logicals(bpq_tanner *t, int n_logicals, const uint8_t *L_host);

/* Copy the graph's device tables to `device` (synchronous; allocates device
 * memory owned by the handle).  Required before any GPU entry point.
 * Errors: ECUDA, ENOMEM, ESTATE if already uploaded. */
int bpq_tanner_upload(bpq_tanner *t, int device);

/* Sizes: N qubits, M checks, E edges (non-identity entries), K logical
 * qubits (-1 if unknown).  Any output pointer may be NULL. */
int bpq_tanner_info(const bpq_tanner *t, int *N, int *M, int *E, int *K);

/* The message layout the decode kernels use for this graph (host only, no
 * GPU needed): 0 generic (slots by check order, per-edge Pauli selects);
 * 1 split (no Y entries and at most two X and two Z edges per qubit: the
 * edge's Pauli is fixed by its slot); 2 split without padding (every check
 * of degree 4 and every qubit with two X and two Z edges, e.g. the toric
 * codes).  Results do not depend on the layout.  Errors: EINVAL (NULL). */
int bpq_tanner_layout(const bpq_tanner *t, int *layout);

/* Check-major CSR of the graph on the host: chk_ptr[M+1], chk_var[E],
 * pauli[E]; edges of check i are chk_ptr[i] .. chk_ptr[i+1]-1 in increasing
 * qubit order.  This is also the edge order of bpq_decode_trace. */
int bpq_tanner_export(const bpq_tanner *t, int32_t *chk_ptr, int32_t *chk_var, uint8_t *pauli);

/* The 2K logical operators used by bpq_check_logical (2K x N codes, host).
 * Errors: ESTATE when none are known. */
int bpq_tanner_logicals(const bpq_tanner *t, uint8_t *L_host);

void bpq_free_tanner(bpq_tanner *t);

/* ---------------------------------------------------------------- sampling */

/* i.i.d. single-qubit Pauli channel (Sec. IV: depolarising p/3 each; the
 * biased channel of Sec. IV-B3 likewise), shots shot0 .. shot0+B-1.
 * Generator: Philox4x64-10 (Salmon et al., SC 2011), key (seed, 0), counter
 * (shot, j / 4, 0, 0), word j % 4 is qubit j's draw u; u < floor(px 2^64)
 * -> X, < floor((px+py) 2^64) -> Y, < floor((px+py+pz) 2^64) -> Z, else I
 * (sums in double, in that order).  err_dev: B x N codes; syn_dev: B x W
 * packed words, s_i = XOR_j <E_j, H_ij> (Sec. II-A).  Either output may be
 * NULL only if B == 0.  Errors: EINVAL (px, py, pz < 0 or sum >= 1, B < 0),
 * ESTATE, ECUDA. */
int bpq_sample(const bpq_tanner *t, double px, double py, double pz, uint64_t seed, uint64_t shot0,
               int B, uint8_t *err_dev, uint32_t *syn_dev, void *stream);

/* ---------------------------------------------------------------- decoding */

/* Bytes of device scratch that bpq_decode needs (a shot work queue and an
 * error word); the caller allocates it, it need not be initialised, and
 * concurrent decodes need separate scratch. */
size_t bpq_decode_workspace_bytes(void);

/* Decode B shots (Sec. II-B1 with the variant rules of Sec. III; flooding
 * schedule, Algorithm 2's control flow for every variant):
 *   prior LLR Pi = ln(p^I / p^W); m(0) = lambda(Pi) (eq. (init));
 *   per iteration t = 1..max_iter: [EWAInit, t > 1: Pi(t) = alpha Pi(0) +
 *   (1-alpha) Q(t-1)]; check-to-variable update (eq. (h_update)); posterior
 *   Q (eq. (p_update) / (mombp1)-(mombp2) / (boost)); variable-to-check
 *   update lambda_{H_ij}(Q - own anticommuting message) (eqs. (v_update),
 *   (mombp5)); hard decision; stop as soon as <H, E^> = s.
 * syn_dev: B x W packed syndromes.  prior_dev: N x 3 float probabilities
 * (p^X, p^Y, p^Z) per qubit, each in (0, 1) with sum < 1, shared by all
 * shots.  params: NULL = bpq_default_params(variant).  max_iter in
 * [1, 255].  Outputs: est_dev B x N Pauli codes (the decision of the last
 * iteration run), conv_dev B flags (1 = syndrome matched), iters_dev B
 * iteration counts (1 .. max_iter).  work_dev: bpq_decode_workspace_bytes()
 * of device scratch.  Shots are independent: any split of a batch gives the
 * same per-shot results.  Errors: EINVAL, ESTATE, ECUDA; a device-side
 * failure is reported by bpq_decode_status. */
int bpq_decode(const bpq_tanner *t, const uint32_t *syn_dev, const float *prior_dev, int variant,
               const bpq_params *params, int max_iter, int B, uint8_t *est_dev, uint8_t *conv_dev,
               uint8_t *iters_dev, void *work_dev, void *stream);

/* Synchronize `stream` and read the device error word a decode left in
 * work_dev: 0 = no error; nonzero = a bounded wait inside the kernel gave up
 * (the outputs of that launch are then invalid). */
int bpq_decode_status(const void *work_dev, void *stream, int *device_error);

/* bpq_decode with host buffers: copies syn_host (B x W words) and
 * prior_host (N x 3) to the device, decodes, copies est/conv/iters back to
 * the host buffers, and synchronizes `stream` before returning.  dev_buf is
 * caller-owned device memory of at least bpq_decode_host_bytes(t, B) bytes.
 * Host buffers should be pinned for the copies to run asynchronously.  From
 * B >= 131072 the batch is cut into up to 8 chunks whose host-to-device
 * copies, decodes and device-to-host copies overlap; the chunks decode
 * alternately on `stream` and on a library stream (so that one chunk's last
 * shots overlap the next chunk), and the copies run on two more library
 * streams, all three per device, created on first use and kept (calls from
 * several host threads on one device share them).  Errors: as bpq_decode,
 * plus EINVAL (NULL host buffers, dev_buf smaller than
 * bpq_decode_host_bytes(t, B) or not 16-byte aligned) and ECUDA (a copy or
 * the synchronization failed). */
size_t bpq_decode_host_bytes(const bpq_tanner *t, int B);
int bpq_decode_host(const bpq_tanner *t, const uint32_t *syn_host, const float *prior_host,
                    int variant, const bpq_params *params, int max_iter, int B, uint8_t *est_host,
                    uint8_t *conv_host, uint8_t *iters_host, void *dev_buf, size_t dev_buf_bytes,
                    void *stream);

/* bpq_decode_host for callers that cannot allocate device memory (no
 * cudaMalloc, cudaFree or allocating library call is made): for example a
 * real-time decoding loop that must not allocate once running, or a process
 * whose device memory is owned by another runtime's allocator.  The paper has
 * no counterpart; this is an interface addition.  The device copies of the
 * inputs and outputs and the decoder's shot queue live in one fixed 8 MiB
 * array inside the library (held on every GPU that loads the library until
 * the process exits).  B is limited to bpq_decode_host_noalloc_max_shots(t)
 * (about 16000 toric d = 15 shots); larger batches return BPQ_EINVAL with a
 * message.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.  The cached address does not survive a cudaDeviceReset:
 * resetting a device after that first call is not supported.  With CUDA's
 * default lazy module loading, the first launch of each decode kernel (one
 * per variant and message layout, see bpq_tanner_layout) loads its module,
 * and the driver may allocate device memory for it: make one warm-up call
 * per variant and code family before the loop that must not allocate, or
 * run with CUDA_MODULE_LOADING=EAGER.  All calls share the one array, which
 * keeps the last call's contents (the shot queue is reset on every call):
 * calls that may overlap on the GPU (other streams, other host threads) race
 * and must be serialised by the caller.  Arguments and errors otherwise as
 * bpq_decode_host; the stream is synchronized before returning. */
int bpq_decode_host_noalloc(const bpq_tanner *t, const uint32_t *syn_host, const float *prior_host, int variant,
                            const bpq_params *params, int max_iter, int B, uint8_t *est_host, uint8_t *conv_host,
                            uint8_t *iters_host, void *stream);
int bpq_decode_host_noalloc_max_shots(const bpq_tanner *t);

/* Per-iteration record for parity checks (small B): runs exactly T
 * iterations without the stopping rule and writes, in check-major edge
 * order (bpq_tanner_export), m_v2c_dev [B][T+1][E] (t = 0 is eq. (init)),
 * m_c2v_dev [B][T][E], Q_dev [B][T][N][3] and dec_dev [B][T][N].  Any
 * record pointer may be NULL.  T in [1, 255].  Errors: as bpq_decode
 * (AEWA-BP has no trace: EINVAL). */
int bpq_decode_trace(const bpq_tanner *t, const uint32_t *syn_dev, const float *prior_dev,
                     int variant, const bpq_params *params, int T, int B, float *m_v2c_dev,
                     float *m_c2v_dev, float *Q_dev, uint8_t *dec_dev, void *work_dev, void *stream);

/* Launch shape of bpq_decode: threads per shot group (a multiple of 32, at
 * most 1024, covering max(N, M) with at most 2 nodes per thread, or at most 4
 * with at most 512 threads) and shot groups per CTA (at most 15, or 32 for
 * one-warp groups).  A shot group decodes one shot at a time, or two with two
 * shots per thread (bpq_set_shots_per_thread; then at most 2 nodes per
 * thread and 28 one-warp groups per CTA).  0 = let the library choose (two
 * nodes per thread, about 256 threads per CTA).  Stored in the
 * handle; bpq_get_launch reports the shape of the plain/Momentum/AdaGrad/
 * EWAInit kernels. */
int bpq_set_launch(bpq_tanner *t, int threads_per_shot, int shots_per_cta);
int bpq_get_launch(const bpq_tanner *t, int *threads_per_shot, int *shots_per_cta, int *ctas);

/* Shots per thread of bpq_decode (an implementation choice; the paper has no
 * GPU design): 1 = each thread works on one shot; 2 = each thread works on
 * the same nodes of two shots, whose messages share 64-bit shared-memory
 * slots and packed f32x2 arithmetic, and each of the two "lanes" takes the
 * next shot from the queue as soon as its own shot stops (split table layout
 * only, see bpq_tanner_layout; plain, Momentum, AdaGrad and EWAInit BP; not
 * the trace, serial, batched or AEWA-BP paths); 0 = automatic (2 where it
 * applies and the batch holds at least 128 shots per resident one-shot shot
 * group, e.g. 77824 toric d = 15 shots on a GB300: a pair's iteration does two
 * shots' work, so smaller batches, whose time is set by their slowest shots,
 * finish sooner with one shot per thread).  Per-shot results are the same
 * bit for bit either way.  bpq_get_shots_per_thread reports what bpq_decode
 * will use for `variant` on large batches.
 * Errors: EINVAL (value outside 0..2, 2 on a table without the split
 * layout, a stored launch shape that does not fit). */
int bpq_set_shots_per_thread(bpq_tanner *t, int shots_per_thread);
int bpq_get_shots_per_thread(const bpq_tanner *t, int variant, int *shots_per_thread);

/* Bounds-checked decoding (a test aid; the paper has no counterpart): with
 * on != 0, bpq_decode and bpq_decode_host run copies of the decode kernels
 * compiled with checks on every shared-memory layout, slot index, table
 * offset and output index.  A failed check sets the device error word that
 * bpq_decode_status reads (value 5), substitutes a safe index and carries on
 * (or, for a layout that does not fit, makes the CTA return before its first
 * barrier); nothing traps.  Results are those of the unchecked kernels when
 * every check passes.  Plain, Momentum, AdaGrad and EWAInit BP, at most two
 * nodes per thread; other launches return EINVAL while it is on. */
int bpq_set_debug_checks(bpq_tanner *t, int on);

/* Autotuner of the launch shape (an addition; the paper has no GPU design):
 * times bpq_decode on the caller's sample batch (same arguments as
 * bpq_decode) for every candidate shape - one or two shots per thread, 1..4
 * nodes per thread (1..2 with two shots per thread), 1..32 shot groups per
 * CTA - and stores the fastest in the handle (as bpq_set_launch and
 * bpq_set_shots_per_thread would).  Synchronizes `stream`; the outputs are
 * those of the last trial.  Reports the chosen shape and its time per
 * launch (any output pointer may be NULL).  Errors: as bpq_decode, plus
 * EINVAL when B < 1 or no shape fits the code; on an error the handle keeps
 * its previous shape. */
int bpq_autotune(bpq_tanner *t, const uint32_t *syn_dev, const float *prior_dev, int variant,
                 const bpq_params *params, int max_iter, int B, uint8_t *est_dev, uint8_t *conv_dev,
                 uint8_t *iters_dev, void *work_dev, void *stream, int *threads_per_shot, int *shots_per_cta,
                 float *best_ms);

/* ---------------------------------------------------------------- serial schedule */

/* Decoding under the serial schedule of Algorithm 1 (Sec. III-A1): in each
 * iteration the qubits are visited in index order and qubit j takes the
 * c->v messages of its checks (eq. (h_update)) from the v->c messages as
 * they stand (already updated in this iteration for the qubits before j),
 * updates its posterior by the variant's rule and sends new v->c messages
 * (eq. (v_update); eq. (mombp5) for Momentum and AdaGrad); the hard
 * decision and syndrome test follow each full sweep.  The kernel runs the
 * sweep's dependency levels in order, all qubits of a level at once, which
 * gives the serial order's result exactly; one warp decodes one shot.
 * variant: plain, Momentum, AdaGrad or EWAInit BP (EINVAL otherwise).
 * Arguments, layouts, ownership, asynchrony and errors as bpq_decode; iters
 * counts sweeps.  EINVAL also when one shot's state does not fit in shared
 * memory (about 10^4 edges for EWAInit-BP).  A warp decodes one shot, or two
 * (bpq_set_serial_shots_per_warp) with the same per-shot results bit for
 * bit. */
int bpq_decode_serial(const bpq_tanner *t, const uint32_t *syn_dev, const float *prior_dev, int variant,
                      const bpq_params *params, int max_iter, int B, uint8_t *est_dev, uint8_t *conv_dev,
                      uint8_t *iters_dev, void *work_dev, void *stream);

/* Shots per warp of bpq_decode_serial (an implementation choice; the paper
 * has no GPU design): 1 = each warp decodes one shot; 2 = each warp decodes
 * two, its lanes working on the same qubit of both, whose messages share
 * 64-bit shared-memory slots and packed f32x2 arithmetic (each shot stops on
 * its own and the warp takes the next one for that half); 0 = automatic (2
 * where shared memory still holds 16 two-shot warps per SM and the batch
 * holds at least 128 shots per resident one-shot warp, e.g. 622592 planar
 * d = 7 shots on a GB300; the kernel is latency-bound, so codes whose
 * two-shot warps fill shared memory sooner, such as toric d = 15, keep one
 * shot per warp).  The trace keeps one shot per warp.
 * Errors: EINVAL (a value outside 0..2); bpq_decode_serial returns EINVAL
 * for 2 when two shots of the code do not fit in shared memory. */
int bpq_set_serial_shots_per_warp(bpq_tanner *t, int shots_per_warp);

/* Per-sweep record of the serial schedule, in bpq_decode_trace's layout:
 * exactly T sweeps, no stopping rule; m_v2c_dev [B][T+1][E] holds each
 * edge's v->c message as sent in that sweep, m_c2v_dev [B][T][E] the c->v
 * message its qubit took.  Errors: as bpq_decode_serial. */
int bpq_decode_serial_trace(const bpq_tanner *t, const uint32_t *syn_dev, const float *prior_dev, int variant,
                            const bpq_params *params, int T, int B, float *m_v2c_dev, float *m_c2v_dev, float *Q_dev,
                            uint8_t *dec_dev, void *work_dev, void *stream);

/* ---------------------------------------------------------------- batched decoding */

/* Many codes in one persistent launch (an interface addition; the paper
 * decodes one code at a time).  Each item is one code's batch: syndromes,
 * prior and outputs exactly as for bpq_decode.  All items share the variant
 * (plain, Momentum, AdaGrad or EWAInit BP), parameters and max_iter.  A CTA
 * of 1024 threads (at 64 registers a thread, the whole register file of an
 * SM) works on one item at a time, split into that code's shot groups (see
 * bpq_set_batch_launch): they take the item's shots one by one from a
 * per-item counter until none are left, and the CTA then moves to another
 * item with shots left, re-staging that code's adjacency.  CTAs start
 * spread over the items in proportion to shots x edges.  Per-shot results
 * equal those of bpq_decode bit for bit. */
typedef struct {
    const bpq_tanner *tanner;  /* uploaded; all items on one device */
    const uint32_t *syn_dev;   /* [B][ceil(M/32)] */
    const float *prior_dev;    /* [N][3] */
    int B;
    uint8_t *est_dev, *conv_dev, *iters_dev;
} bpq_batch_item;

typedef struct bpq_batch bpq_batch; /* opaque plan, library-owned */

/* Device workspace needed by a plan of n_items items (0 if n_items < 1). */
size_t bpq_batch_workspace_bytes(int n_items);

/* Build the plan: per-item counters, descriptors and the CTAs' starting
 * items, copied into work_dev (caller-owned, bpq_batch_workspace_bytes
 * large, to stay untouched while the plan is used).  Synchronizes `stream`.
 * Errors: EINVAL (no items, a NULL buffer, a variant other than the four,
 * max_iter outside [1, 255], too small a workspace), ESTATE (an item's
 * tanner not uploaded, or items on different devices), ECUDA.  Release with
 * bpq_batch_free. */
int bpq_batch_plan(const bpq_batch_item *items, int n_items, int variant, const bpq_params *params, int max_iter,
                   void *work_dev, size_t work_bytes, void *stream, bpq_batch **out);

/* Enqueue one run of the plan on `stream` (a counter reset and one kernel
 * launch; no host synchronization and no allocation, so the call can be
 * captured in a CUDA graph).  Runs of one plan must not overlap.  Errors:
 * EINVAL (NULL plan), ECUDA (the launch failed). */
int bpq_batch_launch(const bpq_batch *b, void *stream);

/* ctas: CTAs per launch; items: n_items; npt_max: the largest nodes per
 * thread of an item; shots: total shots.  Any pointer may be NULL.
 * Errors: EINVAL (NULL plan). */
int bpq_batch_info(const bpq_batch *b, int *ctas, int *items, int *npt_max, long *shots);
void bpq_batch_free(bpq_batch *b);

/* Shape of a code inside the batched kernel and the servers (an
 * implementation choice; the paper has no GPU design), stored in the handle
 * and read when a plan or server is built: nodes_per_thread 1 or 2 sets the
 * threads per shot group (max(N, M) / nodes_per_thread rounded up to a
 * multiple of 32, at most 1024), and the CTA holds as many groups as fit in
 * its 1024 threads (at most 15 multi-warp or 32 one-warp groups) and in
 * 227 KB of shared memory.  0 = automatic: the choice that keeps the most
 * node slots of a CTA busy (groups x max(N, M) / (nodes_per_thread x 1024)),
 * two nodes per thread on a tie.  Independent of bpq_set_launch.
 * Errors: EINVAL (a value outside 0..2, or a shape that does not fit).
 * bpq_get_batch_launch reports the shape for `variant` (any output pointer
 * may be NULL). */
int bpq_set_batch_launch(bpq_tanner *t, int nodes_per_thread);
int bpq_get_batch_launch(const bpq_tanner *t, int variant, int *threads_per_shot, int *shots_per_cta,
                         int *nodes_per_thread);

/* Autotuner of bpq_set_batch_launch: times a one-item plan of the caller's
 * sample (arguments as bpq_decode; work_dev at least
 * bpq_batch_workspace_bytes(1) bytes) with one and with two nodes per
 * thread, and stores the faster in the handle.  Synchronizes `stream`; the
 * outputs are those of the last trial.  Reports the choice and its time per
 * launch (any output pointer may be NULL).  Errors: as bpq_batch_plan and
 * bpq_batch_launch (a workspace below bpq_batch_workspace_bytes(1): EINVAL). */
int bpq_autotune_batch(bpq_tanner *t, const uint32_t *syn_dev, const float *prior_dev, int variant,
                       const bpq_params *params, int max_iter, int B, uint8_t *est_dev, uint8_t *conv_dev,
                       uint8_t *iters_dev, void *work_dev, size_t work_bytes, void *stream,
                       int *nodes_per_thread, float *best_ms);

/* ---------------------------------------------------------------- serving */

/* Continuous-batching decoding server (an interface addition; the paper
 * decodes offline batches).  n_lanes CUDA streams each own a slice of the
 * caller's device memory for max_batch shots (the device-memory budget:
 * at most n_lanes x max_batch shots are on the device at once).  Requests
 * (one syndrome of one of the server's codes each) that have arrived wait
 * in a FIFO; whenever a lane is free, all waiting requests up to max_batch
 * are grouped by code and decoded there by one batched launch (see
 * bpq_batch_plan), with their copies on the lane's stream, so requests that
 * arrive while other lanes are busy run concurrently with them.  A
 * request's result is the one bpq_decode gives for it alone. */
typedef struct bpq_server bpq_server;

size_t bpq_server_device_bytes(const bpq_tanner *const *codes, int n_codes, int n_lanes, int max_batch);

/* codes: uploaded Tanner graphs on one device; priors_dev[c]: [N_c][3]
 * float probabilities of code c.  Creates the lanes' streams, events and
 * pinned host staging.  Errors: EINVAL, ESTATE, ECUDA. */
int bpq_server_create(const bpq_tanner *const *codes, const float *const *priors_dev, int n_codes, int variant,
                      const bpq_params *params, int max_iter, int n_lanes, int max_batch, void *dev_mem,
                      size_t dev_bytes, bpq_server **out);

/* Serve a request trace in real time (host wall clock from the call):
 * request r is decoding code code[r], becomes available at arrival_s[r]
 * seconds (non-decreasing), its packed syndrome is syn_host[syn_off[r] ..
 * + ceil(M/32)), and its outputs go to est_host[est_off[r] .. + N] (within
 * est_bytes), conv_host[r], iters_host[r].  done_s[r] receives the time at
 * which the host saw the request finish; latency = done_s - arrival_s.
 * lanes_used (may be NULL): the largest number of lanes busy at once (slot
 * server: its CTAs).  Slot server: when est_host, conv_host and iters_host
 * are page-locked (cudaHostAlloc or cudaHostRegister), est_host starts on a
 * 16-byte boundary and every est_off is a multiple of 16, the kernel writes
 * each result into them directly and the host only reads the completion
 * queue; otherwise results pass through the rings and the host copies them
 * out.  Returns when every request is done; on an error it first stops the
 * serving kernel, so nothing is written to the outputs after it returns.
 * Errors: EINVAL (NULL arrays, a code index out of range, decreasing
 * arrival times, an estimate outside est_bytes), ECUDA. */
int bpq_server_replay(bpq_server *s, int n_req, const int *code, const double *arrival_s, const uint32_t *syn_host,
                      const int64_t *syn_off, uint8_t *est_host, const int64_t *est_off, size_t est_bytes,
                      uint8_t *conv_host, uint8_t *iters_host, double *done_s, int *lanes_used);

/* Slot-granular continuous batching (an interface addition; the paper
 * decodes offline batches).  A persistent kernel of resident CTAs decodes
 * single-shot requests as they arrive: each code has a ring of
 * slots_per_code request slots in mapped pinned host memory (allocated here
 * and owned by the server); bpq_server_replay admits a request that has
 * arrived into the next free slot of its code's ring (writing its syndrome
 * there and publishing the code's request count with a release store), and a
 * shot group that finishes a shot claims the next published request of its
 * CTA's current code at once.  A CTA whose code has nothing to claim moves
 * to another code with published requests (re-staging that code's
 * adjacency).  Results come back through a completion queue in mapped
 * memory, and a slot is free again once its result has been read, so the
 * rings are the admission budget: at most n_codes x slots_per_code requests
 * are in flight.  Every device-side wait is bounded: the kernel returns
 * after about idle_timeout_us of finding nothing to claim, and replay
 * relaunches it (a CUDA graph captured at creation) while requests remain.
 * A request's result is the one bpq_decode gives for its syndrome alone.
 * Plain, Momentum, AdaGrad or EWAInit BP.  dev_mem: at least
 * bpq_server_slot_device_bytes(n_codes) of caller-owned device memory (the
 * per-code descriptors, claim counters and status).  lanes_used of replay
 * reports the serving grid's CTAs.  Errors: EINVAL, ESTATE, ECUDA (also a
 * device-side bounded wait that gave up). */
size_t bpq_server_slot_device_bytes(int n_codes);
/* Counters of the slot server's last replay (for tuning): CTA code switches,
 * scans that found no code with requests to claim, and claims that found
 * the CTA's code empty.  Synchronizes.  Errors: EINVAL (not a slot server),
 * ECUDA. */
int bpq_server_slot_stats(bpq_server *s, long *code_switches, long *empty_scans, long *empty_claims);
/* The slot server's host loop in its last replay: turns that admitted or
 * completed something, and the seconds they spent admitting requests and
 * reading completions (any pointer may be NULL).  Errors: EINVAL (not a
 * slot server). */
int bpq_server_host_stats(const bpq_server *s, long *turns, double *admit_s, double *complete_s);
int bpq_server_create_slots(const bpq_tanner *const *codes, const float *const *priors_dev, int n_codes, int variant,
                            const bpq_params *params, int max_iter, int slots_per_code, int idle_timeout_us,
                            void *dev_mem, size_t dev_bytes, bpq_server **out);

/* launches (may be NULL): the number of decode kernels the server has
 * launched since its creation (lane server: one batched kernel per dispatch
 * to a lane; slot server: one serving kernel per replay, plus one per
 * relaunch after an idle period).  Errors: EINVAL. */
int bpq_server_stats(const bpq_server *s, long *launches);

void bpq_server_free(bpq_server *s);

/* ---------------------------------------------------------------- differentiable decoding */

/* Unrolled decoders with trainable parameters (an extension in the
 * direction of neural BP named in the paper's conclusion): T flooding
 * iterations without the stopping rule, where iteration t has its own
 * parameters.
 *   model BPQ_TRAIN_EWAINIT: EWAInit-BP (Algorithm 2) with EWA weight
 *     alpha_t, Pi^(t) = alpha_t Pi^(0) + (1 - alpha_t) Q^(t-1) (eq. (EWAInit));
 *   model BPQ_TRAIN_MOMENTUM: Momentum-BP (eqs. (mombp1)-(mombp3)) with step
 *     alpha_t and momentum rate gamma_t, g^(t) = gamma_t g^(t-1) +
 *     (1 - gamma_t)(Q^(t-1) - Pi^(0) - S^(t)), Q^(t) = Q^(t-1) - alpha_t g^(t).
 * Both damp the variable-to-check messages as (1 - beta_t) lambda(...) +
 * beta_t m^(t-1) and scale each check-to-variable message by a weight w_e
 * (E weights in the check-major edge order of bpq_tanner_export).  Constant
 * alpha (and gamma), beta_t = 0, w_e = 1 is EWAInit-BP (Momentum-BP).
 * Loss (loss may be NULL: the posterior loss):
 *   BPQ_TRAIN_LOSS_POSTERIOR: the mean over shots and qubits of -log
 *     softmax(0, -Q_X, -Q_Y, -Q_Z)[true Pauli] of the final posterior;
 *   BPQ_TRAIN_LOSS_COSET: the mean over shots and iterations t = 1..T of
 *     mean_i -log P_t(<E^, H_i> = s_i) + mean_L -log P_t(<E^, L> = <E, L>)
 *     over the checks H_i and the caller's logical operators L
 *     (logicals_dev [n_logicals][N] Pauli codes, 1..4 of them, e.g.
 *     bpq_tanner_logicals), where E^ follows the product of iteration t's
 *     posterior marginals (P(W) proportional to e^{-Q_W}, Q_I = 0) and E is
 *     the true error: the probability that every iteration's soft decision
 *     satisfies the syndrome and lies in the true error's coset (P taken at
 *     least 1e-30, with no gradient below).
 * Inputs: syn_dev [B][ceil(M/32)],
 * err_dev [B][N] Pauli codes (the true errors), prior_dev [N][3];
 * alpha_dev, beta_dev, gamma_dev [T] (gamma ignored, may be NULL, for
 * EWAInit), w_dev [E] (device float).  Codes of up to 1024 nodes; T <= 255.
 * The forward pass stores a checkpoint every ckpt_every iterations in
 * work_dev; bpq_train_backward (same inputs, after the forward on the same
 * workspace) recomputes each segment from its checkpoint and writes
 * d loss / d alpha, beta, w (and gamma for Momentum; grad_gamma_dev may be
 * NULL for EWAInit).  Results are deterministic.  Q_dev (optional) receives
 * Q^(T) [B][N][3].  Errors: EINVAL (unknown model, sizes, NULL buffers,
 * too small a workspace, a checkpoint segment too long for shared memory),
 * ESTATE, ECUDA. */
enum bpq_train_model { BPQ_TRAIN_EWAINIT = 0, BPQ_TRAIN_MOMENTUM = 1 };
enum bpq_train_loss_kind { BPQ_TRAIN_LOSS_POSTERIOR = 0, BPQ_TRAIN_LOSS_COSET = 1 };
typedef struct {
    int kind;                     /* bpq_train_loss_kind */
    const uint8_t *logicals_dev;  /* coset loss: [n_logicals][N] Pauli codes (device) */
    int n_logicals;               /* coset loss: 1..4 */
} bpq_train_loss;
size_t bpq_train_workspace_bytes(const bpq_tanner *t, int model, int B, int T, int ckpt_every);
int bpq_train_forward(const bpq_tanner *t, int model, const uint32_t *syn_dev, const uint8_t *err_dev,
                      const float *prior_dev, int B, int T, int ckpt_every, const float *alpha_dev,
                      const float *beta_dev, const float *gamma_dev, const float *w_dev, float msg_clip,
                      const bpq_train_loss *loss, float *loss_dev, float *Q_dev, void *work_dev, size_t work_bytes,
                      void *stream);
int bpq_train_backward(const bpq_tanner *t, int model, const uint32_t *syn_dev, const uint8_t *err_dev,
                       const float *prior_dev, int B, int T, int ckpt_every, const float *alpha_dev,
                       const float *beta_dev, const float *gamma_dev, const float *w_dev, float msg_clip,
                       const bpq_train_loss *loss, float *grad_alpha_dev, float *grad_beta_dev,
                       float *grad_gamma_dev, float *grad_w_dev, void *work_dev, size_t work_bytes, void *stream);

/* ---------------------------------------------------------------- evaluation */

/* Success criterion of Sec. IV: E^ in E S.  For each shot the residual
 * R = E^ E (Pauli product, phase ignored) is classified: fail_dev[b] = 0 if R
 * is a stabilizer, 1 if R anticommutes with some check (a detected error),
 * 2 if R commutes with every check but anticommutes with a logical
 * operator (an undetected error).  Errors: EINVAL, ESTATE (no logicals). */
int bpq_check_logical(const bpq_tanner *t, const uint8_t *err_dev, const uint8_t *est_dev, int B,
                      uint8_t *fail_dev, void *stream);

/* ---------------------------------------------------------------- misc */

/* Throughput probe used to measure the roofline denominators on the running
 * GPU (not part of the paper's method): launches `blocks` x `threads`
 * threads, each running `iters` rounds of 8 independent chains of
 * which = 0: MUFU ex2 (one SFU op per link), which = 1: fused multiply-add.
 * Time it with events on `stream`; ops = blocks * threads * iters * 8.
 * sink_dev: one float of device memory the kernel may write. */
int bpq_probe_peak(int which, int blocks, int threads, int iters, float *sink_dev, void *stream);

const char *bpq_last_error(void);
int bpq_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BPQ_H */
