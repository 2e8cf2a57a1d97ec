/*
 * bsd.h -- C ABI of the GB300 beam search decoder for quantum LDPC codes.
 *
 * The decoding problem is the triple (H in F2^{M x N}, A in F2^{K x N},
 * p in (0,1)^N) of the paper's App. A: columns are error sources, rows of H
 * are detectors, rows of A are logical observables.  Given a syndrome
 * s = H e the decoder returns a correction e^ with (when it converges)
 * H e^ = s, and the observable flips A e^.  The method is BP-guided beam
 * search: min-sum belief propagation (App. A, Eqs. 1-4), masked BP (Alg. 2)
 * and the beam search controller (Alg. 3 with App. B), run on the GPU for
 * every beam candidate of every syndrome.
 *
 * Conventions
 *   - Every function returns BSD_OK (0) or a negative BSD_ERR_* code; no
 *     function aborts the process.  bsd_error_string() names a code.
 *   - Bit vectors are little-endian uint32 words: bit i of a length-L vector
 *     is bit (i % 32) of word i / 32; a vector takes ceil(L/32) words and
 *     padding bits above L must be zero on input and are written as zero.
 *   - Buffers marked "device" are CUDA device pointers on the decoder's
 *     device; buffers marked "host" are ordinary (preferably pinned) host
 *     memory.  The caller owns every input and output buffer; the decoder
 *     owns only its internal copies of (H, A, p) and its workspace.
 *   - Decoding is asynchronous and stream-ordered, like a CUDA call on the
 *     given stream (NULL = the legacy default stream), except where stated.
 *   - A decoder handle is not thread-safe: one call at a time per handle.
 *   - Arithmetic: edge messages are stored in single precision and every sum
 *     is formed in single precision in the order fixed by the readings below,
 *     so results do not depend on launch configuration or scheduling.
 *
 * Readings of points the paper leaves open (shared with the test oracle):
 *   min-sum scale alpha on D (ms_scale, 1 = Eq. 1 as printed); sign(x) = -1
 *   iff x < 0; a minimum over no other unmasked neighbour is llr_clamp; every
 *   stored E_{j->i} is clamped to [-llr_clamp, llr_clamp]; the sums of
 *   Eqs. 2-3 start at Lambda_j and add the detector messages in ascending
 *   order of value; sum_LLR covers the iterations actually run in that call;
 *   argmin ties go to the lowest index; pruning keeps the top beam_width under
 *   (score descending, canonical index ascending) where the canonical index
 *   of a child is 2 * (rank of its parent) + val; scores and weights are
 *   summed exactly on the fixed-point grid 2^-16.
 */
#ifndef BSD_H
#define BSD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BSD_PARAMS_VERSION 3u

/* return codes */
#define BSD_OK               0
#define BSD_ERR_INVALID_ARG (-1)   /* bad pointer, size, index, prior or parameter */
#define BSD_ERR_CUDA        (-2)   /* a CUDA runtime call failed */
#define BSD_ERR_OOM         (-3)   /* device or host allocation failed */
#define BSD_ERR_TIMEOUT     (-4)   /* a bounded device-side wait gave up */
#define BSD_ERR_UNSUPPORTED (-5)   /* valid input outside what this build handles */
#define BSD_ERR_DEVICE      (-6)   /* a device-side check recorded an error */
#define BSD_ERR_SCRATCH     (-7)   /* bsd_decode_noalloc: one shot needs more than the static scratch */

/* message storage precision (bsd_params.msg_precision): the E messages are
   stored in this format (rounded to nearest even, zero stored as +0, L_MAX
   taken at its stored value); all arithmetic is single precision */
#define BSD_FP32 0
#define BSD_FP16 1
#define BSD_BF16 2

/* per-shot status words written by bsd_decode */
#define BSD_STATUS_CONVERGED_SEED 1u  /* returned e^ comes from the seed BP (Alg. 3, first BP run) */
#define BSD_STATUS_CONVERGED_BEAM 2u  /* returned e^ comes from a masked BP round (Alg. 2/3)    */
#define BSD_STATUS_FAILED         4u  /* no e^ with H e^ = s was found: e^ is the hard decision
                                         of the best path of the final set, fixed values filled */
#define BSD_STATUS_NEAR_TIE       8u  /* with 16-bit messages: an argmin (next_pos) margin of a
                                         visited candidate or a pruning margin of a round lay
                                         strictly inside (0, tie_guard_rel) */
#define BSD_STATUS_FP32_RERUN    16u  /* the shot was decoded again with single-precision messages
                                         because of a near tie; outputs and iteration count are
                                         those of the re-run (bits 1/2/4 from it, 8 kept) */

typedef struct bsd_decoder bsd_decoder;

/* Decoder parameters.  max_rounds .. num_results are the five parameters of
   Alg. 3 (Table I lists the paper's presets). */
typedef struct {
    uint32_t struct_version;   /* must be BSD_PARAMS_VERSION */
    int32_t  max_rounds;       /* rounds of branching, >= 0 */
    int32_t  beam_width;       /* paths kept per round, 1..64 */
    int32_t  initial_iters;    /* seed BP iterations, >= 1 */
    int32_t  iters_per_round;  /* masked BP iterations per child, >= 1 */
    int32_t  num_results;      /* valid solutions to collect before returning, 1..64 */
    float    ms_scale;         /* alpha in D = alpha * (-1)^s * prod sign * min; (0, 1] */
    float    llr_clamp;        /* L_MAX > 0 */
    int32_t  msg_precision;    /* BSD_FP32, BSD_FP16 or BSD_BF16 */
    float    tie_guard_rel;    /* near-tie margin for 16-bit messages: > 0 this value, 0 the
                                  default (1e-3 for FP16, 1e-2 for BF16), < 0 no near-tie
                                  re-runs; with BSD_FP32 only a positive value flags shots */
    int64_t  workspace_bytes;  /* device workspace budget; 0 = library default (4 GiB) */
    int32_t  group_warps;      /* threads per BP candidate: 0 chosen by the library (and by
                                  bsd_autotune), 1 one warp per candidate, 2..16 a block of
                                  that many warps per candidate (codes without the small engine's
                                  layout, or forced); results do not depend on it */
    int32_t  small_batch;      /* chunks of at most this many shots launch a second graph whose
                                  grids are sized to them (low latency for single syndromes):
                                  0 the default 32, -1 never, else 1..65536 */
    int32_t  batch_slots;      /* codes without the small engine's layout (detector error models),
                                  with the scale alpha and num_results = 1: the seed BP of many
                                  shots runs at once over this many slots, messages streamed
                                  through device memory with the shots contiguous; 0 the library
                                  default (codes of at least 16384 edges: 2048 slots; smaller
                                  codes: none), -1 never, else 256..65536 (rounded
                                  down to a multiple of 256); at most a quarter of the workspace;
                                  results do not depend on it */
} bsd_params;

/* Fill *out with the library defaults: beam8_230iters, ms_scale 1,
   llr_clamp 1e4, FP32, tie_guard_rel 0.  Returns BSD_ERR_INVALID_ARG if out is NULL. */
int bsd_params_default(bsd_params *out);

/* Fill *out with a Table I preset ("beam8_230iters", "beam32_340iters",
   "beam64_640iters", "beam64_32res_640iters"); other fields take the
   defaults.  Returns BSD_ERR_INVALID_ARG for an unknown name or NULL. */
int bsd_params_preset(const char *name, bsd_params *out);

/* Create a decoder for (H, A, p) on CUDA device `device`.
 *   H_row_ptr[M+1], H_col_idx[nnz]  host CSR of H; column indices of a row
 *                                    strictly ascending, each in [0, N)
 *   A_row_ptr[K+1], A_col_idx[nnzA] host CSR of A (K may be 0)
 *   priors[N]                        host, each strictly inside (0, 1);
 *                                    Lambda_j = log((1 - p_j) / p_j) (App. A)
 *   params                           see bsd_params
 * The inputs are copied; the caller may free them after the call.  Device
 * memory for the graph and the workspace is allocated here (synchronously).
 * Errors: BSD_ERR_INVALID_ARG (sizes, indices, priors, parameters),
 * BSD_ERR_UNSUPPORTED (a size beyond this build's limits), BSD_ERR_OOM,
 * BSD_ERR_CUDA.  On error *out is set to NULL. */
int bsd_create(int32_t M, int32_t N, int32_t K,
               const int32_t *H_row_ptr, const int32_t *H_col_idx,
               const int32_t *A_row_ptr, const int32_t *A_col_idx,
               const double *priors, const bsd_params *params,
               int device, bsd_decoder **out);

/* Decode B syndromes with the beam search decoder (Alg. 3).
 *   d_syndromes    device, B x ceil(M/32) words, read only
 *   d_corrections  device, B x ceil(N/32) words, e^ per shot
 *   d_obs_flips    device, B x ceil(K/32) words, A e^ per shot (may be NULL if K = 0)
 *   d_status       device, B words, one BSD_STATUS_* value per shot
 *   d_iters        device, B words or NULL: BP iterations the sequential
 *                  algorithm runs up to its return (seed plus every visited
 *                  child), capped at 2^32 - 1
 *   cuda_stream    cudaStream_t or NULL
 * Shots are independent; results do not depend on B or on how the batch is
 * split.  Returns BSD_ERR_INVALID_ARG for NULL buffers or B < 0, else the
 * launch status (BSD_ERR_CUDA).  Device-side errors are reported by
 * bsd_sync_error. */
int bsd_decode(bsd_decoder *dec, const uint32_t *d_syndromes, int64_t B,
               uint32_t *d_corrections, uint32_t *d_obs_flips,
               uint32_t *d_status, uint32_t *d_iters, void *cuda_stream);

/* bsd_decode on host buffers (same layouts): copies the syndromes in,
 * decodes and copies the results back, synchronising the stream before it
 * returns.  h_iters may be NULL.  Pinned host memory gives asynchronous
 * copies; pageable memory works but copies synchronously. */
int bsd_decode_host(bsd_decoder *dec, const uint32_t *h_syndromes, int64_t B,
                    uint32_t *h_corrections, uint32_t *h_obs_flips,
                    uint32_t *h_status, uint32_t *h_iters, void *cuda_stream);

/* Allocation-free variant of bsd_decode.  The paper has no counterpart: this
 * entry point exists for callers that must not allocate device memory when
 * they decode -- for example code whose device memory is owned by another
 * allocator (a framework's caching allocator), or a latency-critical loop
 * that may not take the driver's allocation locks or risk an allocation
 * failure mid-run.  Such a caller creates the decoder once at set-up
 * (bsd_create allocates there) and then decodes through this function, which
 * calls no cudaMalloc, cudaFree or other allocating routine.  Instead of the
 * decoder's own workspace it uses one file-scope static device array of
 * BSD_NOALLOC_SCRATCH_BYTES that every device loading the library holds
 * until the process exits.
 *   Arguments, layouts and results are those of bsd_decode; the results are
 *   identical to bsd_decode's.  Batches of any size are decoded in chunks
 *   that fit the array.
 *   The first call on a device looks up the array's device address on that
 *   device (cudaGetSymbolAddress); make that first call before any stream
 *   capture on the device.
 *   Unlike bsd_decode, the call is not fully asynchronous: with max_rounds
 *   > 0, after the seed pass of each chunk it copies the chunk's count of
 *   shots that need beam rounds to the host and synchronises the stream to
 *   read it, so the calling thread waits for each chunk's seed pass (the
 *   beam rounds of the last chunk are still in flight when it returns).
 *   All calls on a device share the one array, and it keeps the contents the
 *   last call left: each call clears the counters it needs zeroed, but calls
 *   whose work overlaps on the GPU (two streams, two host threads, two
 *   decoders at once) race on the array and corrupt each other's results.
 *   Serialise them.
 *   Decoders with 16-bit messages and near-tie re-runs are not served here
 *   (BSD_ERR_UNSUPPORTED): the re-run needs buffers of its own.
 *   Returns BSD_ERR_SCRATCH when the beam state of a single shot (two banks
 *   of 2 * beam_width edge-message snapshots plus bookkeeping) exceeds the
 *   array, BSD_ERR_INVALID_ARG as bsd_decode does, and BSD_ERR_CUDA when the
 *   address lookup or a launch fails.  Opt-in kernel timing does not apply. */
#define BSD_NOALLOC_SCRATCH_BYTES (32u << 20)
int bsd_decode_noalloc(const bsd_decoder *dec, const uint32_t *d_syndromes, int64_t B,
                       uint32_t *d_corrections, uint32_t *d_obs_flips,
                       uint32_t *d_status, uint32_t *d_iters, void *cuda_stream);

/* Single-syndrome request loop (low-latency decoding).  bsd_serve_start
 * keeps one candidate group of the decoder's kernels resident on its device,
 * polling a mailbox in host-mapped memory; bsd_serve_decode posts one
 * syndrome and waits for the answer.  A syndrome whose first BP run ends the
 * search (Alg. 3: it converges, with num_results = 1, or max_rounds = 0) is
 * answered by the loop itself -- the same kernels, operations and order as
 * bsd_decode, so the outputs are identical -- with no launch and no stream
 * wait; any other is decoded by the regular path (bsd_decode_host on a stream
 * of the loop's own), so every answer equals bsd_decode's.
 *   idle_ms     the loop leaves after this many milliseconds without a
 *               request (1..60000) and bsd_serve_decode starts it again;
 *               every wait of the loop is bounded by it or by the stop flag
 *   h_syndrome  host, WM words; h_correction host, WN words; h_obs_flips
 *               host, WK words (NULL allowed when K = 0); h_status host, one
 *               word; h_iters host, one word or NULL -- as bsd_decode_host
 *               for B = 1
 * bsd_serve_start runs one regular decode first, so the regular path's
 * buffers exist before the loop is resident, then allocates the mailbox
 * (pinned, mapped) and two streams; a decoder already serving returns
 * BSD_OK.  bsd_serve_decode returns BSD_ERR_INVALID_ARG when the decoder is
 * not serving, BSD_ERR_TIMEOUT when no answer comes within 2 s.
 * bsd_serve_stop ends the loop and frees what start allocated (BSD_OK when
 * not serving); bsd_destroy, bsd_set_weights and bsd_autotune call it.
 * While serving, the decoder's other calls may run on other streams; one
 * that allocates device memory (a first decode of a larger batch) may wait
 * for the loop's idle limit.  Calls on one decoder are not thread-safe. */
int bsd_serve_start(bsd_decoder *dec, int32_t idle_ms);
int bsd_serve_decode(bsd_decoder *dec, const uint32_t *h_syndrome, uint32_t *h_correction,
                     uint32_t *h_obs_flips, uint32_t *h_status, uint32_t *h_iters);
int bsd_serve_stop(bsd_decoder *dec);

/* Plain min-sum BP (App. A, Eqs. 1-3) from E(0) = Lambda for exactly T
 * iterations per syndrome, with no stopping rule; writes the posterior LLRs
 * Lambda_j(T) (device, B x N floats) and, if d_sum_llr is not NULL, the sums
 * over t = 1..T of Lambda_j(t) (device, B x N floats).  Used to measure the
 * LLRs against a double-precision reference.  T in [1, 100000]. */
int bsd_bp_llr(bsd_decoder *dec, const uint32_t *d_syndromes, int64_t B, int32_t T,
               float *d_llr, float *d_sum_llr, void *cuda_stream);

/* Synchronise the decoder's last stream, read and clear the device-side
 * error word: BSD_OK, BSD_ERR_TIMEOUT or BSD_ERR_DEVICE. */
int bsd_sync_error(bsd_decoder *dec);

/* Sizes and launch shape: any pointer may be NULL.  chunk_shots is the
 * number of shots decoded per internal pass (bounded by the workspace). */
int bsd_get_info(const bsd_decoder *dec, int32_t *M, int32_t *N, int32_t *K, int32_t *n_edges,
                 int64_t *chunk_shots, int64_t *workspace_bytes);

/* The batched seed BP of a decoder (the paper has no counterpart: it is how
 * this library runs the first BP run of Alg. 3 for many syndromes at once):
 * *slots = the slots of its workspace (0: none), *active = 1 if the current
 * launch shape uses them.  Any pointer may be NULL. */
int bsd_get_batch(const bsd_decoder *dec, int32_t *slots, int32_t *active);

/* Where the single-warp engine keeps a candidate's messages in shared memory
 * (a layout choice of this library; the paper's Eqs. 1-3 do not depend on
 * it).  For codes with every row of degree 6 and every column of degree 3
 * (the bivariate bicycle codes) the pair h of row i is at word plane[h] + 2 i
 * with plane[h] = h (64 ceil(M / 32) + 12), and the error-node pass reads the
 * k-th edge of column j at col_word[3 j + k].
 * The rows' edge orders and the columns' k orders are searched so that both
 * passes touch 32 distinct banks per access; bsd_create builds the same
 * placement for codes of at most 160 columns and 96 rows.  Host only; nothing
 * is allocated on a device.
 *   M, N, H_row_ptr, H_col_idx  host, H in CSR as for bsd_create
 *   plane      host int32[3]: out, the plane bases
 *   edge_word  host int32[E]: out, the word of CSR edge e (E = H_row_ptr[M])
 *   col_word   host int32[3 N]: out
 *   extent     host int32: out, the words spanned
 *   excess     host int32: out, the error-pass bank loads above three that
 *              remain (0: every access conflict-free)
 * Errors: BSD_ERR_INVALID_ARG (null pointer, bad CSR), BSD_ERR_UNSUPPORTED
 * (another degree structure). */
int bsd_small_layout(int32_t M, int32_t N, const int32_t *H_row_ptr, const int32_t *H_col_idx, int32_t *plane,
                     int32_t *edge_word, int32_t *col_word, int32_t *extent, int32_t *excess);

/* Where the generic engines keep a candidate's messages (a layout choice of
 * this library, for codes with every column of degree at most 6): each row's
 * edges permuted inside the row's storage window, each column's edges in the
 * k slots of the padded column table (colK = 3 for a largest column degree of
 * 3 or less, else 6), chosen so that the 32 lanes of an error-pass access
 * meet distinct banks where possible.  bsd_create builds the same placement.
 * Host only; nothing is allocated on a device.
 *   M, N, H_row_ptr, H_col_idx  host, H in CSR as for bsd_create
 *   edge_word  host int32[E]: out, the element of CSR edge e
 *   slot_edge  host int32[colK * N]: out, the CSR edge in slot k of column j
 *              at [k * N + j], -1 for an empty slot
 *   colK       host int32: out, 3 or 6
 *   excess     host int32: out, the bank loads above each 32-column group's
 *              largest degree that the search leaves
 * Errors: BSD_ERR_INVALID_ARG (null pointer, bad CSR), BSD_ERR_UNSUPPORTED
 * (a column of degree above 6, or more than 2^20 edges). */
int bsd_generic_layout(int32_t M, int32_t N, const int32_t *H_row_ptr, const int32_t *H_col_idx,
                       int32_t *edge_word, int32_t *slot_edge, int32_t *colK, int32_t *excess);

/* Opt-in timing of this library's kernels (not part of the method): while
 * enabled, every kernel launch made by bsd_decode / bsd_decode_host is
 * bracketed by two CUDA events recorded on the decode stream.  Enabling costs
 * two event records per launch.  Returns BSD_ERR_INVALID_ARG for NULL. */
int bsd_profile_enable(bsd_decoder *dec, int enable);

/* Synchronise the decode stream, then return and reset, since the previous
 * read: the summed event-timed duration in milliseconds and the launch count
 * of each kernel kind (index 0: seed BP, 1: expand + masked BP of a round,
 * 2: per-shot selection of a round), the full BP iterations executed on the
 * device (index 0: seed candidates, 1: round candidates, counting children
 * evaluated after a shot's first success, 2: the part of index 0 run by the
 * batched seed BP of bsd_params.batch_slots), the number of kernels of this
 * library that ran for this decoder (counted on the device, with or without
 * timing enabled), and the message updates done by first-iteration screens
 * of seed runs (with every Lambda_j > 0, the scale alpha and one result, a
 * seed run first forms e^(1) from the columns next to flipped detectors
 * only, since no other column can flip at t = 1; a run that converges there
 * ends after that partial iteration, which is counted here and not as a full
 * iteration).  While timing is enabled the kernels are launched one by one so
 * that events can bracket them; otherwise each chunk runs as one CUDA graph.
 * Any pointer may be NULL. */
int bsd_profile_read(bsd_decoder *dec, double ms[3], int64_t launches[3], uint64_t exec_iters[3],
                     uint64_t *kernel_launches, uint64_t *screen_updates);

/* Kernel kinds timed while timing is enabled: 0..2 as above, then the
 * unrolled decoder's passes (bsd_unrolled_forward / _backward): 3 check pass,
 * 4 error-node pass, 5 error-node adjoint, 6 check adjoint, 7 its other
 * kernels (bit planes, initial messages, loss and gradient reductions), then
 * the batched seed BP: 8 its check pass, 9 its error-node pass, 10 its
 * stopping test and refill, and 11 the first-iteration screen of seed runs. */
#define BSD_PROFILE_KINDS 12

/* Synchronise the stream of the last timed launch, then return and reset the
 * summed event-timed milliseconds and launch counts of every kind. */
int bsd_profile_read_kinds(bsd_decoder *dec, double ms[BSD_PROFILE_KINDS], int64_t launches[BSD_PROFILE_KINDS]);

/* Weighted min-sum: replace the scale alpha of Eq. 1 by a weight per edge and
 * iteration, D_{i->j}(t) = w[t', e] * (-1)^{s'_i} * prod sign * min, with
 * t' = min(t, T) - 1 and t counted from 1 in every BP call (the seed run and
 * every child's masked run alike).  Weights come from training the unrolled
 * decoder (bsd_unrolled_forward / bsd_unrolled_backward).
 *   h_weights  host, float [T][E], E in the CSR edge order of H given to
 *              bsd_create; copied, so the caller keeps ownership.  Each
 *              weight must be finite with |w| <= 1e6.
 *   T          rows; 0 (h_weights ignored) returns to the scale ms_scale.
 * Waits for the work queued on the stream of the decoder's last call, then
 * re-selects the kernels.  Errors: BSD_ERR_INVALID_ARG (bad weights),
 * BSD_ERR_UNSUPPORTED (16-bit message storage), BSD_ERR_OOM, BSD_ERR_CUDA;
 * on error the decoder keeps its previous weights. */
int bsd_set_weights(bsd_decoder *dec, const float *h_weights, int32_t T);

/* ---- Differentiation: unrolled weighted min-sum ---------------------------
 * T flooding iterations of Eqs. 1-3 with weights w[t][e] in place of the
 * scale (t = 1..T, no stopping rule), on B shots of the decoder's problem, and
 * the loss
 *     loss = sum_{t=1..T} mean_{b,j} BCE(sigmoid(-Lambda_j(t)), e_j)
 * (binary cross entropy between the error probability the posterior assigns
 * and the true error).  The backward gives dloss/dw with the readings: sign()
 * has zero derivative, d|x|/dx = sign(x) with 0 at 0, a minimum over the other
 * edges passes its derivative to the lowest-index edge holding it, a message
 * clamped to +-L_MAX passes none, the minimum over no edge is the constant
 * L_MAX.  The decoder supplies H, the priors and L_MAX (single-precision
 * message storage only; else BSD_ERR_UNSUPPORTED); its beam parameters and
 * weights are not used.
 *
 * Workspace: device memory of bsd_unrolled_workspace() bytes, 256-byte
 * aligned, owned by the caller.  The forward stores E at the checkpoints
 * t = 0, k, 2k, ... (k = ckpt_every, 1 <= k <= T) and the bit planes of the
 * batch there; the backward recomputes each segment of k iterations from its
 * checkpoint.  A backward needs the forward of the same (B, T, k, weights,
 * workspace) before it, with the workspace untouched in between.
 *
 * Memory: about (ceil(T/k) + k + 4) * E * Bp + k * N * Bp floats, Bp = B
 * rounded up to a multiple of 512. */
int bsd_unrolled_workspace(const bsd_decoder *dec, int64_t B, int32_t T, int32_t ckpt_every, int64_t *bytes);

/*   d_syndromes  device, B x ceil(M/32) words (bitpacked like bsd_decode)
 *   d_errors     device, B x ceil(N/32) words: the true errors e
 *   d_weights    device, float [T][E] (CSR edge order)
 *   d_loss       device, float [T + 1]: [0] the loss, [t] the term of iteration t
 *   d_llr        device, float [T][B][N] Lambda_j(t), or NULL
 * Asynchronous on cuda_stream.  Errors: BSD_ERR_INVALID_ARG (sizes, NULL
 * buffers, a workspace too small or misaligned), BSD_ERR_UNSUPPORTED,
 * BSD_ERR_CUDA. */
int bsd_unrolled_forward(const bsd_decoder *dec, const uint32_t *d_syndromes, const uint32_t *d_errors, int64_t B,
                         int32_t T, int32_t ckpt_every, const float *d_weights, float *d_loss, float *d_llr,
                         void *d_work, int64_t work_bytes, void *cuda_stream);

/*   d_grad_loss     device, float [T + 1]: the derivative of the caller's
 *                   objective with respect to the entries of the forward's
 *                   loss vector -- [0] the total, [t] the term of iteration t
 *                   ({1, 0, ..., 0} for the loss itself; {0, c_1, ..., c_T}
 *                   for an objective that weights iteration t by c_t)
 *   d_grad_weights  device, float [T][E]: overwritten with the derivative of
 *                   that objective with respect to the weights
 * Asynchronous on cuda_stream; same errors as the forward.  Weight gradients
 * are sums over the batch taken in a fixed order: the result is deterministic. */
int bsd_unrolled_backward(const bsd_decoder *dec, int64_t B, int32_t T, int32_t ckpt_every, const float *d_weights,
                          const float *d_grad_loss, float *d_grad_weights, void *d_work, int64_t work_bytes,
                          void *cuda_stream);

/* Launch-shape autotuner: decode the caller's sample batch with every launch
 * shape the code can use -- one warp per candidate with 8, 4, 2 or 1
 * candidates per block, then a block of 2, 4, 8 or 16 warps per candidate
 * (fewer edges per thread) -- time each (the fastest of three decodes after
 * two untimed ones, CUDA events on cuda_stream) and keep the fastest.
 * Decoding results do not depend on the shape.  Synchronous.
 *   d_syndromes  device, B x ceil(M/32) words: a sample of the workload
 *   report       host, report_cap entries (may be NULL with report_cap 0):
 *                the shapes timed and their milliseconds, in order
 *   n_report     host (may be NULL): the number of shapes timed
 * Errors: BSD_ERR_INVALID_ARG, BSD_ERR_OOM (scratch outputs for B shots),
 * BSD_ERR_CUDA; on error the decoder keeps a valid shape. */
typedef struct {
    int32_t group_warps;       /* 1: a warp per candidate; >= 2: a block of that many warps */
    int32_t warps_per_block;   /* block size in warps */
    float   ms;                /* decode time of the sample */
} bsd_shape_timing;

int bsd_autotune(bsd_decoder *dec, const uint32_t *d_syndromes, int64_t B, void *cuda_stream,
                 bsd_shape_timing *report, int32_t report_cap, int32_t *n_report);

/* The decoder's current launch shape (either pointer may be NULL). */
int bsd_get_shape(const bsd_decoder *dec, int32_t *group_warps, int32_t *warps_per_block);

/* ---- Detector error models as text ----------------------------------------
 * Reads the common text format of detector error models into the decoding
 * problem (H, A, p) of App. A: one column per error mechanism, in the order
 * met.  Understood: error(p) with D<k> / L<k> targets and '^' separators (a
 * mechanism's effect is the XOR of its parts; a target listed twice cancels),
 * detector, logical_observable, shift_detectors, repeat N { ... } (nested),
 * instruction tags in brackets (ignored), comments.  M (K) is one more than
 * the largest detector (observable) index met or declared.
 *   flags     0, or BSD_DEM_MERGE: merge mechanisms with identical detector and
 *             observable sets, p = p1 (1 - p2) + p2 (1 - p1)
 *   err_line  host (may be NULL): the 1-based line of the first error
 * Errors: BSD_ERR_INVALID_ARG (syntax, a probability outside [0, 1]),
 * BSD_ERR_UNSUPPORTED (an unknown instruction, an index beyond 2^31 - 2),
 * BSD_ERR_OOM.  The handle owns host memory only. */
#define BSD_DEM_MERGE 1
typedef struct bsd_dem bsd_dem;
int bsd_dem_parse(const char *text, int64_t len, int32_t flags, bsd_dem **out, int64_t *err_line);
/* Sizes of the parsed problem: rows M, columns N, observables K, nonzeros of H and A. */
int bsd_dem_sizes(const bsd_dem *dem, int32_t *M, int32_t *N, int32_t *K, int64_t *nnz_H, int64_t *nnz_A);
/* Fill caller-owned host arrays: H_row_ptr[M+1], H_col_idx[nnz_H], A_row_ptr[K+1],
 * A_col_idx[nnz_A], priors[N]; the CSR column indices of every row ascend,
 * as bsd_create requires. */
int bsd_dem_fill(const bsd_dem *dem, int32_t *H_row_ptr, int32_t *H_col_idx, int32_t *A_row_ptr,
                 int32_t *A_col_idx, double *priors);
void bsd_dem_free(bsd_dem *dem);

/* Static text for a return code. */
const char *bsd_error_string(int code);

/* The CUDA runtime's name and description of the most recent CUDA call made
 * by this library on the calling thread that failed, with the library source
 * line that checked it ("" if none): the reason behind a BSD_ERR_CUDA.  The text stays valid until the next call of
 * this function on the same thread. */
const char *bsd_last_cuda_error(void);

/* Release the decoder's device memory.  NULL is ignored. */
void bsd_destroy(bsd_decoder *dec);

#ifdef __cplusplus
}
#endif

#endif /* BSD_H */
