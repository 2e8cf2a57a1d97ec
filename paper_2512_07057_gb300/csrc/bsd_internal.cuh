// bsd_internal.cuh -- device data layout shared by the kernels and the host API.
//
// Layout in HBM (all read-only graph tables are tiny and stay L1/L2 resident):
//   row_ptr[M+1]          CSR of H; CSR edge e of row i lies in [row_ptr[i], row_ptr[i+1])
//   row_col[E]            column of CSR edge e
//   col_ptr[N+1]          per error node j, its edges in col_edge/col_row[col_ptr[j] ..)
//   col_edge[E]           CSR edge id of each (column, k) pair, rows ascending
//   col_row[E]            detector (row) of that edge
//   lam[N]                Lambda_j = log((1-p_j)/p_j) rounded to float
//   lamE[Epad]            clamp(Lambda_{col(e)}), the seed's E(0) in CSR order, storage format
//   hcol[N][WM]           column j of H as an M-bit set (syndrome flip for v = 1)
//   acol[N][WK]           column j of A as a K-bit set (observable flips)
//   lamq[N]               Lambda_j on the 2^-16 fixed-point grid (weights)
//   rs0[M]                the detector records of E(0) (a seed run's first check pass, up to the syndrome)
//   D0[Epad]              the check messages of E(0) with the scale alpha, before the syndrome sign
//   colER[colK][Npad]     (word, row) of the edge in slot k of column j at the
//                         generic engines' placement, (-1, -1) for an empty slot
//   lamEc[Npad]           clamp(Lambda_j) in the storage format (E(0) of every edge of column j)
//
// Workspace (one decoder):
//   seed store, S entries: the snapshot (E, s', mask, vals, e^, record) of
//   every shot of a chunk of S shots whose seed BP did not end the search;
//   beam window, A entries: the active shots of the current beam pass
//   (entries pass*A .. pass*A + A - 1 of the seed store), with two banks of
//   2w child slots each; round r writes bank r % 2 and reads its parents from
//   bank (r - 1) % 2 (or the seed store for r = 1) through a rank -> slot
//   table, so surviving paths are never copied.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "bsd.h"

namespace bsd {

constexpr int kMaxColDeg = 16;   // the generic engines' largest column degree bound
constexpr int kMaxBeam = 64;
constexpr int kSmallMaxCpl = 5;   // the single-warp engine's largest code: 5 words of columns
constexpr int kSmallMaxRpl = 3;   // and 3 of rows
constexpr int kMaxResults = 64;
constexpr double kFixScale = 65536.0;   // fixed-point grid 2^-16 for scores and weights

struct DevGraph {
    int M, N, K, E;
    int WM, WN, WK;        // words of M, N, K bits
    int Epad, Npad;        // E rounded up to a multiple of 8, N to a multiple of 4
    int msg_bytes;         // bytes of a stored message: 4 (float), 2 (binary16 / bfloat16)
    int prec;              // 0 float, 1 binary16, 2 bfloat16
    int max_col_deg, max_row_deg;
    int all_lam_pos;       // every Lambda_j > 0 (all p_j < 1/2)
    int det_bytes;         // per-warp detector-side shared memory (set with the engine)
    const int* row_ptr;
    const int* row_col;    // [E] column of CSR edge e
    const int* col_ptr;
    const int* col_edge;
    const int* col_row;
    const float* lam;
    const void* lamE;      // E(0) in the storage format
    const uint32_t* hcol;
    const uint32_t* acol;
    const long long* lamq;
    const float4* rs0;     // [M] detector records of E(0): (min1, min2, argmin edge, parity of negatives)
    const float* D0;       // [Epad] check messages of E(0) with scale alpha, before the syndrome sign
    const int2* colER;     // [colK][Npad] (word, row) of the edge in slot k of column j, (-1, -1): empty
    int colK;              // 3 or 6 (the generic engines' degree bound), 0 when colER is absent
    const void* lamEc;     // [Npad] E(0) of column j (clamp(Lambda_j)) in the storage format
    // the columns ordered by degree (batched seed BP): colperm[q] is the
    // column at position q, the columns of degree d hold positions
    // [dstart[d], dstart[d + 1]), and the (edge, row) pairs of the column at
    // position q of degree d are colseq[dbase[d] + (q - dstart[d]) * d + k]
    const int* colperm;    // [N]
    const int2* colseq;    // [E]
    // first-iteration screen: per column j its colRDk (D0 of the edge, row)
    // pairs, rows ascending, padded with (+inf, -1); colRDk = 4, 6 or 16 for
    // the degree bounds 3, 6 and 16 (two pairs per float4)
    const float4* colRD;   // [Npad][colRDk / 2]
    int colRDk;
    int dstart[kMaxColDeg + 2];
    int dbase[kMaxColDeg + 2];
    // the single-warp engine's shared-memory placement of a candidate's
    // messages (codes with every row of degree 6 and every column of degree
    // 3; bsd_layout.cu): the pair h of row i at word h small_plane_stride(M)
    // + 2 i, and scol[3 j + k] = (word << 16) | row for the k-th edge of
    // column j; sD0 and slamE hold D0 and E(0) at those words (Epad covers
    // the placement)
    const uint32_t* scol;  // [3 N], null when the code has no such placement
    const float* sD0;      // [Epad]
    const void* slamE;     // [Epad] in the storage format
    const uint4* slamh;    // [32 WN] with the placement: per column slot j the bits of Lambda_j and the
                           // (at most 3) words of column j of H; zero past N
};

struct DecCfg {
    int max_rounds, w, initial_iters, iters_per_round, num_results;
    float alpha, L;        // L: L_MAX as the storage format holds it
    double tie_guard;      // near-tie margin (0: no flags)
    const float* weights;  // optional [wT][Epad]: w_{e,t} in place of alpha (weighted engines only)
    const float* sweights; // the same weights at the single-warp engine's words (when DevGraph::scol is set)
    int wT;                // iteration t of a BP call uses row min(t, wT) - 1
};

// the single-warp engine's placement of a code's messages (bsd_layout.cu):
// plane bases A[0..2], the word of every CSR edge, the per-(column, k) table,
// the words spanned and the bank loads above three the search left (0: both
// passes conflict-free); false when the code is not of row degree 6 and
// column degree 3
struct SmallLayout {
    int A[4];
    std::vector<int> addr;
    std::vector<uint32_t> col;
    int extent;
    int excess;
};
bool small_layout(int M, int N, const int* row_ptr, const int* col_idx, SmallLayout* out);
// the generic engines' placement of a candidate's messages for column degree
// bounds up to 6 (bsd_layout.cu): pos[e] = the word of CSR edge e inside its
// row's storage window [row_ptr[i], row_ptr[i + 1]); kedge[k * N + j] = the
// CSR edge in slot k of column j (-1: a hole); excess = bank loads above each
// column group's largest degree left by the search; false for codes beyond
// kGenericLayoutMaxEdges edges or with a column above colK
struct GenericLayout {
    std::vector<int> pos;
    std::vector<int> kedge;
    int excess;
};
constexpr int kGenericLayoutMaxEdges = 1 << 20;
bool generic_layout(int M, int N, const int* row_ptr, const int* col_idx, int colK, GenericLayout* out);
// the placement's plane stride for codes of M rows (the engine holds
// ceil(M / 32) rows per lane); every plane spans 2 M <= 64 ceil(M / 32) words
__host__ __device__ constexpr int small_plane_stride_rpl(int rpl) { return 64 * rpl + 12; }
inline int small_plane_stride(int M) { return small_plane_stride_rpl((M + 31) / 32); }

struct SlotMeta {
    long long S;           // sum over U of q(|sum_LLR_j|), q = round(x * 2^16)
    int iters;             // iterations run by this BP call (>= 1)
    int next_pos;          // least reliable unmasked node, -1 if none
    int success;           // H e^ = s' at the last iteration
    int flags;             // bit 0: argmin margin inside (0, tie_guard)
};

struct Outputs {
    uint32_t* corr;        // [B][WN]
    uint32_t* obs;         // [B][WK] (may be null when K = 0)
    uint32_t* status;      // [B]
    uint32_t* iters;       // [B] or null
};

// device-resident description of the chunk being decoded: kernels read their
// buffers from here, so one instantiated CUDA graph serves every call
struct RunDesc {
    const uint32_t* synd;
    Outputs out;
    long long chunk_base;  // index of the chunk's first shot in the caller's batch
    long long chunk_n;     // shots in the chunk
    int pass;              // current beam pass
    int round;             // current beam round of the pass (graph launches read it from here)
    int win_base;          // batched seed BP: first entry of the fail list in the current window
};

// per-chunk counters (reset by k_begin_chunk)
struct Counters {
    int claim_seed;
    int n_active;          // seed-store entries written by k_seed
    int err;
    int n_queue;           // shots the first-iteration screen passed on to the seed BP
    // batched seed BP (bsd_batch.cu)
    int bs_claim;          // queue entries handed to slots so far
    int bs_run;            // the batch has active slots: another iteration runs
    int bs_active_next;    // active slots after the current retirement (counted by its blocks)
    int bs_done_blocks;    // blocks of the current retirement that have finished
    int n_fail;            // shots passed on to the per-candidate seed kernel
    // followed by 3 * (max_rounds + 2) ints for the current pass:
    // claim_round[r], claim_select[r], work_count[r] (reset by k_pass_end)
};

struct Work {
    long long S;           // shots per chunk = seed-store entries
    long long S1;          // with the batched seed BP: shots per chunk (>= S); the shots it hands on are
                           // decoded from the seed on in windows of S
    long long A;           // active entries per beam pass
    int SB;                // words per slot bit record: sp[WM] mask[WN] vals[WN] ehat[WN]
    int* queue;            // [S1] chunk-local shots the screen passed on to the seed BP
    // batched seed BP over slots (bsd_batch.cu); bs_slots = 0: not used
    int bs_slots;          // Bs, a multiple of kBsChunk
    unsigned char* bsE;    // [Epad][Bs] messages in the storage format, shots contiguous
    float2* bsR;           // [M][Bs] detector records (min1, min2) with the row's sign parity in bit 31
    int* bs_shot;          // [Bs] chunk-local shot in the slot, -1 when empty
    int* bs_t;             // [Bs] iterations the slot's shot has run
    int* bs_nl;            // [Bs] columns with e^_j(t) = 1 found in the current iteration
    int* bs_list;          // [kBsList][Bs] those columns
    int* fail;             // [S1] shots the batch passes on to the per-candidate seed kernel
    // seed store [S]
    unsigned char* seedE;  // [S][Epad] messages in the storage format
    uint32_t* seedBits;    // [S][SB]
    SlotMeta* seedMeta;    // [S]
    int* seed_shot;        // [S] chunk-local shot of a seed-store entry
    // beam window [A]
    unsigned char* slotE;  // [2][A][2w][Epad] messages in the storage format
    uint32_t* slotBits;    // [2][A][2w][SB]
    SlotMeta* slotMeta;    // [2][A][2w]
    int* shot_of;          // [A] chunk-local shot of a window entry
    int* set_size;         // [A]
    uint8_t* set_idx;      // [A][w] child index (in the parent bank) of the path of rank k
    unsigned long long* iters_acc;   // [A]
    int* done;             // [A]
    uint32_t* res_bits;    // [A][num_results][WN]
    long long* res_w;      // [A][num_results]
    int* res_origin;       // [A][num_results]: 0 = seed, 1 = masked BP round
    int* res_n;            // [A]
    int* near;             // [A] a near-tie met by this shot's search so far
    unsigned long long* first_ok;  // [A] (round stamp << 32) | ~c of the lowest-index successful child so far
    int2* items;           // [2][A * 2w] (window entry, child index) for rounds >= 2
    Counters* ctr;
    int* round_ctr;        // 3 * (max_rounds + 2) ints after ctr
    RunDesc* desc;
    unsigned long long* stats;   // [5]: executed full BP iterations (seed, rounds), kernel launches, message
                                 // updates of first-iteration screens, seed iterations run by the batch
                                 // (included in [0]); never reset by a chunk
};

// batched seed BP: slots per block of its passes, and the columns with
// e^_j = 1 a slot can list in one iteration (a shot with more is passed on to
// the per-candidate seed kernel)
constexpr int kBsChunk = 256;
constexpr int kBsList = 64;
constexpr int kStats = 5;

// true if e is an error; the error and the source line of the call are then
// kept as the calling thread's most recent CUDA failure (bsd_last_cuda_error)
bool cuda_failed_at(cudaError_t e, const char* file, int line);
#define CUDA_FAILED(x) ::bsd::cuda_failed_at((x), __FILE__, __LINE__)

// workspace layout for S seed entries and A window entries starting at base
// (base may be null to size it); returns the bytes used.  The counters and the
// run descriptor come first, in the first head_bytes(cfg) bytes.
size_t work_layout(const DevGraph& g, const DecCfg& cfg, long long S, long long A, char* base, Work* w,
                   int bs_slots = 0, long long S1 = 0);
size_t work_head_bytes(const DecCfg& cfg);

// host-side launch helpers (bsd_kernels.cu)
struct LaunchShape {
    int warps_per_block;
    int group_warps;       // warps per BP candidate: 1 (a warp) or the whole block
    int select_warps;      // block size of the selection kernel, in warps (<= 8)
    int grid_seed, grid_round, grid_select;
    int screen;            // a first-iteration screen kernel runs before the seed BP
    int grid_screen;       // its blocks of 8 warps (one shot per warp)
    int dv_screen;         // its column degree bound: 0 -> 3, 1 -> 6, 2 -> 16
    size_t smem_screen;
    size_t smem_bp;        // dynamic shared memory of the seed / round kernels
    size_t smem_select;
    int dv;                // engine id
    int batch;             // the seed BP runs batched over slots (when the workspace has them)
    int grid_bs;           // blocks of the batched passes (persistent)
};

// optional callbacks around every kernel launch; kinds 0 seed, 1 round,
// 2 select, 3..6 the unrolled decoder's check / error / error adjoint / check
// adjoint passes, 7 its other kernels, 8..10 the batched seed BP's check pass,
// error-node pass and retirement, 11 the first-iteration screen
constexpr int kProfKinds = BSD_PROFILE_KINDS;
struct LaunchHooks {
    void (*before)(void* ctx, int kind);
    void (*after)(void* ctx, int kind);
    void* ctx;
};

// choose the engine and launch shape; group_warps 0 = automatic, 1 = a warp
// per candidate, >= 2 = a block of that many warps per candidate;
// warps_per_block 0 = automatic (warp engines only)
int configure_kernels(DevGraph& g, const DecCfg& cfg, int device, int group_warps, int warps_per_block,
                      LaunchShape* ls);

// decode one chunk: reset counters and set the run descriptor, then the seed
// kernel and as many beam passes as the chunk has active windows.  With a
// graph (built by build_graph) the passes run under a conditional WHILE node;
// without one, n_active is read back after the seed kernel.
int launch_chunk(const DevGraph& g, const DecCfg& cfg, const Work& w, const LaunchShape& ls,
                 const uint32_t* synd, long long chunk_base, long long chunk_n, const Outputs& out,
                 void* stream, const LaunchHooks* hooks, void* graph_exec, int* host_n_active);
// build and instantiate the per-chunk graph (seed kernel + WHILE over beam passes)
int build_graph(const DevGraph& g, const DecCfg& cfg, const Work& w, const LaunchShape& ls, void** graph_exec);

// batched seed BP (bsd_batch.cu): slots that fit a byte budget (0: none)
int batch_slots_for(const DevGraph& g, long long budget);
// add its nodes after `dep` (begin, WHILE the batch has active slots {check
// pass, error-node pass, retirement}); *last is the node that follows
int add_batch_nodes(cudaGraph_t graph, cudaGraphNode_t dep, cudaGraphNode_t* last, const DevGraph& g,
                    const DecCfg& cfg, const Work& w, const LaunchShape& ls, int screened);
// the same kernels launched one by one, reading the batch's state back to the
// host (into *host_word) every few iterations
int launch_batch_direct(const DevGraph& g, const DecCfg& cfg, const Work& w, const LaunchShape& ls, int screened,
                        cudaStream_t s, const LaunchHooks* hk, int* host_word);
// grid of the batched passes for this device
int batch_grid(int device);
void destroy_graph(void* graph_exec);
// the mailbox of the single-syndrome request loop, in host-mapped memory;
// the syndrome [WM], correction [WN] and observable flips [WK] words follow it
struct ServeBox {
    uint32_t req;          // host: number of the latest request (its syndrome written first)
    uint32_t stop;         // host: nonzero ends the loop
    uint32_t done;         // device: number of the last answered request (outputs written first)
    uint32_t state;        // device: 1 looping, 2 left after the idle limit, 3 left on stop
    uint32_t status;       // device: the answer's status, 0 when the beam search must decide
    uint32_t iters;        // device: the answer's BP iterations
    uint32_t pad[2];
};
int launch_serve(const DevGraph& g, const DecCfg& cfg, const LaunchShape& ls, ServeBox* box, uint32_t last,
                 unsigned long long idle_ns, void* stream);
int launch_bp_llr(const DevGraph& g, const DecCfg& cfg, const LaunchShape& ls, const uint32_t* synd,
                  long long B, int T, float* llr, float* sum_llr, void* stream);
// single-precision re-runs of near-tie shots
int launch_collect_flagged(const uint32_t* status, long long B, long long* list, int* count, void* stream);
int launch_gather_rows(const uint32_t* src, const long long* list, int n, int W, uint32_t* dst, void* stream);
int launch_scatter_results(const long long* list, int n, int WN, int WK, const Outputs& from, const Outputs& to,
                           void* stream);

// the decoder's device graph, configuration and device (bsd_api.cu)
int decoder_graph(const bsd_decoder* dec, const DevGraph** g, const DecCfg** cfg, int* device);
// the decoder's timing hooks on `stream` when kernel timing is enabled
bool decoder_hooks(const bsd_decoder* dec, void* stream, LaunchHooks* hk);

}  // namespace bsd
