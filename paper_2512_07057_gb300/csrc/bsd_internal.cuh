// bsd_internal.cuh -- device data layout shared by the kernels and the host API.
//
// Layout in HBM (all read-only graph tables are tiny and stay L1/L2 resident):
//   row_ptr[M+1]          CSR of H; CSR edge e of row i lies in [row_ptr[i], row_ptr[i+1])
//   col_ptr[N+1]          per error node j, its edges in col_edge/col_row[col_ptr[j] ..)
//   col_edge[E]           CSR edge id of each (column, k) pair, rows ascending
//   col_row[E]            detector (row) of that edge
//   lam[N]                Lambda_j = log((1-p_j)/p_j) rounded to float
//   lamE[E]               clamp(Lambda_{col(e)}), the seed's E(0) in CSR order
//   hcol[N][WM]           column j of H as an M-bit set (syndrome flip for v = 1)
//   acol[N][WK]           column j of A as a K-bit set (observable flips)
//   lamq[N]               Lambda_j on the 2^-16 fixed-point grid (weights)
//
// Beam state per chunk of C shots (workspace):
//   two banks of 2w child slots per active shot; round r writes bank r % 2
//   and reads its parents from bank (r - 1) % 2 through set_idx, so surviving
//   paths are never copied.  A slot holds the edge-message snapshot (Epad
//   floats), the bit vectors s', mask, vals, e^ and a SlotMeta record.
#pragma once
#include <cstdint>

namespace bsd {

constexpr int kMaxBeam = 64;
constexpr int kMaxResults = 64;
constexpr double kFixScale = 65536.0;   // fixed-point grid 2^-16 for scores and weights

struct DevGraph {
    int M, N, K, E;
    int WM, WN, WK;        // words of M, N, K bits
    int Epad, Npad;        // E, N rounded up to a multiple of 4
    int max_col_deg, max_row_deg;
    int all_lam_pos;       // every Lambda_j > 0 (all p_j < 1/2)
    int det_bytes;         // per-warp detector-side shared memory (set with the engine)
    const int* row_ptr;
    const int* col_ptr;
    const int* col_edge;
    const int* col_row;
    const float* lam;
    const float* lamE;
    const uint32_t* hcol;
    const uint32_t* acol;
    const long long* lamq;
};

struct DecCfg {
    int max_rounds, w, initial_iters, iters_per_round, num_results;
    float alpha, L;
};

struct SlotMeta {
    long long S;           // sum over U of q(|sum_LLR_j|), q = round(x * 2^16)
    int iters;             // iterations run by this BP call (>= 1)
    int next_pos;          // least reliable unmasked node, -1 if none
    int success;           // H e^ = s' at the last iteration
    int pad;
};

// per-chunk counters (zeroed before each chunk)
struct Counters {
    int claim_seed;
    int n_active;
    int err;
    int pad;
    // followed by 3 * (max_rounds + 2) ints: claim_round[r], claim_select[r], work_count[r]
};

struct Work {
    long long C;           // chunk capacity in shots
    int SB;                // words per slot bit record: sp[WM] mask[WN] vals[WN] ehat[WN]
    float* slotE;          // [2][C][2w][Epad]
    uint32_t* slotBits;    // [2][C][2w][SB]
    SlotMeta* slotMeta;    // [2][C][2w]
    int* shot_of;          // [C] chunk-local shot of an active entry
    int* set_size;         // [C]
    uint8_t* set_idx;      // [C][w] child index (in the parent bank) of the path of rank k
    unsigned long long* iters_acc;   // [C]
    int* done;             // [C]
    uint32_t* res_bits;    // [C][num_results][WN]
    long long* res_w;      // [C][num_results]
    int* res_origin;       // [C][num_results]: 0 = seed, 1 = masked BP round
    int* res_n;            // [C]
    int2* items;           // [2][C * 2w] (active entry, child index)
    Counters* ctr;
    int* round_ctr;        // 3 * (max_rounds + 2) ints after ctr
    unsigned long long* stats;   // [2] executed BP iterations: seed, beam rounds (not reset per chunk)
};

struct Outputs {
    uint32_t* corr;        // [B][WN]
    uint32_t* obs;         // [B][WK] (may be null when K = 0)
    uint32_t* status;      // [B]
    uint32_t* iters;       // [B] or null
};

// host-side launch helpers (bsd_kernels.cu)
struct LaunchShape {
    int warps_per_block;
    int grid_seed, grid_round, grid_select;
    size_t smem_bp;        // dynamic shared memory of the seed / round kernels
    size_t smem_select;
    int dv;                // compiled column-degree bound used
};

// optional callbacks around every kernel launch (kind: 0 seed, 1 round, 2 select)
struct LaunchHooks {
    void (*before)(void* ctx, int kind);
    void (*after)(void* ctx, int kind);
    void* ctx;
};

int configure_kernels(DevGraph& g, const DecCfg& cfg, int device, LaunchShape* ls);
int launch_chunk(const DevGraph& g, const DecCfg& cfg, const Work& w, const LaunchShape& ls,
                 const uint32_t* synd, long long chunk_base, long long chunk_n, const Outputs& out,
                 void* stream, const LaunchHooks* hooks);
int launch_bp_llr(const DevGraph& g, const DecCfg& cfg, const LaunchShape& ls, const uint32_t* synd,
                  long long B, int T, float* llr, float* sum_llr, void* stream);

}  // namespace bsd
