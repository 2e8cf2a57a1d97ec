// bsd_api.cu -- host side of the C ABI declared in include/bsd.h.
//
// bsd_create validates (H, A, p) and the Alg. 3 parameters, builds the
// device graph tables (CSR, per-column edge lists, column bitsets of H and A,
// prior LLRs) and sizes the beam workspace; bsd_decode splits a batch into
// chunks that fit the workspace and launches, per chunk, the seed kernel and
// two kernels per beam round, all on the caller's stream.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "bsd.h"
#include "bsd_internal.cuh"

using namespace bsd;

struct bsd_decoder {
    int device = 0;
    bsd_params prm{};
    DevGraph g{};
    DecCfg cfg{};
    LaunchShape ls{};
    void* graph_mem = nullptr;
    size_t graph_bytes = 0;
    void* work_mem = nullptr;
    size_t work_bytes = 0;
    size_t ctr_bytes = 0;
    Work w{};
    void* io_mem = nullptr;        // device staging for bsd_decode_host
    size_t io_bytes = 0;
    cudaStream_t last_stream = nullptr;
    void* graph = nullptr;                   // instantiated per-chunk graph (or null)
    int* h_nactive = nullptr;                // pinned: active entries of a chunk (launch path without graph)
    // opt-in kernel timing
    bool prof = false;
    cudaStream_t prof_stream = nullptr;
    std::vector<cudaEvent_t> ev;             // event pool
    size_t ev_used = 0;
    struct Rec { int kind; size_t e0, e1; };
    std::vector<Rec> recs;
    int open_kind = -1;
    size_t open_ev = 0;
    double ms[kProfKinds] = {};
    long long launches[kProfKinds] = {};
    // 16-bit messages: a single-precision decoder for near-tie re-runs
    bsd_decoder* twin = nullptr;
    void* rr_mem = nullptr;                  // flagged list, count, gathered syndromes, re-run outputs
    long long rr_cap = 0;                    // capacity of the flagged list
    float* weights_mem = nullptr;            // [wT][Epad] weights of weighted min-sum (bsd_set_weights),
                                             // then the same at the single-warp engine's words
    int small_excess = -1;                   // single-warp placement: bank loads above three left (-1: none)
    int small_extent = 0;                    // words it spans
    std::vector<int> small_addr;             // its word of every CSR edge
    std::vector<int> generic_pos;            // the generic engines' word of every CSR edge (empty: CSR order)
    // the single-syndrome request loop (bsd_serve_*)
    ServeBox* serve_h = nullptr;             // mailbox, host-mapped (null when not serving)
    ServeBox* serve_d = nullptr;             // its device address
    cudaStream_t serve_stream = nullptr;     // the loop's stream
    cudaStream_t serve_fb = nullptr;         // the regular path for answers left to the beam search
    uint32_t serve_seq = 0;                  // number of the latest request
    unsigned long long serve_idle_ns = 0;
    void* graph_small = nullptr;             // the same graph with grids sized for chunks of <= small_n shots
    int small_n = 0;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (CUDA_FAILED(cudaGetDevice(&prev))) prev = -1;
        ok = !CUDA_FAILED(cudaSetDevice(dev));
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
inline int words_of(long long bits) { return (int)((bits + 31) / 32); }

// default of the batched seed BP: codes with at least this many edges, and
// this many slots
constexpr long long kBatchMinEdges = 16384;
constexpr int kBatchDefaultSlots = 2048;

const char* kPresetNames[] = {"beam8_230iters", "beam32_340iters", "beam64_640iters", "beam64_32res_640iters"};
// Table I: max_rounds, beam_width, initial_iters, iters_per_round, num_results
const int kPresetVals[][5] = {{10, 8, 30, 20, 1}, {10, 32, 40, 30, 1}, {20, 64, 40, 30, 1}, {20, 64, 40, 30, 32}};

int validate_params(const bsd_params* p)
{
    if (!p) return BSD_ERR_INVALID_ARG;
    if (p->struct_version != BSD_PARAMS_VERSION) return BSD_ERR_INVALID_ARG;
    if (p->max_rounds < 0 || p->max_rounds > 10000) return BSD_ERR_INVALID_ARG;
    if (p->beam_width < 1 || p->beam_width > kMaxBeam) return BSD_ERR_INVALID_ARG;
    if (p->initial_iters < 1 || p->initial_iters > 1000000) return BSD_ERR_INVALID_ARG;
    if (p->iters_per_round < 1 || p->iters_per_round > 1000000) return BSD_ERR_INVALID_ARG;
    if (p->num_results < 1 || p->num_results > kMaxResults) return BSD_ERR_INVALID_ARG;
    if (!(p->ms_scale > 0.f) || !(p->ms_scale <= 4.f)) return BSD_ERR_INVALID_ARG;
    if (!(p->llr_clamp > 0.f) || !std::isfinite(p->llr_clamp)) return BSD_ERR_INVALID_ARG;
    if (p->msg_precision != BSD_FP32 && p->msg_precision != BSD_FP16 && p->msg_precision != BSD_BF16)
        return BSD_ERR_UNSUPPORTED;
    if (!std::isfinite(p->tie_guard_rel)) return BSD_ERR_INVALID_ARG;
    if (p->workspace_bytes < 0) return BSD_ERR_INVALID_ARG;
    if (p->group_warps < 0 || p->group_warps > 16 || p->small_batch < -1 || p->small_batch > 65536)
        return BSD_ERR_INVALID_ARG;
    if (p->batch_slots < -1 || (p->batch_slots > 0 && p->batch_slots < kBsChunk) || p->batch_slots > 65536)
        return BSD_ERR_INVALID_ARG;
    return BSD_OK;
}

template <class T>
T* carve(char*& p, size_t count)
{
    T* r = reinterpret_cast<T*>(p);
    p += align256(sizeof(T) * (count > 0 ? count : 1));
    return r;
}


// launch grids for a chunk of at most n shots: the persistent kernels claim
// their work, so fewer blocks suffice and none of them starts only to find
// nothing to claim
LaunchShape small_shape(const LaunchShape& ls, const DecCfg& cfg, int n)
{
    LaunchShape s = ls;
    const long long per_block = ls.group_warps >= 2 ? 1 : ls.warps_per_block;
    auto cap = [](long long v, int full) { return (int)(v < 1 ? 1 : (v < full ? v : full)); };
    s.grid_seed = cap((n + per_block - 1) / per_block, ls.grid_seed);
    // no first-iteration screen and no batched seed BP: for a few shots their
    // extra launches cost more latency than they save
    s.screen = 0;
    s.batch = 0;
    s.grid_round = cap(((long long)n * 2 * cfg.w + per_block - 1) / per_block, ls.grid_round);
    s.grid_select = cap((n + ls.select_warps - 1) / ls.select_warps, ls.grid_select);
    return s;
}

// (re)build the decoder's graphs from its current graph, configuration and
// shape; a graph that cannot be built leaves the direct-launch path
void rebuild_graphs(bsd_decoder* dec)
{
    if (dec->graph) destroy_graph(dec->graph);
    if (dec->graph_small) destroy_graph(dec->graph_small);
    dec->graph = dec->graph_small = nullptr;
    if (build_graph(dec->g, dec->cfg, dec->w, dec->ls, &dec->graph) != 0) dec->graph = nullptr;
    if (dec->small_n > 0 &&
        build_graph(dec->g, dec->cfg, dec->w, small_shape(dec->ls, dec->cfg, dec->small_n), &dec->graph_small) != 0)
        dec->graph_small = nullptr;
}
}  // namespace

namespace bsd {
namespace {
thread_local cudaError_t t_last_cuda_error = cudaSuccess;
thread_local const char* t_last_cuda_file = "";
thread_local int t_last_cuda_line = 0;
thread_local char t_last_cuda_text[320];
}  // namespace

bool cuda_failed_at(cudaError_t e, const char* file, int line)
{
    if (e == cudaSuccess) return false;
    t_last_cuda_error = e;
    t_last_cuda_file = file;
    t_last_cuda_line = line;
    return true;
}
}  // namespace bsd

extern "C" {

const char* bsd_last_cuda_error(void)
{
    const cudaError_t e = bsd::t_last_cuda_error;
    if (e == cudaSuccess) return "";
    const char* f = strrchr(bsd::t_last_cuda_file, '/');
    snprintf(bsd::t_last_cuda_text, sizeof(bsd::t_last_cuda_text), "%s: %s (%s:%d)", cudaGetErrorName(e),
             cudaGetErrorString(e), f ? f + 1 : bsd::t_last_cuda_file, bsd::t_last_cuda_line);
    return bsd::t_last_cuda_text;
}

const char* bsd_error_string(int code)
{
    switch (code) {
        case BSD_OK: return "ok";
        case BSD_ERR_INVALID_ARG: return "invalid argument";
        case BSD_ERR_CUDA: return "CUDA runtime error";
        case BSD_ERR_OOM: return "out of memory";
        case BSD_ERR_TIMEOUT: return "device-side wait timed out";
        case BSD_ERR_UNSUPPORTED: return "unsupported size or option";
        case BSD_ERR_DEVICE: return "device-side check failed";
        case BSD_ERR_SCRATCH: return "one shot needs more scratch than the static array holds";
        default: return "unknown error";
    }
}

int bsd_params_default(bsd_params* out)
{
    if (!out) return BSD_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    out->struct_version = BSD_PARAMS_VERSION;
    out->max_rounds = 10;
    out->beam_width = 8;
    out->initial_iters = 30;
    out->iters_per_round = 20;
    out->num_results = 1;
    out->ms_scale = 1.0f;
    out->llr_clamp = 1.0e4f;
    out->msg_precision = BSD_FP32;
    out->workspace_bytes = 0;
    return BSD_OK;
}

int bsd_params_preset(const char* name, bsd_params* out)
{
    if (!name || !out) return BSD_ERR_INVALID_ARG;
    for (int k = 0; k < 4; ++k) {
        if (std::strcmp(name, kPresetNames[k]) == 0) {
            bsd_params_default(out);
            out->max_rounds = kPresetVals[k][0];
            out->beam_width = kPresetVals[k][1];
            out->initial_iters = kPresetVals[k][2];
            out->iters_per_round = kPresetVals[k][3];
            out->num_results = kPresetVals[k][4];
            return BSD_OK;
        }
    }
    return BSD_ERR_INVALID_ARG;
}

void bsd_destroy(bsd_decoder* dec)
{
    if (!dec) return;
    bsd_serve_stop(dec);
    {
        DeviceGuard dg(dec->device);
        if (dec->graph_mem) cudaFree(dec->graph_mem);
        if (dec->work_mem) cudaFree(dec->work_mem);
        if (dec->io_mem) cudaFree(dec->io_mem);
        if (dec->graph) destroy_graph(dec->graph);
        if (dec->graph_small) destroy_graph(dec->graph_small);
        if (dec->h_nactive) cudaFreeHost(dec->h_nactive);
        if (dec->rr_mem) cudaFree(dec->rr_mem);
        if (dec->weights_mem) cudaFree(dec->weights_mem);
        for (cudaEvent_t e : dec->ev) cudaEventDestroy(e);
    }
    if (dec->twin) bsd_destroy(dec->twin);
    delete dec;
}

int bsd_create(int32_t M, int32_t N, int32_t K, const int32_t* H_row_ptr, const int32_t* H_col_idx,
               const int32_t* A_row_ptr, const int32_t* A_col_idx, const double* priors, const bsd_params* params,
               int device, bsd_decoder** out)
{
    if (!out) return BSD_ERR_INVALID_ARG;
    *out = nullptr;
    if (M < 1 || N < 1 || K < 0 || !H_row_ptr || !H_col_idx || !priors) return BSD_ERR_INVALID_ARG;
    if (K > 0 && (!A_row_ptr || !A_col_idx)) return BSD_ERR_INVALID_ARG;
    int rc = validate_params(params);
    if (rc) return rc;
    // ---- validate H and A
    if (H_row_ptr[0] != 0) return BSD_ERR_INVALID_ARG;
    for (int i = 0; i < M; ++i) {
        if (H_row_ptr[i + 1] < H_row_ptr[i]) return BSD_ERR_INVALID_ARG;
        for (int e = H_row_ptr[i]; e < H_row_ptr[i + 1]; ++e) {
            if (H_col_idx[e] < 0 || H_col_idx[e] >= N) return BSD_ERR_INVALID_ARG;
            if (e > H_row_ptr[i] && H_col_idx[e] <= H_col_idx[e - 1]) return BSD_ERR_INVALID_ARG;
        }
    }
    const long long E = H_row_ptr[M];
    if (E < 1 || E > (1ll << 30)) return E < 1 ? BSD_ERR_INVALID_ARG : BSD_ERR_UNSUPPORTED;
    if (K > 0) {
        if (A_row_ptr[0] != 0) return BSD_ERR_INVALID_ARG;
        for (int i = 0; i < K; ++i) {
            if (A_row_ptr[i + 1] < A_row_ptr[i]) return BSD_ERR_INVALID_ARG;
            for (int e = A_row_ptr[i]; e < A_row_ptr[i + 1]; ++e)
                if (A_col_idx[e] < 0 || A_col_idx[e] >= N) return BSD_ERR_INVALID_ARG;
        }
    }
    for (int j = 0; j < N; ++j)
        if (!(priors[j] > 0.0 && priors[j] < 1.0)) return BSD_ERR_INVALID_ARG;

    bsd_decoder* dec = new (std::nothrow) bsd_decoder();
    if (!dec) return BSD_ERR_OOM;
    dec->device = device;
    dec->prm = *params;
    DeviceGuard dg(device);
    if (!dg.ok) { delete dec; return BSD_ERR_CUDA; }

    // ---- host tables
    const int WM = words_of(M), WN = words_of(N), WK = words_of(K);
    // the single-warp engine's placement of the messages, for the codes it
    // can run (at most 5 words of columns, 3 of rows); Epad covers it
    SmallLayout sl;
    const bool has_sl = N <= 32 * kSmallMaxCpl && M <= 32 * kSmallMaxRpl && small_layout(M, N, H_row_ptr, H_col_idx, &sl);
    int Epad = (int)((E + 7) / 8 * 8);
    if (has_sl) Epad = std::max(Epad, (sl.extent + 7) / 8 * 8);
    const int Npad = (N + 3) / 4 * 4;
    const int prec = params->msg_precision;
    const int msg_bytes = prec == BSD_FP32 ? 4 : 2;
    std::vector<int> col_ptr(N + 1, 0), col_edge(E), col_row(E);
    for (long long e = 0; e < E; ++e) col_ptr[H_col_idx[e] + 1]++;
    for (int j = 0; j < N; ++j) col_ptr[j + 1] += col_ptr[j];
    {
        std::vector<int> fill(N, 0);
        for (int i = 0; i < M; ++i)
            for (int e = H_row_ptr[i]; e < H_row_ptr[i + 1]; ++e) {
                const int j = H_col_idx[e];
                const int k = col_ptr[j] + fill[j]++;
                col_edge[k] = e;
                col_row[k] = i;
            }
    }
    int max_col = 0, max_row = 0;
    for (int j = 0; j < N; ++j) max_col = std::max(max_col, col_ptr[j + 1] - col_ptr[j]);
    for (int i = 0; i < M; ++i) max_row = std::max(max_row, H_row_ptr[i + 1] - H_row_ptr[i]);
    // a stored message is the nearest value of the storage format (ties to
    // even); L_MAX is taken at its stored value
    auto store_round = [prec](float x) -> float {
        if (prec == BSD_FP16) return __half2float(__float2half_rn(x));
        if (prec == BSD_BF16) return __bfloat162float(__float2bfloat16_rn(x));
        return x;
    };
    const float L = store_round(params->llr_clamp);
    std::vector<float> lam(Npad, 0.f), lamE(Epad, 0.f);
    std::vector<long long> lamq(N);
    int all_pos = 1;
    for (int j = 0; j < N; ++j) {
        // prior LLR (App. A): Lambda_j = log((1 - p_j) / p_j)
        lam[j] = (float)std::log((1.0 - priors[j]) / priors[j]);
        lamq[j] = (long long)std::llrint((double)lam[j] * kFixScale);
        if (!(lam[j] > 0.f)) all_pos = 0;
    }
    for (long long e = 0; e < E; ++e) lamE[e] = store_round(std::fmin(std::fmax(lam[H_col_idx[e]], -L), L));
    // E(0) in the storage format (a zero stored as +0)
    std::vector<unsigned char> lamE_st((size_t)Epad * msg_bytes, 0);
    for (int e = 0; e < Epad; ++e) {
        const float v = lamE[e] == 0.f ? 0.f : lamE[e];
        if (prec == BSD_FP32) {
            std::memcpy(&lamE_st[(size_t)e * 4], &v, 4);
        } else {
            const unsigned short b = prec == BSD_FP16 ? __half_as_ushort(__float2half_rn(v))
                                                     : __bfloat16_as_ushort(__float2bfloat16_rn(v));
            std::memcpy(&lamE_st[(size_t)e * 2], &b, 2);
        }
    }
    // detector records of E(0), the same for every seed run up to the syndrome
    // sign: the two smallest stored |E(0)| from L_MAX, the edge of the
    // smallest (first on ties) and the parity of the negative messages,
    // formed by the same comparisons as the engines' detector pass
    std::vector<float4> rs0(M);
    for (int i = 0; i < M; ++i) {
        float m1 = L, m2 = L;
        int id = -1;
        unsigned neg = 0;
        for (int e = H_row_ptr[i]; e < H_row_ptr[i + 1]; ++e) {
            const float x = lamE[e] == 0.f ? 0.f : lamE[e];
            const float a = std::fabs(x);
            if (a < m1) { m2 = m1; m1 = a; id = e; }
            else if (a < m2) { m2 = a; }
            neg ^= (x < 0.f) ? 1u : 0u;
        }
        float fid, fneg;
        std::memcpy(&fid, &id, 4);
        std::memcpy(&fneg, &neg, 4);
        rs0[i] = make_float4(m1, m2, fid, fneg);
    }
    // the first check messages of a seed run, before the syndrome sign:
    // alpha * (the minimum over the other edges) with the sign of the others'
    // parity, formed as the small engine forms them (its t = 1 detector pass
    // only flips the sign bit when s_i = 1)
    std::vector<float> D0(Epad, 0.f);
    for (int i = 0; i < M; ++i) {
        const float m1 = rs0[i].x, m2 = rs0[i].y;
        unsigned neg;
        std::memcpy(&neg, &rs0[i].w, 4);
        const float d1 = params->ms_scale * m1, d2 = params->ms_scale * m2;
        for (int e = H_row_ptr[i]; e < H_row_ptr[i + 1]; ++e) {
            const float x = lamE[e] == 0.f ? 0.f : lamE[e];
            float d = (std::fabs(x) == m1) ? d2 : d1;
            if ((neg ^ (x < 0.f ? 1u : 0u)) & 1u) d = -d;
            D0[e] = d;
        }
    }
    // D0 and E(0) at the single-warp engine's words
    std::vector<float> sD0;
    std::vector<unsigned char> slamE_st;
    if (has_sl) {
        sD0.assign(Epad, 0.f);
        slamE_st.assign((size_t)Epad * msg_bytes, 0);
        for (long long e = 0; e < E; ++e) {
            sD0[sl.addr[e]] = D0[e];
            std::memcpy(&slamE_st[(size_t)sl.addr[e] * msg_bytes], &lamE_st[(size_t)e * msg_bytes], msg_bytes);
        }
    }
    // the generic engines' column table: (edge, row) of the k-th edge of column
    // j at [k][j], (-1, -1) past the column's degree, for degree bounds 3 and 6
    const int colK = max_col <= 3 ? 3 : max_col <= 6 ? 6 : 0;
    std::vector<int2> colER((size_t)colK * Npad, make_int2(-1, -1));
    // the generic engines keep a candidate's messages at the words of their
    // own placement (bsd_layout.cu: each row's edges permuted inside the row's
    // window, each column's edges in the k slots of a colouring), so that the
    // 32 lanes of an error-pass access meet distinct banks where possible
    GenericLayout gl;
    const bool has_gl = colK > 0 && generic_layout(M, N, H_row_ptr, H_col_idx, colK, &gl);
    if (has_gl) {
        std::vector<int> erow(E);
        for (int i = 0; i < M; ++i)
            for (int e = H_row_ptr[i]; e < H_row_ptr[i + 1]; ++e) erow[e] = i;
        for (int k = 0; k < colK; ++k)
            for (int j = 0; j < N; ++j) {
                const int e = gl.kedge[(size_t)k * N + j];
                if (e >= 0) colER[(size_t)k * Npad + j] = make_int2(gl.pos[e], erow[e]);
            }
    } else {
        for (int j = 0; j < N && colK > 0; ++j)
            for (int k = 0; k < col_ptr[j + 1] - col_ptr[j]; ++k)
                colER[(size_t)k * Npad + j] = make_int2(col_edge[col_ptr[j] + k], col_row[col_ptr[j] + k]);
    }
    // E(0) of column j in the storage format (every edge of the column holds it)
    std::vector<unsigned char> lamEc_st((size_t)Npad * msg_bytes, 0);
    for (int j = 0; j < N; ++j) {
        const int e = col_ptr[j + 1] > col_ptr[j] ? col_edge[col_ptr[j]] : -1;
        if (e >= 0) std::memcpy(&lamEc_st[(size_t)j * msg_bytes], &lamE_st[(size_t)e * msg_bytes], msg_bytes);
        else {
            // a column with no edge: its E(0) is never read, but keep the value
            const float v = store_round(std::fmin(std::fmax(lam[j], -L), L));
            if (prec == BSD_FP32) std::memcpy(&lamEc_st[(size_t)j * 4], &v, 4);
        }
    }
    // the first-iteration screen's column table: per column the check message
    // of E(0) on each of its edges (D0, before the syndrome sign) and the edge's
    // row, padded to the engines' degree bound with (+inf, -1)
    const int rdk = max_col <= 3 ? 4 : max_col <= 6 ? 6 : max_col <= kMaxColDeg ? kMaxColDeg : 0;
    std::vector<float> colRD((size_t)Npad * rdk * 2, 0.f);
    for (int j = 0; j < Npad && rdk > 0; ++j) {
        const int deg = j < N ? col_ptr[j + 1] - col_ptr[j] : 0;
        for (int k = 0; k < rdk; ++k) {
            float d = INFINITY;
            int r = -1;
            if (k < deg) {
                d = D0[col_edge[col_ptr[j] + k]];
                r = col_row[col_ptr[j] + k];
            }
            colRD[((size_t)j * rdk + k) * 2] = d;
            std::memcpy(&colRD[((size_t)j * rdk + k) * 2 + 1], &r, 4);
        }
    }
    // the columns ordered by degree, each column's (edge, row) pairs contiguous
    // in the order of the column lists (the batched seed BP walks runs of
    // columns of one degree)
    std::vector<int> colperm, dstart(kMaxColDeg + 2, 0), dbase(kMaxColDeg + 2, 0);
    std::vector<int2> colseq;
    if (max_col <= kMaxColDeg) {
        colperm.reserve(N);
        colseq.reserve(E);
        for (int d = 0; d <= kMaxColDeg; ++d) {
            dstart[d] = (int)colperm.size();
            dbase[d] = (int)colseq.size();
            for (int j = 0; j < N; ++j) {
                if (col_ptr[j + 1] - col_ptr[j] != d) continue;
                colperm.push_back(j);
                for (int k = col_ptr[j]; k < col_ptr[j + 1]; ++k) colseq.push_back(make_int2(col_edge[k], col_row[k]));
            }
        }
        dstart[kMaxColDeg + 1] = (int)colperm.size();
        dbase[kMaxColDeg + 1] = (int)colseq.size();
    }
    std::vector<uint32_t> hcol((size_t)N * WM, 0u), acol((size_t)N * (WK > 0 ? WK : 1), 0u);
    for (int i = 0; i < M; ++i)
        for (int e = H_row_ptr[i]; e < H_row_ptr[i + 1]; ++e)
            hcol[(size_t)H_col_idx[e] * WM + (i >> 5)] |= 1u << (i & 31);
    for (int i = 0; i < K; ++i)
        for (int e = A_row_ptr[i]; e < A_row_ptr[i + 1]; ++e)
            acol[(size_t)A_col_idx[e] * WK + (i >> 5)] ^= 1u << (i & 31);

    // ---- device graph
    size_t gb = 0;
    gb += align256(sizeof(int) * (M + 1));
    gb += align256(sizeof(int) * E);
    gb += align256(sizeof(int) * (N + 1));
    gb += 2 * align256(sizeof(int) * E);
    gb += align256(sizeof(float) * Npad);
    gb += align256((size_t)msg_bytes * Epad);
    gb += align256(sizeof(uint32_t) * hcol.size());
    gb += align256(sizeof(uint32_t) * acol.size());
    gb += align256(sizeof(long long) * N);
    gb += align256(sizeof(float4) * M);
    gb += align256(sizeof(float) * Epad);
    gb += align256(sizeof(int2) * colER.size());
    gb += align256(lamEc_st.size());
    gb += align256(sizeof(int) * colperm.size());
    gb += align256(sizeof(int2) * colseq.size());
    gb += align256(sizeof(float) * colRD.size());
    // the single-warp engine's per-column record: Lambda_j and column j of H in one 16-byte load
    std::vector<uint32_t> slamh;
    if (has_sl) {
        slamh.assign((size_t)4 * 32 * WN, 0u);
        for (int j = 0; j < N; ++j) {
            std::memcpy(&slamh[(size_t)4 * j], &lam[j], sizeof(float));
            for (int q = 0; q < WM && q < 3; ++q) slamh[(size_t)4 * j + 1 + q] = hcol[(size_t)j * WM + q];
        }
    }
    if (has_sl) {
        gb += align256(sizeof(uint32_t) * sl.col.size());
        gb += align256(sizeof(float) * sD0.size());
        gb += align256(slamE_st.size());
        gb += align256(sizeof(uint32_t) * slamh.size());
    }
    if (CUDA_FAILED(cudaMalloc(&dec->graph_mem, gb))) { bsd_destroy(dec); return BSD_ERR_OOM; }
    dec->graph_bytes = gb;
    char* p = (char*)dec->graph_mem;
    int* d_row_ptr = carve<int>(p, M + 1);
    int* d_row_col = carve<int>(p, E);
    int* d_col_ptr = carve<int>(p, N + 1);
    int* d_col_edge = carve<int>(p, E);
    int* d_col_row = carve<int>(p, E);
    float* d_lam = carve<float>(p, Npad);
    unsigned char* d_lamE = carve<unsigned char>(p, (size_t)msg_bytes * Epad);
    uint32_t* d_hcol = carve<uint32_t>(p, hcol.size());
    uint32_t* d_acol = carve<uint32_t>(p, acol.size());
    long long* d_lamq = carve<long long>(p, N);
    float4* d_rs0 = carve<float4>(p, M);
    float* d_D0 = carve<float>(p, Epad);
    int2* d_colER = colER.empty() ? nullptr : carve<int2>(p, colER.size());
    unsigned char* d_lamEc = carve<unsigned char>(p, lamEc_st.size());
    int* d_colperm = colperm.empty() ? nullptr : carve<int>(p, colperm.size());
    int2* d_colseq = colseq.empty() ? nullptr : carve<int2>(p, colseq.size());
    float* d_colRD = colRD.empty() ? nullptr : carve<float>(p, colRD.size());
    uint32_t* d_scol = has_sl ? carve<uint32_t>(p, sl.col.size()) : nullptr;
    float* d_sD0 = has_sl ? carve<float>(p, sD0.size()) : nullptr;
    unsigned char* d_slamE = has_sl ? carve<unsigned char>(p, slamE_st.size()) : nullptr;
    uint32_t* d_slamh = has_sl ? carve<uint32_t>(p, slamh.size()) : nullptr;
    bool ok = !CUDA_FAILED(cudaMemcpy(d_row_ptr, H_row_ptr, sizeof(int) * (M + 1), cudaMemcpyHostToDevice)) &&
              !CUDA_FAILED(cudaMemcpy(d_row_col, H_col_idx, sizeof(int) * E, cudaMemcpyHostToDevice)) &&
              !CUDA_FAILED(cudaMemcpy(d_col_ptr, col_ptr.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice)) &&
              !CUDA_FAILED(cudaMemcpy(d_col_edge, col_edge.data(), sizeof(int) * E, cudaMemcpyHostToDevice)) &&
              !CUDA_FAILED(cudaMemcpy(d_col_row, col_row.data(), sizeof(int) * E, cudaMemcpyHostToDevice)) &&
              !CUDA_FAILED(cudaMemcpy(d_lam, lam.data(), sizeof(float) * Npad, cudaMemcpyHostToDevice)) &&
              !CUDA_FAILED(cudaMemcpy(d_lamE, lamE_st.data(), lamE_st.size(), cudaMemcpyHostToDevice)) &&
              !CUDA_FAILED(cudaMemcpy(d_hcol, hcol.data(), sizeof(uint32_t) * hcol.size(), cudaMemcpyHostToDevice)) &&
              !CUDA_FAILED(cudaMemcpy(d_acol, acol.data(), sizeof(uint32_t) * acol.size(), cudaMemcpyHostToDevice)) &&
              !CUDA_FAILED(cudaMemcpy(d_lamq, lamq.data(), sizeof(long long) * N, cudaMemcpyHostToDevice)) &&
              !CUDA_FAILED(cudaMemcpy(d_rs0, rs0.data(), sizeof(float4) * M, cudaMemcpyHostToDevice)) &&
              !CUDA_FAILED(cudaMemcpy(d_D0, D0.data(), sizeof(float) * Epad, cudaMemcpyHostToDevice)) &&
              (colER.empty() ||
               !CUDA_FAILED(cudaMemcpy(d_colER, colER.data(), sizeof(int2) * colER.size(), cudaMemcpyHostToDevice))) &&
              !CUDA_FAILED(cudaMemcpy(d_lamEc, lamEc_st.data(), lamEc_st.size(), cudaMemcpyHostToDevice)) &&
              (colperm.empty() ||
               !CUDA_FAILED(cudaMemcpy(d_colperm, colperm.data(), sizeof(int) * colperm.size(), cudaMemcpyHostToDevice))) &&
              (colseq.empty() ||
               !CUDA_FAILED(cudaMemcpy(d_colseq, colseq.data(), sizeof(int2) * colseq.size(), cudaMemcpyHostToDevice))) &&
              (colRD.empty() ||
               !CUDA_FAILED(cudaMemcpy(d_colRD, colRD.data(), sizeof(float) * colRD.size(), cudaMemcpyHostToDevice))) &&
              (!has_sl ||
               (!CUDA_FAILED(cudaMemcpy(d_scol, sl.col.data(), sizeof(uint32_t) * sl.col.size(), cudaMemcpyHostToDevice)) &&
                !CUDA_FAILED(cudaMemcpy(d_sD0, sD0.data(), sizeof(float) * sD0.size(), cudaMemcpyHostToDevice)) &&
                !CUDA_FAILED(cudaMemcpy(d_slamE, slamE_st.data(), slamE_st.size(), cudaMemcpyHostToDevice)) &&
                !CUDA_FAILED(cudaMemcpy(d_slamh, slamh.data(), sizeof(uint32_t) * slamh.size(), cudaMemcpyHostToDevice))));
    if (!ok) { bsd_destroy(dec); return BSD_ERR_CUDA; }

    DevGraph& g = dec->g;
    g.M = M; g.N = N; g.K = K; g.E = (int)E;
    g.WM = WM; g.WN = WN; g.WK = WK;
    g.Epad = Epad; g.Npad = Npad;
    g.msg_bytes = msg_bytes; g.prec = prec;
    g.max_col_deg = max_col; g.max_row_deg = max_row;
    g.all_lam_pos = all_pos;
    g.row_ptr = d_row_ptr; g.row_col = d_row_col; g.col_ptr = d_col_ptr; g.col_edge = d_col_edge; g.col_row = d_col_row;
    g.lam = d_lam; g.lamE = d_lamE; g.hcol = d_hcol; g.acol = d_acol; g.lamq = d_lamq; g.rs0 = d_rs0; g.D0 = d_D0;
    g.colER = d_colER; g.colK = colK; g.lamEc = d_lamEc;
    g.colperm = d_colperm; g.colseq = d_colseq;
    g.colRD = reinterpret_cast<const float4*>(d_colRD); g.colRDk = rdk;
    for (int d = 0; d < kMaxColDeg + 2; ++d) { g.dstart[d] = dstart[d]; g.dbase[d] = dbase[d]; }
    g.scol = d_scol; g.sD0 = d_sD0; g.slamE = d_slamE; g.slamh = reinterpret_cast<const uint4*>(d_slamh);
    if (has_gl) dec->generic_pos = gl.pos;
    if (has_sl) {
        dec->small_excess = sl.excess;
        dec->small_extent = sl.extent;
        dec->small_addr = sl.addr;
    }

    DecCfg& cfg = dec->cfg;
    cfg.max_rounds = params->max_rounds;
    cfg.w = params->beam_width;
    cfg.initial_iters = params->initial_iters;
    cfg.iters_per_round = params->iters_per_round;
    cfg.num_results = params->num_results;
    cfg.alpha = params->ms_scale;
    cfg.L = L;
    // near-tie margin: the given value, the precision's default for 16-bit
    // messages when 0, no flags when negative (or 0 with single precision)
    const float tg = params->tie_guard_rel;
    cfg.tie_guard = tg > 0.f ? (double)tg : (tg == 0.f && prec == BSD_FP16) ? 1e-3 : (tg == 0.f && prec == BSD_BF16) ? 1e-2 : 0.0;
    cfg.weights = nullptr;         // the scale alpha until bsd_set_weights
    cfg.sweights = nullptr;
    cfg.wT = 0;

    rc = configure_kernels(g, cfg, device, params->group_warps, 0, &dec->ls);
    if (rc) { bsd_destroy(dec); return rc == -5 ? BSD_ERR_UNSUPPORTED : BSD_ERR_CUDA; }

    // ---- workspace: a seed store of S shots and a beam window of A active
    // entries (two banks of 2w child slots each), about 1 : 4 in bytes
    const int W2 = 2 * cfg.w;
    const int SB = WM + 3 * WN;
    const int NR = cfg.num_results;
    const double seed_b = (double)msg_bytes * Epad + sizeof(uint32_t) * (double)SB + sizeof(SlotMeta) + 4.0;
    const double win_b = 2.0 * W2 * ((double)msg_bytes * Epad + sizeof(uint32_t) * (double)SB + sizeof(SlotMeta)) +
                         12.0 + cfg.w + 8.0 + NR * (4.0 * WN + 12.0) + 4.0 + 2.0 * W2 * sizeof(int2);
    long long budget = params->workspace_bytes > 0 ? params->workspace_bytes : (4ll << 30);
    // the batched seed BP's slots: the requested count, or by default for
    // codes of at least kBatchMinEdges edges kBatchDefaultSlots (measured on
    // GB300: on the 35k-edge synthetic DEM the batch decodes 1.8x faster than
    // one candidate per block of warps in single precision, on the 6912-edge
    // phenomenological DEM 1.6x slower, where the per-iteration launches
    // dominate); at most a quarter of the workspace
    int bs_slots = 0;
    const bool bs_default = params->batch_slots == 0 && E >= kBatchMinEdges;
    if (dec->ls.batch && (params->batch_slots > 0 || bs_default)) {
        const long long cap = budget / 4;
        const int fit = batch_slots_for(g, cap);
        const int want = params->batch_slots > 0 ? params->batch_slots / kBsChunk * kBsChunk
                                                 : kBatchDefaultSlots;
        bs_slots = want < fit ? want : fit;
        if (bs_slots > 0) {
            Work probe{};
            const size_t with = work_layout(g, cfg, 1, 1, nullptr, &probe, bs_slots);
            const size_t without = work_layout(g, cfg, 1, 1, nullptr, nullptr);
            budget -= (long long)(with - without);
        }
    }
    long long A = (long long)(0.8 * (double)budget / win_b);
    if (A < 1) A = 1;
    long long S = (long long)(((double)budget - (double)A * win_b) / seed_b);
    if (S > (1ll << 22)) S = 1ll << 22;
    if (S < A) S = A;
    if (A > (1ll << 22)) A = 1ll << 22;
    // with the batched seed BP a chunk can hold far more shots than the seed
    // store: only the shots it hands on need an entry, and they are decoded
    // in windows of S
    const long long S1 = bs_slots > 0 ? (1ll << 22) : 0;
    for (;;) {
        const size_t wb = work_layout(g, cfg, S, A, nullptr, nullptr, bs_slots, S1);
        if (cudaMalloc(&dec->work_mem, wb) == cudaSuccess) { dec->work_bytes = wb; break; }
        cudaGetLastError();
        dec->work_mem = nullptr;
        if (S == 1 && A == 1) { bsd_destroy(dec); return BSD_ERR_OOM; }
        S = S > 1 ? S / 2 : 1;
        A = A > 1 ? A / 2 : 1;
    }
    Work& w = dec->w;
    work_layout(g, cfg, S, A, (char*)dec->work_mem, &w, bs_slots, S1);
    dec->ctr_bytes = work_head_bytes(cfg);
    if (CUDA_FAILED(cudaMemset(dec->work_mem, 0, dec->ctr_bytes)) ||
        CUDA_FAILED(cudaMallocHost(&dec->h_nactive, sizeof(int)))) {
        bsd_destroy(dec);
        return BSD_ERR_CUDA;
    }
    // the per-chunk graph: seed kernel + WHILE over beam passes; without it
    // decoding falls back to plain launches
    dec->small_n = params->small_batch > 0 ? params->small_batch : (params->small_batch == 0 ? 32 : 0);
    rebuild_graphs(dec);
    // 16-bit messages with near-tie flags: shots flagged by the 16-bit run are
    // decoded again by a single-precision twin
    if (prec != BSD_FP32 && cfg.tie_guard > 0.0) {
        bsd_params p2 = *params;
        p2.msg_precision = BSD_FP32;
        p2.tie_guard_rel = -1.f;
        p2.workspace_bytes = budget / 4 > (256ll << 20) ? budget / 4 : (256ll << 20);
        const int rc2 = bsd_create(M, N, K, H_row_ptr, H_col_idx, A_row_ptr, A_col_idx, priors, &p2, device,
                                   &dec->twin);
        if (rc2 != BSD_OK) { bsd_destroy(dec); return rc2; }
    }
    *out = dec;
    return BSD_OK;
}

// decode again, in single precision, every shot of [d_synd, B) whose status
// carries the near-tie flag; outputs land where the 16-bit run put them
static int rerun_flagged(bsd_decoder* dec, const uint32_t* d_synd, long long B, const Outputs& o, cudaStream_t s)
{
    if (!dec->twin || B <= 0) return BSD_OK;
    const DevGraph& g = dec->g;
    const int WKo = g.WK > 0 ? g.WK : 1;
    const long long R = 65536;
    if (dec->rr_cap < B) {
        if (dec->rr_mem) cudaFree(dec->rr_mem);
        dec->rr_mem = nullptr;
        dec->rr_cap = 0;
        const size_t need = align256(sizeof(long long) * (size_t)B) + 256 +
                            align256(sizeof(uint32_t) * (size_t)R * (g.WM + g.WN + WKo + 2));
        if (CUDA_FAILED(cudaMalloc(&dec->rr_mem, need))) { cudaGetLastError(); return BSD_ERR_OOM; }
        dec->rr_cap = B;
    }
    char* p = (char*)dec->rr_mem;
    long long* list = carve<long long>(p, (size_t)dec->rr_cap);
    int* count = reinterpret_cast<int*>(p);
    p += 256;
    uint32_t* gs = carve<uint32_t>(p, (size_t)R * g.WM);
    uint32_t* gc = carve<uint32_t>(p, (size_t)R * g.WN);
    uint32_t* go = carve<uint32_t>(p, (size_t)R * WKo);
    uint32_t* gst = carve<uint32_t>(p, (size_t)R);
    uint32_t* git = carve<uint32_t>(p, (size_t)R);
    if (launch_collect_flagged(o.status, B, list, count, s) != 0 ||
        CUDA_FAILED(cudaMemcpyAsync(dec->h_nactive, count, sizeof(int), cudaMemcpyDeviceToHost, s)) ||
        CUDA_FAILED(cudaStreamSynchronize(s)))
        return BSD_ERR_CUDA;
    const long long n = *dec->h_nactive;
    for (long long off = 0; off < n; off += R) {
        const int m = (int)((n - off) < R ? (n - off) : R);
        if (launch_gather_rows(d_synd, list + off, m, g.WM, gs, s) != 0) return BSD_ERR_CUDA;
        const int rc = bsd_decode(dec->twin, gs, m, gc, g.K > 0 ? go : nullptr, gst, git, s);
        if (rc != BSD_OK) return rc;
        Outputs from{gc, g.K > 0 ? go : nullptr, gst, git};
        if (launch_scatter_results(list + off, m, g.WN, g.WK, from, o, s) != 0) return BSD_ERR_CUDA;
    }
    return BSD_OK;
}

// ---- opt-in kernel timing: events around every launch on the decode stream
static size_t prof_event(bsd_decoder* d)
{
    if (d->ev_used == d->ev.size()) {
        cudaEvent_t e;
        if (CUDA_FAILED(cudaEventCreate(&e))) return (size_t)-1;
        d->ev.push_back(e);
    }
    return d->ev_used++;
}

static void prof_before(void* ctx, int kind)
{
    bsd_decoder* d = (bsd_decoder*)ctx;
    const size_t e = prof_event(d);
    if (e == (size_t)-1) return;
    cudaEventRecord(d->ev[e], d->prof_stream);
    d->open_kind = kind;
    d->open_ev = e;
}

static void prof_after(void* ctx, int kind)
{
    bsd_decoder* d = (bsd_decoder*)ctx;
    if (d->open_kind != kind) return;
    const size_t e = prof_event(d);
    if (e == (size_t)-1) return;
    cudaEventRecord(d->ev[e], d->prof_stream);
    d->recs.push_back({kind, d->open_ev, e});
    d->open_kind = -1;
}

static void prof_collect(bsd_decoder* d)
{
    for (const auto& r : d->recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, d->ev[r.e0], d->ev[r.e1]) == cudaSuccess) {
            d->ms[r.kind] += ms;
            d->launches[r.kind] += 1;
        }
    }
    d->recs.clear();
    d->ev_used = 0;
}

// shots per chunk: the seed store, or with the batched seed BP the larger
// chunk whose handed-on shots it decodes in windows of the seed store
static long long chunk_of(const bsd_decoder* dec)
{
    return (dec->ls.batch && dec->w.bs_slots > 0) ? dec->w.S1 : dec->w.S;
}

static int decode_impl(bsd_decoder* dec, const uint32_t* d_synd, long long base, long long n, const Outputs& o,
                       cudaStream_t s)
{
    LaunchHooks hk{prof_before, prof_after, dec};
    dec->prof_stream = s;
    // a small chunk (at most S shots: no batched seed BP) runs the small-chunk
    // graph, or its kernels one by one while timing is enabled
    const bool small = dec->small_n > 0 && n <= dec->small_n && n <= dec->w.S;
    if (dec->prof || (small ? !dec->graph_small : !dec->graph)) {
        const LaunchShape ls = small ? small_shape(dec->ls, dec->cfg, dec->small_n) : dec->ls;
        return launch_chunk(dec->g, dec->cfg, dec->w, ls, d_synd, base, n, o, s, dec->prof ? &hk : nullptr, nullptr,
                            dec->h_nactive)
                   ? BSD_ERR_CUDA
                   : BSD_OK;
    }
    void* gx = small ? dec->graph_small : dec->graph;
    return launch_chunk(dec->g, dec->cfg, dec->w, dec->ls, d_synd, base, n, o, s, dec->prof ? &hk : nullptr, gx,
                        dec->h_nactive)
               ? BSD_ERR_CUDA
               : BSD_OK;
}

int bsd_decode(bsd_decoder* dec, const uint32_t* d_syndromes, int64_t B, uint32_t* d_corrections,
               uint32_t* d_obs_flips, uint32_t* d_status, uint32_t* d_iters, void* cuda_stream)
{
    if (!dec || B < 0) return BSD_ERR_INVALID_ARG;
    if (B == 0) return BSD_OK;
    if (!d_syndromes || !d_corrections || !d_status || (dec->g.K > 0 && !d_obs_flips)) return BSD_ERR_INVALID_ARG;
    DeviceGuard dg(dec->device);
    if (!dg.ok) return BSD_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    dec->last_stream = s;
    Outputs o{d_corrections, dec->g.K > 0 ? d_obs_flips : nullptr, d_status, d_iters};
    const long long C = chunk_of(dec);
    for (long long base = 0; base < B; base += C) {
        const long long n = (B - base) < C ? (B - base) : C;
        const int rc = decode_impl(dec, d_syndromes, base, n, o, s);
        if (rc) return rc;
    }
    return rerun_flagged(dec, d_syndromes, B, o, s);
}

int bsd_decode_host(bsd_decoder* dec, const uint32_t* h_syndromes, int64_t B, uint32_t* h_corrections,
                    uint32_t* h_obs_flips, uint32_t* h_status, uint32_t* h_iters, void* cuda_stream)
{
    if (!dec || B < 0) return BSD_ERR_INVALID_ARG;
    if (B == 0) return BSD_OK;
    if (!h_syndromes || !h_corrections || !h_status || (dec->g.K > 0 && !h_obs_flips)) return BSD_ERR_INVALID_ARG;
    DeviceGuard dg(dec->device);
    if (!dg.ok) return BSD_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    dec->last_stream = s;
    const DevGraph& g = dec->g;
    // host chunks: the seed store, or for the batched seed BP up to 2^18 shots
    const long long C = chunk_of(dec) > dec->w.S ? (chunk_of(dec) < (1ll << 18) ? chunk_of(dec) : (1ll << 18))
                                                  : dec->w.S;
    const size_t need = align256(sizeof(uint32_t) * C * g.WM) + align256(sizeof(uint32_t) * C * g.WN) +
                        align256(sizeof(uint32_t) * C * (g.WK > 0 ? g.WK : 1)) + 2 * align256(sizeof(uint32_t) * C);
    if (dec->io_bytes < need) {
        if (dec->io_mem) cudaFree(dec->io_mem);
        dec->io_mem = nullptr;
        dec->io_bytes = 0;
        if (CUDA_FAILED(cudaMalloc(&dec->io_mem, need))) { cudaGetLastError(); return BSD_ERR_OOM; }
        dec->io_bytes = need;
    }
    char* p = (char*)dec->io_mem;
    uint32_t* d_s = carve<uint32_t>(p, C * g.WM);
    uint32_t* d_c = carve<uint32_t>(p, C * g.WN);
    uint32_t* d_o = carve<uint32_t>(p, C * (g.WK > 0 ? g.WK : 1));
    uint32_t* d_st = carve<uint32_t>(p, C);
    uint32_t* d_it = carve<uint32_t>(p, C);
    Outputs o{d_c, g.K > 0 ? d_o : nullptr, d_st, h_iters ? d_it : nullptr};
    for (long long base = 0; base < B; base += C) {
        const long long n = (B - base) < C ? (B - base) : C;
        if (CUDA_FAILED(cudaMemcpyAsync(d_s, h_syndromes + base * g.WM, sizeof(uint32_t) * n * g.WM, cudaMemcpyHostToDevice, s)))
            return BSD_ERR_CUDA;
        int rc = decode_impl(dec, d_s, 0, n, o, s);
        if (rc) return rc;
        // a re-run needs iteration counts to scatter: use the staging buffer
        Outputs o_rr{d_c, g.K > 0 ? d_o : nullptr, d_st, d_it};
        if (dec->twin && (rc = rerun_flagged(dec, d_s, n, o_rr, s)) != BSD_OK) return rc;
        bool ok = !CUDA_FAILED(cudaMemcpyAsync(h_corrections + base * g.WN, d_c, sizeof(uint32_t) * n * g.WN,
                                  cudaMemcpyDeviceToHost, s)) &&
                  !CUDA_FAILED(cudaMemcpyAsync(h_status + base, d_st, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, s));
        if (ok && g.K > 0)
            ok = !CUDA_FAILED(cudaMemcpyAsync(h_obs_flips + base * g.WK, d_o, sizeof(uint32_t) * n * g.WK, cudaMemcpyDeviceToHost,
                                 s));
        if (ok && h_iters)
            ok = !CUDA_FAILED(cudaMemcpyAsync(h_iters + base, d_it, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, s));
        if (!ok) return BSD_ERR_CUDA;
    }
    return !CUDA_FAILED(cudaStreamSynchronize(s)) ? BSD_OK : BSD_ERR_CUDA;
}

int bsd_bp_llr(bsd_decoder* dec, const uint32_t* d_syndromes, int64_t B, int32_t T, float* d_llr, float* d_sum_llr,
               void* cuda_stream)
{
    if (!dec || B < 0 || T < 1 || T > 100000) return BSD_ERR_INVALID_ARG;
    if (B == 0) return BSD_OK;
    if (!d_syndromes || !d_llr) return BSD_ERR_INVALID_ARG;
    DeviceGuard dg(dec->device);
    if (!dg.ok) return BSD_ERR_CUDA;
    dec->last_stream = (cudaStream_t)cuda_stream;
    return launch_bp_llr(dec->g, dec->cfg, dec->ls, d_syndromes, B, T, d_llr, d_sum_llr, cuda_stream) ? BSD_ERR_CUDA
                                                                                                      : BSD_OK;
}

int bsd_sync_error(bsd_decoder* dec)
{
    if (!dec) return BSD_ERR_INVALID_ARG;
    DeviceGuard dg(dec->device);
    if (!dg.ok) return BSD_ERR_CUDA;
    if (CUDA_FAILED(cudaStreamSynchronize(dec->last_stream))) return BSD_ERR_CUDA;
    Counters c;
    if (CUDA_FAILED(cudaMemcpy(&c, dec->w.ctr, sizeof(c), cudaMemcpyDeviceToHost))) return BSD_ERR_CUDA;
    if (c.err != 0) {
        const int zero = 0;
        cudaMemcpy(&dec->w.ctr->err, &zero, sizeof(int), cudaMemcpyHostToDevice);
        return c.err == 1 ? BSD_ERR_TIMEOUT : BSD_ERR_DEVICE;
    }
    return BSD_OK;
}

// switch the decoder to another launch shape (kernels, graph); results do not change
static int apply_shape(bsd_decoder* dec, int group_warps, int warps_per_block)
{
    DevGraph g = dec->g;
    LaunchShape ls{};
    const int rc = configure_kernels(g, dec->cfg, dec->device, group_warps, warps_per_block, &ls);
    if (rc) return rc == -5 ? BSD_ERR_UNSUPPORTED : BSD_ERR_CUDA;
    dec->g = g;
    dec->ls = ls;
    rebuild_graphs(dec);
    return BSD_OK;
}

int bsd_get_shape(const bsd_decoder* dec, int32_t* group_warps, int32_t* warps_per_block)
{
    if (!dec) return BSD_ERR_INVALID_ARG;
    if (group_warps) *group_warps = dec->ls.group_warps;
    if (warps_per_block) *warps_per_block = dec->ls.warps_per_block;
    return BSD_OK;
}

int bsd_autotune(bsd_decoder* dec, const uint32_t* d_syndromes, int64_t B, void* cuda_stream,
                 bsd_shape_timing* report, int32_t report_cap, int32_t* n_report)
{
    if (!dec || !d_syndromes || B < 1 || report_cap < 0 || (report_cap > 0 && !report)) return BSD_ERR_INVALID_ARG;
    if (dec->serve_h && bsd_serve_stop(dec) != BSD_OK) return BSD_ERR_CUDA;   // it runs the current kernels
    DeviceGuard dg(dec->device);
    if (!dg.ok) return BSD_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (CUDA_FAILED(cudaStreamSynchronize(dec->last_stream)) || CUDA_FAILED(cudaStreamSynchronize(s)))
        return BSD_ERR_CUDA;
    const DevGraph& g0 = dec->g;
    const int WKo = g0.WK > 0 ? g0.WK : 1;
    void* mem = nullptr;
    const size_t need = sizeof(uint32_t) * (size_t)B * (size_t)(g0.WN + WKo + 2);
    if (CUDA_FAILED(cudaMalloc(&mem, need))) return BSD_ERR_OOM;
    uint32_t* d_c = (uint32_t*)mem;
    uint32_t* d_o = d_c + (size_t)B * g0.WN;
    uint32_t* d_st = d_o + (size_t)B * WKo;
    uint32_t* d_it = d_st + B;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (CUDA_FAILED(cudaEventCreate(&e0)) || CUDA_FAILED(cudaEventCreate(&e1))) {
        if (e0) cudaEventDestroy(e0);
        cudaFree(mem);
        return BSD_ERR_CUDA;
    }
    // candidate shapes: warps per block of the one-warp engines, then blocks
    // of 2 .. 16 warps per candidate; shapes the code cannot use are skipped
    const int cand[][2] = {{1, 8}, {1, 4}, {1, 2}, {1, 1}, {2, 0}, {4, 0}, {8, 0}, {16, 0}};
    const int prev_gw = dec->ls.group_warps >= 2 ? dec->ls.group_warps : 1;
    const int prev_wpb = dec->ls.group_warps >= 2 ? 0 : dec->ls.warps_per_block;
    int best = -1, nrep = 0, rc = BSD_OK;
    float best_ms = 0.f;
    for (int c = 0; c < (int)(sizeof(cand) / sizeof(cand[0])) && rc == BSD_OK; ++c) {
        const int r = apply_shape(dec, cand[c][0], cand[c][1]);
        if (r == BSD_ERR_UNSUPPORTED) continue;
        if (r != BSD_OK) { rc = r; break; }
        // two untimed decodes (first-touch, caches), then the fastest of three
        float ms = 0.f;
        for (int rep = 0; rep < 5 && rc == BSD_OK; ++rep) {
            if (rep >= 2 && CUDA_FAILED(cudaEventRecord(e0, s))) { rc = BSD_ERR_CUDA; break; }
            rc = bsd_decode(dec, d_syndromes, B, d_c, g0.K > 0 ? d_o : nullptr, d_st, d_it, s);
            if (rc != BSD_OK) break;
            if (rep >= 2) {
                float t = 0.f;
                if (CUDA_FAILED(cudaEventRecord(e1, s)) || CUDA_FAILED(cudaEventSynchronize(e1)) ||
                    CUDA_FAILED(cudaEventElapsedTime(&t, e0, e1))) { rc = BSD_ERR_CUDA; break; }
                ms = (rep == 2 || t < ms) ? t : ms;
            }
        }
        if (rc != BSD_OK) break;
        if (nrep < report_cap) report[nrep] = bsd_shape_timing{dec->ls.group_warps, dec->ls.warps_per_block, ms};
        ++nrep;
        if (best < 0 || ms < best_ms) { best = c; best_ms = ms; }
    }
    if (CUDA_FAILED(cudaStreamSynchronize(s)) && rc == BSD_OK) rc = BSD_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(mem);
    // keep the fastest shape (or the previous one if nothing could be timed)
    const int r2 = best >= 0 && rc == BSD_OK ? apply_shape(dec, cand[best][0], cand[best][1])
                                             : apply_shape(dec, prev_gw, prev_wpb);
    if (n_report) *n_report = nrep;
    return rc != BSD_OK ? rc : r2;
}

int bsd_set_weights(bsd_decoder* dec, const float* h_weights, int32_t T)
{
    if (!dec || T < 0 || (T > 0 && !h_weights)) return BSD_ERR_INVALID_ARG;
    if (dec->serve_h && bsd_serve_stop(dec) != BSD_OK) return BSD_ERR_CUDA;   // it runs the current kernels
    if (T > 0 && dec->g.prec != BSD_FP32) return BSD_ERR_UNSUPPORTED;
    const size_t E = (size_t)dec->g.E, Epad = (size_t)dec->g.Epad;
    for (size_t k = 0; k < (size_t)T * E; ++k)
        if (!std::isfinite(h_weights[k]) || std::fabs(h_weights[k]) > 1e6f) return BSD_ERR_INVALID_ARG;
    DeviceGuard dg(dec->device);
    if (!dg.ok) return BSD_ERR_CUDA;
    // work already queued on the decoder's stream uses the current kernels and weights
    if (CUDA_FAILED(cudaStreamSynchronize(dec->last_stream))) return BSD_ERR_CUDA;
    float* d_w = nullptr;
    // [T][Epad] at the generic engines' words, then (for codes the
    // single-warp engine can run) [T][Epad] at that engine's words
    const bool two = dec->g.scol != nullptr;
    const bool gperm = !dec->generic_pos.empty();
    if (T > 0) {
        std::vector<float> hw((size_t)T * Epad * (two ? 2 : 1), 0.f);
        for (size_t t = 0; t < (size_t)T; ++t) {
            if (gperm) {
                for (size_t e = 0; e < E; ++e) hw[t * Epad + (size_t)dec->generic_pos[e]] = h_weights[t * E + e];
            } else {
                std::memcpy(hw.data() + t * Epad, h_weights + t * E, sizeof(float) * E);
            }
            if (two)
                for (size_t e = 0; e < E; ++e)
                    hw[((size_t)T + t) * Epad + (size_t)dec->small_addr[e]] = h_weights[t * E + e];
        }
        if (CUDA_FAILED(cudaMalloc(&d_w, sizeof(float) * hw.size()))) return BSD_ERR_OOM;
        if (CUDA_FAILED(cudaMemcpy(d_w, hw.data(), sizeof(float) * hw.size(), cudaMemcpyHostToDevice))) {
            cudaFree(d_w);
            return BSD_ERR_CUDA;
        }
    }
    DecCfg cfg = dec->cfg;
    cfg.weights = d_w;
    cfg.sweights = (d_w && two) ? d_w + (size_t)T * Epad : nullptr;
    cfg.wT = T;
    DevGraph g = dec->g;
    LaunchShape ls{};
    // keep the decoder's launch shape (engine family, block size)
    const int rc = configure_kernels(g, cfg, dec->device, dec->ls.group_warps >= 2 ? dec->ls.group_warps : 1,
                                     dec->ls.group_warps >= 2 ? 0 : dec->ls.warps_per_block, &ls);
    if (rc) {
        if (d_w) cudaFree(d_w);
        return rc == -5 ? BSD_ERR_UNSUPPORTED : BSD_ERR_CUDA;
    }
    if (dec->weights_mem) cudaFree(dec->weights_mem);
    dec->g = g;
    dec->cfg = cfg;
    dec->ls = ls;
    dec->weights_mem = d_w;
    rebuild_graphs(dec);
    return BSD_OK;
}

int bsd_profile_enable(bsd_decoder* dec, int enable)
{
    if (!dec) return BSD_ERR_INVALID_ARG;
    dec->prof = enable != 0;
    return BSD_OK;
}

int bsd_profile_read(bsd_decoder* dec, double ms[3], int64_t launches[3], uint64_t exec_iters[3],
                     uint64_t* kernel_launches, uint64_t* screen_updates)
{
    if (!dec) return BSD_ERR_INVALID_ARG;
    DeviceGuard dg(dec->device);
    if (!dg.ok) return BSD_ERR_CUDA;
    if (CUDA_FAILED(cudaStreamSynchronize(dec->last_stream))) return BSD_ERR_CUDA;
    prof_collect(dec);
    unsigned long long st[kStats] = {};
    if (CUDA_FAILED(cudaMemcpy(st, dec->w.stats, sizeof(st), cudaMemcpyDeviceToHost)) ||
        CUDA_FAILED(cudaMemset(dec->w.stats, 0, sizeof(st))))
        return BSD_ERR_CUDA;
    for (int k = 0; k < 3; ++k) {
        if (ms) ms[k] = dec->ms[k];
        if (launches) launches[k] = dec->launches[k];
        dec->ms[k] = 0;
        dec->launches[k] = 0;
    }
    if (exec_iters) { exec_iters[0] = st[0]; exec_iters[1] = st[1]; exec_iters[2] = st[4]; }
    if (kernel_launches) *kernel_launches = st[2];
    if (screen_updates) *screen_updates = st[3];
    return BSD_OK;
}

int bsd_profile_read_kinds(bsd_decoder* dec, double ms[BSD_PROFILE_KINDS], int64_t launches[BSD_PROFILE_KINDS])
{
    if (!dec) return BSD_ERR_INVALID_ARG;
    DeviceGuard dg(dec->device);
    if (!dg.ok) return BSD_ERR_CUDA;
    if (CUDA_FAILED(cudaStreamSynchronize(dec->prof_stream))) return BSD_ERR_CUDA;
    prof_collect(dec);
    for (int k = 0; k < kProfKinds; ++k) {
        if (ms) ms[k] = dec->ms[k];
        if (launches) launches[k] = dec->launches[k];
        dec->ms[k] = 0;
        dec->launches[k] = 0;
    }
    return BSD_OK;
}

}  // extern "C"

namespace bsd {
// read-only view of a decoder for the allocation-free entry point (bsd_noalloc.cu)
int decoder_view(const bsd_decoder* dec, const DevGraph** g, const DecCfg** cfg, const LaunchShape** ls,
                 int* device)
{
    if (!dec) return BSD_ERR_INVALID_ARG;
    if (dec->twin) return BSD_ERR_UNSUPPORTED;   // near-tie re-runs need buffers of their own
    *g = &dec->g;
    *cfg = &dec->cfg;
    *ls = &dec->ls;
    *device = dec->device;
    return BSD_OK;
}

bool decoder_hooks(const bsd_decoder* dec, void* stream, LaunchHooks* hk)
{
    bsd_decoder* d = const_cast<bsd_decoder*>(dec);   // the timing records are not part of the decoder's state
    if (!d || !d->prof) return false;
    d->prof_stream = (cudaStream_t)stream;
    *hk = LaunchHooks{prof_before, prof_after, d};
    return true;
}

int decoder_graph(const bsd_decoder* dec, const DevGraph** g, const DecCfg** cfg, int* device)
{
    if (!dec) return BSD_ERR_INVALID_ARG;
    *g = &dec->g;
    *cfg = &dec->cfg;
    *device = dec->device;
    return BSD_OK;
}
}  // namespace bsd

extern "C" {

int bsd_get_info(const bsd_decoder* dec, int32_t* M, int32_t* N, int32_t* K, int32_t* n_edges, int64_t* chunk_shots,
                 int64_t* workspace_bytes)
{
    if (!dec) return BSD_ERR_INVALID_ARG;
    if (M) *M = dec->g.M;
    if (N) *N = dec->g.N;
    if (K) *K = dec->g.K;
    if (n_edges) *n_edges = dec->g.E;
    if (chunk_shots) *chunk_shots = dec->w.S;
    if (workspace_bytes) *workspace_bytes = (int64_t)dec->work_bytes;
    return BSD_OK;
}

int bsd_get_batch(const bsd_decoder* dec, int32_t* slots, int32_t* active)
{
    if (!dec) return BSD_ERR_INVALID_ARG;
    if (slots) *slots = dec->w.bs_slots;
    if (active) *active = (dec->ls.batch && dec->w.bs_slots > 0) ? 1 : 0;
    return BSD_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------
// single-syndrome request loop
// ----------------------------------------------------------------------------
namespace {

constexpr double kServeWaitSeconds = 2.0;     // the host's bound on one answer

// the decoder's streams are the caller's or the legacy stream once the
// loop's own are gone (later calls synchronise dec->last_stream)
void serve_drop_streams(bsd_decoder* dec)
{
    if (dec->last_stream == dec->serve_stream || dec->last_stream == dec->serve_fb) dec->last_stream = nullptr;
    if (dec->serve_stream) cudaStreamDestroy(dec->serve_stream);
    if (dec->serve_fb) cudaStreamDestroy(dec->serve_fb);
    dec->serve_stream = dec->serve_fb = nullptr;
}

int serve_launch(bsd_decoder* dec)
{
    ServeBox* b = dec->serve_h;
    __atomic_store_n(&b->stop, 0u, __ATOMIC_RELAXED);
    __atomic_store_n(&b->state, 0u, __ATOMIC_RELAXED);
    // answer whatever came after the last answered request
    const uint32_t last = __atomic_load_n(&b->done, __ATOMIC_ACQUIRE);
    __atomic_thread_fence(__ATOMIC_SEQ_CST);
    return launch_serve(dec->g, dec->cfg, dec->ls, dec->serve_d, last, dec->serve_idle_ns, dec->serve_stream)
               ? BSD_ERR_CUDA
               : BSD_OK;
}

}  // namespace

extern "C" {

int bsd_serve_start(bsd_decoder* dec, int32_t idle_ms)
{
    if (!dec || idle_ms < 1 || idle_ms > 60000) return BSD_ERR_INVALID_ARG;
    if (dec->serve_h) return BSD_OK;
    DeviceGuard dg(dec->device);
    if (!dg.ok) return BSD_ERR_CUDA;
    const DevGraph& g = dec->g;
    if (CUDA_FAILED(cudaStreamCreateWithFlags(&dec->serve_fb, cudaStreamNonBlocking))) return BSD_ERR_CUDA;
    // one regular decode first: every buffer the regular path allocates on
    // first use exists before the loop is resident (an allocation may wait
    // for the whole device)
    std::vector<uint32_t> zs(g.WM, 0u), zc(g.WN), zo(g.WK > 0 ? g.WK : 1), zst(1), zit(1);
    int rc = bsd_decode_host(dec, zs.data(), 1, zc.data(), g.K > 0 ? zo.data() : nullptr, zst.data(), zit.data(),
                             dec->serve_fb);
    if (rc == BSD_OK && CUDA_FAILED(cudaStreamSynchronize(dec->serve_fb))) rc = BSD_ERR_CUDA;
    const size_t bytes = sizeof(ServeBox) + sizeof(uint32_t) * (size_t)(g.WM + g.WN + (g.WK > 0 ? g.WK : 1));
    void* h = nullptr;
    void* d = nullptr;
    if (rc == BSD_OK && CUDA_FAILED(cudaHostAlloc(&h, bytes, cudaHostAllocMapped))) rc = BSD_ERR_OOM;
    if (rc == BSD_OK) {
        std::memset(h, 0, bytes);
        if (CUDA_FAILED(cudaHostGetDevicePointer(&d, h, 0)) ||
            CUDA_FAILED(cudaStreamCreateWithFlags(&dec->serve_stream, cudaStreamNonBlocking)))
            rc = BSD_ERR_CUDA;
    }
    if (rc == BSD_OK) {
        dec->serve_h = (ServeBox*)h;
        dec->serve_d = (ServeBox*)d;
        dec->serve_seq = 0;
        dec->serve_idle_ns = (unsigned long long)idle_ms * 1000000ull;
        rc = serve_launch(dec);
        if (rc == BSD_OK) return BSD_OK;
        dec->serve_h = dec->serve_d = nullptr;
    }
    serve_drop_streams(dec);
    if (h) cudaFreeHost(h);
    return rc;
}

int bsd_serve_decode(bsd_decoder* dec, const uint32_t* h_syndrome, uint32_t* h_correction, uint32_t* h_obs_flips,
                     uint32_t* h_status, uint32_t* h_iters)
{
    if (!dec || !dec->serve_h || !h_syndrome || !h_correction || !h_status || (dec->g.K > 0 && !h_obs_flips))
        return BSD_ERR_INVALID_ARG;
    DeviceGuard dg(dec->device);
    if (!dg.ok) return BSD_ERR_CUDA;
    const DevGraph& g = dec->g;
    ServeBox* b = dec->serve_h;
    uint32_t* words = reinterpret_cast<uint32_t*>(b + 1);
    // a loop that left after its idle limit runs again
    if (__atomic_load_n(&b->state, __ATOMIC_ACQUIRE) >= 2u) {
        if (CUDA_FAILED(cudaStreamSynchronize(dec->serve_stream))) return BSD_ERR_CUDA;
        if (serve_launch(dec) != BSD_OK) return BSD_ERR_CUDA;
    }
    std::memcpy(words, h_syndrome, sizeof(uint32_t) * (size_t)g.WM);
    uint32_t seq = dec->serve_seq + 1;
    if (seq == 0u) seq = 1u;                      // 0 is the mailbox's initial number
    dec->serve_seq = seq;
    __atomic_store_n(&b->req, seq, __ATOMIC_RELEASE);
    const auto t0 = std::chrono::steady_clock::now();
    while (__atomic_load_n(&b->done, __ATOMIC_ACQUIRE) != seq) {
        if (__atomic_load_n(&b->state, __ATOMIC_ACQUIRE) >= 2u) {
            // the loop reached its idle limit before it saw this request
            if (CUDA_FAILED(cudaStreamSynchronize(dec->serve_stream))) return BSD_ERR_CUDA;
            if (__atomic_load_n(&b->done, __ATOMIC_ACQUIRE) == seq) break;
            if (serve_launch(dec) != BSD_OK) return BSD_ERR_CUDA;
        }
        if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > kServeWaitSeconds)
            return BSD_ERR_TIMEOUT;
    }
    const uint32_t status = __atomic_load_n(&b->status, __ATOMIC_ACQUIRE);
    if (status == 0u)                             // the beam search decides: the regular path
        return bsd_decode_host(dec, h_syndrome, 1, h_correction, h_obs_flips, h_status, h_iters, dec->serve_fb);
    std::memcpy(h_correction, words + g.WM, sizeof(uint32_t) * (size_t)g.WN);
    if (g.K > 0) std::memcpy(h_obs_flips, words + g.WM + g.WN, sizeof(uint32_t) * (size_t)g.WK);
    *h_status = status;
    if (h_iters) *h_iters = __atomic_load_n(&b->iters, __ATOMIC_RELAXED);
    return BSD_OK;
}

int bsd_serve_stop(bsd_decoder* dec)
{
    if (!dec) return BSD_ERR_INVALID_ARG;
    if (!dec->serve_h) return BSD_OK;
    DeviceGuard dg(dec->device);
    if (!dg.ok) return BSD_ERR_CUDA;
    __atomic_store_n(&dec->serve_h->stop, 1u, __ATOMIC_RELEASE);
    // the loop reads the stop flag on every poll and leaves within one answer
    int rc = CUDA_FAILED(cudaStreamSynchronize(dec->serve_stream)) ? BSD_ERR_CUDA : BSD_OK;
    if (CUDA_FAILED(cudaStreamSynchronize(dec->serve_fb))) rc = BSD_ERR_CUDA;
    serve_drop_streams(dec);
    cudaFreeHost(dec->serve_h);
    dec->serve_h = dec->serve_d = nullptr;
    return rc;
}

}  // extern "C"
