// bsd_kernels.cu -- sm_103a kernels of the BP-guided beam search decoder.
//
// One warp owns one BP candidate (the seed path of a shot, or one child of a
// beam round) and keeps its whole state in shared memory: the edge messages
// E_{j->i}, a compact 8-byte per-detector record (min1, min2 with the sign
// parity in both sign bits) standing in for the detector-to-error messages
// D_{i->j} (the single-warp engine keeps D per edge instead), sum_LLR, and
// the bit vectors s', mask, vals, e^ and the running syndrome parity.
//
// Kernels (all persistent: warps claim work with one atomic per item and
// exit when the item counter runs out, so uneven iteration counts balance):
//   k_screen<DV>  (generic engines, every Lambda_j > 0, one result) a warp per
//                 shot forms e^(1) from the columns next to flipped detectors;
//                 finalises the shots that converge there, queues the rest
//   k_seed<DV>    the seed BP of every shot in a chunk, or of the queued ones
//                 (Alg. 3, first BP run)
//   k_round<DV>   expand + masked BP for every child of round r (Alg. 2)
//   k_select      per shot: first success in visit order, results, top-w
//                 pruning and the work list of round r + 1 (Alg. 3, App. B)
//   k_bp_llr<DV>  plain BP for a fixed number of iterations (LLR measurement)
//
// Arithmetic follows the readings stated in include/bsd.h: D = alpha * sign *
// min with the minimum over no other unmasked neighbour equal to L_MAX;
// E clamped to [-L_MAX, L_MAX]; the sums of Eqs. 2-3 start at Lambda_j and
// add the incoming messages in ascending order; every add and multiply is a
// single IEEE round-to-nearest operation (__fadd_rn / __fmul_rn, so no FMA
// contraction); scores and weights are summed exactly on a 2^-16 grid.
//
// Masked nodes: the messages of a masked error node are set to +L_MAX when it
// is masked.  A +L_MAX input never lowers a minimum below that of the other
// inputs and never flips a sign, so the check pass needs no mask test; the
// error-node pass skips masked nodes, whose messages therefore stay +L_MAX.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>

#include "bsd_device.cuh"
#include "bsd_internal.cuh"

namespace bsd {

// bytes and 16-byte vectors of one E snapshot (Epad is a multiple of 8)
__host__ __device__ __forceinline__ size_t snap_bytes(const DevGraph& g) { return (size_t)g.Epad * (size_t)g.msg_bytes; }
__host__ __device__ __forceinline__ int snap_vec16(const DevGraph& g) { return (int)(snap_bytes(g) / 16); }

// Early abort of a beam child (num_results = 1): once a child of the same shot
// with a lower canonical index has succeeded in this round, this child's
// result can no longer be the first success in visit order and is never read.
// The shot's key holds (round stamp << 32) | ~c of the lowest successful index
// c so far (atomicMax); a run loads it at the start of an iteration and
// checks it at the end, so the load's latency hides behind the iteration.
struct AbortCheck {
    const unsigned long long* key;   // null: never abort
    unsigned long long stamp;        // this round's stamp << 32
    unsigned c;                      // this child's canonical index
    __device__ __forceinline__ bool hit(unsigned long long v) const
    {
        return (v & 0xffffffff00000000ull) == stamp && (0xffffffffu - (unsigned)v) < c;
    }
};

// copy n16 16-byte vectors (the E snapshot) with the threads of a candidate group
template <class G>
__device__ __forceinline__ void group_copy16(const G& grp, void* dst, const void* src, int n16)
{
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (int q = grp.rank(); q < n16; q += grp.size()) d[q] = s[q];
}


// ----------------------------------------------------------------------------
// candidate groups: the threads that process one BP candidate together.
// WarpGroup is one warp (a block holds several candidates); BlockGroup is a
// whole block (one candidate per block), for codes whose per-candidate state
// leaves room for only a few warps per SM.  Every row and column is computed
// by one thread and every reduction is exact (minima with index ties, integer
// sums, XOR), so both give the same results bit for bit.
// ----------------------------------------------------------------------------
struct ArgRec {                // per-warp partial of the argmin / score reduction
    float best, second;
    int bj, pad;
    unsigned long long s;
};

struct WarpGroup {
    static constexpr bool kBlock = false;
    __device__ static WarpGroup make(char*) { return WarpGroup{}; }
    __device__ __forceinline__ int rank() const { return threadIdx.x & 31; }
    __device__ __forceinline__ int size() const { return 32; }
    __device__ __forceinline__ int warp() const { return 0; }
    __device__ __forceinline__ int nwarps() const { return 1; }
    __device__ __forceinline__ int index() const { return threadIdx.x >> 5; }       // candidate slot of the block
    __device__ __forceinline__ int per_block() const { return blockDim.x >> 5; }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
    __device__ __forceinline__ bool any(bool p) const { return __any_sync(FULLMASK, p); }
    __device__ __forceinline__ int bcast(int v) const { return __shfl_sync(FULLMASK, v, 0); }
    __device__ __forceinline__ uint32_t xor_all(uint32_t v) const
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v ^= __shfl_xor_sync(FULLMASK, v, o);
        return v;
    }
};

struct BlockGroup {
    static constexpr bool kBlock = true;
    ArgRec* rec;               // shared scratch: one record per warp (16 at most)
    __device__ static BlockGroup make(char* scratch) { return BlockGroup{reinterpret_cast<ArgRec*>(scratch)}; }
    __device__ __forceinline__ int rank() const { return threadIdx.x; }
    __device__ __forceinline__ int size() const { return blockDim.x; }
    __device__ __forceinline__ int warp() const { return threadIdx.x >> 5; }
    __device__ __forceinline__ int nwarps() const { return blockDim.x >> 5; }
    __device__ __forceinline__ int index() const { return 0; }
    __device__ __forceinline__ int per_block() const { return 1; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ bool any(bool p) const { return __syncthreads_or(p ? 1 : 0) != 0; }
    __device__ __forceinline__ int bcast(int v) const
    {
        if (threadIdx.x == 0) rec[0].bj = v;
        __syncthreads();
        const int r = rec[0].bj;
        __syncthreads();
        return r;
    }
    __device__ __forceinline__ uint32_t xor_all(uint32_t v) const
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v ^= __shfl_xor_sync(FULLMASK, v, o);
        if ((threadIdx.x & 31) == 0) rec[threadIdx.x >> 5].pad = (int)v;
        __syncthreads();
        uint32_t r = 0;
        for (int q = 0; q < nwarps(); ++q) r ^= (uint32_t)rec[q].pad;
        __syncthreads();
        return r;
    }
};

// shared scratch a candidate group needs beyond the candidate's own state

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// per-warp shared-memory footprint of one BP candidate
// detector-side region: M records of 16 bytes (GenericEngine), or one D
// message per edge and at least M records (SmallEngine); g.det_bytes is set
// with the engine choice
__host__ __device__ inline size_t det_region_bytes(const DevGraph& g) { return (size_t)g.det_bytes; }

__host__ __device__ inline size_t warp_smem_bytes(const DevGraph& g)
{
    return align16((size_t)g.msg_bytes * (size_t)g.Epad) + det_region_bytes(g) +
           align16(sizeof(float) * (size_t)g.Npad) + align16(sizeof(uint32_t) * (size_t)(2 * g.WM + 3 * g.WN));
}

struct WarpState {
    void* E;           // [Epad] E_{j->i} in the storage format, CSR edge order
    float2* rs;        // [M]    (min1, min2), s'_i xor the parity of the negative messages in both sign bits
    float* D;          // [Epad] D_{i->j} per CSR edge (same storage as rs)
    float* sumllr;     // [Npad]
    uint32_t* sp;      // [WM] s' = s with the columns of nodes fixed to 1 folded in
    uint32_t* par;     // [WM] s' xor H e^ (zero iff converged)
    uint32_t* mask;    // [WN]
    uint32_t* vals;    // [WN]
    uint32_t* ehat;    // [WN]
};

__device__ inline WarpState carve(char* base, const DevGraph& g)
{
    WarpState s;
    char* p = base;
    s.E = p;                                 p += align16((size_t)g.msg_bytes * (size_t)g.Epad);
    s.rs = reinterpret_cast<float2*>(p);
    s.D = reinterpret_cast<float*>(p);       p += det_region_bytes(g);
    s.sumllr = reinterpret_cast<float*>(p);  p += align16(sizeof(float) * (size_t)g.Npad);
    uint32_t* b = reinterpret_cast<uint32_t*>(p);
    s.sp = b;
    s.par = b + g.WM;
    s.mask = b + 2 * g.WM;
    s.vals = b + 2 * g.WM + g.WN;
    s.ehat = b + 2 * g.WM + 2 * g.WN;
    return s;
}

// round(x * 2^16) to the nearest integer, ties to even: scaling a float by a
// power of two is exact, so single precision gives the value double would
// (GB300's double-precision pipe is narrow)
__device__ inline unsigned long long fixq(float x)
{
    return (unsigned long long)__float2ll_rn(__fmul_rn(x, (float)kFixScale));
}

// ----------------------------------------------------------------------------
// BP iterations on one candidate (Eqs. 1-4 with the masking of Alg. 2)
// ----------------------------------------------------------------------------
// Runs up to max_iters flooding iterations from the messages in st.E.  With
// stop = true it returns at the first t with H e^(t) = s' (Alg. 2).  On return
// st.ehat holds e^(t) of the last iteration (masked positions 0), st.sumllr
// holds the sum over the iterations run of Lambda_j(t).  With kPostOut,
// Lambda_j(max_iters) is written to post_out.
template <int DV, int P, bool W, bool kPostOut, class G>
__device__ int bp_iterate(const G& grp, const DevGraph& g, const DecCfg& cfg, const WarpState& st, int max_iters,
                          bool stop, int* success, float* post_out, bool from_prior, const AbortCheck& ab)
{
    using S = Store<P>;
    using T = typename S::T;
    T* const E = reinterpret_cast<T*>(st.E);
    const int lane = threadIdx.x & 31;
    const float alpha = cfg.alpha;
    const float L = cfg.L;
    int iters = 0;
    int ok = 0;
    for (int t = 1; t <= max_iters; ++t) {
        unsigned long long ab_key = 0ull;
        if (ab.key != nullptr && grp.rank() == 0) ab_key = *((volatile const unsigned long long*)ab.key);
        for (int q = grp.rank(); q < g.WM; q += grp.size()) st.par[q] = st.sp[q];
        // weighted min-sum: row min(t, wT) - 1 of the weights in place of alpha
        const float* wt = W ? cfg.weights + (size_t)((t < cfg.wT ? t : cfg.wT) - 1) * (size_t)g.Epad : nullptr;

        // a run from E(0) (seed, LLRs): the first check pass is the
        // precomputed E(0) record of each row with the syndrome bit folded into
        // the sign parity, and E(0) itself (clamp(Lambda), the same on every
        // edge of a column) is read from the graph, not from the candidate
        const bool prior = from_prior && t == 1;
        if (prior) {
            for (int i = grp.rank(); i < g.M; i += grp.size()) {
                const float4 r = __ldg(g.rs0 + i);
                const uint32_t sb = (((st.sp[i >> 5] >> (i & 31)) ^ __float_as_uint(r.w)) & 1u) << 31;
                st.rs[i] = make_float2(__uint_as_float(__float_as_uint(r.x) | sb),
                                       __uint_as_float(__float_as_uint(r.y) | sb));
            }
        }
        // ---- detector pass (Eq. 1): min1, min2 and the sign parity per row
        // (8-byte records: the error pass tells the edge holding the minimum
        // by its magnitude -- where the minimum is attained twice, min2 =
        // min1, so this equals the lowest-index argmin rule)
        for (int i = prior ? g.M : grp.rank(); i < g.M; i += grp.size()) {
            const int rb = __ldg(g.row_ptr + i), re = __ldg(g.row_ptr + i + 1);
            float m1 = L, m2 = L;
            uint32_t sg = ((st.sp[i >> 5] >> (i & 31)) & 1u) << 31;
            // branch-free: the runner-up is min(m2, max(m1, a)); a stored
            // message is never -0 (a clamped sum that starts at Lambda_j), so
            // its sign bit is exactly x < 0
            // (four messages per step; past the row's end a lane takes
            // +L_MAX, which changes neither minimum nor the parity)
            for (int e = rb; e < re; e += 4) {
                float x[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) x[u] = (e + u < re) ? S::ld(E, e + u) : L;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float a = fabsf(x[u]);
                    m2 = fminf(m2, fmaxf(m1, a));
                    m1 = fminf(m1, a);
                    sg ^= __float_as_uint(x[u]);
                }
            }
            sg &= 0x80000000u;
            st.rs[i] = make_float2(__uint_as_float(__float_as_uint(m1) | sg), __uint_as_float(__float_as_uint(m2) | sg));
        }
        grp.sync();

        // D_{i->j} of column j's edges in ascending order (padding +inf last),
        // with their CSR edge ids; returns the column's degree
        auto gather = [&](int j, float (&v)[DV], int (&ed)[DV]) -> int {
            // the column's edges: from the padded (edge, row) table for degree
            // bounds up to 6 (one coalesced load per slot), else from the
            // column lists
            int kb = 0, deg = 0;
            if constexpr (DV > 6) {
                kb = __ldg(g.col_ptr + j);
                deg = __ldg(g.col_ptr + j + 1) - kb;
            }
            // E(0) is the same on every edge of a column: one load
            const float x0 = prior ? S::ld(reinterpret_cast<const T*>(g.lamEc), j) : 0.f;
#pragma unroll
            for (int k = 0; k < DV; ++k) {
                int e = -1, r = 0;
                if constexpr (DV <= 6) {
                    const int2 er = __ldg(g.colER + (size_t)k * g.Npad + j);
                    e = er.x;
                    r = er.y;
                    deg += (e >= 0) ? 1 : 0;
                } else if (k < deg) {
                    e = __ldg(g.col_edge + kb + k);
                    r = __ldg(g.col_row + kb + k);
                }
                if (e >= 0) {
                    const float2 r2 = st.rs[r];
                    const float x = prior ? x0 : S::ld(E, e);
                    // the minimum over the row's other edges: min2 on an edge
                    // holding the minimum, min1 elsewhere; sign: the row's
                    // parity without the edge's own sign
                    const float m = (fabsf(x) == fabsf(r2.x)) ? fabsf(r2.y) : fabsf(r2.x);
                    const uint32_t sg = (__float_as_uint(r2.x) ^ __float_as_uint(x)) & 0x80000000u;
                    const float d = __fmul_rn(W ? __ldg(wt + e) : alpha, m);
                    v[k] = __uint_as_float(__float_as_uint(d) ^ sg);
                    ed[k] = e;
                } else {
                    v[k] = INFINITY;
                    ed[k] = -1;
                }
            }
            // ascending order of value (exchange network)
#pragma unroll
            for (int a = 0; a < DV; ++a) {
#pragma unroll
                for (int k = 0; k + 1 < DV - a; ++k) {
                    if (v[k] > v[k + 1]) {
                        const float tv = v[k]; v[k] = v[k + 1]; v[k + 1] = tv;
                        const int te = ed[k]; ed[k] = ed[k + 1]; ed[k + 1] = te;
                    }
                }
            }
            return deg;
        };
        auto flip_rows = [&](int j, int deg) {                 // s' xor H e^: the rows of column j
            if constexpr (DV <= 6) {
                // the column's slots of the padded table (a slot may be a hole)
#pragma unroll
                for (int k = 0; k < DV; ++k) {
                    const int r = __ldg(g.colER + (size_t)k * g.Npad + j).y;
                    if (r >= 0) atomicXor(&st.par[r >> 5], 1u << (r & 31));
                }
            } else {
                for (int k = 0; k < deg; ++k) {
                    const int r = __ldg(g.col_row + __ldg(g.col_ptr + j) + k);
                    atomicXor(&st.par[r >> 5], 1u << (r & 31));
                }
            }
        };

        // ---- error-node pass (Eqs. 2-4) and syndrome parity; each warp owns
        // whole 32-column words of e^ (one column per lane)
        auto column = [&](int jb) -> uint32_t {
            const int j = jb + lane;
            uint32_t ebit = 0;
            const bool act = (j < g.N) && !((st.mask[jb >> 5] >> lane) & 1u);
            if (act) {
                float v[DV];
                int ed[DV];
                const int deg = gather(j, v, ed);
                const float lj = __ldg(g.lam + j);
#pragma unroll
                for (int k = 0; k < DV; ++k) {                    // Eq. 2: leave d_i out
                    if (k < deg) {
                        float acc = lj;
#pragma unroll
                        for (int k2 = 0; k2 < DV; ++k2)
                            if (k2 != k && k2 < deg) acc = __fadd_rn(acc, v[k2]);
                        S::st(E, ed[k], fminf(fmaxf(acc, -L), L));
                    }
                }
                float post = lj;                                  // Eq. 3
#pragma unroll
                for (int k = 0; k < DV; ++k)
                    if (k < deg) post = __fadd_rn(post, v[k]);
                // a run from E(0) starts its sums here (0 + post, as a sum from zero)
                st.sumllr[j] = __fadd_rn(prior ? 0.f : st.sumllr[j], post);
                if (kPostOut && t == max_iters) post_out[j] = post;
                ebit = (post <= 0.f) ? 1u : 0u;                   // Eq. 4
                if (ebit) flip_rows(j, deg);
            }
            return ebit;
        };
        for (int jb = 32 * grp.warp(); jb < g.N; jb += 32 * grp.nwarps()) {
            const uint32_t bal = __ballot_sync(FULLMASK, column(jb));
            if (lane == 0) st.ehat[jb >> 5] = bal;
        }
        grp.sync();

        // ---- stopping rule: H e^(t) = s'
        uint32_t nz = 0;
        for (int q = grp.rank(); q < g.WM; q += grp.size()) nz |= st.par[q];
        ok = !grp.any(nz != 0u);
        iters = t;
        grp.sync();
        if (ok && stop) break;
        if (ab.key != nullptr && grp.any(grp.rank() == 0 && ab.hit(ab_key))) { ok = 0; break; }
    }
    *success = ok;
    return iters;
}

// reduction of per-thread (two smallest |sum_LLR|, node of the smallest, sum
// of q(|sum_LLR|)) over a candidate group: the smaller value wins, equal
// values go to the lower node index; every step is exact, so the result does
// not depend on the group's shape.  *tie is set when the relative margin
// between the smallest and the second smallest lies strictly inside
// (0, guard).
__device__ __forceinline__ void merge_argmin(float& best, float& second, int& bj, float ob, float os, int oj)
{
    second = fminf(fmaxf(best, ob), fminf(second, os));
    if (oj >= 0 && (bj < 0 || ob < best || (ob == best && oj < bj))) { best = ob; bj = oj; }
}

template <class G>
__device__ inline void reduce_argmin_score(const G& grp, float best, float second, int bj, unsigned long long s,
                                           double guard, int* next_pos, long long* S, int* tie)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(FULLMASK, best, o);
        const float os = __shfl_xor_sync(FULLMASK, second, o);
        const int oj = __shfl_xor_sync(FULLMASK, bj, o);
        merge_argmin(best, second, bj, ob, os, oj);
        s += __shfl_xor_sync(FULLMASK, s, o);
    }
    if constexpr (G::kBlock) {
        if ((threadIdx.x & 31) == 0) grp.rec[threadIdx.x >> 5] = ArgRec{best, second, bj, 0, s};
        __syncthreads();
        best = INFINITY; second = INFINITY; bj = -1; s = 0;
        for (int q = 0; q < grp.nwarps(); ++q) {
            const ArgRec r = grp.rec[q];
            merge_argmin(best, second, bj, r.best, r.second, r.bj);
            s += r.s;
        }
        __syncthreads();
    }
    *next_pos = bj;
    *S = (long long)s;
    int t = 0;
    if (guard > 0.0 && bj >= 0 && second != INFINITY) {
        const double den = fabs((double)second) > 1.0 ? fabs((double)second) : 1.0;
        const double gap = ((double)second - (double)best) / den;
        t = (gap > 0.0 && gap < guard) ? 1 : 0;
    }
    *tie = t;
}

// per-lane update of (smallest, second smallest, node of the smallest); nodes
// arrive in ascending order, so the lowest index keeps ties
__device__ __forceinline__ void two_smallest(float a, int j, float* best, float* second, int* bj)
{
    if (*bj < 0 || a < *best) {
        *second = *best;
        *best = a;
        *bj = j;
    } else if (a < *second) {
        *second = a;
    }
}

// least reliable unmasked node (lowest index on ties) and the score numerator
template <class G>
__device__ inline void argmin_and_score(const G& grp, const DevGraph& g, const WarpState& st, double guard,
                                        int* next_pos, long long* S, int* tie)
{
    float best = INFINITY, second = INFINITY;
    int bj = -1;
    unsigned long long s = 0;
    for (int j = grp.rank(); j < g.N; j += grp.size()) {
        if ((st.mask[j >> 5] >> (j & 31)) & 1u) continue;
        const float a = fabsf(st.sumllr[j]);
        two_smallest(a, j, &best, &second, &bj);
        s += fixq(a);
    }
    reduce_argmin_score(grp, best, second, bj, s, guard, next_pos, S, tie);
}

// ----------------------------------------------------------------------------
// BP engines: how one warp runs the iterations of one candidate
// ----------------------------------------------------------------------------
// GenericEngine: any code whose column degree is at most DV; graph tables
// are read from global memory (L1-resident) and sum_LLR lives in shared memory.
template <int DV, int P, bool W = false, class G = WarpGroup>
struct GenericEngine {
    using Grp = G;
    // blocks of up to 16 warps: for column degrees up to 6 the kernels fit in
    // 64 registers, so two such blocks stay resident on an SM; one warp per
    // candidate: 80 registers, three 8-warp blocks
    static constexpr int kMinBlocks = (DV <= 6) ? (G::kBlock ? 2 : 3) : 1;
    static constexpr int kMaxThreads = G::kBlock ? 512 : 256;
    static constexpr int kPrec = P;
    static constexpr bool kPriorStart = true;   // runs from E(0) need no copy of E(0)
    static constexpr bool kPriorSetsSums = true;  // ... nor cleared sums: their first iteration sets them
    G grp;
    __device__ void load_graph(const DevGraph&) {}
    // E(0) in this engine's message layout (the CSR edge order)
    static __device__ const void* prior_E(const DevGraph& g) { return g.lamE; }
    // the sentinel +L_MAX on every message of the newly fixed node j (at the
    // words of the padded column table for degree bounds up to 6, which may
    // have holes; at the CSR edges for the column lists)
    __device__ void fix_node(const DevGraph& g, const WarpState& st, int j, float L) const
    {
        typename Store<P>::T* const E = reinterpret_cast<typename Store<P>::T*>(st.E);
        if constexpr (DV <= 6) {
            for (int k = grp.rank(); k < DV; k += grp.size()) {
                const int e = __ldg(g.colER + (size_t)k * g.Npad + j).x;
                if (e >= 0) Store<P>::st(E, e, L);
            }
        } else {
            for (int q = __ldg(g.col_ptr + j) + grp.rank(); q < __ldg(g.col_ptr + j + 1); q += grp.size())
                Store<P>::st(E, __ldg(g.col_edge + q), L);
        }
    }
    __device__ void clear_sums(const DevGraph& g, const WarpState& st)
    {
        for (int j = grp.rank(); j < g.N; j += grp.size()) st.sumllr[j] = 0.f;
    }
    // (kAtomicStop selects the small engine's form of the stopping rule; the
    // generic engines have one form)
    template <bool kPostOut = false, bool kAtomicStop = false>
    __device__ int run(const DevGraph& g, const DecCfg& cfg, const WarpState& st, int max_iters, bool stop,
                       int* success, float* post_out, bool from_prior = false, const AbortCheck& ab = AbortCheck{})
    {
        return bp_iterate<DV, P, W, kPostOut>(grp, g, cfg, st, max_iters, stop, success, post_out, from_prior, ab);
    }
    __device__ void argmin_score(const DevGraph& g, const WarpState& st, double guard, int* np, long long* S,
                                 int* tie)
    {
        argmin_and_score(grp, g, st, guard, np, S, tie);
    }
    __device__ void write_sums(const DevGraph& g, const WarpState& st, float* dst)
    {
        for (int j = grp.rank(); j < g.N; j += grp.size()) dst[j] = st.sumllr[j];
    }
};

// SmallEngine: codes with every column of degree exactly 3, every row of
// degree exactly RD = 6, N <= 32*CPL, M <= 32*RPL and fewer than 65536 edges
// -- the bivariate bicycle codes.  A candidate's messages E and D sit at the
// words of the code's placement (bsd_layout.cu): the pair h of row i at
// h kPlane + 2 i, so the detector pass moves 32 consecutive pairs per access,
// and the error pass gathers and scatters through a per-(column, k) word
// table chosen to put the 32 lanes in 32 distinct banks.  Each lane keeps its
// columns' words, sum_LLR and mask bits in registers for the warp's lifetime.
// The stopping rule forms H e^ from the columns of H of the lane's columns
// with e^_j = 1 and three warp XOR reductions, with no shared-memory atomics
// (kAtomicStop: XOR of the set columns' rows into shared words instead, which
// the seed kernel uses: most of its runs stop after one or two iterations,
// where the reductions' latency is not hidden).  The warp's e^ words stay in
// registers and are written once, after the last iteration.
// The detector pass writes D_{i->j} itself for every edge, so the
// error-node pass gathers one 4-byte message per edge; the ascending-order
// sums of three messages are formed from min / max / median directly.  Every
// value it produces is the one GenericEngine produces (same operations, same
// order; the placement only permutes where a row's edges and a column's
// edges are kept, and neither pass depends on that order).
template <int CPL, int RPL, int RD, int P, bool W = false>
struct SmallEngine {
    using Grp = WarpGroup;
    static constexpr int kMinBlocks = 2;   // at most 128 registers: two 8-warp blocks per SM
    static constexpr int kMaxThreads = 256;
    static constexpr int kPrec = P;
    static constexpr bool kPriorStart = !W;  // unweighted runs from E(0) start from the table D0
    static constexpr bool kPriorSetsSums = false;
    WarpGroup grp;
    using S = Store<P>;
    static_assert(RD == 6, "the placement holds rows of degree 6");
    static_assert(RPL <= 3, "the per-column record holds at most three words of a column of H");
    static constexpr int kPlane = small_plane_stride_rpl(RPL);   // words between a row's pairs
    uint32_t ci[CPL][3];   // (word << 16) | row of the k-th edge of column lane + 32 c
    float sum[CPL];
    uint32_t mb;           // bit c: column lane + 32 c is masked or beyond N

    __device__ void load_graph(const DevGraph& g)
    {
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int j = lane + 32 * c;
            ci[c][0] = ci[c][1] = ci[c][2] = 0u;
            if (j < g.N) {
#pragma unroll
                for (int k = 0; k < 3; ++k) ci[c][k] = __ldg(g.scol + 3 * j + k);
            }
        }
    }
    static __device__ const void* prior_E(const DevGraph& g) { return g.slamE; }
    __device__ void fix_node(const DevGraph& g, const WarpState& st, int j, float L) const
    {
        const int lane = threadIdx.x & 31;
        if (lane < 3)
            Store<P>::st(reinterpret_cast<typename Store<P>::T*>(st.E), __ldg(g.scol + 3 * j + lane) >> 16, L);
    }
    __device__ void clear_sums(const DevGraph&, const WarpState&)
    {
#pragma unroll
        for (int c = 0; c < CPL; ++c) sum[c] = 0.f;
    }
    template <bool kPostOut = false, bool kAtomicStop = false>
    __device__ int run(const DevGraph& g, const DecCfg& cfg, const WarpState& st, int max_iters, bool stop,
                       int* success, float* post_out, bool from_prior = false, const AbortCheck& ab = AbortCheck{})
    {
        const int lane = threadIdx.x & 31;
        const float alpha = cfg.alpha;
        const float L = cfg.L;
        typename S::T* const E = reinterpret_cast<typename S::T*>(st.E);
        mb = 0u;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int j = lane + 32 * c;
            if (j >= g.N || ((st.mask[c] >> lane) & 1u)) mb |= 1u << c;
        }
        // s'_i of the lane's rows in bit 31 (s' is fixed for the whole run)
        uint32_t sb[RPL];
#pragma unroll
        for (int r = 0; r < RPL; ++r) sb[r] = (lane + 32 * r < g.M) ? ((st.sp[r] >> lane) & 1u) << 31 : 0u;
        const uint32_t spw = lane < RPL ? st.sp[lane] : 0u;
        int iters = 0;
        int ok = 0;
        uint32_t bal[CPL];     // e^ words of the last iteration (the same in every lane)
#pragma unroll
        for (int c = 0; c < CPL; ++c) bal[c] = 0u;
        for (int t = 1; t <= max_iters; ++t) {
            unsigned long long ab_key = 0ull;
            if (ab.key != nullptr && lane == 0) ab_key = *((volatile const unsigned long long*)ab.key);
            if (kAtomicStop && lane < RPL) st.par[lane] = spw;
            // weighted min-sum: row min(t, wT) - 1 of the weights in place of alpha
            const float* wt = W ? cfg.sweights + (size_t)((t < cfg.wT ? t : cfg.wT) - 1) * (size_t)g.Epad : nullptr;
            // ---- detector pass (Eq. 1); a run from E(0) takes its first check
            // messages from the table D0, flipping the sign where s_i = 1
            if (!W && from_prior && t == 1) {
#pragma unroll
                for (int r = 0; r < RPL; ++r) {
                    const int i = lane + 32 * r;
                    if (i < g.M) {
                        const uint32_t sb = ((st.sp[i >> 5] >> (i & 31)) & 1u) << 31;
#pragma unroll
                        for (int h = 0; h < RD / 2; ++h) {
                            const int wd = h * kPlane + 2 * i;
                            const float2 v = __ldg(reinterpret_cast<const float2*>(g.sD0 + wd));
                            *reinterpret_cast<float2*>(st.D + wd) =
                                make_float2(__uint_as_float(__float_as_uint(v.x) ^ sb),
                                            __uint_as_float(__float_as_uint(v.y) ^ sb));
                        }
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < ((!W && from_prior && t == 1) ? 0 : RPL); ++r) {
                const int i = lane + 32 * r;
                if (i < g.M) {
                    float x[RD];
#pragma unroll
                    for (int h = 0; h < RD / 2; ++h) {
                        const float2 x2 = S::ld2(E, h * kPlane + 2 * i);
                        x[2 * h] = x2.x;
                        x[2 * h + 1] = x2.y;
                    }
                    // the two smallest magnitudes m1 <= m2 of min(|x|, L_MAX)
                    // (R3; m2 = m1 when the minimum is attained twice): the
                    // pairs (lo, hi) of edges 2h, 2h + 1; m1 and the runner-up
                    // among the lo; m2 = min(runner-up, every hi), since a hi
                    // is never below its own lo
                    float lo[RD / 2], hi[RD / 2];
#pragma unroll
                    for (int h = 0; h < RD / 2; ++h) {
                        lo[h] = fminf(fabsf(x[2 * h]), fabsf(x[2 * h + 1]));
                        hi[h] = fmaxf(fabsf(x[2 * h]), fabsf(x[2 * h + 1]));
                    }
                    // (three pairs: t <= u the pair minima lo0, lo1 in order;
                    // the runner-up among the lo is min(u, max(t, lo2)); the
                    // caps at L_MAX folded into three-input minima)
                    const float t = fminf(lo[0], lo[1]), u = fmaxf(lo[0], lo[1]);
                    const float m1 = fmin3(t, lo[2], L);
                    const float m2 = fminf(fmin3(u, fmaxf(t, lo[2]), hi[0]), fmin3(hi[1], hi[2], L));
                    // sign parity in bit 31: a stored message is never -0 (it is
                    // a clamped sum of terms that starts at Lambda_j or the
                    // sentinel), so its sign bit is exactly x < 0
                    uint32_t nb = sb[r];
#pragma unroll
                    for (int k = 0; k < RD; ++k) nb ^= __float_as_uint(x[k]);
                    nb &= 0x80000000u;
                    // D_{i->j} for every edge of the row: alpha * (minimum over the
                    // others), which is m2 for an edge holding the minimum and m1
                    // otherwise; sign = s'_i xor parity of all signs xor the
                    // edge's own sign.  The row's part of the sign is applied to
                    // both candidates once (negating a factor negates the
                    // product exactly), the edge's own per edge.
                    const float m1s = __uint_as_float(__float_as_uint(m1) | nb);
                    const float m2s = __uint_as_float(__float_as_uint(m2) | nb);
                    const float d1 = W ? m1s : __fmul_rn(alpha, m1s), d2 = W ? m2s : __fmul_rn(alpha, m2s);
#pragma unroll
                    for (int h = 0; h < RD / 2; ++h) {
                        const int wd = h * kPlane + 2 * i;
                        float dd[2];
                        float2 w2 = make_float2(alpha, alpha);
                        if (W) w2 = __ldg(reinterpret_cast<const float2*>(wt + wd));
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int k = 2 * h + u;
                            const float sel = (fabsf(x[k]) == m1) ? d2 : d1;
                            const float d = W ? __fmul_rn(u ? w2.y : w2.x, sel) : sel;
                            dd[u] = __uint_as_float(__float_as_uint(d) ^ (__float_as_uint(x[k]) & 0x80000000u));
                        }
                        *reinterpret_cast<float2*>(st.D + wd) = make_float2(dd[0], dd[1]);
                    }
                }
            }
            __syncwarp();
            // ---- error-node pass (Eqs. 2-4); hx: the XOR of the columns of H
            // of the lane's columns with e^_j = 1, reduced over the warp into
            // H e^ after the pass (the code's M bits fill RPL words)
            uint32_t hx[RPL];
#pragma unroll
            for (int q = 0; q < RPL; ++q) hx[q] = 0u;
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                // every column is computed; a masked column or one beyond N
                // stores nothing
                const bool inr = (lane + 32 * c) < g.N;
                const bool act = !((mb >> c) & 1u);
                float v[3];
                int ed[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    ed[k] = (int)(ci[c][k] >> 16);
                    v[k] = st.D[ed[k]];
                }
                // Lambda_j and column j of H in one 16-byte record (zero past N)
                const uint4 lh = __ldg(g.slamh + lane + 32 * c);
                const float l = __uint_as_float(lh.x);
                // Eq. 2: each message leaves its own detector out; the other two
                // are added in ascending order.  Messages are stored unclamped:
                // the detector pass reads min(|E|, L_MAX) and the sign, which is
                // what a clamp at store time (R4) would leave, and |E| stays below
                // Lambda_j + 3 alpha L_MAX.  A masked column stores nothing: its
                // messages hold the sentinel +L_MAX from the moment it was fixed.
                const float e0 = __fadd_rn(__fadd_rn(l, fminf(v[1], v[2])), fmaxf(v[1], v[2]));
                const float e1 = __fadd_rn(__fadd_rn(l, fminf(v[0], v[2])), fmaxf(v[0], v[2]));
                const float e2 = __fadd_rn(__fadd_rn(l, fminf(v[0], v[1])), fmaxf(v[0], v[1]));
                if (act) {
                    S::st(E, ed[0], e0);
                    S::st(E, ed[1], e1);
                    S::st(E, ed[2], e2);
                }
                // Eq. 3 in ascending order: smallest, median, largest
                const float lo01 = fminf(v[0], v[1]), hi01 = fmaxf(v[0], v[1]);
                const float a0 = fminf(lo01, v[2]);
                const float a2 = fmaxf(hi01, v[2]);
                const float a1 = fmaxf(lo01, fminf(hi01, v[2]));
                const float post = __fadd_rn(__fadd_rn(__fadd_rn(l, a0), a1), a2);
                sum[c] = __fadd_rn(sum[c], post);           // unused for masked columns
                if (kPostOut && t == max_iters && inr) post_out[lane + 32 * c] = post;
                const uint32_t ebit = (act && post <= 0.f) ? 1u : 0u;                // Eq. 4
                if (kAtomicStop) {
                    if (ebit) {
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const int r = (int)(ci[c][k] & 0xffffu);
                            atomicXor(&st.par[r >> 5], 1u << (r & 31));
                        }
                    }
                } else {
                    // column j of H where e^_j = 1
                    const uint32_t em = 0u - ebit;
                    const uint32_t hw[3] = {lh.y, lh.z, lh.w};
#pragma unroll
                    for (int q = 0; q < RPL; ++q) hx[q] ^= hw[q] & em;
                }
                bal[c] = __ballot_sync(FULLMASK, ebit);
            }
            // stopping rule: H e^ = s' word by word (every lane gets the same
            // reductions, so the decision needs no vote)
            if (kAtomicStop) {
                __syncwarp();
                uint32_t nz = 0;
                if (lane < RPL) nz = st.par[lane];
                ok = !__any_sync(FULLMASK, nz != 0u);
            } else {
                uint32_t nz = 0u;
#pragma unroll
                for (int q = 0; q < RPL; ++q) nz |= __reduce_xor_sync(FULLMASK, hx[q]) ^ st.sp[q];
                __syncwarp();
                ok = (nz == 0u);
            }
            iters = t;
            if (ok && stop) break;
            if (ab.key != nullptr && __any_sync(FULLMASK, lane == 0 && ab.hit(ab_key))) { ok = 0; break; }
        }
        // e^ of the last iteration run
#pragma unroll
        for (int c = 0; c < CPL; ++c)
            if (lane == c && iters > 0) st.ehat[c] = bal[c];
        *success = ok;
        return iters;
    }
    __device__ void argmin_score(const DevGraph&, const WarpState&, double guard, int* np, long long* S,
                                 int* tie)
    {
        const int lane = threadIdx.x & 31;
        float best = INFINITY, second = INFINITY;
        int bj = -1;
        unsigned long long s = 0;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            if ((mb >> c) & 1u) continue;
            const float a = fabsf(sum[c]);
            two_smallest(a, lane + 32 * c, &best, &second, &bj);
            s += fixq(a);
        }
        reduce_argmin_score(grp, best, second, bj, s, guard, np, S, tie);
    }
    __device__ void write_sums(const DevGraph& g, const WarpState&, float* dst)
    {
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int c = 0; c < CPL; ++c)
            if (lane + 32 * c < g.N) dst[lane + 32 * c] = sum[c];
    }
};

// write one shot's outputs: e^, A e^, status, iteration count
// (kSparse: A e^ from the set bits of e^, for the seed kernel, where e^ is
// long and sparse)
template <class G = WarpGroup, bool kSparse = false>
__device__ void finalize_shot(const DevGraph& g, const Outputs& out, long long gb, const uint32_t* ehat,
                              uint32_t status, unsigned long long iters, const G& grp = G{})
{
    uint32_t* corr = out.corr + gb * g.WN;
    for (int q = grp.rank(); q < g.WN; q += grp.size()) corr[q] = ehat[q];
    if (out.obs != nullptr) {
        for (int wq = 0; wq < g.WK; ++wq) {
            uint32_t acc = 0;
            if constexpr (kSparse) {
                // over the set bits of e^ only (bits past N are never set)
                for (int q = grp.rank(); q < g.WN; q += grp.size()) {
                    uint32_t bits = ehat[q];
                    while (bits != 0u) {
                        const int b = __ffs(bits) - 1;
                        bits &= bits - 1u;
                        acc ^= __ldg(g.acol + (size_t)(32 * q + b) * g.WK + wq);
                    }
                }
            } else {
                for (int j = grp.rank(); j < g.N; j += grp.size())
                    if ((ehat[j >> 5] >> (j & 31)) & 1u) acc ^= __ldg(g.acol + (size_t)j * g.WK + wq);
            }
            acc = grp.xor_all(acc);
            if (grp.rank() == 0) out.obs[gb * g.WK + wq] = acc;
        }
    }
    if (grp.rank() == 0) {
        out.status[gb] = status;
        if (out.iters != nullptr) out.iters[gb] = iters > 0xffffffffull ? 0xffffffffu : (uint32_t)iters;
    }
}

// weight of a bit vector on the 2^-16 grid: sum of q(Lambda_j) over its support
__device__ inline long long vector_weight(const DevGraph& g, const uint32_t* bits)
{
    const int lane = threadIdx.x & 31;
    unsigned long long s = 0;
    for (int j = lane; j < g.N; j += 32)
        if ((bits[j >> 5] >> (j & 31)) & 1u) s += (unsigned long long)__ldg(g.lamq + j);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULLMASK, s, o);
    return (long long)s;
}

__device__ inline int* round_ctr(const Work& w, int r) { return w.round_ctr + 3 * r; }

// slot of child c of window entry a in bank `bank`
__device__ inline size_t slot_index(const Work& w, int bank, int a, int c, int W2)
{
    return ((size_t)bank * (size_t)w.A + (size_t)a) * (size_t)W2 + (size_t)c;
}

// the parent of the rank-k path of window entry a in round r: the seed-store
// entry for r = 1, else the slot of the previous round that won rank k
struct SlotRef {
    const unsigned char* E;   // snapshot, Epad messages in the storage format
    const uint32_t* bits;
    const SlotMeta* meta;
};

__device__ inline SlotRef parent_ref(const DevGraph& g, const DecCfg& cfg, const Work& w, int r, long long pbase,
                                     int a, int k)
{
    SlotRef s;
    if (r == 1) {
        const size_t e = (size_t)(pbase + a);
        s.E = w.seedE + e * snap_bytes(g);
        s.bits = w.seedBits + e * (size_t)w.SB;
        s.meta = w.seedMeta + e;
    } else {
        const size_t e = slot_index(w, (r - 1) & 1, a, w.set_idx[(size_t)a * cfg.w + k], 2 * cfg.w);
        s.E = w.slotE + e * snap_bytes(g);
        s.bits = w.slotBits + e * (size_t)w.SB;
        s.meta = w.slotMeta + e;
    }
    return s;
}

// entries of the current pass's window: [pbase, pbase + count)
__device__ inline int window(const Work& w, long long* pbase)
{
    const int pass = *((volatile int*)&w.desc->pass);
    const long long n_active = *((volatile int*)&w.ctr->n_active);
    *pbase = (long long)pass * w.A;
    long long cnt = n_active - *pbase;
    if (cnt > w.A) cnt = w.A;
    return cnt > 0 ? (int)cnt : 0;
}

// ----------------------------------------------------------------------------
// chunk set-up and pass advance (one warp each)
// ----------------------------------------------------------------------------
__device__ inline void count_launch(const Work& w)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&w.stats[2], 1ull);
}

__global__ void k_begin_chunk(Work w, int n_round_ints, const uint32_t* synd, Outputs out, long long base,
                              long long n)
{
    count_launch(w);
    for (int q = threadIdx.x; q < n_round_ints; q += blockDim.x) w.round_ctr[q] = 0;
    // early-abort keys of the window entries this chunk can use (stamps grow
    // within a chunk, so only a new chunk needs them cleared)
    const long long na = n < w.A ? n : w.A;
    for (long long q = threadIdx.x; q < na; q += blockDim.x) w.first_ok[q] = 0ull;
    if (threadIdx.x == 0) {
        w.ctr->claim_seed = 0;
        w.ctr->n_active = 0;
        w.ctr->n_queue = 0;
        w.ctr->err = 0;
        w.ctr->bs_claim = 0;
        w.ctr->bs_run = 0;
        w.ctr->bs_active_next = 0;
        w.ctr->bs_done_blocks = 0;
        w.ctr->n_fail = 0;
        RunDesc d;
        d.synd = synd;
        d.out = out;
        d.chunk_base = base;
        d.chunk_n = n;
        d.pass = 0;
        d.round = 1;
        d.win_base = 0;
        *w.desc = d;
    }
}

// after the last round of a pass: move to the next window, reset the per-pass
// counters and, under a graph, set the WHILE condition (another window left)
__global__ void k_pass_end(Work w, int n_round_ints, cudaGraphConditionalHandle cond, int use_cond)
{
    count_launch(w);
    for (int q = threadIdx.x; q < n_round_ints; q += blockDim.x) w.round_ctr[q] = 0;
    if (threadIdx.x == 0) {
        const int pass = w.desc->pass + 1;
        w.desc->pass = pass;
        w.desc->round = 1;
        if (use_cond) cudaGraphSetConditional(cond, ((long long)pass * w.A < (long long)w.ctr->n_active) ? 1u : 0u);
    }
}

// graph only, after the seed kernel: enter the loop over beam passes only if
// some shot of the chunk needs beam rounds
__global__ void k_pass_gate(Work w, cudaGraphConditionalHandle cond)
{
    count_launch(w);
    if (threadIdx.x == 0) cudaGraphSetConditional(cond, w.ctr->n_active > 0 ? 1u : 0u);
}

// graph only, at the start of a pass: the loop over rounds begins with round 1
__global__ void k_rounds_begin(Work w, cudaGraphConditionalHandle cond)
{
    count_launch(w);
    if (threadIdx.x == 0) {
        w.desc->round = 1;
        cudaGraphSetConditional(cond, 1u);
    }
}

// graph only, after the selection of round r: run round r + 1 only if it has
// children to expand (a shot with none left was finalised by the selection)
__global__ void k_round_end(Work w, int max_rounds, cudaGraphConditionalHandle cond)
{
    count_launch(w);
    if (threadIdx.x == 0) {
        const int r = w.desc->round;
        const int more = (r < max_rounds && *((volatile int*)(w.round_ctr + 3 * (r + 1) + 2)) > 0) ? 1 : 0;
        w.desc->round = r + 1;
        cudaGraphSetConditional(cond, (unsigned)more);
    }
}

// batched seed BP: the shots it hands on are decoded from the seed on in
// windows of at most S shots (the seed store); graph only: enter the loop
// over windows if there is any
__global__ void k_win_gate(Work w, cudaGraphConditionalHandle cond)
{
    count_launch(w);
    if (threadIdx.x == 0) {
        w.desc->win_base = 0;
        cudaGraphSetConditional(cond, *((volatile int*)&w.ctr->n_fail) > 0 ? 1u : 0u);
    }
}

// start of a window: the per-window counters and early-abort keys start
// afresh, as at the start of a chunk (base < 0: keep the window base)
__global__ void k_win_begin(Work w, int n_round_ints, int base)
{
    count_launch(w);
    for (int q = threadIdx.x; q < n_round_ints; q += blockDim.x) w.round_ctr[q] = 0;
    for (long long q = threadIdx.x; q < w.A; q += blockDim.x) w.first_ok[q] = 0ull;
    if (threadIdx.x == 0) {
        w.ctr->claim_seed = 0;
        w.ctr->n_active = 0;
        w.desc->pass = 0;
        w.desc->round = 1;
        if (base >= 0) w.desc->win_base = base;
    }
}

// end of a window: graph only, another window if the fail list goes on
__global__ void k_win_end(Work w, cudaGraphConditionalHandle cond)
{
    count_launch(w);
    if (threadIdx.x == 0) {
        const long long nb = (long long)w.desc->win_base + w.S;
        w.desc->win_base = (int)(nb < 0x7fffffffll ? nb : 0x7fffffffll);
        cudaGraphSetConditional(cond, nb < (long long)*((volatile int*)&w.ctr->n_fail) ? 1u : 0u);
    }
}

// ----------------------------------------------------------------------------
// first-iteration screen of the seed runs (generic engines)
// ----------------------------------------------------------------------------
// With every Lambda_j > 0, the scale alpha and one result, E(0) carries no
// negative sign, so at t = 1 a detector i with s_i = 0 sends
// D_{i->j}(1) = alpha min_{j' != j} Lambda_{j'} > 0 to every neighbour, and a
// column none of whose detectors is flipped has Lambda_j(1) > 0, e^_j(1) = 0.
// One warp per shot forms e^(1) from the columns next to flipped detectors
// (each once), by the operations and in the order of the seed BP's first
// iteration (its check messages are the create-time table D0 of E(0) with the
// syndrome sign, the values bp_iterate forms from the E(0) records; the sums
// of Eq. 3 in ascending order), and tests H e^(1) = s.  A shot
// that converges (or has s = 0) is finalised here: its seed BP would stop at
// t = 1 with this e^, and a converged seed with one result reads neither E(1)
// nor sum_LLR.  The others go to the seed BP through the queue.  The state of
// a warp is four bit vectors, so many shots are in flight per SM.
constexpr int kScreenWarps = 8;
constexpr int kMaxFlip = 128;

__host__ __device__ inline size_t screen_warp_words(const DevGraph& g)
{
    return 2 * (size_t)g.WN + 2 * (size_t)g.WM + 2 * (size_t)kMaxFlip;
}

template <int DV>
__global__ void k_screen(DevGraph g, DecCfg cfg, Work w)
{
    extern __shared__ __align__(16) uint32_t ssm[];
    const int lane = threadIdx.x & 31;
    uint32_t* seen = ssm + (size_t)(threadIdx.x >> 5) * screen_warp_words(g);
    uint32_t* eh = seen + g.WN;
    uint32_t* sp = eh + g.WN;
    uint32_t* par = sp + g.WM;
    int* fst = reinterpret_cast<int*>(par + g.WM);    // [kMaxFlip] flipped detectors, then their first edges
    int* foff = fst + kMaxFlip;                       // [kMaxFlip] their edges' offsets in the shot's list
    count_launch(w);
    const RunDesc* dp = w.desc;
    const long long n = dp->chunk_n;
    const long long nw = (long long)gridDim.x * kScreenWarps;
    unsigned long long upd = 0;                  // message updates formed (lane)
    for (long long b = (long long)blockIdx.x * kScreenWarps + (threadIdx.x >> 5); b < n; b += nw) {
        const long long gb = dp->chunk_base + b;
        const uint32_t* s = dp->synd + gb * g.WM;
        uint32_t nz = 0;
        for (int q = lane; q < g.WM; q += 32) {
            const uint32_t x = s[q];
            sp[q] = x;
            par[q] = x;
            nz |= x;
        }
        for (int q = lane; q < g.WN; q += 32) { seen[q] = 0u; eh[q] = 0u; }
        __syncwarp();
        bool conv = !__any_sync(FULLMASK, nz != 0u);
        if (!conv) {
            // the flipped detectors, in order (a shot with more than kMaxFlip
            // goes to the seed BP unscreened)
            int nflip = 0;
            for (int q0 = 0; q0 < g.WM; q0 += 32) {
                const int q = q0 + lane;
                const uint32_t word = q < g.WM ? sp[q] : 0u;
                const int c = __popc(word);
                int incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(FULLMASK, incl, o);
                    if (lane >= o) incl += y;
                }
                int k = nflip + incl - c;
                if (k + c <= kMaxFlip) {
                    for (uint32_t w2 = word; w2 != 0u; w2 &= w2 - 1u) fst[k++] = 32 * q + __ffs(w2) - 1;
                }
                nflip += __shfl_sync(FULLMASK, incl, 31);
            }
            if (nflip <= kMaxFlip) {
                __syncwarp();
                // each flipped detector's first edge and its edges' offset in
                // the shot's list of (detector, edge) pairs
                int tot = 0;
                for (int k0 = 0; k0 < nflip; k0 += 32) {
                    const int k = k0 + lane;
                    int rb = 0, d = 0;
                    if (k < nflip) {
                        const int i = fst[k];
                        rb = __ldg(g.row_ptr + i);
                        d = __ldg(g.row_ptr + i + 1) - rb;
                    }
                    int incl = d;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(FULLMASK, incl, o);
                        if (lane >= o) incl += y;
                    }
                    if (k < nflip) {
                        fst[k] = rb;
                        foff[k] = tot + incl - d;
                    }
                    tot += __shfl_sync(FULLMASK, incl, 31);
                }
                __syncwarp();
                // one (detector, edge) pair per lane: the column on the edge
                for (int t = lane; t < tot; t += 32) {
                    int lo = 0, hi = nflip - 1;                    // last detector with foff <= t
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (foff[mid] <= t) lo = mid; else hi = mid - 1;
                    }
                    const int e0 = fst[lo] + (t - foff[lo]);
                    const int j = __ldg(g.row_col + e0);
                    const uint32_t bit = 1u << (j & 31);
                    if (atomicOr(&seen[j >> 5], bit) & bit) continue;   // another flipped detector has it
                    // D_{i'->j}(1) on the column's edges: the check message of
                    // E(0) on the edge (the same for every shot: E(0) > 0 on
                    // every edge, so it is alpha times the row's minimum over the
                    // other edges, positive) with the syndrome bit of its row as
                    // the sign; two (message, row) pairs per 16-byte load, padding
                    // (+inf, -1) past the column's degree
                    constexpr int KD = DV == 3 ? 4 : DV;
                    const float4* cr = g.colRD + (size_t)j * (KD / 2);
                    float v[KD];
                    int rr[KD];
                    int deg = 0;
#pragma unroll
                    for (int h = 0; h < KD / 2; ++h) {
                        const float4 q = __ldg(cr + h);
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int r = __float_as_int(u ? q.w : q.y);
                            const float d = u ? q.z : q.x;
                            const int rs = r >= 0 ? r : 0;
                            const uint32_t si = (r >= 0) ? (sp[rs >> 5] >> (rs & 31)) & 1u : 0u;
                            v[2 * h + u] = __uint_as_float(__float_as_uint(d) ^ (si << 31));
                            rr[2 * h + u] = r;
                            deg += (r >= 0) ? 1 : 0;
                        }
                    }
#pragma unroll
                    for (int a = 0; a < KD; ++a) {
#pragma unroll
                        for (int k = 0; k + 1 < KD - a; ++k) {
                            if (v[k] > v[k + 1]) { const float tv = v[k]; v[k] = v[k + 1]; v[k + 1] = tv; }
                        }
                    }
                    float post = __ldg(g.lam + j);               // Eq. 3 in ascending order
#pragma unroll
                    for (int k = 0; k < KD; ++k)
                        if (k < deg) post = __fadd_rn(post, v[k]);
                    upd += (unsigned long long)deg;
                    if (post <= 0.f) {                            // Eq. 4
                        atomicOr(&eh[j >> 5], bit);
#pragma unroll
                        for (int k = 0; k < KD; ++k)
                            if (rr[k] >= 0) atomicXor(&par[rr[k] >> 5], 1u << (rr[k] & 31));
                    }
                }
                __syncwarp();
                nz = 0;
                for (int q = lane; q < g.WM; q += 32) nz |= par[q];
                conv = !__any_sync(FULLMASK, nz != 0u);
            }
        }
        if (conv) {
            finalize_shot<WarpGroup, true>(g, dp->out, gb, eh, ST_SEED, 1ull);
        } else if (lane == 0) {
            const int k = atomicAdd(&w.ctr->n_queue, 1);
            w.queue[k] = (int)b;
        }
        __syncwarp();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) upd += __shfl_xor_sync(FULLMASK, upd, o);
    if (lane == 0 && upd != 0ull) atomicAdd(&w.stats[3], upd);
}

// ----------------------------------------------------------------------------
// seed BP
// ----------------------------------------------------------------------------
template <class Eng>
__global__ void __launch_bounds__(Eng::kMaxThreads, Eng::kMinBlocks) k_seed(DevGraph g, DecCfg cfg, Work w,
                                                                             int screened)
{
    extern __shared__ __align__(16) char smem[];
    Eng eng;
    eng.grp = Eng::Grp::make(smem + warp_smem_bytes(g));
    const auto& grp = eng.grp;
    const WarpState st = carve(smem + (size_t)grp.index() * warp_smem_bytes(g), g);
    const RunDesc* dp = w.desc;                  // read fields when needed (keeps registers free)
    count_launch(w);
    eng.load_graph(g);
    unsigned long long seed_iters = 0;           // BP iterations (group rank 0)
    // a warp claims its shots kBatch at a time (one atomic per batch on the
    // chunk's counter, which a million one-iteration seeds would otherwise
    // hit a million times); a block candidate one at a time
    constexpr int kBatch = Eng::Grp::kBlock ? 1 : 4;
    // the shots: every shot of the chunk (screened = 0), those the screen
    // passed on (1), or those the batched seed BP passed on (2)
    const int wb = screened == 2 ? *((volatile int*)&w.desc->win_base) : 0;
    const int* list = screened == 2 ? w.fail + wb : w.queue;
    int nq = screened ? *((volatile int*)&w.ctr->n_queue) : 0;
    if (screened == 2) {
        // the current window of the fail list: at most S shots (the seed store)
        const long long left = (long long)*((volatile int*)&w.ctr->n_fail) - wb;
        nq = (int)(left < w.S ? (left > 0 ? left : 0) : w.S);
    }
    int kcur = 0, kend = 0;                      // claimed slots [kcur, kend), the same in the whole group
    for (;;) {
        if (kcur >= kend) {
            int base = 0;
            if (grp.rank() == 0) base = atomicAdd(&w.ctr->claim_seed, kBatch);
            kcur = grp.bcast(base);
            kend = kcur + kBatch;
        }
        const int k = kcur++;
        // after a screen, the shots it passed on; else every shot of the chunk
        const int b = !screened ? k : (k < nq ? list[k] : (int)dp->chunk_n);
        if (b >= dp->chunk_n) break;
        const long long gb = dp->chunk_base + b;
        const uint32_t* s = dp->synd + gb * g.WM;
        uint32_t nz = 0;
        for (int q = grp.rank(); q < g.WM; q += grp.size()) {
            const uint32_t x = s[q];
            st.sp[q] = x;
            nz |= x;
        }
        for (int q = grp.rank(); q < g.WN; q += grp.size()) { st.mask[q] = 0u; st.vals[q] = 0u; st.ehat[q] = 0u; }
        grp.sync();
        // s = 0 with every Lambda_j > 0: D > 0 at t = 1, so e^(1) = 0 and the
        // seed converges after one iteration (exact, no BP needed)
        if (!grp.any(nz != 0u) && cfg.num_results == 1 && g.all_lam_pos) {
            finalize_shot<typename Eng::Grp, true>(g, dp->out, gb, st.ehat, ST_SEED, 1ull, grp);
            grp.sync();
            continue;
        }
        if (!Eng::kPriorStart) group_copy16(grp, st.E, Eng::prior_E(g), snap_vec16(g));
        if (!Eng::kPriorSetsSums) eng.clear_sums(g, st);
        grp.sync();
        int succ = 0;
        const int it = eng.template run<false, true>(g, cfg, st, cfg.initial_iters, true, &succ, nullptr, true);
        if (grp.rank() == 0) seed_iters += (unsigned long long)it;
        grp.sync();
        if ((succ && cfg.num_results == 1) || cfg.max_rounds == 0) {
            finalize_shot<typename Eng::Grp, true>(g, dp->out, gb, st.ehat, succ ? ST_SEED : ST_FAILED,
                                                   (unsigned long long)it, grp);
            grp.sync();
            continue;
        }
        int np, tie;
        long long S;
        eng.argmin_score(g, st, cfg.tie_guard, &np, &S, &tie);
        int a = 0;
        if (grp.rank() == 0) a = atomicAdd(&w.ctr->n_active, 1);
        a = grp.bcast(a);
        // the seed path (Alg. 3): snapshot, s' = s, no fixed node, e^, next_pos
        group_copy16(grp, w.seedE + (size_t)a * snap_bytes(g), st.E, snap_vec16(g));
        uint32_t* bits = w.seedBits + (size_t)a * (size_t)w.SB;
        for (int q = grp.rank(); q < g.WM; q += grp.size()) bits[q] = st.sp[q];
        for (int q = grp.rank(); q < g.WN; q += grp.size()) {
            bits[g.WM + q] = 0u;
            bits[g.WM + g.WN + q] = 0u;
            bits[g.WM + 2 * g.WN + q] = st.ehat[q];
        }
        if (grp.rank() == 0) {
            SlotMeta m;
            m.S = 0; m.iters = it; m.next_pos = np; m.success = succ; m.flags = tie;
            w.seedMeta[a] = m;
            w.seed_shot[a] = b;
        }
        grp.sync();
    }
    if (grp.rank() == 0 && seed_iters != 0ull) atomicAdd(&w.stats[0], seed_iters);
}

// ----------------------------------------------------------------------------
// one beam round: expand every child and run masked BP (Alg. 2)
// ----------------------------------------------------------------------------
template <class Eng>
__global__ void __launch_bounds__(Eng::kMaxThreads, Eng::kMinBlocks) k_round(DevGraph g, DecCfg cfg, Work w, int r)
{
    extern __shared__ __align__(16) char smem[];
    count_launch(w);
    if (r <= 0) r = *((volatile int*)&w.desc->round);   // graph launches: the round counter
    long long pbase;
    const int cnt = window(w, &pbase);
    if (cnt == 0) return;
    const int pass = *((volatile int*)&w.desc->pass);
    Eng eng;
    eng.grp = Eng::Grp::make(smem + warp_smem_bytes(g));
    const auto& grp = eng.grp;
    const WarpState st = carve(smem + (size_t)grp.index() * warp_smem_bytes(g), g);
    const int W2 = 2 * cfg.w;
    int* rc = round_ctr(w, r);
    // round 1: two children of every window entry; later rounds: the work list
    const int nitems = (r == 1) ? 2 * cnt : *((volatile int*)(rc + 2));
    const int2* items = w.items + (size_t)(r & 1) * (size_t)w.A * (size_t)W2;
    const int cb = r & 1;
    eng.load_graph(g);
    for (;;) {
        int it = 0;
        if (grp.rank() == 0) it = atomicAdd(&rc[0], 1);
        it = grp.bcast(it);
        if (it >= nitems) break;
        const int2 item = (r == 1) ? make_int2(it >> 1, it & 1) : items[it];
        const int a = item.x, c = item.y;
        const int k = c >> 1, v = c & 1;
        const SlotRef par = parent_ref(g, cfg, w, r, pbase, a, k);
        const int pos = par.meta->next_pos;
        if (pos < 0) continue;                     // a path with no unmasked node has no children
        const size_t cslot = slot_index(w, cb, a, c, W2);
        // s' of the child: flip the detectors of pos when it is fixed to 1
        for (int q = grp.rank(); q < g.WM; q += grp.size()) {
            uint32_t x = par.bits[q];
            if (v) x ^= __ldg(g.hcol + (size_t)pos * g.WM + q);
            st.sp[q] = x;
        }
        for (int q = grp.rank(); q < g.WN; q += grp.size()) {
            uint32_t m = par.bits[g.WM + q];
            uint32_t vv = par.bits[g.WM + g.WN + q];
            if (q == (pos >> 5)) {
                m |= 1u << (pos & 31);
                if (v) vv |= 1u << (pos & 31);
            }
            st.mask[q] = m;
            st.vals[q] = vv;
        }
        // warm start from the parent's snapshot
        group_copy16(grp, st.E, par.E, snap_vec16(g));
        eng.clear_sums(g, st);
        grp.sync();
        eng.fix_node(g, st, pos, cfg.L);
        grp.sync();
        // with num_results = 1, only the first success in visit order matters:
        // a child stops once a lower-index sibling of this round has succeeded
        AbortCheck ab{};
        if (cfg.num_results == 1) {
            ab.key = w.first_ok + a;
            ab.stamp = (unsigned long long)(pass * (cfg.max_rounds + 1) + r) << 32;
            ab.c = (unsigned)c;
        }
        int succ = 0;
        const int iters = eng.run(g, cfg, st, cfg.iters_per_round, true, &succ, nullptr, false, ab);
        int superseded = 0;
        if (grp.rank() == 0) {
            atomicAdd(&w.stats[1], (unsigned long long)iters);
            if (ab.key != nullptr) {
                if (succ) atomicMax(w.first_ok + a, ab.stamp | (0xffffffffull - (unsigned)c));
                else superseded = ab.hit(*((volatile const unsigned long long*)ab.key)) ? 1 : 0;
            }
        }
        // a superseded child's slot is never read: record only that it exists
        if (grp.bcast(superseded)) {
            if (grp.rank() == 0) {
                SlotMeta m;
                m.S = 0; m.iters = iters; m.next_pos = -1; m.success = 0; m.flags = 0;
                w.slotMeta[cslot] = m;
            }
            grp.sync();
            continue;
        }
        grp.sync();
        for (int q = grp.rank(); q < g.WN; q += grp.size()) st.ehat[q] = (st.ehat[q] & ~st.mask[q]) | st.vals[q];
        grp.sync();
        int np, tie;
        long long S;
        eng.argmin_score(g, st, cfg.tie_guard, &np, &S, &tie);
        group_copy16(grp, w.slotE + cslot * snap_bytes(g), st.E, snap_vec16(g));
        uint32_t* cbits = w.slotBits + cslot * (size_t)w.SB;
        for (int q = grp.rank(); q < g.WM; q += grp.size()) cbits[q] = st.sp[q];
        for (int q = grp.rank(); q < g.WN; q += grp.size()) {
            cbits[g.WM + q] = st.mask[q];
            cbits[g.WM + g.WN + q] = st.vals[q];
            cbits[g.WM + 2 * g.WN + q] = st.ehat[q];
        }
        if (grp.rank() == 0) {
            SlotMeta m;
            m.S = S; m.iters = iters; m.next_pos = np; m.success = succ; m.flags = tie;
            w.slotMeta[cslot] = m;
        }
        grp.sync();
    }
}

// ----------------------------------------------------------------------------
// per-shot selection after round r
// ----------------------------------------------------------------------------
struct SelScratch {
    double score[2 * kMaxBeam];
    int iters[2 * kMaxBeam];
    int flags[2 * kMaxBeam];     // bit0 exists, bit1 success, bit2 argmin near-tie
};

__device__ void finalize_results(const DevGraph& g, const DecCfg& cfg, const Work& w, const Outputs& out,
                                 int a, long long gb, unsigned long long total, uint32_t extra)
{
    const int n = w.res_n[a];
    const long long* rw = w.res_w + (size_t)a * cfg.num_results;
    int bi = 0;
    for (int q = 1; q < n; ++q)
        if (rw[q] < rw[bi]) bi = q;
    const uint32_t st = (w.res_origin[(size_t)a * cfg.num_results + bi] == 0) ? ST_SEED : ST_BEAM;
    finalize_shot(g, out, gb, w.res_bits + ((size_t)a * cfg.num_results + bi) * g.WN, st | extra, total);
}

__global__ void __launch_bounds__(256) k_select(DevGraph g, DecCfg cfg, Work w, int r)
{
    extern __shared__ __align__(16) char smem[];
    count_launch(w);
    if (r <= 0) r = *((volatile int*)&w.desc->round);   // graph launches: the round counter
    long long pbase;
    const int cnt = window(w, &pbase);
    if (cnt == 0) return;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    SelScratch* sc = reinterpret_cast<SelScratch*>(smem) + wid;
    const int W2 = 2 * cfg.w;
    const RunDesc d = *w.desc;
    int* rc = round_ctr(w, r);
    const int cb = r & 1;
    int acur = 0, aend = 0;                      // window entries claimed four at a time
    for (;;) {
        if (acur >= aend) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&rc[1], 4);
            acur = __shfl_sync(FULLMASK, base, 0);
            aend = acur + 4;
        }
        const int a = acur++;
        if (a >= cnt) break;
        if (r == 1) {
            // a new window entry: the seed path is its only path (Alg. 3)
            const size_t e = (size_t)(pbase + a);
            const SlotMeta sm = w.seedMeta[e];
            if (sm.success) {                  // num_results > 1: the seed result opens `results`
                const uint32_t* eb = w.seedBits + e * (size_t)w.SB + g.WM + 2 * g.WN;
                uint32_t* rb = w.res_bits + (size_t)a * cfg.num_results * g.WN;
                for (int q = lane; q < g.WN; q += 32) rb[q] = eb[q];
                const long long W = vector_weight(g, eb);
                if (lane == 0) {
                    w.res_w[(size_t)a * cfg.num_results] = W;
                    w.res_origin[(size_t)a * cfg.num_results] = 0;
                }
            }
            if (lane == 0) {
                w.shot_of[a] = w.seed_shot[e];
                w.set_size[a] = 1;
                w.iters_acc[a] = (unsigned long long)sm.iters;
                w.done[a] = 0;
                w.res_n[a] = sm.success ? 1 : 0;
                w.near[a] = sm.flags & 1;      // the seed path branches on its argmin
            }
            __syncwarp();
        } else if (w.done[a]) {
            continue;
        }
        const long long gb = d.chunk_base + w.shot_of[a];
        const int npar = w.set_size[a];
        const int nch = 2 * npar;
        // gather the children of this round in canonical order c = 2 * rank + val
        for (int c = lane; c < nch; c += 32) {
            const int pnp = parent_ref(g, cfg, w, r, pbase, a, c >> 1).meta->next_pos;
            int fl = 0, it = 0;
            double scv = 0.0;
            if (pnp >= 0) {
                const SlotMeta m = w.slotMeta[slot_index(w, cb, a, c, W2)];
                fl = 1 | (m.success ? 2 : 0) | ((m.flags & 1) << 2);
                it = m.iters;
                scv = ((double)m.S / kFixScale) / (double)m.iters;
            }
            sc->flags[c] = fl;
            sc->iters[c] = it;
            sc->score[c] = scv;
        }
        __syncwarp();
        unsigned long long acc = w.iters_acc[a];
        bool done = false;
        // near-tie record: argmin margins of the children the sequential
        // algorithm visits, and the pruning margin of the round
        int near = w.near[a];
        auto near_upto = [&](int last) {
            int f = 0;
            for (int c = lane; c <= last && c < nch; c += 32) f |= (sc->flags[c] >> 2) & 1;
            return __any_sync(FULLMASK, f != 0) ? 1 : 0;
        };
        if (cfg.num_results == 1) {
            // Alg. 3: the first successful child in visit order ends the search
            int first = 0x7fffffff;
            for (int c = lane; c < nch; c += 32)
                if ((sc->flags[c] & 3) == 3 && c < first) first = c;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) first = min(first, __shfl_xor_sync(FULLMASK, first, o));
            if (first != 0x7fffffff) {
                unsigned long long sum = 0;
                for (int c = lane; c <= first; c += 32)
                    if (sc->flags[c] & 1) sum += (unsigned long long)sc->iters[c];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(FULLMASK, sum, o);
                const uint32_t* eb = w.slotBits + slot_index(w, cb, a, first, W2) * (size_t)w.SB + g.WM + 2 * g.WN;
                near |= near_upto(first);
                finalize_shot(g, d.out, gb, eb, ST_BEAM | (near ? ST_NEAR : 0u), acc + sum);
                done = true;
            }
        } else {
            // results collection in visit order (dedupe by equality, App. B)
            unsigned long long sum = 0;
            for (int c = 0; c < nch && !done; ++c) {
                const int fl = sc->flags[c];
                if (!(fl & 1)) continue;
                sum += (unsigned long long)sc->iters[c];
                if (!(fl & 2)) continue;
                const uint32_t* eb = w.slotBits + slot_index(w, cb, a, c, W2) * (size_t)w.SB + g.WM + 2 * g.WN;
                const int nres = w.res_n[a];
                bool dup = false;
                for (int q = 0; q < nres && !dup; ++q) {
                    const uint32_t* rb = w.res_bits + ((size_t)a * cfg.num_results + q) * g.WN;
                    bool eq = true;
                    for (int x = lane; x < g.WN; x += 32) eq = eq && (rb[x] == eb[x]);
                    dup = __all_sync(FULLMASK, eq);
                }
                if (!dup) {
                    uint32_t* rb = w.res_bits + ((size_t)a * cfg.num_results + nres) * g.WN;
                    for (int x = lane; x < g.WN; x += 32) rb[x] = eb[x];
                    const long long W = vector_weight(g, eb);
                    __syncwarp();
                    if (lane == 0) {
                        w.res_w[(size_t)a * cfg.num_results + nres] = W;
                        w.res_origin[(size_t)a * cfg.num_results + nres] = 1;
                        w.res_n[a] = nres + 1;
                    }
                    __syncwarp();
                    if (nres + 1 >= cfg.num_results) {
                        near |= near_upto(c);
                        finalize_results(g, cfg, w, d.out, a, gb, acc + sum, near ? ST_NEAR : 0u);
                        done = true;
                    }
                }
            }
        }
        if (!done) {
            unsigned long long sum = 0;
            int nex = 0;
            for (int c = lane; c < nch; c += 32) {
                if (sc->flags[c] & 1) { sum += (unsigned long long)sc->iters[c]; ++nex; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sum += __shfl_xor_sync(FULLMASK, sum, o);
                nex += __shfl_xor_sync(FULLMASK, nex, o);
            }
            acc += sum;
            near |= near_upto(nch - 1);
            // rank of each existing child under (score desc, canonical index asc)
            int myrank[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = lane + 32 * q;
                myrank[q] = -1;
                if (c < nch && (sc->flags[c] & 1)) {
                    const double s0 = sc->score[c];
                    int rk = 0;
                    for (int c2 = 0; c2 < nch; ++c2) {
                        if (!(sc->flags[c2] & 1)) continue;
                        const double s2 = sc->score[c2];
                        rk += (s2 > s0 || (s2 == s0 && c2 < c)) ? 1 : 0;
                    }
                    myrank[q] = rk;
                }
            }
            // the kept paths of a round before the last, and how many of them
            // have a node left to branch on (their children make round r + 1)
            const bool last = (r >= cfg.max_rounds || nex == 0);
            int keep = 0, tot = 0;
            if (!last) {
                __syncwarp();
                keep = nex < cfg.w ? nex : cfg.w;
                if (cfg.tie_guard > 0.0 && nex > keep) {
                    // pruning margin: last kept (rank keep-1) against first dropped (rank keep)
                    double s_in = -INFINITY, s_out = -INFINITY;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (myrank[q] == keep - 1) s_in = sc->score[lane + 32 * q];
                        if (myrank[q] == keep) s_out = sc->score[lane + 32 * q];
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        s_in = fmax(s_in, __shfl_xor_sync(FULLMASK, s_in, o));
                        s_out = fmax(s_out, __shfl_xor_sync(FULLMASK, s_out, o));
                    }
                    const double den = fabs(s_in) > 1.0 ? fabs(s_in) : 1.0;
                    const double gap = (s_in - s_out) / den;
                    if (gap > 0.0 && gap < cfg.tie_guard) near = 1;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (myrank[q] >= 0 && myrank[q] < keep)
                        w.set_idx[(size_t)a * cfg.w + myrank[q]] = (uint8_t)(lane + 32 * q);
                __syncwarp();
                int cntp = 0;
                for (int k = lane; k < keep; k += 32) {
                    const int c = w.set_idx[(size_t)a * cfg.w + k];
                    cntp += (w.slotMeta[slot_index(w, cb, a, c, W2)].next_pos >= 0) ? 1 : 0;
                }
                tot = cntp;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(FULLMASK, tot, o);
            }
            if (last || tot == 0) {
                // the search ends here: the last round, no child, or no kept
                // path with a node left (the next round would have no child)
                if (cfg.num_results > 1 && w.res_n[a] > 0) {
                    finalize_results(g, cfg, w, d.out, a, gb, acc, near ? ST_NEAR : 0u);
                } else {
                    // no valid solution: the best path of the final set
                    int best = 0x7fffffff;
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (myrank[q] == 0) best = lane + 32 * q;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(FULLMASK, best, o));
                    const uint32_t* eb;
                    if (best != 0x7fffffff)
                        eb = w.slotBits + slot_index(w, cb, a, best, W2) * (size_t)w.SB + g.WM + 2 * g.WN;
                    else
                        eb = parent_ref(g, cfg, w, r, pbase, a, 0).bits + g.WM + 2 * g.WN;
                    finalize_shot(g, d.out, gb, eb, ST_FAILED | (near ? ST_NEAR : 0u), acc);
                }
                done = true;
            } else {
                // the kept slots become the next round's parents: two children per
                // kept path that has a next_pos
                int wbase = 0;
                if (lane == 0) {
                    w.set_size[a] = keep;
                    w.iters_acc[a] = acc;
                    w.near[a] = near;
                    wbase = atomicAdd(&round_ctr(w, r + 1)[2], 2 * tot);
                }
                wbase = __shfl_sync(FULLMASK, wbase, 0);
                if (lane == 0) {
                    int2* items = w.items + (size_t)((r + 1) & 1) * (size_t)w.A * (size_t)W2;
                    int o = 0;
                    for (int k = 0; k < keep; ++k) {
                        const int c = w.set_idx[(size_t)a * cfg.w + k];
                        if (w.slotMeta[slot_index(w, cb, a, c, W2)].next_pos >= 0) {
                            items[wbase + o] = make_int2(a, 2 * k);
                            items[wbase + o + 1] = make_int2(a, 2 * k + 1);
                            o += 2;
                        }
                    }
                }
            }
        }
        if (done && lane == 0) w.done[a] = 1;
        __syncwarp();
    }
}

// ----------------------------------------------------------------------------
// plain BP for a fixed number of iterations (LLR measurement)
// ----------------------------------------------------------------------------
template <class Eng>
__global__ void __launch_bounds__(Eng::kMaxThreads, Eng::kMinBlocks) k_bp_llr(DevGraph g, DecCfg cfg,
                                                                           const uint32_t* __restrict__ synd,
                                                                           long long B, int T, float* llr,
                                                                           float* sum_llr)
{
    extern __shared__ __align__(16) char smem[];
    Eng eng;
    eng.grp = Eng::Grp::make(smem + warp_smem_bytes(g));
    const auto& grp = eng.grp;
    const WarpState st = carve(smem + (size_t)grp.index() * warp_smem_bytes(g), g);
    eng.load_graph(g);
    const long long nw = (long long)gridDim.x * grp.per_block();
    for (long long b = (long long)blockIdx.x * grp.per_block() + grp.index(); b < B; b += nw) {
        for (int q = grp.rank(); q < g.WM; q += grp.size()) st.sp[q] = synd[b * g.WM + q];
        for (int q = grp.rank(); q < g.WN; q += grp.size()) { st.mask[q] = 0u; st.vals[q] = 0u; }
        if (!Eng::kPriorStart) group_copy16(grp, st.E, Eng::prior_E(g), snap_vec16(g));
        if (!Eng::kPriorSetsSums) eng.clear_sums(g, st);
        grp.sync();
        int succ;
        eng.template run<true>(g, cfg, st, T, false, &succ, llr + b * g.N, true);
        grp.sync();
        if (sum_llr != nullptr) eng.write_sums(g, st, sum_llr + b * g.N);
        grp.sync();
    }
}

// ----------------------------------------------------------------------------
// host-side launch helpers
// ----------------------------------------------------------------------------
// engine id = 3 * kind + storage precision, or 15 + kind for weighted min-sum;
// kinds: 0..2 generic with column degree bound 3 / 6 / 16, 3: small (CPL 3,
// RPL 2, row degree 6), 4: small (CPL 5, RPL 3, row degree 6); precision 0
// float, 1 binary16, 2 bfloat16
#define BSD_KIND_ALIASES(P, SFX)                          \
    using Generic3##SFX = GenericEngine<3, P>;            \
    using Generic6##SFX = GenericEngine<6, P>;            \
    using Generic16##SFX = GenericEngine<16, P>;          \
    using Small326##SFX = SmallEngine<3, 2, 6, P>;        \
    using Small536##SFX = SmallEngine<5, 3, 6, P>;
BSD_KIND_ALIASES(0, _f32)
BSD_KIND_ALIASES(1, _f16)
BSD_KIND_ALIASES(2, _bf16)
// weighted min-sum (per-edge, per-iteration weights), single-precision messages: id 15 + kind
using Generic3_w = GenericEngine<3, 0, true>;
using Generic6_w = GenericEngine<6, 0, true>;
using Generic16_w = GenericEngine<16, 0, true>;
using Small326_w = SmallEngine<3, 2, 6, 0, true>;
using Small536_w = SmallEngine<5, 3, 6, 0, true>;
constexpr int kWeightedEngine = 15;
// a block of warps per candidate (generic engines only): id 20 + 4 * kind + (0 float, 1 binary16,
// 2 bfloat16, 3 weighted float)
#define BSD_BLOCK_ALIASES(DV)                                                   \
    using Block##DV##_f32 = GenericEngine<DV, 0, false, BlockGroup>;            \
    using Block##DV##_f16 = GenericEngine<DV, 1, false, BlockGroup>;            \
    using Block##DV##_bf16 = GenericEngine<DV, 2, false, BlockGroup>;           \
    using Block##DV##_w = GenericEngine<DV, 0, true, BlockGroup>;
BSD_BLOCK_ALIASES(3)
BSD_BLOCK_ALIASES(6)
BSD_BLOCK_ALIASES(16)
constexpr int kBlockEngine = 20;
#define BSD_ENGINES(X)                                                                          \
    X(0, Generic3_f32) X(1, Generic3_f16) X(2, Generic3_bf16)                                   \
    X(3, Generic6_f32) X(4, Generic6_f16) X(5, Generic6_bf16)                                   \
    X(6, Generic16_f32) X(7, Generic16_f16) X(8, Generic16_bf16)                                \
    X(9, Small326_f32) X(10, Small326_f16) X(11, Small326_bf16)                                 \
    X(12, Small536_f32) X(13, Small536_f16) X(14, Small536_bf16)                                \
    X(15, Generic3_w) X(16, Generic6_w) X(17, Generic16_w) X(18, Small326_w) X(19, Small536_w)  \
    X(20, Block3_f32) X(21, Block3_f16) X(22, Block3_bf16) X(23, Block3_w)                      \
    X(24, Block6_f32) X(25, Block6_f16) X(26, Block6_bf16) X(27, Block6_w)                      \
    X(28, Block16_f32) X(29, Block16_f16) X(30, Block16_bf16) X(31, Block16_w)

template <class Eng>
static int set_attrs(size_t smem_bp)
{
    if (CUDA_FAILED(cudaFuncSetAttribute(k_seed<Eng>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bp)) ||
        CUDA_FAILED(cudaFuncSetAttribute(k_round<Eng>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bp)) ||
        CUDA_FAILED(cudaFuncSetAttribute(k_bp_llr<Eng>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bp)))
        return -2;
    return 0;
}

template <class Eng>
static int occupancy(int threads, size_t smem_bp, int* bps)
{
    int a = 0, b = 0;
    if (CUDA_FAILED(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_round<Eng>, threads, smem_bp))) return -2;
    if (CUDA_FAILED(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_seed<Eng>, threads, smem_bp))) return -2;
    *bps = a < b ? a : b;
    return 0;
}

// can the small engine run this code? (column degree 3, row degree 6, with
// the placement of its messages built)
static bool small_fits(const DevGraph& g, int cpl, int rpl)
{
    if (g.scol == nullptr) return false;
    if (g.max_col_deg != 3 || g.max_row_deg != 6 || g.E != 3 * g.N || g.E != 6 * g.M) return false;
    if (g.E >= 65536 || g.M >= 65536) return false;
    return g.WN == cpl && (g.M + 31) / 32 == rpl;
}

int configure_kernels(DevGraph& g, const DecCfg& cfg, int device, int group_warps, int warps_per_block,
                      LaunchShape* ls)
{
    if (cfg.weights != nullptr && g.prec != 0) return -5;   // weights: single-precision messages only
    if (group_warps < 0 || group_warps > 16 || warps_per_block < 0 || warps_per_block > 8) return -5;
    int gkind;                                               // generic kind: column degree bound 3 / 6 / 16
    if (g.max_col_deg <= 3) gkind = 0;
    else if (g.max_col_deg <= 6) gkind = 1;
    else if (g.max_col_deg <= 16) gkind = 2;
    else return -5;
    if (gkind < 2 && g.colK != (gkind == 0 ? 3 : 6)) return -5;   // the column table matches the engine
    int skind = -1;                                          // small engine kind, if the code has its layout
    if (small_fits(g, 3, 2)) skind = 3;
    else if (small_fits(g, 5, 3)) skind = 4;
    int max_optin = 0, sms = 0;
    if (CUDA_FAILED(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device)) ||
        CUDA_FAILED(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)))
        return -2;
    // per-candidate state with the generic engine's detector records
    g.det_bytes = (int)align16(sizeof(float2) * (size_t)g.M);
    const size_t generic_bytes = warp_smem_bytes(g);
    // automatic choice: the small engine where it fits; otherwise a warp per
    // candidate while eight or more candidates fit on an SM, a block of 8
    // warps per candidate beyond
    int gw = group_warps;
    if (gw == 0) gw = (skind >= 0 || generic_bytes * 8 <= (size_t)max_optin) ? 1 : 8;
    const bool weighted = cfg.weights != nullptr;
    int eng, wpb;
    if (gw >= 2) {
        eng = kBlockEngine + 4 * gkind + (weighted ? 3 : g.prec);
        wpb = gw;
    } else {
        const int kind = skind >= 0 ? skind : gkind;
        eng = weighted ? kWeightedEngine + kind : 3 * kind + g.prec;
        // the small engine keeps D per edge in float; the generic one a record per detector
        const size_t recs = sizeof(float2) * (size_t)g.M, msgs = sizeof(float) * (size_t)g.Epad;
        g.det_bytes = (int)align16(kind >= 3 && msgs > recs ? msgs : recs);
        const size_t per_warp = warp_smem_bytes(g);
        if (per_warp > (size_t)max_optin) return -5;
        wpb = warps_per_block > 0 ? warps_per_block : (int)((96 * 1024) / per_warp);
        if (wpb > 8) wpb = 8;
        if (wpb < 1) wpb = 1;
        if (per_warp * (size_t)wpb > (size_t)max_optin) return -5;
    }
    const size_t per_cand = warp_smem_bytes(g);
    ls->group_warps = gw >= 2 ? gw : 1;
    ls->warps_per_block = wpb;
    ls->smem_bp = gw >= 2 ? per_cand + 16 * sizeof(ArgRec) : per_cand * (size_t)wpb;
    if (ls->smem_bp > (size_t)max_optin) return -5;
    // the selection kernel handles one shot per warp in blocks of at most 8 warps
    ls->select_warps = wpb < 8 ? wpb : 8;
    ls->smem_select = sizeof(SelScratch) * (size_t)ls->select_warps;
    ls->dv = eng;
    const int threads = 32 * wpb;
    int rc = 0, bps_bp = 0, bps_sel = 0;
    // The dynamic shared-memory limit is a property of the kernel, shared by
    // every decoder that launches it; it is raised to the device maximum so
    // that no decoder created later can lower it below what an earlier one
    // launches with (a CUDA graph keeps the value it was instantiated with,
    // a direct launch checks the current one).
    switch (eng) {
#define X(id, E)                                                                \
    case id:                                                                    \
        rc = set_attrs<E>((size_t)max_optin);                       \
        if (!rc) rc = occupancy<E>(threads, ls->smem_bp, &bps_bp);  \
        break;
        BSD_ENGINES(X)
#undef X
        default: return -5;
    }
    if (rc) return rc;
    if (CUDA_FAILED(cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin)) ||
        CUDA_FAILED(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps_sel, k_select, 32 * ls->select_warps,
                                                                  ls->smem_select)))
        return -2;
    if (bps_bp < 1 || bps_sel < 1) return -5;
    // the first-iteration screen: generic engines, the scale alpha, every
    // Lambda_j > 0, one result
    ls->screen = 0;
    ls->grid_screen = 0;
    ls->smem_screen = sizeof(uint32_t) * screen_warp_words(g) * kScreenWarps;
    if (eng < 9 || eng >= kBlockEngine) {                   // not a small engine
        if (!weighted && g.all_lam_pos && cfg.num_results == 1 && ls->smem_screen <= (size_t)max_optin) {
            void* kf = gkind == 0 ? (void*)k_screen<3> : gkind == 1 ? (void*)k_screen<6> : (void*)k_screen<16>;
            int bps_scr = 0;
            // a screen warp's state is a few KB of bit sets and lists: prefer the
            // shared-memory carveout that lets the register file, not the
            // carveout, bound the resident blocks
            if (CUDA_FAILED(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin)) ||
                CUDA_FAILED(cudaFuncSetAttribute(kf, cudaFuncAttributePreferredSharedMemoryCarveout,
                                                 cudaSharedmemCarveoutMaxShared)) ||
                CUDA_FAILED(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps_scr, kf, 32 * kScreenWarps,
                                                                          ls->smem_screen)))
                return -2;
            if (bps_scr >= 1) {
                ls->screen = 1;
                ls->grid_screen = sms * bps_scr;
                ls->dv_screen = gkind;
            }
        }
    }
    ls->grid_seed = sms * bps_bp;
    ls->grid_round = sms * bps_bp;
    ls->grid_select = sms * bps_sel;
    // the batched seed BP: generic engines with the scale alpha and one result
    // (the shots it finishes need no snapshot; the others are decoded again by
    // the per-candidate seed kernel)
    ls->batch = (eng < 9 || eng >= kBlockEngine) && !weighted && cfg.num_results == 1 ? 1 : 0;
    ls->grid_bs = batch_grid(device);
    return 0;
}

static void* screen_func(const LaunchShape& ls)
{
    return ls.dv_screen == 0 ? (void*)k_screen<3> : ls.dv_screen == 1 ? (void*)k_screen<6> : (void*)k_screen<16>;
}

static void launch_screen(const DevGraph& g, const DecCfg& cfg, const Work& w, const LaunchShape& ls, cudaStream_t s)
{
    const dim3 grid((unsigned)ls.grid_screen), block(32 * kScreenWarps);
    if (ls.dv_screen == 0) k_screen<3><<<grid, block, ls.smem_screen, s>>>(g, cfg, w);
    else if (ls.dv_screen == 1) k_screen<6><<<grid, block, ls.smem_screen, s>>>(g, cfg, w);
    else k_screen<16><<<grid, block, ls.smem_screen, s>>>(g, cfg, w);
}

template <class Eng>
static int launch_chunk_t(const DevGraph& g, const DecCfg& cfg, const Work& w, const LaunchShape& ls,
                          const uint32_t* synd, long long base, long long n, const Outputs& out, cudaStream_t s,
                          const LaunchHooks* hk, cudaGraphExec_t gx, int* host_n_active)
{
    const int threads = 32 * ls.warps_per_block;
    const int nri = 3 * (cfg.max_rounds + 2);
    k_begin_chunk<<<1, 128, 0, s>>>(w, nri, synd, out, base, n);
    if (CUDA_FAILED(cudaGetLastError())) return -2;
    if (gx != nullptr) return !CUDA_FAILED(cudaGraphLaunch(gx, s)) ? 0 : -2;
    if (ls.screen) {
        if (hk) hk->before(hk->ctx, 11);
        launch_screen(g, cfg, w, ls, s);
        if (hk) hk->after(hk->ctx, 11);
    }
    // the seed kernel on its shots, then exactly the beam passes they need
    // (without a graph the number of active entries is read back)
    auto seed_and_passes = [&](int seed_src) -> int {
        if (hk) hk->before(hk->ctx, 0);
        k_seed<Eng><<<ls.grid_seed, threads, ls.smem_bp, s>>>(g, cfg, w, seed_src);
        if (hk) hk->after(hk->ctx, 0);
        if (CUDA_FAILED(cudaGetLastError())) return -2;
        if (cfg.max_rounds == 0) return 0;
        if (CUDA_FAILED(cudaMemcpyAsync(host_n_active, &w.ctr->n_active, sizeof(int), cudaMemcpyDeviceToHost, s)) ||
            CUDA_FAILED(cudaStreamSynchronize(s)))
            return -2;
        const long long passes = (*host_n_active + w.A - 1) / w.A;
        for (long long p = 0; p < passes; ++p) {
            for (int r = 1; r <= cfg.max_rounds; ++r) {
                if (hk) hk->before(hk->ctx, 1);
                k_round<Eng><<<ls.grid_round, threads, ls.smem_bp, s>>>(g, cfg, w, r);
                if (hk) { hk->after(hk->ctx, 1); hk->before(hk->ctx, 2); }
                k_select<<<ls.grid_select, 32 * ls.select_warps, ls.smem_select, s>>>(g, cfg, w, r);
                if (hk) hk->after(hk->ctx, 2);
            }
            k_pass_end<<<1, 128, 0, s>>>(w, nri, cudaGraphConditionalHandle{}, 0);
            if (CUDA_FAILED(cudaGetLastError())) return -2;
        }
        return 0;
    };
    if (!(ls.batch && w.bs_slots > 0)) return seed_and_passes(ls.screen);
    // batched seed BP over the chunk, then the shots it handed on in windows
    // of at most S (the seed store)
    if (launch_batch_direct(g, cfg, w, ls, ls.screen, s, hk, host_n_active)) return -2;
    if (CUDA_FAILED(cudaMemcpyAsync(host_n_active, &w.ctr->n_fail, sizeof(int), cudaMemcpyDeviceToHost, s)) ||
        CUDA_FAILED(cudaStreamSynchronize(s)))
        return -2;
    const long long n_fail = *host_n_active;
    for (long long wb = 0; wb < n_fail; wb += w.S) {
        k_win_begin<<<1, 128, 0, s>>>(w, nri, (int)wb);
        if (CUDA_FAILED(cudaGetLastError())) return -2;
        const int rc = seed_and_passes(2);
        if (rc) return rc;
    }
    return 0;
}

int launch_chunk(const DevGraph& g, const DecCfg& cfg, const Work& w, const LaunchShape& ls, const uint32_t* synd,
                 long long base, long long n, const Outputs& out, void* stream, const LaunchHooks* hooks,
                 void* graph_exec, int* host_n_active)
{
    cudaStream_t s = (cudaStream_t)stream;
    cudaGraphExec_t gx = (cudaGraphExec_t)graph_exec;
    switch (ls.dv) {
#define X(id, E) \
    case id: return launch_chunk_t<E>(g, cfg, w, ls, synd, base, n, out, s, hooks, gx, host_n_active);
        BSD_ENGINES(X)
#undef X
        default: return -5;
    }
}

// ---- the per-chunk graph: k_seed, then WHILE(another window) { rounds, k_pass_end }
static int add_kernel(cudaGraph_t graph, cudaGraphNode_t* node, const cudaGraphNode_t* dep, void* func, int grid,
                      int block, size_t smem, void** args)
{
    cudaKernelNodeParams p{};
    p.func = func;
    p.gridDim = dim3((unsigned)grid);
    p.blockDim = dim3((unsigned)block);
    p.sharedMemBytes = (unsigned)smem;
    p.kernelParams = args;
    return !CUDA_FAILED(cudaGraphAddKernelNode(node, graph, dep, dep ? 1 : 0, &p)) ? 0 : -2;
}

// WHILE (a window of active shots left) { round 1, WHILE (the next round has
// children) { round r, selection, round end }, pass end }, after `dep` in
// `graph`: a chunk runs exactly the passes and rounds it needs
template <class Eng>
static int add_beam_nodes(cudaGraph_t graph, cudaGraphNode_t dep, cudaGraphNode_t* last, DevGraph& g, DecCfg& cfg,
                          Work& w, const LaunchShape& ls)
{
    const int threads = 32 * ls.warps_per_block;
    int nri = 3 * (cfg.max_rounds + 2);
    int rc = 0;
    cudaGraphConditionalHandle cpass, cround;
    cudaGraphNode_t gate, wpass, rbegin, wround, pend;
    cudaGraphNodeParams cp{};
    if (CUDA_FAILED(cudaGraphConditionalHandleCreate(&cpass, graph, 0, cudaGraphCondAssignDefault))) rc = -2;
    if (!rc) {
        void* gargs[] = {&w, &cpass};
        rc = add_kernel(graph, &gate, &dep, (void*)k_pass_gate, 1, 32, 0, gargs);
    }
    if (!rc) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cpass;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        if (CUDA_FAILED(cudaGraphAddNode(&wpass, graph, &gate, nullptr, 1, &cp))) rc = -2;
    }
    cudaGraph_t body = rc ? nullptr : cp.conditional.phGraph_out[0];
    if (!rc && CUDA_FAILED(cudaGraphConditionalHandleCreate(&cround, body, 0, 0))) rc = -2;
    if (!rc) {
        void* bargs[] = {&w, &cround};
        rc = add_kernel(body, &rbegin, nullptr, (void*)k_rounds_begin, 1, 32, 0, bargs);
    }
    cudaGraphNodeParams cr{};
    if (!rc) {
        cr.type = cudaGraphNodeTypeConditional;
        cr.conditional.handle = cround;
        cr.conditional.type = cudaGraphCondTypeWhile;
        cr.conditional.size = 1;
        if (CUDA_FAILED(cudaGraphAddNode(&wround, body, &rbegin, nullptr, 1, &cr))) rc = -2;
    }
    if (!rc) {
        // kernel parameters are copied when a node is added; round 0 means
        // "read the round counter"
        cudaGraph_t rbody = cr.conditional.phGraph_out[0];
        cudaGraphNode_t nr, ns, ne;
        int r0 = 0, maxr = cfg.max_rounds;
        void* rargs[] = {&g, &cfg, &w, &r0};
        rc = add_kernel(rbody, &nr, nullptr, (void*)k_round<Eng>, ls.grid_round, threads, ls.smem_bp, rargs);
        if (!rc) rc = add_kernel(rbody, &ns, &nr, (void*)k_select, ls.grid_select, 32 * ls.select_warps,
                                    ls.smem_select, rargs);
        void* eargs[] = {&w, &maxr, &cround};
        if (!rc) rc = add_kernel(rbody, &ne, &ns, (void*)k_round_end, 1, 32, 0, eargs);
    }
    if (!rc) {
        int use = 1;
        void* pargs[] = {&w, &nri, &cpass, &use};
        rc = add_kernel(body, &pend, &wround, (void*)k_pass_end, 1, 128, 0, pargs);
    }
    if (!rc) *last = wpass;
    return rc;
}

template <class Eng>
static int build_graph_t(const DevGraph& g0, const DecCfg& cfg0, const Work& w0, const LaunchShape& ls,
                         cudaGraphExec_t* out)
{
    DevGraph g = g0;
    DecCfg cfg = cfg0;
    Work w = w0;
    const int threads = 32 * ls.warps_per_block;
    int nri = 3 * (cfg.max_rounds + 2);
    cudaGraph_t graph = nullptr;
    if (CUDA_FAILED(cudaGraphCreate(&graph, 0))) return -2;
    int rc = 0;
    cudaGraphNode_t seed, scr, last;
    const bool batched = ls.batch && w.bs_slots > 0;
    int screened = batched ? 2 : ls.screen;
    void* sargs[] = {&g, &cfg, &w, &screened};
    void* cargs[] = {&g, &cfg, &w};
    if (ls.screen)
        rc = add_kernel(graph, &scr, nullptr, screen_func(ls), ls.grid_screen, 32 * kScreenWarps, ls.smem_screen,
                        cargs);
    if (!batched) {
        // seed, then the beam passes
        if (!rc)
            rc = add_kernel(graph, &seed, ls.screen ? &scr : nullptr, (void*)k_seed<Eng>, ls.grid_seed, threads,
                            ls.smem_bp, sargs);
        if (!rc && cfg.max_rounds > 0) rc = add_beam_nodes<Eng>(graph, seed, &last, g, cfg, w, ls);
    } else {
        // the batched seed BP over the chunk, then WHILE (shots handed on
        // remain) { window start, the seed kernel on at most S of them, the
        // beam passes, window end }
        cudaGraphNode_t bs, wgate, wwin;
        cudaGraphConditionalHandle cwin;
        if (!rc) rc = add_batch_nodes(graph, ls.screen ? scr : nullptr, &bs, g, cfg, w, ls, ls.screen);
        if (!rc && CUDA_FAILED(cudaGraphConditionalHandleCreate(&cwin, graph, 0, cudaGraphCondAssignDefault)))
            rc = -2;
        if (!rc) {
            void* gargs[] = {&w, &cwin};
            rc = add_kernel(graph, &wgate, &bs, (void*)k_win_gate, 1, 32, 0, gargs);
        }
        cudaGraphNodeParams cp{};
        if (!rc) {
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = cwin;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            if (CUDA_FAILED(cudaGraphAddNode(&wwin, graph, &wgate, nullptr, 1, &cp))) rc = -2;
        }
        if (!rc) {
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            cudaGraphNode_t wbeg, wend;
            int keep = -1;
            void* bargs[] = {&w, &nri, &keep};
            rc = add_kernel(body, &wbeg, nullptr, (void*)k_win_begin, 1, 128, 0, bargs);
            if (!rc)
                rc = add_kernel(body, &seed, &wbeg, (void*)k_seed<Eng>, ls.grid_seed, threads, ls.smem_bp, sargs);
            cudaGraphNode_t tail = seed;
            if (!rc && cfg.max_rounds > 0) rc = add_beam_nodes<Eng>(body, seed, &tail, g, cfg, w, ls);
            void* eargs[] = {&w, &cwin};
            if (!rc) rc = add_kernel(body, &wend, &tail, (void*)k_win_end, 1, 32, 0, eargs);
        }
    }
    cudaGraphExec_t gx = nullptr;
    if (!rc && CUDA_FAILED(cudaGraphInstantiate(&gx, graph, 0))) rc = -2;
    cudaGraphDestroy(graph);
    if (rc) {
        cudaGetLastError();
        return rc;
    }
    *out = gx;
    return 0;
}

int build_graph(const DevGraph& g, const DecCfg& cfg, const Work& w, const LaunchShape& ls, void** graph_exec)
{
    cudaGraphExec_t gx = nullptr;
    int rc;
    switch (ls.dv) {
#define X(id, E) \
    case id: rc = build_graph_t<E>(g, cfg, w, ls, &gx); break;
        BSD_ENGINES(X)
#undef X
        default: rc = -5;
    }
    *graph_exec = rc ? nullptr : (void*)gx;
    return rc;
}

void destroy_graph(void* graph_exec)
{
    if (graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)graph_exec);
}

// ---- workspace layout
static inline size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

size_t work_head_bytes(const DecCfg& cfg)
{
    return a256(sizeof(Counters) + sizeof(int) * 3 * (size_t)(cfg.max_rounds + 2)) + a256(sizeof(RunDesc)) +
           a256(kStats * sizeof(unsigned long long));
}

size_t work_layout(const DevGraph& g, const DecCfg& cfg, long long S, long long A, char* base, Work* w,
                   int bs_slots, long long S1)
{
    if (bs_slots <= 0 || S1 < S) S1 = S;
    const size_t W2 = 2 * (size_t)cfg.w;
    const size_t SB = (size_t)g.WM + 3 * (size_t)g.WN;
    const size_t NR = (size_t)cfg.num_results;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = base ? base + off : nullptr;
        off += a256(bytes > 0 ? bytes : 1);
        return p;
    };
    char* ctr = take(sizeof(Counters) + sizeof(int) * 3 * (size_t)(cfg.max_rounds + 2));
    char* desc = take(sizeof(RunDesc));
    char* stats = take(kStats * sizeof(unsigned long long));
    Work v{};
    v.S = S;
    v.S1 = S1;
    v.A = A;
    v.SB = (int)SB;
    v.ctr = reinterpret_cast<Counters*>(ctr);
    v.round_ctr = ctr ? reinterpret_cast<int*>(ctr + sizeof(Counters)) : nullptr;
    v.desc = reinterpret_cast<RunDesc*>(desc);
    v.stats = reinterpret_cast<unsigned long long*>(stats);
    v.seedE = (unsigned char*)take((size_t)S * snap_bytes(g));
    v.seedBits = (uint32_t*)take(sizeof(uint32_t) * (size_t)S * SB);
    v.seedMeta = (SlotMeta*)take(sizeof(SlotMeta) * (size_t)S);
    v.seed_shot = (int*)take(sizeof(int) * (size_t)S);
    v.queue = (int*)take(sizeof(int) * (size_t)S1);
    v.slotE = (unsigned char*)take(2 * (size_t)A * W2 * snap_bytes(g));
    v.slotBits = (uint32_t*)take(sizeof(uint32_t) * 2 * (size_t)A * W2 * SB);
    v.slotMeta = (SlotMeta*)take(sizeof(SlotMeta) * 2 * (size_t)A * W2);
    v.shot_of = (int*)take(sizeof(int) * (size_t)A);
    v.set_size = (int*)take(sizeof(int) * (size_t)A);
    v.done = (int*)take(sizeof(int) * (size_t)A);
    v.set_idx = (uint8_t*)take((size_t)A * (size_t)cfg.w);
    v.iters_acc = (unsigned long long*)take(sizeof(unsigned long long) * (size_t)A);
    v.res_bits = (uint32_t*)take(sizeof(uint32_t) * (size_t)A * NR * (size_t)g.WN);
    v.res_w = (long long*)take(sizeof(long long) * (size_t)A * NR);
    v.res_origin = (int*)take(sizeof(int) * (size_t)A * NR);
    v.res_n = (int*)take(sizeof(int) * (size_t)A);
    v.first_ok = (unsigned long long*)take(sizeof(unsigned long long) * (size_t)A);
    v.near = (int*)take(sizeof(int) * (size_t)A);
    v.items = (int2*)take(sizeof(int2) * 2 * (size_t)A * W2);
    // the batched seed BP's slots and the shots it passes on
    v.bs_slots = bs_slots;
    if (bs_slots > 0) {
        const size_t Bs = (size_t)bs_slots;
        v.bsE = (unsigned char*)take(Bs * (size_t)g.Epad * (size_t)g.msg_bytes);
        v.bsR = (float2*)take(sizeof(float2) * Bs * (size_t)g.M);
        v.bs_shot = (int*)take(sizeof(int) * Bs);
        v.bs_t = (int*)take(sizeof(int) * Bs);
        v.bs_nl = (int*)take(sizeof(int) * Bs);
        v.bs_list = (int*)take(sizeof(int) * Bs * (size_t)kBsList);
        v.fail = (int*)take(sizeof(int) * (size_t)S1);
    }
    if (w) *w = v;
    return off;
}

template <class Eng>
static void launch_llr_t(const DevGraph& g, const DecCfg& cfg, const LaunchShape& ls, const uint32_t* synd,
                         long long B, int T, float* llr, float* sum_llr, cudaStream_t s, int blocks)
{
    k_bp_llr<Eng><<<blocks, 32 * ls.warps_per_block, ls.smem_bp, s>>>(g, cfg, synd, B, T, llr, sum_llr);
}

// ----------------------------------------------------------------------------
// request loop for single syndromes (low-latency mode): one candidate group
// stays resident and answers requests posted in host-mapped memory, so a
// syndrome whose seed BP ends the search (Alg. 3: the first BP run converges,
// with one result) costs no launch and no host-side stream wait
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_acquire_sys(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_sys(uint32_t* p, uint32_t v)
{
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The loop answers a request (ServeBox::req != the last answered number) by
// the seed BP of its syndrome -- the same engine, operations and order as
// k_seed, so the outputs are identical -- and writes e^, A e^, status and
// iterations, or status 0 when the beam search must decide (the host then
// takes the regular path).  Every wait is bounded: the loop leaves when the
// host sets ServeBox::stop or when no request comes for idle_ns.
template <class Eng>
__global__ void __launch_bounds__(Eng::kMaxThreads, Eng::kMinBlocks) k_serve(DevGraph g, DecCfg cfg, ServeBox* box,
                                                                           uint32_t last, unsigned long long idle_ns)
{
    extern __shared__ __align__(16) char smem[];
    Eng eng;
    eng.grp = Eng::Grp::make(smem + warp_smem_bytes(g));
    const auto& grp = eng.grp;
    const WarpState st = carve(smem, g);
    eng.load_graph(g);
    volatile uint32_t* const synd = reinterpret_cast<volatile uint32_t*>(box + 1);
    uint32_t* const obuf = reinterpret_cast<uint32_t*>(box + 1) + g.WM;
    const Outputs out{obuf, g.K > 0 ? obuf + g.WN : nullptr, &box->status, &box->iters};
    if (grp.rank() == 0) st_release_sys(&box->state, 1u);
    for (;;) {
        int what = 0;                             // 1 request, 2 stop, 3 idle
        if (grp.rank() == 0) {
            const unsigned long long t0 = global_ns();
            for (;;) {
                if (ld_acquire_sys(&box->stop) != 0u) { what = 2; break; }
                const uint32_t r = ld_acquire_sys(&box->req);
                if (r != last) { last = r; what = 1; break; }
                if (global_ns() - t0 > idle_ns) { what = 3; break; }
                __nanosleep(32);                  // each poll crosses to host memory
            }
        }
        what = grp.bcast(what);
        if (what != 1) {
            if (grp.rank() == 0) st_release_sys(&box->state, what == 2 ? 3u : 2u);
            return;
        }
        uint32_t nz = 0;
        for (int q = grp.rank(); q < g.WM; q += grp.size()) {
            const uint32_t x = synd[q];
            st.sp[q] = x;
            nz |= x;
        }
        for (int q = grp.rank(); q < g.WN; q += grp.size()) { st.mask[q] = 0u; st.vals[q] = 0u; st.ehat[q] = 0u; }
        grp.sync();
        if (!grp.any(nz != 0u) && cfg.num_results == 1 && g.all_lam_pos) {
            // s = 0 with every Lambda_j > 0: the seed converges at t = 1 with e^ = 0
            finalize_shot<typename Eng::Grp, true>(g, out, 0, st.ehat, ST_SEED, 1ull, grp);
        } else {
            if (!Eng::kPriorStart) group_copy16(grp, st.E, Eng::prior_E(g), snap_vec16(g));
            if (!Eng::kPriorSetsSums) eng.clear_sums(g, st);
            grp.sync();
            int succ = 0;
            const int it = eng.run(g, cfg, st, cfg.initial_iters, true, &succ, nullptr, true);
            grp.sync();
            if ((succ && cfg.num_results == 1) || cfg.max_rounds == 0)
                finalize_shot<typename Eng::Grp, true>(g, out, 0, st.ehat, succ ? ST_SEED : ST_FAILED,
                                                       (unsigned long long)it, grp);
            else if (grp.rank() == 0)
                box->status = 0u;
        }
        __threadfence_system();
        grp.sync();
        if (grp.rank() == 0) st_release_sys(&box->done, last);
    }
}

template <class Eng>
static int launch_serve_t(const DevGraph& g, const DecCfg& cfg, const LaunchShape& ls, ServeBox* box,
                          uint32_t last, unsigned long long idle_ns, cudaStream_t s)
{
    const bool block = ls.group_warps >= 2;
    const size_t smem = block ? ls.smem_bp : warp_smem_bytes(g);
    if (CUDA_FAILED(cudaFuncSetAttribute(k_serve<Eng>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return -2;
    k_serve<Eng><<<1, 32 * (block ? ls.group_warps : 1), smem, s>>>(g, cfg, box, last, idle_ns);
    return CUDA_FAILED(cudaGetLastError()) ? -2 : 0;
}

int launch_serve(const DevGraph& g, const DecCfg& cfg, const LaunchShape& ls, ServeBox* box, uint32_t last,
                 unsigned long long idle_ns, void* stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    switch (ls.dv) {
#define X(id, E) \
    case id: return launch_serve_t<E>(g, cfg, ls, box, last, idle_ns, s);
        BSD_ENGINES(X)
#undef X
        default: return -5;
    }
}

int launch_bp_llr(const DevGraph& g, const DecCfg& cfg, const LaunchShape& ls, const uint32_t* synd, long long B,
                  int T, float* llr, float* sum_llr, void* stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    long long blocks = (B + ls.warps_per_block - 1) / ls.warps_per_block;
    if (blocks > ls.grid_round) blocks = ls.grid_round;
    if (blocks < 1) blocks = 1;
    switch (ls.dv) {
#define X(id, E) \
    case id: launch_llr_t<E>(g, cfg, ls, synd, B, T, llr, sum_llr, s, (int)blocks); break;
        BSD_ENGINES(X)
#undef X
        default: return -5;
    }
    return CUDA_FAILED(cudaGetLastError()) ? -2 : 0;
}

}  // namespace bsd

// ----------------------------------------------------------------------------
// single-precision re-runs of near-tie shots (16-bit messages)
// ----------------------------------------------------------------------------
namespace bsd {

__global__ void k_collect_flagged(const uint32_t* __restrict__ status, long long B, long long* list, int* count)
{
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < B; b += (long long)gridDim.x * blockDim.x)
        if (status[b] & ST_NEAR) list[atomicAdd(count, 1)] = b;
}

__global__ void k_gather_rows(const uint32_t* __restrict__ src, const long long* __restrict__ list, int n, int W,
                              uint32_t* __restrict__ dst)
{
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < (long long)n * W;
         k += (long long)gridDim.x * blockDim.x) {
        const long long i = k / W, q = k % W;
        dst[k] = src[list[i] * W + q];
    }
}

__global__ void k_scatter_results(const long long* __restrict__ list, int n, int WN, int WK, Outputs from, Outputs to)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long b = list[i];
        for (int q = 0; q < WN; ++q) to.corr[b * WN + q] = from.corr[i * WN + q];
        if (to.obs != nullptr)
            for (int q = 0; q < WK; ++q) to.obs[b * WK + q] = from.obs[i * WK + q];
        to.status[b] = from.status[i] | ST_NEAR | ST_RERUN;
        if (to.iters != nullptr) to.iters[b] = from.iters[i];
    }
}

int launch_collect_flagged(const uint32_t* status, long long B, long long* list, int* count, void* stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (CUDA_FAILED(cudaMemsetAsync(count, 0, sizeof(int), s))) return -2;
    long long blocks = (B + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_collect_flagged<<<(int)(blocks > 0 ? blocks : 1), 256, 0, s>>>(status, B, list, count);
    return CUDA_FAILED(cudaGetLastError()) ? -2 : 0;
}

int launch_gather_rows(const uint32_t* src, const long long* list, int n, int W, uint32_t* dst, void* stream)
{
    long long blocks = ((long long)n * W + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_gather_rows<<<(int)(blocks > 0 ? blocks : 1), 256, 0, (cudaStream_t)stream>>>(src, list, n, W, dst);
    return CUDA_FAILED(cudaGetLastError()) ? -2 : 0;
}

int launch_scatter_results(const long long* list, int n, int WN, int WK, const Outputs& from, const Outputs& to,
                           void* stream)
{
    long long blocks = ((long long)n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_scatter_results<<<(int)(blocks > 0 ? blocks : 1), 256, 0, (cudaStream_t)stream>>>(list, n, WN, WK, from, to);
    return CUDA_FAILED(cudaGetLastError()) ? -2 : 0;
}

}  // namespace bsd
