// bsd_batch.cu -- the seed BP of many shots at once, messages streamed
// through HBM with the shots contiguous.
//
// The seed BP of a shot (Alg. 3, first BP run: Eqs. 1-4 from E(0) = Lambda
// with the stopping rule) reads the same graph for every shot.  Here Bs slots
// each hold one shot and every pass walks the graph once for all of them: the
// messages live in [Epad][Bs] (edge e of slot b at e * Bs + b), so the 32
// threads of a warp -- 32 slots of one row or one column -- read and write 32
// consecutive messages, and every graph table entry is one broadcast load for
// the whole warp.  Per iteration:
//   k_bs_check   per (row i, slot): the two smallest magnitudes of the row's
//                messages (capped at L_MAX) and the parity of their signs with
//                s_i, written as the record (min1, min2) with the parity in
//                both sign bits (Eq. 1 before the per-edge selection);
//   k_bs_var     per (column j, slot): D_{i->j} from the record and the edge's
//                own message (min2 where |E_{j->i}| = min1, else min1; the
//                parity without the edge's own sign; times alpha), then
//                Eqs. 2-3 in ascending order and Eq. 4; a column with
//                e^_j(t) = 1 is added to the slot's list;
//   k_bs_retire  per slot: H e^(t) = s from the listed columns (a stopping
//                test needs only the few ones of e^); a converged shot gets
//                its outputs, a shot at initial_iters without convergence (or
//                with more ones than the list holds) goes to the list of shots
//                the per-candidate seed kernel decodes again from scratch
//                (its snapshot and sum_LLR feed the beam); a finished slot
//                takes the next queued shot.
// A slot's first iteration reads the precomputed records of E(0) and E(0)
// itself from the graph tables, as the per-candidate engines do.  Every
// operation is the one the per-candidate generic engine performs on the same
// values in the same order (minimum with the lowest-index rule replaced by the
// equivalent magnitude test, since a tie for the minimum makes min2 = min1),
// so outputs and iteration counts are bit-identical.  Messages are stored
// clamped to [-L_MAX, L_MAX] in the decoder's storage format.
#include "bsd_device.cuh"
#include "bsd_internal.cuh"

namespace bsd {

namespace {

__device__ __forceinline__ bool batch_running(const Work& w)
{
    return *((volatile const int*)&w.ctr->bs_run) != 0;
}

// the slots of a block and the contiguous range of items (rows or columns) it covers
struct BsRange {
    int b;            // this thread's slot
    int lo, hi;       // items [lo, hi)
};

// the error-node pass gives each thread two adjacent slots (b, b + 1): one
// 8-byte (FP32) or 4-byte (16-bit) load moves the message of an edge for
// both, one 16-byte load their detector records, and the graph-table loads
// serve both (more bytes in flight per instruction for a pass that waits on
// memory); the check pass keeps one slot per thread (more warps in flight)
constexpr int kBsThreads = kBsChunk / 2;
// messages of a row the check pass loads before it reduces them
constexpr int kBsRowBatch = 8;

template <int SPT>
__device__ __forceinline__ BsRange bs_range(const Work& w, int items)
{
    const int nch = w.bs_slots / kBsChunk;
    const int groups = (gridDim.x + nch - 1) / nch;      // item groups
    const int c = blockIdx.x % nch, grp = blockIdx.x / nch;
    const int per = (items + groups - 1) / groups;
    BsRange r;
    r.b = c * kBsChunk + SPT * threadIdx.x;
    r.lo = grp * per;
    r.hi = min(items, r.lo + per);
    return r;
}

}  // namespace

// fill the slots with the first queued shots (every shot of the chunk when no
// screen ran) and open the loop
__global__ void k_bs_begin(Work w, int screened, cudaGraphConditionalHandle cond, int use_cond)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&w.stats[2], 1ull);
    const long long chunk_n = w.desc->chunk_n;
    const int nq = screened ? *((volatile int*)&w.ctr->n_queue) : (int)chunk_n;
    const int Bs = w.bs_slots;
    for (int b = threadIdx.x; b < Bs; b += blockDim.x) {
        w.bs_shot[b] = b < nq ? (screened ? w.queue[b] : b) : -1;
        w.bs_t[b] = 0;
        w.bs_nl[b] = 0;
    }
    if (threadIdx.x == 0) {
        const int n0 = nq < Bs ? nq : Bs;
        w.ctr->bs_claim = n0;
        w.ctr->bs_run = n0 > 0 ? 1 : 0;
        w.ctr->bs_active_next = 0;
        w.ctr->bs_done_blocks = 0;
        w.ctr->n_fail = 0;
        if (use_cond) cudaGraphSetConditional(cond, n0 > 0 ? 1u : 0u);
    }
}

// Eq. 1, first half: the record of every (row, slot)
template <int P>
__global__ void __launch_bounds__(kBsChunk) k_bs_check(DevGraph g, DecCfg cfg, Work w)
{
    if (!batch_running(w)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&w.stats[2], 1ull);
    using S = Store<P>;
    using T = typename S::T;
    const BsRange rg = bs_range<1>(w, g.M);
    const int b = rg.b;
    const int Bs = w.bs_slots;
    const int shot = w.bs_shot[b];
    if (shot < 0) return;
    const bool fresh = w.bs_t[b] == 0;
    const uint32_t* s = w.desc->synd + (w.desc->chunk_base + shot) * (long long)g.WM;
    const T* E = reinterpret_cast<const T*>(w.bsE);
    const float L = cfg.L;
    uint32_t sw = 0;
    int sq = -1;
    for (int i = rg.lo; i < rg.hi; ++i) {
        if ((i >> 5) != sq) { sq = i >> 5; sw = __ldg(s + sq); }
        uint32_t nb = (sw >> (i & 31)) & 1u;
        float m1, m2;
        if (fresh) {
            const float4 r = __ldg(g.rs0 + i);
            m1 = r.x;
            m2 = r.y;
            nb ^= __float_as_uint(r.w) & 1u;
        } else {
            // branch-free running pair of smallest magnitudes, capped at L_MAX
            // (R3), eight messages in flight per thread: past the row's end a
            // lane takes +L_MAX, which changes neither minimum nor the parity
            m1 = L;
            m2 = L;
            const int rb = __ldg(g.row_ptr + i), re = __ldg(g.row_ptr + i + 1);
            const T* Eb = E + b;
            uint32_t sg = 0u;
            for (int e = rb; e < re; e += kBsRowBatch) {
                float x[kBsRowBatch];
#pragma unroll
                for (int u = 0; u < kBsRowBatch; ++u)
                    x[u] = (e + u < re) ? S::ld(Eb, (size_t)(e + u) * Bs) : L;
#pragma unroll
                for (int u = 0; u < kBsRowBatch; ++u) {
                    const float a = fabsf(x[u]);
                    m2 = fminf(m2, fmaxf(m1, a));
                    m1 = fminf(m1, a);
                    sg ^= __float_as_uint(x[u]);
                }
            }
            // a stored message is never -0 (a clamped sum that starts at
            // Lambda_j), so its sign bit is exactly x < 0
            nb ^= sg >> 31;
        }
        const uint32_t sb = nb << 31;
        w.bsR[(size_t)i * Bs + b] = make_float2(__uint_as_float(__float_as_uint(m1) | sb),
                                                __uint_as_float(__float_as_uint(m2) | sb));
    }
}

// Eq. 1 per edge, Eqs. 2-4 per (column, slot), for a run of columns of
// degree D (positions [q0, q1) of the degree-sorted column order) and the
// thread's two slots; every lane of a warp holds the same column, so the
// degree is warp-uniform.  The next column's (edge, row) pairs are loaded
// while the current one is computed.  A slot without a shot computes values
// no one reads and lists nothing.
template <int D, int P>
__device__ __forceinline__ void bs_var_run(const DevGraph& g, const DecCfg& cfg, const Work& w, int b, bool act0,
                                           bool act1, bool fresh0, bool fresh1, int q0, int q1)
{
    using S = Store<P>;
    using T = typename S::T;
    T* const E = reinterpret_cast<T*>(w.bsE);
    const size_t Bs = (size_t)w.bs_slots;
    const float alpha = cfg.alpha, L = cfg.L;
    const int2* seq = g.colseq + g.dbase[D] + (size_t)(q0 - g.dstart[D]) * D;
    int2 er[D > 0 ? D : 1], nx[D > 0 ? D : 1];
#pragma unroll
    for (int k = 0; k < D; ++k) er[k] = __ldg(seq + k);
    for (int q = q0; q < q1; ++q) {
        seq += D;
        if (q + 1 < q1) {
#pragma unroll
            for (int k = 0; k < D; ++k) nx[k] = __ldg(seq + k);
        }
        const int j = __ldg(g.colperm + q);
        const float lj = __ldg(g.lam + j);
        // E(0) of a fresh slot: the same on every edge of the column
        const float x0 = (fresh0 || fresh1) ? S::ld(reinterpret_cast<const T*>(g.lamEc), j) : 0.f;
        float v0[D > 0 ? D : 1], v1[D > 0 ? D : 1];
        int e0[D > 0 ? D : 1], e1[D > 0 ? D : 1];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const float4 rec = *reinterpret_cast<const float4*>(w.bsR + (size_t)er[k].y * Bs + b);
            float2 xo = S::ld2(E, (size_t)er[k].x * Bs + b);
            if (fresh0) xo.x = x0;
            if (fresh1) xo.y = x0;
            // the minimum over the row's other edges: min2 on an edge holding
            // the minimum (a tie makes min2 = min1), min1 elsewhere; sign: the
            // row's parity (in the record) without the edge's own sign
            const float m0 = (fabsf(xo.x) == fabsf(rec.x)) ? rec.y : rec.x;
            const float m1 = (fabsf(xo.y) == fabsf(rec.z)) ? rec.w : rec.z;
            const float d0 = __fmul_rn(alpha, m0), d1 = __fmul_rn(alpha, m1);
            v0[k] = __uint_as_float(__float_as_uint(d0) ^ (__float_as_uint(xo.x) & 0x80000000u));
            v1[k] = __uint_as_float(__float_as_uint(d1) ^ (__float_as_uint(xo.y) & 0x80000000u));
            e0[k] = er[k].x;
            e1[k] = er[k].x;
        }
        // ascending order of value (an exchange network of D inputs per slot)
#pragma unroll
        for (int a = 0; a < D; ++a) {
#pragma unroll
            for (int k = 0; k + 1 < D - a; ++k) {
                if (v0[k] > v0[k + 1]) {
                    const float tv = v0[k]; v0[k] = v0[k + 1]; v0[k + 1] = tv;
                    const int te = e0[k]; e0[k] = e0[k + 1]; e0[k + 1] = te;
                }
                if (v1[k] > v1[k + 1]) {
                    const float tv = v1[k]; v1[k] = v1[k + 1]; v1[k + 1] = tv;
                    const int te = e1[k]; e1[k] = e1[k + 1]; e1[k + 1] = te;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {                         // Eq. 2: leave d_i out
            float acc0 = lj, acc1 = lj;
#pragma unroll
            for (int k2 = 0; k2 < D; ++k2) {
                if (k2 != k) {
                    acc0 = __fadd_rn(acc0, v0[k2]);
                    acc1 = __fadd_rn(acc1, v1[k2]);
                }
            }
            S::st(E, (size_t)e0[k] * Bs + b, fminf(fmaxf(acc0, -L), L));
            S::st(E, (size_t)e1[k] * Bs + b + 1, fminf(fmaxf(acc1, -L), L));
        }
        float p0 = lj, p1 = lj;                               // Eq. 3
#pragma unroll
        for (int k = 0; k < D; ++k) {
            p0 = __fadd_rn(p0, v0[k]);
            p1 = __fadd_rn(p1, v1[k]);
        }
        if (act0 && p0 <= 0.f) {                              // Eq. 4
            const int qn = atomicAdd(&w.bs_nl[b], 1);
            if (qn < kBsList) w.bs_list[(size_t)qn * Bs + b] = j;
        }
        if (act1 && p1 <= 0.f) {
            const int qn = atomicAdd(&w.bs_nl[b + 1], 1);
            if (qn < kBsList) w.bs_list[(size_t)qn * Bs + b + 1] = j;
        }
#pragma unroll
        for (int k = 0; k < D; ++k) er[k] = nx[k];
    }
}

template <int DV, int P>
__global__ void __launch_bounds__(kBsThreads) k_bs_var(DevGraph g, DecCfg cfg, Work w)
{
    if (!batch_running(w)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&w.stats[2], 1ull);
    const BsRange rg = bs_range<2>(w, g.N);
    const int b = rg.b;
    const int2 shot = *reinterpret_cast<const int2*>(w.bs_shot + b);
    if (shot.x < 0 && shot.y < 0) return;
    const int2 tt = *reinterpret_cast<const int2*>(w.bs_t + b);
    const bool act0 = shot.x >= 0, act1 = shot.y >= 0;
    const bool fresh0 = tt.x == 0, fresh1 = tt.y == 0;
    // the block's positions of the degree-sorted order, run by run of one degree
#define BS_RUN(DD)                                                                  \
    if constexpr (DD <= DV) {                                                       \
        const int q0 = max(rg.lo, g.dstart[DD]), q1 = min(rg.hi, g.dstart[DD + 1]); \
        if (q0 < q1) bs_var_run<DD, P>(g, cfg, w, b, act0, act1, fresh0, fresh1, q0, q1); \
    }
    BS_RUN(0) BS_RUN(1) BS_RUN(2) BS_RUN(3) BS_RUN(4) BS_RUN(5) BS_RUN(6) BS_RUN(7) BS_RUN(8)
    BS_RUN(9) BS_RUN(10) BS_RUN(11) BS_RUN(12) BS_RUN(13) BS_RUN(14) BS_RUN(15) BS_RUN(16)
#undef BS_RUN
}

// stopping rule, outputs of converged shots, hand-off of the others, refill
__global__ void __launch_bounds__(256) k_bs_retire(DevGraph g, DecCfg cfg, Work w, int screened,
                                                  cudaGraphConditionalHandle cond, int use_cond)
{
    if (!batch_running(w)) {
        // (the loop flag and the graph's condition are always set together;
        // should they ever disagree, the loop still ends here)
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&w.stats[2], 1ull);
    __shared__ int s_last;
    const int lane = threadIdx.x & 31;
    const int Bs = w.bs_slots;
    const RunDesc* dp = w.desc;
    const long long chunk_n = dp->chunk_n;
    const int nq = screened ? *((volatile int*)&w.ctr->n_queue) : (int)chunk_n;
    unsigned long long ran = 0;                   // slot-iterations of this launch (lane 0 of each warp)
    int active = 0;                               // slots holding a shot for the next iteration
    for (int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < Bs; b += gridDim.x * (blockDim.x >> 5)) {
        const int shot = w.bs_shot[b];
        if (shot < 0) continue;
        const int t = w.bs_t[b] + 1;
        const int n = w.bs_nl[b];
        ++ran;
        const long long gb = dp->chunk_base + shot;
        const uint32_t* s = dp->synd + gb * (long long)g.WM;
        bool conv = false;
        if (n <= kBsList) {
            // H e^(t) xor s from the listed columns
            uint32_t nz = 0;
            for (int q = lane; q < g.WM; q += 32) {
                uint32_t acc = __ldg(s + q);
                for (int k = 0; k < n; ++k) acc ^= __ldg(g.hcol + (size_t)w.bs_list[(size_t)k * Bs + b] * g.WM + q);
                nz |= acc;
            }
            conv = !__any_sync(FULLMASK, nz != 0u);
        }
        bool done = true;
        if (conv) {
            // outputs: e^ from the listed columns, A e^, status, iterations
            uint32_t* corr = dp->out.corr + gb * g.WN;
            for (int q = lane; q < g.WN; q += 32) {
                uint32_t word = 0;
                for (int k = 0; k < n; ++k) {
                    const int j = w.bs_list[(size_t)k * Bs + b];
                    if ((j >> 5) == q) word |= 1u << (j & 31);
                }
                corr[q] = word;
            }
            if (dp->out.obs != nullptr) {
                for (int wq = 0; wq < g.WK; ++wq) {
                    uint32_t acc = 0;
                    for (int k = lane; k < n; k += 32)
                        acc ^= __ldg(g.acol + (size_t)w.bs_list[(size_t)k * Bs + b] * g.WK + wq);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_xor_sync(FULLMASK, acc, o);
                    if (lane == 0) dp->out.obs[gb * g.WK + wq] = acc;
                }
            }
            if (lane == 0) {
                dp->out.status[gb] = ST_SEED;
                if (dp->out.iters != nullptr) dp->out.iters[gb] = (uint32_t)t;
            }
        } else if (n > kBsList || t >= cfg.initial_iters) {
            // the seed BP fails (or e^ has more ones than the list holds): the
            // per-candidate seed kernel decodes the shot again from E(0)
            if (lane == 0) w.fail[atomicAdd(&w.ctr->n_fail, 1)] = shot;
        } else {
            done = false;
        }
        __syncwarp();
        if (lane == 0) {
            int next = shot, tn = t;
            if (done) {
                const int k = atomicAdd(&w.ctr->bs_claim, 1);
                next = k < nq ? (screened ? w.queue[k] : k) : -1;
                tn = 0;
            }
            w.bs_shot[b] = next;
            w.bs_t[b] = tn;
            w.bs_nl[b] = 0;
            active += next >= 0 ? 1 : 0;
        }
    }
    if (lane == 0 && ran != 0ull) {
        atomicAdd(&w.stats[0], ran);
        atomicAdd(&w.stats[4], ran);
    }
    if (lane == 0 && active != 0) atomicAdd(&w.ctr->bs_active_next, active);
    // the last block to finish decides whether another iteration runs
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&w.ctr->bs_done_blocks, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        const int act = *((volatile int*)&w.ctr->bs_active_next);
        w.ctr->bs_active_next = 0;
        w.ctr->bs_done_blocks = 0;
        w.ctr->bs_run = act > 0 ? 1 : 0;
        if (use_cond) cudaGraphSetConditional(cond, act > 0 ? 1u : 0u);
    }
}

// ----------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------
int batch_slots_for(const DevGraph& g, long long budget)
{
    // per slot: the messages, the detector records, the list and small state
    const long long per = (long long)g.Epad * g.msg_bytes + 8ll * g.M + 4ll * kBsList + 16;
    long long bs = budget / (per > 0 ? per : 1);
    bs = (bs / kBsChunk) * kBsChunk;
    if (bs > 16384) bs = 16384;
    return bs >= kBsChunk ? (int)bs : 0;
}

int batch_grid(int device)
{
    int sms = 0;
    if (CUDA_FAILED(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device))) return 0;
    return 8 * sms;
}

namespace {

// items per thread of the check pass (rows) and the error-node pass (columns)
constexpr int kRowsPerThread = 2;
constexpr int kColsPerThread = 8;

void* check_func(int prec)
{
    return prec == 0 ? (void*)k_bs_check<0> : prec == 1 ? (void*)k_bs_check<1> : (void*)k_bs_check<2>;
}

void* var_func(int dv, int prec)
{
    if (dv <= 3) return prec == 0 ? (void*)k_bs_var<3, 0> : prec == 1 ? (void*)k_bs_var<3, 1> : (void*)k_bs_var<3, 2>;
    if (dv <= 6) return prec == 0 ? (void*)k_bs_var<6, 0> : prec == 1 ? (void*)k_bs_var<6, 1> : (void*)k_bs_var<6, 2>;
    return prec == 0 ? (void*)k_bs_var<16, 0> : prec == 1 ? (void*)k_bs_var<16, 1> : (void*)k_bs_var<16, 2>;
}

// column degree bound of the generic engines (3, 6 or 16)
int dv_of(const DevGraph& g) { return g.max_col_deg <= 3 ? 3 : g.max_col_deg <= 6 ? 6 : 16; }

// blocks of a pass: every slot chunk times groups of about `per` items
// (rows or columns), enough blocks to keep every SM busy
int grid_pass(const Work& w, int items, int per)
{
    const int nch = w.bs_slots / kBsChunk;
    const int groups = (items + per - 1) / per;
    return nch * (groups > 0 ? groups : 1);
}

int grid_retire(const LaunchShape& ls, const Work& w)
{
    const int need = w.bs_slots / 8;           // one warp per slot, 8 warps per block
    return need < ls.grid_bs ? need : ls.grid_bs;
}

int add_node(cudaGraph_t graph, cudaGraphNode_t* node, const cudaGraphNode_t* dep, void* func, int grid, int block,
             void** args)
{
    cudaKernelNodeParams p{};
    p.func = func;
    p.gridDim = dim3((unsigned)grid);
    p.blockDim = dim3((unsigned)block);
    p.sharedMemBytes = 0;
    p.kernelParams = args;
    return !CUDA_FAILED(cudaGraphAddKernelNode(node, graph, dep, dep ? 1 : 0, &p)) ? 0 : -2;
}

}  // namespace

int add_batch_nodes(cudaGraph_t graph, cudaGraphNode_t dep, cudaGraphNode_t* last, const DevGraph& g0,
                    const DecCfg& cfg0, const Work& w0, const LaunchShape& ls, int screened)
{
    DevGraph g = g0;
    DecCfg cfg = cfg0;
    Work w = w0;
    cudaGraphConditionalHandle cond;
    if (CUDA_FAILED(cudaGraphConditionalHandleCreate(&cond, graph, 0, cudaGraphCondAssignDefault))) return -2;
    int use = 1;
    cudaGraphNode_t nb, nw;
    void* bargs[] = {&w, &screened, &cond, &use};
    int rc = add_node(graph, &nb, dep ? &dep : nullptr, (void*)k_bs_begin, 1, 256, bargs);
    cudaGraphNodeParams cp{};
    if (!rc) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        if (CUDA_FAILED(cudaGraphAddNode(&nw, graph, &nb, nullptr, 1, &cp))) rc = -2;
    }
    if (!rc) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaGraphNode_t nc, nv, nr;
        void* pargs[] = {&g, &cfg, &w};
        void* rargs[] = {&g, &cfg, &w, &screened, &cond, &use};
        rc = add_node(body, &nc, nullptr, check_func(g.prec), grid_pass(w, g.M, kRowsPerThread), kBsChunk, pargs);
        if (!rc)
            rc = add_node(body, &nv, &nc, var_func(dv_of(g), g.prec), grid_pass(w, g.N, kColsPerThread), kBsThreads,
                          pargs);
        if (!rc) rc = add_node(body, &nr, &nv, (void*)k_bs_retire, grid_retire(ls, w), 256, rargs);
    }
    if (!rc) *last = nw;
    return rc;
}

int launch_batch_direct(const DevGraph& g, const DecCfg& cfg, const Work& w, const LaunchShape& ls, int screened,
                        cudaStream_t s, const LaunchHooks* hk, int* host_word)
{
    const cudaGraphConditionalHandle none{};
    k_bs_begin<<<1, 256, 0, s>>>(w, screened, none, 0);
    if (CUDA_FAILED(cudaGetLastError())) return -2;
    const int gc = grid_pass(w, g.M, kRowsPerThread), gv = grid_pass(w, g.N, kColsPerThread);
    const int gr = grid_retire(ls, w);
    void* cf = check_func(g.prec);
    void* vf = var_func(dv_of(g), g.prec);
    DevGraph gg = g;
    DecCfg cc = cfg;
    Work ww = w;
    int scr = screened, use = 0;
    cudaGraphConditionalHandle h = none;
    void* pargs[] = {&gg, &cc, &ww};
    void* rargs[] = {&gg, &cc, &ww, &scr, &h, &use};
    // kernels return at once when the batch has finished, so a few extra
    // iterations between read-backs of the loop flag cost nothing
    constexpr int kBetweenReads = 8;
    for (;;) {
        for (int k = 0; k < kBetweenReads; ++k) {
            if (hk) hk->before(hk->ctx, 8);
            if (CUDA_FAILED(cudaLaunchKernel(cf, dim3(gc), dim3(kBsChunk), pargs, 0, s))) return -2;
            if (hk) { hk->after(hk->ctx, 8); hk->before(hk->ctx, 9); }
            if (CUDA_FAILED(cudaLaunchKernel(vf, dim3(gv), dim3(kBsThreads), pargs, 0, s))) return -2;
            if (hk) { hk->after(hk->ctx, 9); hk->before(hk->ctx, 10); }
            if (CUDA_FAILED(cudaLaunchKernel((void*)k_bs_retire, dim3(gr), dim3(256), rargs, 0, s))) return -2;
            if (hk) hk->after(hk->ctx, 10);
        }
        if (CUDA_FAILED(cudaMemcpyAsync(host_word, &w.ctr->bs_run, sizeof(int), cudaMemcpyDeviceToHost, s)) ||
            CUDA_FAILED(cudaStreamSynchronize(s)))
            return -2;
        if (*host_word == 0) break;
    }
    return 0;
}

}  // namespace bsd
