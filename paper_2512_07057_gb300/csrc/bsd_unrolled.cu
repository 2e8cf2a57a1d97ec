// bsd_unrolled.cu -- unrolled weighted min-sum: forward, loss and adjoint.
//
// Training the weights w[t][e] of weighted min-sum (a weight per edge and
// iteration in place of the scale of Eq. 1) runs T flooding iterations of
// Eqs. 1-3 on a batch of B shots, with no stopping rule, and differentiates
//     loss = sum_{t=1..T} mean_{b,j} BCE(sigmoid(-Lambda_j(t)), e_j)
// with respect to the weights.
//
// Layout: every per-edge array is [E][Bp] and every per-node array [N][Bp]
// (shots contiguous; Bp = B rounded up to the 512-shot tile of a block), so a
// warp's 32 threads x 4 shots move 512 contiguous bytes of one edge.  The
// passes stream coalesced float4 vectors; the graph tables are read-only and
// cache resident.  Syndromes and true errors are transposed once into bit
// planes [M][Bp/32] and [N][Bp/32].
//
//   check pass (block = row i x 512 shots):
//       D_e(t) = w[t-1][e] * (-1)^{s_i} * prod_{e' != e} sign(E_e') * min_{e' != e} |E_e'|
//   error pass (block = column j x 512 shots):
//       Lambda_j(t) = Lambda_j + sum_{e in N(j)} D_e(t),  E_e(t) = clamp(Lambda_j(t) - D_e(t))
// The forward keeps E at the checkpoints t = 0, k, 2k, ...  The backward
// recomputes each segment of k iterations from its checkpoint, keeping E(t)
// and Lambda(t) of the segment, then runs the adjoint passes from t = T down:
//   error pass adjoint: gLam_j = dloss/dLambda_j(t) + sum_e [|E_e(t)| < L] gE_e
//                       gD_e = gLam_j - [|E_e(t)| < L] gE_e
//   check pass adjoint: gw[t-1][e] += gD_e sigma_e m_e,  gm_e = gD_e w[t-1][e] sigma_e
//                       gE_{i1}(t-1) = sign(E_{i1}) sum_{e != i1} gm_e
//                       gE_{i2}(t-1) = sign(E_{i2}) gm_{i1}
// with i1, i2 the edges of the row holding the smallest and second smallest
// |E(t-1)| (lowest edge index among equal magnitudes), sigma_e = (-1)^{s_i}
// prod_{e' != e} sign(E_e'), and m_e = |E_{i1}| for e != i1, |E_{i2}| for
// e = i1, or the constant L_MAX when no such edge exists (a row of weight 1,
// or every |E| at L_MAX).  sign() has zero derivative, d|x|/dx = sign(x) with
// 0 at 0, and a message at +-L_MAX passes none.  Loss and weight gradients
// are reduced through per-warp partial sums added in a fixed order, so every
// result is deterministic.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "bsd.h"
#include "bsd_internal.cuh"

namespace bsd {
namespace {

constexpr int kThreads = 128;            // threads per block
constexpr int kTile = 4 * kThreads;      // shots per block (4 per thread)
// a row or column of degree <= CAP (4 or 8) keeps its vectors in registers
// between passes; CAP = 0 loads them again
constexpr int kWarps = kThreads / 32;    // partial sums are kept per warp (no block barrier)

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct UArgs {
    const int* row_ptr;
    const int* col_ptr;
    const int* col_edge;
    const float* lam;
    int M, N, E;
    float L;
    long long B, Bp;
    int ntile;
    int T;
    const float* w;          // [T][E]
    const uint32_t* sT;      // [M][Bp/32]
    const uint32_t* yT;      // [N][Bp/32]
};

struct ULayout {
    uint32_t* sT;
    uint32_t* yT;
    float* ck;               // [C][E][Bp]: E at t = c k
    float* seg;              // [k][E][Bp]: E(t0 + 1 .. t0 + k) of the segment being differentiated
    float* lamT;             // [k][N][Bp]: Lambda(t0 + 1 .. t0 + k)
    float* D;                // [E][Bp]
    float* gE[2];            // [E][Bp]
    float* gD;               // [E][Bp]
    float* loss_part;        // [T][N][ntile * kWarps]: per-warp loss sums
    float* gw_part;          // [T][ntile * kWarps][E]: per-warp weight-gradient sums
    size_t bytes;
};

ULayout layout(const DevGraph& g, long long B, int T, int k, char* base)
{
    ULayout u{};
    const long long Bp = (B + kTile - 1) / kTile * kTile;
    const size_t W32 = (size_t)(Bp / 32), EB = (size_t)g.E * (size_t)Bp, NB = (size_t)g.N * (size_t)Bp;
    const int C = (T + k - 1) / k;
    const size_t ntile = (size_t)(Bp / kTile);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = base ? base + off : nullptr;
        off += a256(bytes);
        return p;
    };
    u.sT = (uint32_t*)take(sizeof(uint32_t) * (size_t)g.M * W32);
    u.yT = (uint32_t*)take(sizeof(uint32_t) * (size_t)g.N * W32);
    u.ck = (float*)take(sizeof(float) * EB * (size_t)C);
    u.seg = (float*)take(sizeof(float) * EB * (size_t)k);
    u.lamT = (float*)take(sizeof(float) * NB * (size_t)k);
    u.D = (float*)take(sizeof(float) * EB);
    u.gE[0] = (float*)take(sizeof(float) * EB);
    u.gE[1] = (float*)take(sizeof(float) * EB);
    u.gD = (float*)take(sizeof(float) * EB);
    u.loss_part = (float*)take(sizeof(float) * (size_t)T * (size_t)g.N * ntile * kWarps);
    u.gw_part = (float*)take(sizeof(float) * (size_t)T * ntile * kWarps * (size_t)g.E);
    u.bytes = off;
    return u;
}

__device__ __forceinline__ float4 ld4(const float* base, int row, long long Bp, long long b)
{
    return *reinterpret_cast<const float4*>(base + (size_t)row * (size_t)Bp + (size_t)b);
}
__device__ __forceinline__ void st4(float* base, int row, long long Bp, long long b, float4 v)
{
    *reinterpret_cast<float4*>(base + (size_t)row * (size_t)Bp + (size_t)b) = v;
}
__device__ __forceinline__ float comp(const float4& v, int c) { return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w; }
__device__ __forceinline__ void setc(float4& v, int c, float x)
{
    if (c == 0) v.x = x; else if (c == 1) v.y = x; else if (c == 2) v.z = x; else v.w = x;
}
// the 4 bits of shots b .. b+3 (b a multiple of 4) from a bit plane row
__device__ __forceinline__ uint32_t bits4(const uint32_t* plane, int row, long long Bp, long long b)
{
    return (plane[(size_t)row * (size_t)(Bp / 32) + (size_t)(b >> 5)] >> (b & 31)) & 0xFu;
}
__device__ __forceinline__ float softplus(float x) { return fmaxf(x, 0.f) + log1pf(expf(-fabsf(x))); }
__device__ __forceinline__ float sgn0(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

// sum over the warp; every lane gets the total
__device__ __forceinline__ float warp_sum(float v)
{
_Pragma("unroll")
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// slot of this warp among the per-warp partial sums of a tile
__device__ __forceinline__ int warp_slot() { return (int)blockIdx.x * kWarps + (int)(threadIdx.x >> 5); }

// ---------------------------------------------------------------------------
// batch intake: bitpacked [B][W] words -> bit planes [nbits][Bp/32]
// ---------------------------------------------------------------------------
__global__ void k_u_planes(const uint32_t* __restrict__ src, long long B, int W, int nbits, long long Bp,
                           uint32_t* __restrict__ dst)
{
    // one warp per (32 shots, one source word): lane l loads shot 32 wd + l's
    // word, and the ballot over bit k is row 32 w + k of those 32 shots
    const long long W32 = Bp / 32;
    const long long nwarp = W32 * (long long)W;
    const int lane = threadIdx.x & 31;
    for (long long q = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nwarp;
         q += ((long long)gridDim.x * blockDim.x) >> 5) {
        const long long wd = q / W;
        const int w = (int)(q % W);
        const long long b = 32 * wd + lane;
        const uint32_t v = (b < B) ? src[(size_t)b * W + w] : 0u;
        for (int k = 0; k < 32; ++k) {
            const uint32_t bal = __ballot_sync(0xffffffffu, (v >> k) & 1u);
            const int i = 32 * w + k;
            if (lane == k && i < nbits) dst[(size_t)i * (size_t)W32 + (size_t)wd] = bal;
        }
    }
}

// E(0) = clamp(Lambda_j) on every edge of column j, for every shot
__global__ void k_u_init(UArgs a, float* __restrict__ E0)
{
    const long long b = (long long)blockIdx.x * kTile + 4 * threadIdx.x;
    for (int j = blockIdx.y; j < a.N; j += gridDim.y) {
        const float v = fminf(fmaxf(__ldg(a.lam + j), -a.L), a.L);
        const float4 v4 = make_float4(v, v, v, v);
        for (int q = __ldg(a.col_ptr + j); q < __ldg(a.col_ptr + j + 1); ++q) st4(E0, __ldg(a.col_edge + q), a.Bp, b, v4);
    }
}

// Loops over the edges of a row or column: with CAP > 0 the loop is unrolled
// up to CAP with compile-time indices, so each edge's vector stays in a
// register between passes; with CAP = 0 the vector is loaded again.
#define U_FOR_EDGES(CAP, k, deg, ...)                        \
    if (CAP > 0) {                                          \
        _Pragma("unroll") for (int k = 0; k < CAP; ++k)     \
            if (k < (deg)) { __VA_ARGS__ }                  \
    } else {                                                \
        for (int k = 0; k < (deg); ++k) { __VA_ARGS__ }     \
    }

// ---------------------------------------------------------------------------
// check pass (Eq. 1 with weights): D(t) from E(t-1)
// ---------------------------------------------------------------------------
template <int CAP>
__global__ void __launch_bounds__(kThreads) k_u_check(UArgs a, const float* __restrict__ Ein, float* __restrict__ D,
                                                      int t)
{
    const long long b = (long long)blockIdx.x * kTile + 4 * threadIdx.x;
    const float* wt = a.w + (size_t)(t - 1) * (size_t)a.E;
    for (int i = blockIdx.y; i < a.M; i += gridDim.y) {
        const int rb = __ldg(a.row_ptr + i), deg = __ldg(a.row_ptr + i + 1) - rb;
        const uint32_t s4 = bits4(a.sT, i, a.Bp, b);
        float m1[4], m2[4];
        uint32_t neg[4];
_Pragma("unroll")
        for (int c = 0; c < 4; ++c) { m1[c] = a.L; m2[c] = a.L; neg[c] = (s4 >> c) & 1u; }
        float4 x[CAP > 0 ? CAP : 1];
        U_FOR_EDGES(CAP, k, deg, {
            const float4 v = ld4(Ein, rb + k, a.Bp, b);
            if (CAP > 0) x[CAP > 0 ? k : 0] = v;
_Pragma("unroll")
            for (int c = 0; c < 4; ++c) {
                const float y = comp(v, c), m = fabsf(y);
                m2[c] = fminf(m2[c], fmaxf(m1[c], m));
                m1[c] = fminf(m1[c], m);
                neg[c] ^= (y < 0.f) ? 1u : 0u;
            }
        })
        U_FOR_EDGES(CAP, k, deg, {
            const float4 v = CAP > 0 ? x[CAP > 0 ? k : 0] : ld4(Ein, rb + k, a.Bp, b);
            const float wv = __ldg(wt + rb + k);
            float4 d;
_Pragma("unroll")
            for (int c = 0; c < 4; ++c) {
                const float y = comp(v, c);
                const float m = (fabsf(y) == m1[c]) ? m2[c] : m1[c];
                const float dd = __fmul_rn(wv, m);
                setc(d, c, (neg[c] ^ ((y < 0.f) ? 1u : 0u)) ? -dd : dd);
            }
            st4(D, rb + k, a.Bp, b, d);
        })
    }
}

// ---------------------------------------------------------------------------
// error pass (Eqs. 2-3): Lambda(t), E(t), loss terms
// ---------------------------------------------------------------------------
template <int CAP>
__global__ void __launch_bounds__(kThreads) k_u_var(UArgs a, const float* __restrict__ D, float* __restrict__ Eout,
                                                    float* __restrict__ lamT, float* __restrict__ llr,
                                                    float* __restrict__ loss_part)
{
    const long long b = (long long)blockIdx.x * kTile + 4 * threadIdx.x;
    for (int j = blockIdx.y; j < a.N; j += gridDim.y) {
        const int kb = __ldg(a.col_ptr + j), deg = __ldg(a.col_ptr + j + 1) - kb;
        const float lj = __ldg(a.lam + j);
        float4 post = make_float4(lj, lj, lj, lj);
        float4 x[CAP > 0 ? CAP : 1];
        U_FOR_EDGES(CAP, k, deg, {
            const float4 v = ld4(D, __ldg(a.col_edge + kb + k), a.Bp, b);
            if (CAP > 0) x[CAP > 0 ? k : 0] = v;
            post.x = __fadd_rn(post.x, v.x);
            post.y = __fadd_rn(post.y, v.y);
            post.z = __fadd_rn(post.z, v.z);
            post.w = __fadd_rn(post.w, v.w);
        })
        U_FOR_EDGES(CAP, k, deg, {
            const int e = __ldg(a.col_edge + kb + k);
            const float4 v = CAP > 0 ? x[CAP > 0 ? k : 0] : ld4(D, e, a.Bp, b);
            float4 o;
_Pragma("unroll")
            for (int c = 0; c < 4; ++c) setc(o, c, fminf(fmaxf(__fsub_rn(comp(post, c), comp(v, c)), -a.L), a.L));
            st4(Eout, e, a.Bp, b, o);
        })
        if (lamT) st4(lamT, j, a.Bp, b, post);
        if (llr) {
_Pragma("unroll")
            for (int c = 0; c < 4; ++c)
                if (b + c < a.B) llr[(size_t)(b + c) * (size_t)a.N + j] = comp(post, c);
        }
        if (loss_part) {
            const uint32_t y4 = bits4(a.yT, j, a.Bp, b);
            float l = 0.f;
_Pragma("unroll")
            for (int c = 0; c < 4; ++c) {
                const float p = comp(post, c);
                if (b + c < a.B) l += ((y4 >> c) & 1u) ? softplus(p) : softplus(-p);
            }
            l = warp_sum(l);
            if ((threadIdx.x & 31) == 0) loss_part[(size_t)j * a.ntile * kWarps + warp_slot()] = l;
        }
    }
}

// loss term of iteration t (block t): its partial sums added in a fixed order, in double
__global__ void k_u_loss(const float* __restrict__ loss_part, int N, int nslot, double scale, float* __restrict__ out)
{
    __shared__ double red[256];
    const int t = blockIdx.x;
    const float* p = loss_part + (size_t)t * N * nslot;
    double s = 0.0;
    for (long long q = threadIdx.x; q < (long long)N * nslot; q += blockDim.x) s += (double)p[q];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[1 + t] = (float)(red[0] * scale);
}

// the loss: the T terms added in order
__global__ void k_u_loss_total(int T, float* __restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int t = 0; t < T; ++t) s += (double)out[1 + t];
        out[0] = (float)s;
    }
}

// ---------------------------------------------------------------------------
// adjoint of the error pass at iteration t: gD(t) from gE(t) and the loss
// ---------------------------------------------------------------------------
template <int CAP>
__global__ void __launch_bounds__(kThreads) k_u_bvar(UArgs a, const float* __restrict__ gEin,
                                                     const float* __restrict__ Et, const float* __restrict__ lamT,
                                                     const float* __restrict__ gout, double scale, int t,
                                                     float* __restrict__ gD)
{
    const long long b = (long long)blockIdx.x * kTile + 4 * threadIdx.x;
    // the objective's derivative with respect to the term of iteration t:
    // through the total ([0]) and through the term itself ([t])
    const float gs = (float)(((double)__ldg(gout) + (double)__ldg(gout + t)) * scale);
    for (int j = blockIdx.y; j < a.N; j += gridDim.y) {
        const int kb = __ldg(a.col_ptr + j), deg = __ldg(a.col_ptr + j + 1) - kb;
        const float4 post = ld4(lamT, j, a.Bp, b);
        const uint32_t y4 = bits4(a.yT, j, a.Bp, b);
        float4 gl;
_Pragma("unroll")
        for (int c = 0; c < 4; ++c) {
            // d BCE / d Lambda = sigmoid(Lambda) - 1 + e_j
            const float p = comp(post, c);
            const float sg = 1.f / (1.f + expf(-p));
            setc(gl, c, (b + c < a.B) ? gs * (sg - 1.f + (float)((y4 >> c) & 1u)) : 0.f);
        }
        // gE(t) where the clamp let the derivative through, 0 elsewhere
        auto gE_of = [&](int e) {
            float4 g = ld4(gEin, e, a.Bp, b);
            const float4 v = ld4(Et, e, a.Bp, b);
_Pragma("unroll")
            for (int c = 0; c < 4; ++c)
                if (!(fabsf(comp(v, c)) < a.L)) setc(g, c, 0.f);
            return g;
        };
        float4 ge[CAP > 0 ? CAP : 1];
        if (gEin) {
            U_FOR_EDGES(CAP, k, deg, {
                const float4 g = gE_of(__ldg(a.col_edge + kb + k));
                if (CAP > 0) ge[CAP > 0 ? k : 0] = g;
                gl.x += g.x; gl.y += g.y; gl.z += g.z; gl.w += g.w;
            })
        }
        U_FOR_EDGES(CAP, k, deg, {
            const int e = __ldg(a.col_edge + kb + k);
            float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gEin) g = CAP > 0 ? ge[CAP > 0 ? k : 0] : gE_of(e);
            st4(gD, e, a.Bp, b, make_float4(gl.x - g.x, gl.y - g.y, gl.z - g.z, gl.w - g.w));
        })
    }
}

// ---------------------------------------------------------------------------
// adjoint of the check pass at iteration t: weight gradients and gE(t-1)
// ---------------------------------------------------------------------------
template <int CAP>
__global__ void __launch_bounds__(kThreads) k_u_bcheck(UArgs a, const float* __restrict__ Eprev,
                                                       const float* __restrict__ gD, float* __restrict__ gEprev,
                                                       float* __restrict__ gw_part, int t)
{
    const long long b = (long long)blockIdx.x * kTile + 4 * threadIdx.x;
    const float* wt = a.w + (size_t)(t - 1) * (size_t)a.E;
    for (int i = blockIdx.y; i < a.M; i += gridDim.y) {
        const int rb = __ldg(a.row_ptr + i), deg = __ldg(a.row_ptr + i + 1) - rb;
        const uint32_t s4 = bits4(a.sT, i, a.Bp, b);
        float m1[4], m2[4], v1[4], v2[4];
        int i1[4], i2[4];
        uint32_t neg[4];
_Pragma("unroll")
        for (int c = 0; c < 4; ++c) {
            m1[c] = a.L; m2[c] = a.L; v1[c] = 0.f; v2[c] = 0.f; i1[c] = -1; i2[c] = -1;
            neg[c] = (s4 >> c) & 1u;
        }
        float4 x[CAP > 0 ? CAP : 1];
        // the two smallest magnitudes with their edges (lowest index among equals)
        U_FOR_EDGES(CAP, k, deg, {
            const float4 v = ld4(Eprev, rb + k, a.Bp, b);
            if (CAP > 0) x[CAP > 0 ? k : 0] = v;
_Pragma("unroll")
            for (int c = 0; c < 4; ++c) {
                const float y = comp(v, c), m = fabsf(y);
                if (m < m1[c]) {
                    m2[c] = m1[c]; i2[c] = i1[c]; v2[c] = v1[c];
                    m1[c] = m; i1[c] = k; v1[c] = y;
                } else if (m < m2[c]) {
                    m2[c] = m; i2[c] = k; v2[c] = y;
                }
                neg[c] ^= (y < 0.f) ? 1u : 0u;
            }
        })
        float acc1[4] = {0.f, 0.f, 0.f, 0.f}, g1[4] = {0.f, 0.f, 0.f, 0.f};
        U_FOR_EDGES(CAP, k, deg, {
            const float4 v = CAP > 0 ? x[CAP > 0 ? k : 0] : ld4(Eprev, rb + k, a.Bp, b);
            const float4 g = ld4(gD, rb + k, a.Bp, b);
            const float wv = __ldg(wt + rb + k);
            float gw = 0.f;
_Pragma("unroll")
            for (int c = 0; c < 4; ++c) {
                const float y = comp(v, c);
                const float sig = (neg[c] ^ ((y < 0.f) ? 1u : 0u)) ? -1.f : 1.f;
                const float m = (k == i1[c]) ? m2[c] : m1[c];
                const float gd = comp(g, c);
                gw += gd * sig * m;
                const float gm = gd * wv * sig;
                if (k == i1[c]) g1[c] = gm; else acc1[c] += gm;
            }
            gw = warp_sum(gw);
            if ((threadIdx.x & 31) == 0) gw_part[(size_t)warp_slot() * a.E + rb + k] = gw;
        })
        if (gEprev) {
            U_FOR_EDGES(CAP, k, deg, {
                float4 o;
_Pragma("unroll")
                for (int c = 0; c < 4; ++c) {
                    float r = 0.f;
                    if (k == i1[c]) r = sgn0(v1[c]) * acc1[c];
                    else if (k == i2[c] && i1[c] >= 0) r = sgn0(v2[c]) * g1[c];
                    setc(o, c, r);
                }
                st4(gEprev, rb + k, a.Bp, b, o);
            })
        }
    }
}

// weight gradients: the per-warp partial sums added in a fixed order
__global__ void k_u_gw(const float* __restrict__ gw_part, int T, int ntile, int E, float* __restrict__ grad)
{
    const long long total = (long long)T * E;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long t = q / E, e = q % E;
        const float* p = gw_part + (size_t)t * ntile * E + e;
        float s = 0.f;
        for (int k = 0; k < ntile; ++k) s += p[(size_t)k * E];
        grad[q] = s;
    }
}

// register cache for rows / columns of degree at most 4 or 8, none beyond
int cap_of(int max_deg) { return max_deg <= 4 ? 4 : (max_deg <= 8 ? 8 : 0); }

int grid_y(int items) { return items < 65535 ? (items > 0 ? items : 1) : 65535; }

int check_args(const bsd_decoder* dec, int64_t B, int32_t T, int32_t k, const DevGraph** g, const DecCfg** cfg,
               int* device)
{
    if (!dec || B < 1 || T < 1 || k < 1 || k > T || B > (1ll << 30)) return BSD_ERR_INVALID_ARG;
    if (decoder_graph(dec, g, cfg, device) != BSD_OK) return BSD_ERR_INVALID_ARG;
    if ((*g)->prec != 0) return BSD_ERR_UNSUPPORTED;
    return BSD_OK;
}

UArgs make_args(const DevGraph& g, const DecCfg& cfg, long long B, int T, const float* w, const ULayout& u)
{
    UArgs a{};
    a.row_ptr = g.row_ptr;
    a.col_ptr = g.col_ptr;
    a.col_edge = g.col_edge;
    a.lam = g.lam;
    a.M = g.M; a.N = g.N; a.E = g.E;
    a.L = cfg.L;
    a.B = B;
    a.Bp = (B + kTile - 1) / kTile * kTile;
    a.ntile = (int)(a.Bp / kTile);
    a.T = T;
    a.w = w;
    a.sT = u.sT;
    a.yT = u.yT;
    return a;
}

struct DeviceScope {
    int prev = -1;
    bool ok = false;
    explicit DeviceScope(int dev)
    {
        if (CUDA_FAILED(cudaGetDevice(&prev))) prev = -1;
        ok = !CUDA_FAILED(cudaSetDevice(dev));
    }
    ~DeviceScope()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// event hooks around a launch when the decoder's kernel timing is on
enum { kKindCheck = 3, kKindVar = 4, kKindBVar = 5, kKindBCheck = 6, kKindOther = 7 };
struct Timed {
    const LaunchHooks* hk;
    int kind;
    Timed(const LaunchHooks* h, int k) : hk(h), kind(k) { if (hk) hk->before(hk->ctx, kind); }
    ~Timed() { if (hk) hk->after(hk->ctx, kind); }
};

void launch_check(const UArgs& a, const DevGraph& g, const float* Ein, float* D, int t, cudaStream_t s,
                  const LaunchHooks* hk)
{
    const dim3 grid(a.ntile, grid_y(a.M));
    Timed tm(hk, kKindCheck);
    switch (cap_of(g.max_row_deg)) {
        case 4: k_u_check<4><<<grid, kThreads, 0, s>>>(a, Ein, D, t); break;
        case 8: k_u_check<8><<<grid, kThreads, 0, s>>>(a, Ein, D, t); break;
        default: k_u_check<0><<<grid, kThreads, 0, s>>>(a, Ein, D, t); break;
    }
}

void launch_var(const UArgs& a, const DevGraph& g, const float* D, float* Eout, float* lamT, float* llr,
                float* loss_part, cudaStream_t s, const LaunchHooks* hk)
{
    const dim3 grid(a.ntile, grid_y(a.N));
    Timed tm(hk, kKindVar);
    switch (cap_of(g.max_col_deg)) {
        case 4: k_u_var<4><<<grid, kThreads, 0, s>>>(a, D, Eout, lamT, llr, loss_part); break;
        case 8: k_u_var<8><<<grid, kThreads, 0, s>>>(a, D, Eout, lamT, llr, loss_part); break;
        default: k_u_var<0><<<grid, kThreads, 0, s>>>(a, D, Eout, lamT, llr, loss_part); break;
    }
}

}  // namespace
}  // namespace bsd

using namespace bsd;

extern "C" {

int bsd_unrolled_workspace(const bsd_decoder* dec, int64_t B, int32_t T, int32_t ckpt_every, int64_t* bytes)
{
    const DevGraph* g;
    const DecCfg* cfg;
    int device;
    if (!bytes) return BSD_ERR_INVALID_ARG;
    const int rc = check_args(dec, B, T, ckpt_every, &g, &cfg, &device);
    if (rc) return rc;
    *bytes = (int64_t)layout(*g, B, T, ckpt_every, nullptr).bytes;
    return BSD_OK;
}

int bsd_unrolled_forward(const bsd_decoder* dec, const uint32_t* d_syndromes, const uint32_t* d_errors, int64_t B,
                         int32_t T, int32_t ckpt_every, const float* d_weights, float* d_loss, float* d_llr,
                         void* d_work, int64_t work_bytes, void* cuda_stream)
{
    const DevGraph* g;
    const DecCfg* cfg;
    int device;
    int rc = check_args(dec, B, T, ckpt_every, &g, &cfg, &device);
    if (rc) return rc;
    if (!d_syndromes || !d_errors || !d_weights || !d_loss || !d_work) return BSD_ERR_INVALID_ARG;
    const ULayout u = layout(*g, B, T, ckpt_every, (char*)d_work);
    if (work_bytes < (int64_t)u.bytes || ((uintptr_t)d_work & 255u)) return BSD_ERR_INVALID_ARG;
    DeviceScope ds(device);
    if (!ds.ok) return BSD_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const UArgs a = make_args(*g, *cfg, B, T, d_weights, u);
    const int k = ckpt_every;
    const size_t EB = (size_t)g->E * (size_t)a.Bp;
    LaunchHooks hks;
    const LaunchHooks* hk = decoder_hooks(dec, s, &hks) ? &hks : nullptr;
    {
        Timed tm(hk, kKindOther);
        k_u_planes<<<1024, 256, 0, s>>>(d_syndromes, B, g->WM, g->M, a.Bp, u.sT);
        k_u_planes<<<1024, 256, 0, s>>>(d_errors, B, g->WN, g->N, a.Bp, u.yT);
        k_u_init<<<dim3(a.ntile, grid_y(g->N)), kThreads, 0, s>>>(a, u.ck);
    }
    // E(t) lives in its checkpoint slot at t = c k, else in a scratch buffer
    const float* src = u.ck;
    for (int t = 1; t <= T; ++t) {
        launch_check(a, *g, src, u.D, t, s, hk);
        float* dst = (t % k == 0 && t < T) ? u.ck + (size_t)(t / k) * EB : u.seg;
        launch_var(a, *g, u.D, dst, nullptr, d_llr ? d_llr + (size_t)(t - 1) * (size_t)B * g->N : nullptr,
                   u.loss_part + (size_t)(t - 1) * g->N * a.ntile * kWarps, s, hk);
        src = dst;
    }
    {
        Timed tm(hk, kKindOther);
        k_u_loss<<<T, 256, 0, s>>>(u.loss_part, g->N, a.ntile * kWarps, 1.0 / ((double)B * (double)g->N), d_loss);
        k_u_loss_total<<<1, 32, 0, s>>>(T, d_loss);
    }
    return CUDA_FAILED(cudaGetLastError()) ? BSD_ERR_CUDA : BSD_OK;
}

int bsd_unrolled_backward(const bsd_decoder* dec, int64_t B, int32_t T, int32_t ckpt_every, const float* d_weights,
                          const float* d_grad_loss, float* d_grad_weights, void* d_work, int64_t work_bytes,
                          void* cuda_stream)
{
    const DevGraph* g;
    const DecCfg* cfg;
    int device;
    int rc = check_args(dec, B, T, ckpt_every, &g, &cfg, &device);
    if (rc) return rc;
    if (!d_weights || !d_grad_loss || !d_grad_weights || !d_work) return BSD_ERR_INVALID_ARG;
    const ULayout u = layout(*g, B, T, ckpt_every, (char*)d_work);
    if (work_bytes < (int64_t)u.bytes || ((uintptr_t)d_work & 255u)) return BSD_ERR_INVALID_ARG;
    DeviceScope ds(device);
    if (!ds.ok) return BSD_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const UArgs a = make_args(*g, *cfg, B, T, d_weights, u);
    const int k = ckpt_every;
    const size_t EB = (size_t)g->E * (size_t)a.Bp, NB = (size_t)g->N * (size_t)a.Bp;
    const double scale = 1.0 / ((double)B * (double)g->N);
    const int cap_c = cap_of(g->max_col_deg);
    const dim3 gcol(a.ntile, grid_y(g->N)), grow(a.ntile, grid_y(g->M));
    LaunchHooks hks;
    const LaunchHooks* hk = decoder_hooks(dec, s, &hks) ? &hks : nullptr;
    int cur = 0;                               // gE(t) lives in u.gE[cur]
    const int C = (T + k - 1) / k;
    for (int c = C - 1; c >= 0; --c) {
        const int t0 = c * k, t1 = (t0 + k < T) ? t0 + k : T;
        // recompute E(t) and Lambda(t) of the segment from its checkpoint
        const float* src = u.ck + (size_t)c * EB;
        for (int t = t0 + 1; t <= t1; ++t) {
            launch_check(a, *g, src, u.D, t, s, hk);
            float* dst = u.seg + (size_t)(t - t0 - 1) * EB;
            launch_var(a, *g, u.D, dst, u.lamT + (size_t)(t - t0 - 1) * NB, nullptr, nullptr, s, hk);
            src = dst;
        }
        for (int t = t1; t > t0; --t) {
            const float* Et = u.seg + (size_t)(t - t0 - 1) * EB;
            const float* lamT = u.lamT + (size_t)(t - t0 - 1) * NB;
            const float* gEin = (t == T) ? nullptr : u.gE[cur];
            {
                Timed tm(hk, kKindBVar);
                if (cap_c == 4)
                    k_u_bvar<4><<<gcol, kThreads, 0, s>>>(a, gEin, Et, lamT, d_grad_loss, scale, t, u.gD);
                else if (cap_c == 8)
                    k_u_bvar<8><<<gcol, kThreads, 0, s>>>(a, gEin, Et, lamT, d_grad_loss, scale, t, u.gD);
                else k_u_bvar<0><<<gcol, kThreads, 0, s>>>(a, gEin, Et, lamT, d_grad_loss, scale, t, u.gD);
            }
            const float* Eprev = (t == t0 + 1) ? u.ck + (size_t)c * EB : u.seg + (size_t)(t - t0 - 2) * EB;
            float* gEout = (t > 1) ? u.gE[cur ^ 1] : nullptr;
            float* gwp = u.gw_part + (size_t)(t - 1) * a.ntile * kWarps * g->E;
            {
                Timed tm(hk, kKindBCheck);
                // the check adjoint reloads its vectors (64 registers, 8 blocks per SM):
                // faster than holding them (96 registers, 5 blocks)
                k_u_bcheck<0><<<grow, kThreads, 0, s>>>(a, Eprev, u.gD, gEout, gwp, t);
            }
            cur ^= 1;
        }
    }
    {
        Timed tm(hk, kKindOther);
        k_u_gw<<<1024, 256, 0, s>>>(u.gw_part, T, a.ntile * kWarps, g->E, d_grad_weights);
    }
    return CUDA_FAILED(cudaGetLastError()) ? BSD_ERR_CUDA : BSD_OK;
}

}  // extern "C"
