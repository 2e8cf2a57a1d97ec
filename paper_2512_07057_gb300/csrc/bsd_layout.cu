// bsd_layout.cu -- where the BP engines keep each edge's messages in shared
// memory (host code, run once when a decoder is created).
//
// Generic engines (column degree bound 3 or 6; generic_layout): a row's
// edges occupy the row's window [row_ptr[i], row_ptr[i + 1]) in any order
// (the detector pass reduces the window with order-independent operations),
// and a column's edges may take any k slots of the padded column table (the
// error pass sorts its inputs).  A local search over swaps within rows
// spreads each group of 32 columns over the banks (at most the group's
// largest column degree per bank), and a colouring of the group's
// (column, bank) multigraph then gives each k slot distinct banks; where the
// search leaves a bank above that, each edge takes the free slot whose bank
// is least loaded.  Columns may keep holes in their slots.
//
// Single-warp engine (small_layout):
//
// The single-warp engine (codes with every row of degree 6 and every column of
// degree 3) runs two passes per BP iteration over a candidate's messages in
// shared memory (Eqs. 1-3):
//   detector pass  lane l takes rows i = l + 32 r and loads / stores each
//                  row's messages as three 8-byte pairs;
//   error pass     lane l takes columns j = l + 32 c and gathers / scatters
//                  the message of its k-th edge, k = 0, 1, 2, one 4-byte word
//                  each, from a per-(column, k) address table.
// A warp's shared-memory access costs one wavefront per distinct word in the
// busiest of the 32 banks.  Storing row i's pairs at 6 i, 6 i + 2, 6 i + 4
// makes the detector pass conflict-free but leaves the error pass about 2.3
// wavefronts per access on [[144,12,12]].
//
// Placement used here: pair h of row i at word h P + 2 i, three planes of
// stride P = 64 ceil(M / 32) + 12 (a compile-time constant of the engine,
// which holds ceil(M / 32) rows per lane, so these addresses fold into its
// load and store offsets); every detector-pass access is 32 consecutive
// pairs, conflict-free.  Two choices leave every value the engine computes
// unchanged, and the search below uses them to make the error pass
// conflict-free too:
//   * the order of a row's six edges over its six positions (the two smallest
//     magnitudes and the sign parity of a row do not depend on it, and each
//     edge's outgoing message depends only on its own input and those);
//   * which of a column's three edges is its k-th (the error pass sorts the
//     three incoming messages before it adds them).
// The error-pass access (c, k) is conflict-free when the 32 k-th edges of
// columns 32 c .. 32 c + 31 sit in 32 distinct banks.  If every bank holds at
// most three of the 96 edges of that column group, such a k exists for every
// column (a bipartite multigraph of columns and banks with degrees <= 3 has a
// proper 3-edge-colouring, Koenig's theorem), built here by alternating
// paths.  The row orders are found by a deterministic local search over
// swaps within a row that lowers the bank loads above three, restarted from
// a few seeds; if no run reaches zero the best one is kept (the engine is
// correct for any placement, only slower).  The skew 12 is one for which an
// exact integer program finds a zero-load placement on the [[72,12,6]],
// [[144,12,12]] and [[108,8,10]] bivariate bicycle codes.
#include "bsd_internal.cuh"

#include <algorithm>
#include <cstdint>
#include <vector>

namespace bsd {

namespace {

constexpr int kPlanes = 3;      // pairs per row of degree 6
constexpr int kRowDeg = 6;
constexpr int kColDeg = 3;
constexpr int kTries = 16;      // local-search restarts
constexpr int kSweeps = 200;    // sweeps per restart

struct Rng {                    // xorshift64*: a fixed, reproducible sequence
    uint64_t s;
    uint32_t next()
    {
        s ^= s >> 12;
        s ^= s << 25;
        s ^= s >> 27;
        return (uint32_t)((s * 2685821657736338717ull) >> 32);
    }
    uint32_t below(uint32_t n) { return next() % n; }
};

int mod32(int x) { return ((x % 32) + 32) % 32; }

// proper k-colouring (k = 0..2) of the edges of one column group whose banks
// each hold at most three of its edges, the edge (column u, bank v) list
// given; colour[i] receives the colour of edge i
void colour_group(const std::vector<int>& eu, const std::vector<int>& ev, std::vector<int>* colour)
{
    const int n = (int)eu.size();
    colour->assign(n, -1);
    int atU[32][kColDeg], atV[32][kColDeg];
    for (int a = 0; a < 32; ++a)
        for (int c = 0; c < kColDeg; ++c) atU[a][c] = atV[a][c] = -1;
    for (int i = 0; i < n; ++i) {
        const int u = eu[i], v = ev[i];
        int a = -1, b = -1;
        for (int c = 0; c < kColDeg && a < 0; ++c)
            if (atU[u][c] < 0) a = c;
        for (int c = 0; c < kColDeg && b < 0; ++c)
            if (atV[v][c] < 0) b = c;
        if (atV[v][a] >= 0) {
            // swap colours a and b along the path from v that alternates
            // a, b, a, ...; in a bipartite graph it never reaches u, and
            // afterwards a is free at v (and still free at u)
            std::vector<int> path;
            int x = v, side = 1, c = a;            // side 1: x is a bank
            while ((int)path.size() <= n) {
                const int e = side ? atV[x][c] : atU[x][c];
                if (e < 0) break;
                path.push_back(e);
                x = side ? eu[e] : ev[e];
                side ^= 1;
                c = (c == a) ? b : a;
            }
            for (int e : path) {                   // clear, then set with the other colour
                atU[eu[e]][(*colour)[e]] = -1;
                atV[ev[e]][(*colour)[e]] = -1;
            }
            for (int e : path) {
                const int ce = (*colour)[e] == a ? b : a;
                (*colour)[e] = ce;
                atU[eu[e]][ce] = e;
                atV[ev[e]][ce] = e;
            }
        }
        (*colour)[i] = a;
        atU[u][a] = i;
        atV[v][a] = i;
    }
}

}  // namespace

bool small_layout(int M, int N, const int* row_ptr, const int* col_idx, SmallLayout* out)
{
    if (M < 1 || N < 1) return false;
    for (int i = 0; i < M; ++i)
        if (row_ptr[i + 1] - row_ptr[i] != kRowDeg) return false;
    const int E = row_ptr[M];
    std::vector<int> cdeg(N, 0);
    for (int e = 0; e < E; ++e) cdeg[col_idx[e]]++;
    for (int j = 0; j < N; ++j)
        if (cdeg[j] != kColDeg) return false;
    const int NG = (N + 31) / 32;

    const int P = small_plane_stride(M);
    const int A[kPlanes] = {0, P, 2 * P};
    Rng rng{0x9e3779b97f4a7c15ull};
    int best_ex = -1;
    std::vector<int> best_perm;
    std::vector<int> perm((size_t)M * kRowDeg), cnt((size_t)NG * 32);
    for (int t = 0; t < kTries && best_ex != 0; ++t) {
        auto bank = [&](int i, int q) { return mod32(A[q >> 1] + 2 * i + (q & 1)); };
        auto grp = [&](int i, int q) { return col_idx[row_ptr[i] + perm[(size_t)i * kRowDeg + q]] >> 5; };
        for (int i = 0; i < M; ++i)
            for (int q = 0; q < kRowDeg; ++q) perm[(size_t)i * kRowDeg + q] = q;
        std::fill(cnt.begin(), cnt.end(), 0);
        for (int i = 0; i < M; ++i)
            for (int q = 0; q < kRowDeg; ++q) cnt[(size_t)grp(i, q) * 32 + bank(i, q)]++;
        auto over = [&](int g, int b) { return std::max(0, cnt[(size_t)g * 32 + b] - kColDeg); };
        int ex = 0;
        for (int x : cnt) ex += std::max(0, x - kColDeg);
        std::vector<int> order(M);
        for (int i = 0; i < M; ++i) order[i] = i;
        for (int sw = 0; sw < kSweeps && ex > 0; ++sw) {
            for (int i = M - 1; i > 0; --i) std::swap(order[i], order[rng.below((uint32_t)i + 1)]);
            for (int i : order) {
                for (int a = 0; a < kRowDeg; ++a) {
                    for (int b = a + 1; b < kRowDeg; ++b) {
                        const int ga = grp(i, a), gb = grp(i, b);
                        if (ga == gb) continue;
                        const int ba = bank(i, a), bb = bank(i, b);
                        const int before = over(ga, ba) + over(gb, bb) + over(ga, bb) + over(gb, ba);
                        cnt[(size_t)ga * 32 + ba]--; cnt[(size_t)gb * 32 + bb]--;
                        cnt[(size_t)ga * 32 + bb]++; cnt[(size_t)gb * 32 + ba]++;
                        const int after = over(ga, ba) + over(gb, bb) + over(ga, bb) + over(gb, ba);
                        // keep improvements, and one equal move in four to move on a plateau
                        if (after < before || (after == before && rng.below(4) == 0)) {
                            std::swap(perm[(size_t)i * kRowDeg + a], perm[(size_t)i * kRowDeg + b]);
                            ex += after - before;
                        } else {
                            cnt[(size_t)ga * 32 + ba]++; cnt[(size_t)gb * 32 + bb]++;
                            cnt[(size_t)ga * 32 + bb]--; cnt[(size_t)gb * 32 + ba]--;
                        }
                    }
                }
            }
        }
        if (best_ex < 0 || ex < best_ex) {
            best_ex = ex;
            best_perm = perm;
        }
    }

    // word address of every CSR edge
    out->addr.assign(E, 0);
    for (int i = 0; i < M; ++i)
        for (int q = 0; q < kRowDeg; ++q)
            out->addr[row_ptr[i] + best_perm[(size_t)i * kRowDeg + q]] = A[q >> 1] + 2 * i + (q & 1);
    for (int h = 0; h < kPlanes; ++h) out->A[h] = A[h];
    out->A[3] = 0;
    out->extent = A[kPlanes - 1] + 2 * M;
    out->excess = best_ex;

    // the k order of every column from a colouring per column group
    std::vector<int> erow(E);
    for (int i = 0; i < M; ++i)
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) erow[e] = i;
    std::vector<std::vector<int>> cedges(N);
    for (int e = 0; e < E; ++e) cedges[col_idx[e]].push_back(e);
    out->col.assign((size_t)N * kColDeg, 0u);
    for (int g = 0; g < NG; ++g) {
        std::vector<int> ids, eu, ev, colour;
        for (int j = 32 * g; j < std::min(N, 32 * g + 32); ++j)
            for (int e : cedges[j]) {
                ids.push_back(e);
                eu.push_back(j - 32 * g);
                ev.push_back(out->addr[e] & 31);
            }
        // a bank above three edges (a search that did not reach zero) admits
        // no proper colouring: the group keeps the column lists' order
        int vdeg[32] = {0};
        for (int v : ev) vdeg[v]++;
        bool proper = *std::max_element(vdeg, vdeg + 32) <= kColDeg;
        if (proper) colour_group(eu, ev, &colour);
        // every column must take k = 0, 1, 2 once (the engine reads all three)
        for (size_t x = 0; proper && x < ids.size(); x += kColDeg) {
            int seen = 0;
            for (int y = 0; y < kColDeg; ++y) seen |= colour[x + y] >= 0 ? 1 << colour[x + y] : 8;
            proper = seen == 7;
        }
        if (!proper) {
            colour.resize(ids.size());
            for (size_t x = 0; x < ids.size(); ++x) colour[x] = (int)(x % kColDeg);
        }
        for (size_t x = 0; x < ids.size(); ++x) {
            const int e = ids[x], j = col_idx[e];
            out->col[(size_t)j * kColDeg + colour[x]] = ((uint32_t)out->addr[e] << 16) | (uint32_t)erow[e];
        }
    }
    return true;
}

}  // namespace bsd

namespace bsd {

namespace {

constexpr int kMaxColour = 16;
constexpr int kPatience = 4;

// proper colouring with `ncol` colours of the edges of one column group whose
// banks each hold at most ncol of its edges and whose columns have at most
// ncol edges (Koenig's theorem; alternating paths, as colour_group)
void colour_group_n(const std::vector<int>& eu, const std::vector<int>& ev, int ncol, std::vector<int>* colour)
{
    const int n = (int)eu.size();
    colour->assign(n, -1);
    int atU[32][kMaxColour], atV[32][kMaxColour];
    for (int a = 0; a < 32; ++a)
        for (int c = 0; c < kMaxColour; ++c) atU[a][c] = atV[a][c] = -1;
    for (int i = 0; i < n; ++i) {
        const int u = eu[i], v = ev[i];
        int a = -1, b = -1;
        for (int c = 0; c < ncol && a < 0; ++c)
            if (atU[u][c] < 0) a = c;
        for (int c = 0; c < ncol && b < 0; ++c)
            if (atV[v][c] < 0) b = c;
        if (atV[v][a] >= 0) {
            std::vector<int> path;
            int x = v, side = 1, c = a;
            while ((int)path.size() <= n) {
                const int e = side ? atV[x][c] : atU[x][c];
                if (e < 0) break;
                path.push_back(e);
                x = side ? eu[e] : ev[e];
                side ^= 1;
                c = (c == a) ? b : a;
            }
            for (int e : path) {
                atU[eu[e]][(*colour)[e]] = -1;
                atV[ev[e]][(*colour)[e]] = -1;
            }
            for (int e : path) {
                const int ce = (*colour)[e] == a ? b : a;
                (*colour)[e] = ce;
                atU[eu[e]][ce] = e;
                atV[ev[e]][ce] = e;
            }
        }
        (*colour)[i] = a;
        atU[u][a] = i;
        atV[v][a] = i;
    }
}

}  // namespace

bool generic_layout(int M, int N, const int* row_ptr, const int* col_idx, int colK, GenericLayout* out)
{
    if (M < 1 || N < 1 || colK < 1 || colK > kMaxColour) return false;
    const int E = row_ptr[M];
    if (E > kGenericLayoutMaxEdges) return false;
    std::vector<int> cdeg(N, 0);
    for (int e = 0; e < E; ++e) cdeg[col_idx[e]]++;
    for (int j = 0; j < N; ++j)
        if (cdeg[j] > colK) return false;
    const int NG = (N + 31) / 32;
    std::vector<int> cap(NG, 0);                  // the largest column degree of each group
    for (int j = 0; j < N; ++j) cap[j >> 5] = std::max(cap[j >> 5], cdeg[j]);
    // position of every CSR edge inside its row's storage window: start from
    // the CSR order and swap within rows while the bank loads above each
    // group's cap fall
    std::vector<int> pos(E);
    for (int e = 0; e < E; ++e) pos[e] = e;
    std::vector<int> cnt((size_t)NG * 32, 0);
    for (int e = 0; e < E; ++e) cnt[(size_t)(col_idx[e] >> 5) * 32 + (pos[e] & 31)]++;
    auto over = [&](int g, int b) { return std::max(0, cnt[(size_t)g * 32 + b] - cap[g]); };
    int ex = 0;
    for (int g = 0; g < NG; ++g)
        for (int b = 0; b < 32; ++b) ex += over(g, b);
    Rng rng{0x243f6a8885a308d3ull};
    std::vector<int> order(M);
    for (int i = 0; i < M; ++i) order[i] = i;
    // a bounded effort: at most ~5e7 swap trials, and kPatience sweeps
    // without a lower load end the search
    double per_sweep = 1.0;
    for (int i = 0; i < M; ++i) {
        const double d = row_ptr[i + 1] - row_ptr[i];
        per_sweep += d * (d - 1) / 2;
    }
    const int max_sweeps = (int)std::min<double>(kSweeps, 5e7 / per_sweep);
    int best = ex, stale = 0;
    for (int sw = 0; sw < max_sweeps && ex > 0 && stale < kPatience; ++sw) {
        if (ex < best) { best = ex; stale = 0; } else if (sw > 0) { ++stale; }
        for (int i = M - 1; i > 0; --i) std::swap(order[i], order[rng.below((uint32_t)i + 1)]);
        for (int i : order) {
            for (int a = row_ptr[i]; a < row_ptr[i + 1]; ++a) {
                for (int b = a + 1; b < row_ptr[i + 1]; ++b) {
                    const int ga = col_idx[a] >> 5, gb = col_idx[b] >> 5;
                    if (ga == gb) continue;
                    const int ba = pos[a] & 31, bb = pos[b] & 31;
                    const int before = over(ga, ba) + over(gb, bb) + over(ga, bb) + over(gb, ba);
                    cnt[(size_t)ga * 32 + ba]--; cnt[(size_t)gb * 32 + bb]--;
                    cnt[(size_t)ga * 32 + bb]++; cnt[(size_t)gb * 32 + ba]++;
                    const int after = over(ga, ba) + over(gb, bb) + over(ga, bb) + over(gb, ba);
                    if (after < before || (after == before && rng.below(4) == 0)) {
                        std::swap(pos[a], pos[b]);
                        ex += after - before;
                    } else {
                        cnt[(size_t)ga * 32 + ba]++; cnt[(size_t)gb * 32 + bb]++;
                        cnt[(size_t)ga * 32 + bb]--; cnt[(size_t)gb * 32 + ba]--;
                    }
                }
            }
        }
    }
    out->pos = pos;
    out->excess = ex;
    // the k slot of every column's edges: a proper colouring per group where
    // the loads allow one (holes where a column has fewer edges than colours),
    // else the column lists' order
    std::vector<std::vector<int>> cedges(N);
    for (int e = 0; e < E; ++e) cedges[col_idx[e]].push_back(e);
    out->kedge.assign((size_t)colK * N, -1);
    for (int g = 0; g < NG; ++g) {
        std::vector<int> ids, eu, ev, colour;
        for (int j = 32 * g; j < std::min(N, 32 * g + 32); ++j)
            for (int e : cedges[j]) {
                ids.push_back(e);
                eu.push_back(j - 32 * g);
                ev.push_back(pos[e] & 31);
            }
        int vdeg[32] = {0};
        for (int v : ev) vdeg[v]++;
        bool proper = cap[g] > 0 && *std::max_element(vdeg, vdeg + 32) <= cap[g];
        if (proper) colour_group_n(eu, ev, cap[g], &colour);
        // every column's edges take distinct slots below colK
        if (proper) {
            std::vector<int> seen((size_t)32 * kMaxColour, 0);
            for (size_t x = 0; x < ids.size() && proper; ++x) {
                const int c = colour[x];
                if (c < 0 || c >= colK || seen[(size_t)eu[x] * kMaxColour + c]++) proper = false;
            }
        }
        if (!proper) {
            // greedy: each edge takes the free slot of its column whose bank
            // is least loaded so far
            colour.assign(ids.size(), 0);
            std::vector<int> load((size_t)colK * 32, 0);
            for (size_t x = 0; x < ids.size();) {
                size_t y = x;
                while (y < ids.size() && eu[y] == eu[x]) ++y;
                uint32_t used = 0;
                for (size_t z = x; z < y; ++z) {
                    int bestk = -1;
                    for (int k = 0; k < colK; ++k) {
                        if ((used >> k) & 1u) continue;
                        if (bestk < 0 || load[(size_t)k * 32 + ev[z]] < load[(size_t)bestk * 32 + ev[z]]) bestk = k;
                    }
                    colour[z] = bestk;
                    used |= 1u << bestk;
                    load[(size_t)bestk * 32 + ev[z]]++;
                }
                x = y;
            }
        }
        for (size_t x = 0; x < ids.size(); ++x) out->kedge[(size_t)colour[x] * N + col_idx[ids[x]]] = ids[x];
    }
    return true;
}

}  // namespace bsd

extern "C" int bsd_small_layout(int32_t M, int32_t N, const int32_t* H_row_ptr, const int32_t* H_col_idx,
                                int32_t* plane, int32_t* edge_word, int32_t* col_word, int32_t* extent,
                                int32_t* excess)
{
    if (M < 1 || N < 1 || !H_row_ptr || !H_col_idx || !plane || !edge_word || !col_word || !extent || !excess)
        return BSD_ERR_INVALID_ARG;
    if (H_row_ptr[0] != 0) return BSD_ERR_INVALID_ARG;
    for (int i = 0; i < M; ++i) {
        if (H_row_ptr[i + 1] < H_row_ptr[i]) return BSD_ERR_INVALID_ARG;
        for (int e = H_row_ptr[i]; e < H_row_ptr[i + 1]; ++e) {
            if (H_col_idx[e] < 0 || H_col_idx[e] >= N) return BSD_ERR_INVALID_ARG;
            if (e > H_row_ptr[i] && H_col_idx[e] <= H_col_idx[e - 1]) return BSD_ERR_INVALID_ARG;
        }
    }
    bsd::SmallLayout sl;
    if (!bsd::small_layout(M, N, H_row_ptr, H_col_idx, &sl)) return BSD_ERR_UNSUPPORTED;
    for (int h = 0; h < 3; ++h) plane[h] = sl.A[h];
    for (size_t e = 0; e < sl.addr.size(); ++e) edge_word[e] = sl.addr[e];
    for (size_t q = 0; q < sl.col.size(); ++q) col_word[q] = (int32_t)(sl.col[q] >> 16);
    *extent = sl.extent;
    *excess = sl.excess;
    return BSD_OK;
}

extern "C" int bsd_generic_layout(int32_t M, int32_t N, const int32_t* H_row_ptr, const int32_t* H_col_idx,
                                  int32_t* edge_word, int32_t* slot_edge, int32_t* colK, int32_t* excess)
{
    if (M < 1 || N < 1 || !H_row_ptr || !H_col_idx || !edge_word || !slot_edge || !colK || !excess)
        return BSD_ERR_INVALID_ARG;
    if (H_row_ptr[0] != 0) return BSD_ERR_INVALID_ARG;
    for (int i = 0; i < M; ++i) {
        if (H_row_ptr[i + 1] < H_row_ptr[i]) return BSD_ERR_INVALID_ARG;
        for (int e = H_row_ptr[i]; e < H_row_ptr[i + 1]; ++e) {
            if (H_col_idx[e] < 0 || H_col_idx[e] >= N) return BSD_ERR_INVALID_ARG;
            if (e > H_row_ptr[i] && H_col_idx[e] <= H_col_idx[e - 1]) return BSD_ERR_INVALID_ARG;
        }
    }
    const int E = H_row_ptr[M];
    std::vector<int> cdeg(N, 0);
    for (int e = 0; e < E; ++e) cdeg[H_col_idx[e]]++;
    const int max_col = N > 0 ? *std::max_element(cdeg.begin(), cdeg.end()) : 0;
    if (max_col > 6) return BSD_ERR_UNSUPPORTED;
    const int K = max_col <= 3 ? 3 : 6;
    bsd::GenericLayout gl;
    if (!bsd::generic_layout(M, N, H_row_ptr, H_col_idx, K, &gl)) return BSD_ERR_UNSUPPORTED;
    for (int e = 0; e < E; ++e) edge_word[e] = gl.pos[e];
    for (size_t q = 0; q < gl.kedge.size(); ++q) slot_edge[q] = gl.kedge[q];
    *colK = K;
    *excess = gl.excess;
    return BSD_OK;
}
