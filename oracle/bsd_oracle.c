/*
 * bsd_oracle.c -- plain CPU oracle for the BP-guided beam search decoder.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this code.  It shares no code, header, table or
 * helper with the CUDA library; it is written from the paper directly:
 *
 *   App. A, Eqs. 1-4   min-sum belief propagation (flooding schedule)
 *   Alg. 2             masked_BP
 *   Alg. 3 + App. B    beam search decoder (bounded insert, descending-score
 *                      exploration, num_results termination, minimum weight)
 *
 * It is deliberately slow and literal: every D_{i->j} recomputes its minimum
 * over the other neighbours of d_i, every E_{j->i} re-adds the other incoming
 * messages of e_j, and pruning uses the on-the-fly insert of App. B.
 *
 * The file is compiled twice:
 *   default            real = double  (the reference arithmetic)
 *   -DORACLE_FP32      real = float   (the same algorithm at single precision,
 *                                       used to compare integer decisions such
 *                                       as hard decisions, argmin and pruning
 *                                       with a single-precision implementation
 *                                       taken at the same precision)
 *
 * Readings of points the paper leaves open (each applies to both builds):
 *   R1  D = alpha * (-1)^{s_i} * prod sign * min   (alpha = 1 is Eq. 1 as printed)
 *   R2  sign(x) = -1 iff x < 0
 *   R3  a minimum over an empty set (a check with no other unmasked
 *       neighbour) is L_MAX
 *   R4  every stored E_{j->i} is clamped to [-L_MAX, L_MAX]
 *   R5  the sums of Eqs. 2-3 start from Lambda_j and add the detector messages
 *       in ascending order of value, so the rounded sum depends only on the
 *       multiset of messages (equal inputs give equal outputs at any node)
 *   R6  sum_LLR covers the iterations t = 1..iters actually run by that call
 *   R7  argmin ties go to the lowest index
 *   R8  pruning keeps the top beam_width under (score desc, canonical index
 *       asc); among equal minima the latest inserted path is ejected
 *   R9  a path whose unmasked set is empty has no next_pos and no children
 *   R10 when no return happens, the result is the minimum-weight element of
 *       results if any (CONVERGED), else the hard decision of the best path of
 *       the final set with masked values filled (FAILED)
 *   R11 results are deduplicated by exact equality; equal weights keep the
 *       element found first
 *   R15 16-bit message storage (float build, msg_storage 1 / 2): every stored
 *       E_{j->i}, E(0) included, is the float result rounded to binary16 /
 *       bfloat16 to nearest even, a zero stored as +0, and L_MAX is taken at
 *       its stored value; every sum is formed in float
 *   R16 near-tie flag (tie_guard > 0): set when the seed path (if rounds
 *       follow) or any visited child with a next_pos has a relative margin
 *       between its smallest and second smallest |sum_LLR| strictly inside
 *       (0, tie_guard), or when the score margin between the last kept and
 *       the first dropped child of a round (before the last round) is; exact
 *       ties are not flagged, since R5, R7 and R8 decide them the same way in
 *       any precision
 *   R17 weighted min-sum: a weight w[t'][e] per edge in place of alpha, with
 *       t' = min(t, T) - 1 and t counted from 1 in every BP call
 *   R19 near-tie log (every build): each decision taken in floating point is
 *       logged with its relative margin -- the sign of every Lambda_j(t) and
 *       E_{j->i}(t) formed (|sum| / max(1, sum of |terms|)), every argmin
 *       (second smallest minus smallest over max(1, second)), the order of
 *       each round's kept set and, before the last round, the boundary
 *       between the last kept and the first dropped child ((a - b) /
 *       max(1, |a|)), and the choice of minimum weight among results; a
 *       margin of exactly 0 is an exact tie.  Per shot: the smallest nonzero
 *       margin and the number of exact ties, and on request the decision log
 *       (oracle_decode_logged) that places each one in the run
 *   Score and weight arithmetic:
 *     double build: score = (sum over U of |sum_LLR[j]| added in ascending
 *                   order) / iters; weight = sum of Lambda_j over the support
 *                   added in ascending order.
 *     float build:  each |sum_LLR[j]| (resp. Lambda_j) is taken to the fixed
 *                   point grid 2^-16 (round to nearest even), summed exactly in
 *                   int64, and score = (double)S * 2^-16 / iters.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef ORACLE_FP32
typedef float real;
#define R_ABS fabsf
#else
typedef double real;
#define R_ABS fabs
#endif

#define FIX_SCALE 65536.0

/* ------------------------------------------------------------------------- */
/* public structs (mirrored by the ctypes wrapper)                            */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t max_rounds;
    int32_t beam_width;
    int32_t initial_iters;
    int32_t iters_per_round;
    int32_t num_results;
    int32_t prune_mode;      /* 0: on-the-fly insert (App. B); 1: collect then prune (Alg. 3) */
    double ms_scale;         /* alpha of R1 */
    double llr_clamp;        /* L_MAX of R3/R4 */
    int32_t msg_storage;     /* float build: 0 messages kept in float, 1 binary16, 2 bfloat16 */
    int32_t pad0;
    double tie_guard;        /* near-tie flag threshold on argmin and pruning margins (0: off) */
    const float *weights;    /* optional [weights_iters][E] per-edge weights in place of alpha, CSR edge order */
    int32_t weights_iters;   /* iteration t of a BP call uses row min(t, weights_iters) - 1 */
    int32_t pad1;
} oracle_params;

typedef struct {
    int32_t cap;             /* capacity of the per-child arrays */
    int32_t n;               /* children recorded */
    int32_t *round, *canon, *parent_rank, *val, *pos, *success, *iters, *next_pos, *kept;
    double *score;
    int32_t seed_iters, seed_success, seed_next_pos;
    int32_t ret_round;       /* where the search stopped early: 0 = seed, r = round r, -1 = ran out */
    int32_t ret_canon;       /* canonical index (2 * parent rank + val) of the child that stopped it */
} oracle_trace;

typedef struct {
    int M, N, K, E;
    int *row_ptr, *col_idx, *edge_row;   /* CSR of H; edge e = (edge_row[e], col_idx[e]) */
    int *col_ptr, *col_edge;             /* per column: its CSR edge ids, rows ascending */
    int *a_row_ptr, *a_col_idx;          /* CSR of A */
    double *p;
    real *lam;                           /* Lambda_j = log((1-p_j)/p_j) */
} oracle_graph;

/* ------------------------------------------------------------------------- */
/* graph                                                                      */
/* ------------------------------------------------------------------------- */
void oracle_graph_destroy(oracle_graph *g)
{
    if (!g) return;
    free(g->row_ptr); free(g->col_idx); free(g->edge_row);
    free(g->col_ptr); free(g->col_edge);
    free(g->a_row_ptr); free(g->a_col_idx);
    free(g->p); free(g->lam);
    free(g);
}

oracle_graph *oracle_graph_create(int M, int N, int K,
                                  const int32_t *H_row_ptr, const int32_t *H_col_idx,
                                  const int32_t *A_row_ptr, const int32_t *A_col_idx,
                                  const double *priors)
{
    oracle_graph *g = (oracle_graph *)calloc(1, sizeof(*g));
    int E = H_row_ptr[M];
    g->M = M; g->N = N; g->K = K; g->E = E;
    g->row_ptr = (int *)malloc(sizeof(int) * (M + 1));
    g->col_idx = (int *)malloc(sizeof(int) * (E > 0 ? E : 1));
    g->edge_row = (int *)malloc(sizeof(int) * (E > 0 ? E : 1));
    for (int i = 0; i <= M; ++i) g->row_ptr[i] = H_row_ptr[i];
    for (int i = 0; i < M; ++i)
        for (int e = H_row_ptr[i]; e < H_row_ptr[i + 1]; ++e) {
            g->col_idx[e] = H_col_idx[e];
            g->edge_row[e] = i;
        }
    /* neighbourhoods N(e_j): scan rows in order, so each column lists its
       edges with ascending row index */
    g->col_ptr = (int *)calloc((size_t)N + 1, sizeof(int));
    for (int e = 0; e < E; ++e) g->col_ptr[g->col_idx[e] + 1]++;
    for (int j = 0; j < N; ++j) g->col_ptr[j + 1] += g->col_ptr[j];
    g->col_edge = (int *)malloc(sizeof(int) * (E > 0 ? E : 1));
    int *fill = (int *)calloc((size_t)(N > 0 ? N : 1), sizeof(int));
    for (int e = 0; e < E; ++e) {
        int j = g->col_idx[e];
        g->col_edge[g->col_ptr[j] + fill[j]++] = e;
    }
    free(fill);
    g->a_row_ptr = (int *)malloc(sizeof(int) * (K + 1));
    int EA = A_row_ptr[K];
    g->a_col_idx = (int *)malloc(sizeof(int) * (EA > 0 ? EA : 1));
    for (int i = 0; i <= K; ++i) g->a_row_ptr[i] = A_row_ptr[i];
    for (int e = 0; e < EA; ++e) g->a_col_idx[e] = A_col_idx[e];
    g->p = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    g->lam = (real *)malloc(sizeof(real) * (size_t)(N > 0 ? N : 1));
    for (int j = 0; j < N; ++j) {
        g->p[j] = priors[j];
        /* prior LLR of App. A: Lambda_j = log((1 - p_j) / p_j) */
        g->lam[j] = (real)log((1.0 - priors[j]) / priors[j]);
    }
    return g;
}

/* ------------------------------------------------------------------------- */
/* 16-bit message storage (float build only)                                  */
/* ------------------------------------------------------------------------- */
/* Nearest binary16 value of a float, ties to even, as a float: 10 fraction
   bits for magnitudes from 2^-14 (normal), multiples of 2^-24 below it
   (subnormal), infinity from 65520 up. */
static float round_binary16(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    const uint32_t sign = u & 0x80000000u;
    uint32_t a = u & 0x7fffffffu;
    float ax;
    memcpy(&ax, &a, 4);
    if (a >= 0x7f800000u) return x;
    if (ax >= 65520.0f) {
        a = 0x7f800000u;
    } else if (ax >= 6.103515625e-05f) {            /* 2^-14: keep 10 of 23 fraction bits */
        const uint32_t rem = a & 0x1fffu, base = a & ~0x1fffu;
        a = base;
        if (rem > 0x1000u || (rem == 0x1000u && (base & 0x2000u))) a += 0x2000u;
    } else {                                         /* subnormal: multiples of 2^-24 */
        const float q = nearbyintf(ax * 16777216.0f);
        const float r = q * 5.9604644775390625e-08f;
        memcpy(&a, &r, 4);
    }
    a |= sign;
    float y;
    memcpy(&y, &a, 4);
    return y;
}

/* Nearest bfloat16 value of a float (8 significant bits), ties to even. */
static float round_bfloat16(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7fffffffu) >= 0x7f800000u) return x;
    const uint32_t rem = u & 0xffffu, base = u & 0xffff0000u;
    u = base;
    if (rem > 0x8000u || (rem == 0x8000u && (base & 0x10000u))) u += 0x10000u;
    float y;
    memcpy(&y, &u, 4);
    return y;
}

/* A stored message: rounded to the storage format, and a zero is stored as
   +0 (R2 gives -0 and +0 the same sign, so this changes no decision). */
static real store_msg(const oracle_params *prm, real x)
{
#ifdef ORACLE_FP32
    if (prm->msg_storage == 1) x = round_binary16(x);
    else if (prm->msg_storage == 2) x = round_bfloat16(x);
    if (prm->msg_storage != 0 && x == 0) x = 0;
#else
    (void)prm;
#endif
    return x;
}

/* L_MAX as the storage format holds it */
static real clamp_value(const oracle_params *prm)
{
    return store_msg(prm, (real)prm->llr_clamp);
}

void oracle_round_storage(float *x, int n, int mode)
{
    for (int k = 0; k < n; ++k) x[k] = mode == 1 ? round_binary16(x[k]) : mode == 2 ? round_bfloat16(x[k]) : x[k];
}

/* ------------------------------------------------------------------------- */
/* masked BP (Alg. 2); plain BP is the case with no masked node              */
/* ------------------------------------------------------------------------- */
typedef struct {
    /* inputs */
    const real *E_in;        /* E_{j->i}(0) per CSR edge */
    const uint8_t *masked;   /* N: 1 if e_j appears in pos_val_pairs */
    const uint8_t *val;      /* N: its value v */
    const uint8_t *s;        /* M: the original syndrome */
    int max_iters;
    int stop_on_success;     /* 1: return at the first t with H e(t) = s' (Alg. 2) */
    /* outputs */
    real *E_out;             /* E(t) of the last iteration run */
    real *sum_llr;           /* N: sum over t of Lambda_j(t) (R6); masked: 0 */
    uint8_t *ehat;           /* N: e(t) of the last iteration, masked positions = v */
    real *llr_traj;          /* optional [max_iters][N]: Lambda_j(t) */
    int iters;               /* iterations actually run */
    int success;             /* H e(t) = s' held at the last iteration run */
    int first_success;       /* first t with H e(t) = s', 0 if none */
    double min_gap;          /* smallest relative sign margin met (double build) */
} bp_call;

typedef struct {
    uint8_t *sp;             /* M: syndrome with masked ones folded in */
    real *D;                 /* E: detector-to-error messages */
    real *post;              /* N: Lambda_j(t) */
    real *vbuf;              /* max column degree */
    int *ebuf;
} bp_work;

/* Near-tie log of the decisions taken in floating point (a sign, an argmin,
   a score order, a weight order): the smallest nonzero relative margin, and
   the number of exact ties (margin 0).  R5 and R7 settle an exact tie the
   same way in any precision only when both precisions compute equal values;
   a lower precision can also split an exact tie of this build.

   The relative margin of a sign decision on a sum is |sum| / max(1, sum of
   the magnitudes of its terms); of an order decision between a > b it is
   (a - b) / max(1, |a|). */
static int g_ties_tls_dummy;
static _Thread_local int *g_tie_counter = &g_ties_tls_dummy;

static void margin_note(double *g, int *nties, double value, double scale)
{
    double s = scale > 1.0 ? scale : 1.0;
    double r = fabs(value) / s;
    if (r == 0) { ++*nties; return; }
    if (r < *g) *g = r;
}

static void gap_update(double *g, double value, double scale)
{
    margin_note(g, g_tie_counter, value, scale);
}

/* Decision log (optional, one shot at a time): one record per decision
   group, in the order the sequential algorithm takes them, so that two runs
   of the same shot (double and single precision) can be compared record by
   record up to their first different outcome.
     kind 0  BP iteration t of a call: key = hash of the signs of every
             stored E_{j->i}(t) and of e^(t); margins of the signs of every
             Lambda_j(t) and E_{j->i}(t) formed (Eqs. 2-4)
     kind 1  next_pos of a call (Alg. 3 argmin): key = next_pos; margin
             between the smallest and second smallest |sum_LLR|
     kind 2  the kept set of a round (Alg. 3 pruning, App. B): key = hash of
             the kept canonical indices in rank order; margins between
             consecutive kept scores and, before the last round, between the
             last kept and the first dropped child
     kind 3  the returned element of results (App. B minimum weight): key =
             its index; margins between its weight and every other
   Calls are numbered in visit order: 0 the seed BP, then every child. */
typedef struct {
    int32_t cap, n;
    int32_t *call, *round, *t, *kind, *nties;
    uint64_t *key;
    double *gap;             /* smallest nonzero relative margin of the record (inf if none) */
} oracle_dlog;

static _Thread_local oracle_dlog *g_dlog = NULL;
static _Thread_local int g_call = 0, g_round = 0;

static void log_push(int kind, int t, uint64_t key, double gap, int nties)
{
    oracle_dlog *d = g_dlog;
    if (!d || d->n >= d->cap) return;
    const int k = d->n++;
    d->call[k] = g_call; d->round[k] = g_round; d->t[k] = t; d->kind[k] = kind;
    d->key[k] = key; d->gap[k] = gap; d->nties[k] = nties;
}

/* 64-bit FNV-1a over a sequence of small values */
static uint64_t fnv_add(uint64_t h, uint64_t v)
{
    for (int b = 0; b < 8; ++b) {
        h ^= (v >> (8 * b)) & 0xffu;
        h *= 1099511628211ull;
    }
    return h;
}
#define FNV_INIT 14695981039346656037ull

static void masked_bp(const oracle_graph *g, const oracle_params *prm, bp_call *c, bp_work *w)
{
    const int M = g->M, N = g->N, E = g->E;
    const real alpha = (real)prm->ms_scale;
    const real LMAX = clamp_value(prm);
    uint8_t *sp = w->sp;

    /* syndrome pre-processing: flip s_i for every detector of a node fixed to 1 */
    memcpy(sp, c->s, (size_t)M);
    for (int j = 0; j < N; ++j)
        if (c->masked[j] && c->val[j])
            for (int k = g->col_ptr[j]; k < g->col_ptr[j + 1]; ++k)
                sp[g->edge_row[g->col_edge[k]]] ^= 1;

    /* warm start: E(0) = edge_msgs */
    if (E) memcpy(c->E_out, c->E_in, sizeof(real) * (size_t)E);
    real *Em = c->E_out;
    for (int j = 0; j < N; ++j) c->sum_llr[j] = 0;
    c->iters = 0;
    c->success = 0;
    c->first_success = 0;
    c->min_gap = INFINITY;

    for (int t = 1; t <= c->max_iters; ++t) {
        /* weighted min-sum: w_{e,t} in place of alpha, t counted from 1 in
           every BP call, the last row reused beyond weights_iters */
        const float *wt = NULL;
        if (prm->weights && prm->weights_iters > 0)
            wt = prm->weights + (size_t)((t < prm->weights_iters ? t : prm->weights_iters) - 1) * (size_t)E;
        /* Eq. 1, ignoring masked nodes: D_{i->j} is not formed for a masked j,
           and masked neighbours j' do not enter the product or the minimum */
        for (int i = 0; i < M; ++i) {
            for (int e = g->row_ptr[i]; e < g->row_ptr[i + 1]; ++e) {
                int j = g->col_idx[e];
                if (c->masked[j]) continue;
                real mn = LMAX;                      /* R3 */
                int neg = sp[i];
                for (int e2 = g->row_ptr[i]; e2 < g->row_ptr[i + 1]; ++e2) {
                    if (e2 == e) continue;
                    int j2 = g->col_idx[e2];
                    if (c->masked[j2]) continue;
                    real x = Em[e2];
                    real ax = R_ABS(x);
                    if (ax < mn) mn = ax;
                    if (x < 0) neg ^= 1;             /* R2 */
                }
                real d = (wt ? (real)wt[e] : alpha) * mn;   /* R1 */
                w->D[e] = neg ? -d : d;
            }
        }
        /* Eqs. 2-3 for unmasked nodes, summing in ascending order (R5) */
        double it_gap = INFINITY;
        int it_ties = 0;
        for (int j = 0; j < N; ++j) {
            if (c->masked[j]) { w->post[j] = 0; continue; }
            int deg = g->col_ptr[j + 1] - g->col_ptr[j];
            for (int k = 0; k < deg; ++k) {
                int e = g->col_edge[g->col_ptr[j] + k];
                real v = w->D[e];
                int pos = k;
                while (pos > 0 && w->vbuf[pos - 1] > v) {   /* insertion sort */
                    w->vbuf[pos] = w->vbuf[pos - 1];
                    w->ebuf[pos] = w->ebuf[pos - 1];
                    --pos;
                }
                w->vbuf[pos] = v;
                w->ebuf[pos] = e;
            }
            real post = g->lam[j];
            double scale = fabs((double)g->lam[j]);
            for (int k = 0; k < deg; ++k) {
                post += w->vbuf[k];
                scale += fabs((double)w->vbuf[k]);
            }
            w->post[j] = post;                       /* Eq. 3 */
            margin_note(&it_gap, &it_ties, (double)post, scale);
            for (int k = 0; k < deg; ++k) {          /* Eq. 2: leave d_i out */
                real acc = g->lam[j];
                double sc = fabs((double)g->lam[j]);
                for (int k2 = 0; k2 < deg; ++k2) {
                    if (k2 == k) continue;
                    acc += w->vbuf[k2];
                    sc += fabs((double)w->vbuf[k2]);
                }
                margin_note(&it_gap, &it_ties, (double)acc, sc);
                if (acc > LMAX) acc = LMAX;          /* R4 */
                if (acc < -LMAX) acc = -LMAX;
                Em[w->ebuf[k]] = store_msg(prm, acc);
            }
            c->sum_llr[j] += post;                   /* R6 */
        }
        /* Eq. 4; masked positions are 0 while checking */
        for (int j = 0; j < N; ++j)
            c->ehat[j] = c->masked[j] ? 0 : (uint8_t)(w->post[j] <= 0);
        if (c->llr_traj)
            for (int j = 0; j < N; ++j) c->llr_traj[(size_t)(t - 1) * N + j] = w->post[j];
        if (it_gap < c->min_gap) c->min_gap = it_gap;
        *g_tie_counter += it_ties;
        if (g_dlog) {
            uint64_t h = FNV_INIT;
            for (int e = 0; e < E; ++e) h = fnv_add(h, Em[e] < 0);
            for (int j = 0; j < N; ++j) h = fnv_add(h, c->ehat[j]);
            log_push(0, t, h, it_gap, it_ties);
        }
        c->iters = t;
        /* stopping rule: H e(t) = s' */
        int ok = 1;
        for (int i = 0; i < M && ok; ++i) {
            int par = sp[i];
            for (int e = g->row_ptr[i]; e < g->row_ptr[i + 1]; ++e) par ^= c->ehat[g->col_idx[e]];
            if (par) ok = 0;
        }
        c->success = ok;
        if (ok && !c->first_success) c->first_success = t;
        if (ok && c->stop_on_success) break;
    }
    /* masked positions take their fixed values */
    for (int j = 0; j < N; ++j)
        if (c->masked[j]) c->ehat[j] = c->val[j];
}

/* ------------------------------------------------------------------------- */
/* score, weight, argmin                                                     */
/* ------------------------------------------------------------------------- */
static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

#ifdef ORACLE_FP32
static int64_t fixq(real x) { return (int64_t)llrint((double)x * FIX_SCALE); }
#endif

/* sum over U of |sum_LLR[j]|, divided by iters (Alg. 3) */
static double path_score(const oracle_graph *g, const real *sum_llr, const uint8_t *masked,
                         int iters, double *tmp)
{
#ifdef ORACLE_FP32
    (void)tmp;
    int64_t S = 0;
    for (int j = 0; j < g->N; ++j)
        if (!masked[j]) S += fixq(R_ABS(sum_llr[j]));
    return ((double)S / FIX_SCALE) / (double)iters;
#else
    int n = 0;
    for (int j = 0; j < g->N; ++j)
        if (!masked[j]) tmp[n++] = fabs(sum_llr[j]);
    qsort(tmp, (size_t)n, sizeof(double), cmp_double);
    double S = 0;
    for (int k = 0; k < n; ++k) S += tmp[k];
    return S / (double)iters;
#endif
}

/* wt(e) = sum_j e_j log((1-p_j)/p_j)  (App. B) */
static double error_weight(const oracle_graph *g, const uint8_t *e, double *tmp)
{
#ifdef ORACLE_FP32
    (void)tmp;
    int64_t S = 0;
    for (int j = 0; j < g->N; ++j)
        if (e[j]) S += fixq(g->lam[j]);
    return (double)S;
#else
    int n = 0;
    for (int j = 0; j < g->N; ++j)
        if (e[j]) tmp[n++] = g->lam[j];
    qsort(tmp, (size_t)n, sizeof(double), cmp_double);
    double S = 0;
    for (int k = 0; k < n; ++k) S += tmp[k];
    return S;
#endif
}

/* least reliable unmasked node: argmin |sum_LLR[j]|, lowest index on ties (R7);
   also reports the gap to the runner-up for near-tie logging */
static int least_reliable(const oracle_graph *g, const real *sum_llr, const uint8_t *masked,
                          double *gap_rel)
{
    int best = -1;
    real bv = 0, second = 0;
    int have_second = 0;
    for (int j = 0; j < g->N; ++j) {
        if (masked[j]) continue;
        real v = R_ABS(sum_llr[j]);
        if (best < 0 || v < bv) {
            if (best >= 0) { second = bv; have_second = 1; }
            best = j; bv = v;
        } else if (!have_second || v < second) {
            second = v; have_second = 1;
        }
    }
    if (gap_rel) {
        *gap_rel = INFINITY;
        if (best >= 0 && have_second) {
            double s = fabs((double)second) > 1.0 ? fabs((double)second) : 1.0;
            *gap_rel = ((double)second - (double)bv) / s;
        }
    }
    return best;
}

/* ------------------------------------------------------------------------- */
/* beam search (Alg. 3)                                                       */
/* ------------------------------------------------------------------------- */
typedef struct {
    real *E;                 /* edge_msgs */
    uint8_t *masked, *val;   /* pos_val_pairs as node flags */
    int next_pos;
    double score;
    int canon;               /* insertion order within the round */
    int trace_idx;
    uint8_t *ehat;           /* last hard decision, masked filled (R10) */
} path_t;

typedef struct {
    const oracle_graph *g;
    const oracle_params *prm;
    bp_work w;
    bp_call c;
    double *tmp;
    path_t *cur, *nxt;       /* beam_width (or 2*beam_width in collect mode) paths */
    int ncur, nnxt, cap;
    real *E_seed;
    real *sum_llr;
    uint8_t *ehat;
    uint8_t *cmask, *cval;   /* child's pos_val_pairs */
    uint8_t *results;        /* num_results * N */
    double *res_w;
    int nres;
    int res_from_round, res_from_canon;
    double *rscore;          /* scores of the current round's children, for the pruning margin */
    int *rcanon;
    int nr;
    int near_tie;            /* an argmin or pruning margin fell in (0, tie_guard) */
} dec_ctx;

static void path_alloc(path_t *p, int E, int N)
{
    p->E = (real *)malloc(sizeof(real) * (size_t)(E > 0 ? E : 1));
    p->masked = (uint8_t *)malloc((size_t)N);
    p->val = (uint8_t *)malloc((size_t)N);
    p->ehat = (uint8_t *)malloc((size_t)N);
}

static void path_free(path_t *p)
{
    free(p->E); free(p->masked); free(p->val); free(p->ehat);
}

static void path_swap(path_t *a, path_t *b)
{
    path_t t = *a; *a = *b; *b = t;
}

static dec_ctx *ctx_new(const oracle_graph *g, const oracle_params *prm)
{
    dec_ctx *x = (dec_ctx *)calloc(1, sizeof(*x));
    int N = g->N, M = g->M, E = g->E;
    int maxdeg = 1;
    for (int j = 0; j < N; ++j) {
        int d = g->col_ptr[j + 1] - g->col_ptr[j];
        if (d > maxdeg) maxdeg = d;
    }
    x->g = g; x->prm = prm;
    x->w.sp = (uint8_t *)malloc((size_t)(M > 0 ? M : 1));
    x->w.D = (real *)malloc(sizeof(real) * (size_t)(E > 0 ? E : 1));
    x->w.post = (real *)malloc(sizeof(real) * (size_t)(N > 0 ? N : 1));
    x->w.vbuf = (real *)malloc(sizeof(real) * (size_t)maxdeg);
    x->w.ebuf = (int *)malloc(sizeof(int) * (size_t)maxdeg);
    x->tmp = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    x->cap = prm->beam_width > 0 ? prm->beam_width : 1;
    if (prm->prune_mode == 1) x->cap *= 2;
    x->cur = (path_t *)calloc((size_t)x->cap + 1, sizeof(path_t));
    x->nxt = (path_t *)calloc((size_t)x->cap + 1, sizeof(path_t));
    for (int k = 0; k <= x->cap; ++k) { path_alloc(&x->cur[k], E, N); path_alloc(&x->nxt[k], E, N); }
    x->E_seed = (real *)malloc(sizeof(real) * (size_t)(E > 0 ? E : 1));
    x->sum_llr = (real *)malloc(sizeof(real) * (size_t)(N > 0 ? N : 1));
    x->ehat = (uint8_t *)malloc((size_t)(N > 0 ? N : 1));
    x->cmask = (uint8_t *)malloc((size_t)(N > 0 ? N : 1));
    x->cval = (uint8_t *)malloc((size_t)(N > 0 ? N : 1));
    int nr = prm->num_results > 0 ? prm->num_results : 1;
    x->results = (uint8_t *)malloc((size_t)nr * (size_t)(N > 0 ? N : 1));
    x->res_w = (double *)malloc(sizeof(double) * (size_t)nr);
    x->rscore = (double *)malloc(sizeof(double) * (size_t)(2 * x->cap + 2));
    x->rcanon = (int *)malloc(sizeof(int) * (size_t)(2 * x->cap + 2));
    return x;
}

/* near-tie flag: a decision margin strictly between 0 and tie_guard */
static void tie_check(dec_ctx *x, double gap_rel)
{
    if (x->prm->tie_guard > 0 && gap_rel > 0 && gap_rel < x->prm->tie_guard) x->near_tie = 1;
}

/* margin at the pruning boundary of a round: the relative score gap between
   the last kept child (rank w-1) and the first dropped one (rank w); inf when
   the round has no more than w children (nothing is dropped) */
static double pruning_margin(dec_ctx *x, int w)
{
    if (x->nr <= w) return INFINITY;
    /* rank the round's children by (score desc, canonical index asc) */
    for (int a = 1; a < x->nr; ++a)
        for (int k = a; k > 0; --k) {
            const int before = x->rscore[k] > x->rscore[k - 1] ||
                               (x->rscore[k] == x->rscore[k - 1] && x->rcanon[k] < x->rcanon[k - 1]);
            if (!before) break;
            double ts = x->rscore[k]; x->rscore[k] = x->rscore[k - 1]; x->rscore[k - 1] = ts;
            int tc = x->rcanon[k]; x->rcanon[k] = x->rcanon[k - 1]; x->rcanon[k - 1] = tc;
        }
    const double s0 = x->rscore[w - 1], s1 = x->rscore[w];
    const double den = fabs(s0) > 1.0 ? fabs(s0) : 1.0;
    return (s0 - s1) / den;
}

static void ctx_free(dec_ctx *x)
{
    if (!x) return;
    free(x->w.sp); free(x->w.D); free(x->w.post); free(x->w.vbuf); free(x->w.ebuf);
    free(x->tmp);
    for (int k = 0; k <= x->cap; ++k) { path_free(&x->cur[k]); path_free(&x->nxt[k]); }
    free(x->cur); free(x->nxt);
    free(x->E_seed); free(x->sum_llr); free(x->ehat); free(x->cmask); free(x->cval);
    free(x->results); free(x->res_w);
    free(x->rscore); free(x->rcanon);
    free(x);
}

/* add a valid solution to results (dedupe R11); returns 1 when |results| reached num_results */
static int results_insert(dec_ctx *x, const uint8_t *e, int round, int canon, double *min_gap)
{
    const int N = x->g->N;
    for (int r = 0; r < x->nres; ++r)
        if (memcmp(x->results + (size_t)r * N, e, (size_t)N) == 0) return x->nres >= x->prm->num_results;
    memcpy(x->results + (size_t)x->nres * N, e, (size_t)N);
    x->res_w[x->nres] = error_weight(x->g, e, x->tmp);
    if (x->nres == 0) { x->res_from_round = round; x->res_from_canon = canon; }
    x->nres++;
    (void)min_gap;
    return x->nres >= x->prm->num_results;
}

/* minimum-weight element of results (first found on equal weight) */
static int results_best(dec_ctx *x, double *min_gap)
{
    int best = 0;
    for (int r = 1; r < x->nres; ++r)
        if (x->res_w[r] < x->res_w[best]) best = r;
    if (x->nres > 1) {
        /* an equal weight is an exact tie, settled by the order found (R11) */
        double g = INFINITY;
        int nt = 0;
        for (int r = 0; r < x->nres; ++r)
            if (r != best) margin_note(&g, &nt, x->res_w[r] - x->res_w[best], fabs(x->res_w[best]));
        if (min_gap && g < *min_gap) *min_gap = g;
        *g_tie_counter += nt;
        log_push(3, 0, (uint64_t)best, g, nt);
    }
    return best;
}

/* order of the current set: score descending, canonical index ascending (R8) */
static int path_before(const path_t *a, const path_t *b)
{
    if (a->score != b->score) return a->score > b->score;
    return a->canon < b->canon;
}

static void sort_paths(path_t *ps, int n)
{
    for (int a = 1; a < n; ++a) {
        int k = a;
        while (k > 0 && path_before(&ps[k], &ps[k - 1])) { path_swap(&ps[k], &ps[k - 1]); --k; }
    }
}

static void trace_child(oracle_trace *tr, int round, int canon, int prank, int val, int pos,
                        int success, int iters, int next_pos, double score, int *idx)
{
    *idx = -1;
    if (!tr || tr->n >= tr->cap) return;
    int k = tr->n++;
    tr->round[k] = round; tr->canon[k] = canon; tr->parent_rank[k] = prank; tr->val[k] = val;
    tr->pos[k] = pos; tr->success[k] = success; tr->iters[k] = iters; tr->next_pos[k] = next_pos;
    tr->score[k] = score; tr->kept[k] = -1;
    *idx = k;
}

/* Decode one syndrome.  s: M bytes (0/1).  Outputs: ehat N bytes, status
   (1 = converged in the seed BP, 2 = converged in a masked BP round, 4 = failed),
   iters = BP iterations run by the sequential algorithm up to its return. */
static void decode_one(dec_ctx *x, const uint8_t *s, uint8_t *out_e, int32_t *status,
                       int64_t *iters_total, double *min_gap, int32_t *n_ties, oracle_trace *tr)
{
    int ties = 0;
    g_tie_counter = &ties;
    g_call = 0;
    g_round = 0;
    const oracle_graph *g = x->g;
    const oracle_params *prm = x->prm;
    const int N = g->N, E = g->E;
    const int w = prm->beam_width;
    double gap = INFINITY;
    int64_t total = 0;
    x->nres = 0;
    x->res_from_round = -1;
    x->res_from_canon = -1;
    if (tr) { tr->n = 0; tr->ret_round = -1; tr->ret_canon = -1; }

    /* seed: plain BP from E(0) = Lambda for initial_iters iterations */
    for (int e = 0; e < E; ++e) {
        real l = g->lam[g->col_idx[e]];
        const real lmax = clamp_value(prm);
        if (l > lmax) l = lmax;
        if (l < -lmax) l = -lmax;
        x->E_seed[e] = store_msg(prm, l);
    }
    memset(x->cmask, 0, (size_t)N);
    memset(x->cval, 0, (size_t)N);
    path_t *seed = &x->cur[0];
    bp_call *c = &x->c;
    c->E_in = x->E_seed; c->masked = x->cmask; c->val = x->cval; c->s = s;
    c->max_iters = prm->initial_iters; c->stop_on_success = 1;
    c->E_out = seed->E; c->sum_llr = x->sum_llr; c->ehat = seed->ehat; c->llr_traj = NULL;
    masked_bp(g, prm, c, &x->w);
    if (c->min_gap < gap) gap = c->min_gap;
    total += c->iters;
    double agap;
    seed->next_pos = least_reliable(g, x->sum_llr, x->cmask, &agap);
    if (agap == 0) ++*g_tie_counter;
    else if (agap < gap) gap = agap;
    log_push(1, 0, (uint64_t)(int64_t)seed->next_pos, agap == 0 ? INFINITY : agap, agap == 0);
    seed->score = 0;
    seed->canon = 0;
    memset(seed->masked, 0, (size_t)N);
    memset(seed->val, 0, (size_t)N);
    if (tr) { tr->seed_iters = c->iters; tr->seed_success = c->success; tr->seed_next_pos = seed->next_pos; }
    int done = 0;
    x->near_tie = 0;
    if (c->success) {
        if (results_insert(x, seed->ehat, 0, 0, &gap)) {
            done = 1;
            if (tr) { tr->ret_round = 0; tr->ret_canon = 0; }
        }
    }
    if (!done && prm->max_rounds > 0) tie_check(x, agap);   /* the seed path will branch on next_pos */
    x->ncur = 1;

    for (int r = 1; r <= prm->max_rounds && !done; ++r) {
        x->nnxt = 0;
        x->nr = 0;
        g_round = r;
        for (int pr = 0; pr < x->ncur && !done; ++pr) {
            path_t *par = &x->cur[pr];
            if (par->next_pos < 0) continue;                       /* R9 */
            for (int v = 0; v <= 1 && !done; ++v) {
                const int canon = 2 * pr + v;   /* visit order: parents by rank, val 0 then 1 */
                /* nextp.pos_val_pairs = path.pos_val_pairs + (next_pos, v) */
                memcpy(x->cmask, par->masked, (size_t)N);
                memcpy(x->cval, par->val, (size_t)N);
                x->cmask[par->next_pos] = 1;
                x->cval[par->next_pos] = (uint8_t)v;
                /* candidate slot: a free entry of nxt (index nnxt, or the spare) */
                path_t *ch = &x->nxt[x->nnxt < x->cap ? x->nnxt : x->cap];
                c->E_in = par->E; c->masked = x->cmask; c->val = x->cval; c->s = s;
                c->max_iters = prm->iters_per_round; c->stop_on_success = 1;
                c->E_out = ch->E; c->sum_llr = x->sum_llr; c->ehat = ch->ehat; c->llr_traj = NULL;
                ++g_call;
                masked_bp(g, prm, c, &x->w);
                if (c->min_gap < gap) gap = c->min_gap;
                total += c->iters;
                int succ = c->success;
                memcpy(ch->masked, x->cmask, (size_t)N);
                memcpy(ch->val, x->cval, (size_t)N);
                ch->next_pos = least_reliable(g, x->sum_llr, x->cmask, &agap);
                if (ch->next_pos >= 0 && agap == 0) ++*g_tie_counter;
                else if (ch->next_pos >= 0 && agap < gap) gap = agap;
                log_push(1, 0, (uint64_t)(int64_t)ch->next_pos, agap == 0 ? INFINITY : agap,
                         ch->next_pos >= 0 && agap == 0);
                ch->score = path_score(g, x->sum_llr, x->cmask, c->iters, x->tmp);
                ch->canon = canon;
                if (ch->next_pos >= 0) tie_check(x, agap);
                x->rscore[x->nr] = ch->score;
                x->rcanon[x->nr] = canon;
                x->nr++;
                trace_child(tr, r, canon, pr, v, par->next_pos, succ, c->iters, ch->next_pos,
                            ch->score, &ch->trace_idx);
                if (succ && results_insert(x, ch->ehat, r, canon, &gap)) {
                    done = 1;
                    if (tr) { tr->ret_round = r; tr->ret_canon = canon; }
                    break;
                }
                /* insert nextp into next_set */
                if (prm->prune_mode == 1 || x->nnxt < w) {
                    if (ch != &x->nxt[x->nnxt]) path_swap(ch, &x->nxt[x->nnxt]);
                    x->nnxt++;
                } else if (w > 0) {
                    /* on-the-fly bounded insert (App. B): replace the minimum
                       (latest inserted among equal minima) when strictly better */
                    int mi = 0;
                    for (int k = 1; k < x->nnxt; ++k) {
                        if (x->nxt[k].score < x->nxt[mi].score ||
                            (x->nxt[k].score == x->nxt[mi].score && x->nxt[k].canon > x->nxt[mi].canon))
                            mi = k;
                    }
                    if (ch->score > x->nxt[mi].score) path_swap(ch, &x->nxt[mi]);
                }
            }
        }
        if (done) break;
        /* the round's pruning decisions: the boundary between kept and
           dropped (before the last round; it flags a near tie, R16) and the
           order of the kept set (the visit order of the next round, and in
           the last round the path R10 falls back to) */
        double pg = INFINITY;
        int pties = 0;
        if (r < prm->max_rounds) {
            const double bm = pruning_margin(x, w);
            tie_check(x, bm);
            if (bm < INFINITY) margin_note(&pg, &pties, bm, 1.0);
        }
        /* the new set, explored next round in descending score (App. B) */
        sort_paths(x->nxt, x->nnxt);
        if (prm->prune_mode == 1 && x->nnxt > w) x->nnxt = w;     /* Alg. 3: keep the top beam_width */
        for (int k = 0; k + 1 < x->nnxt; ++k)
            margin_note(&pg, &pties, x->nxt[k].score - x->nxt[k + 1].score, fabs(x->nxt[k].score));
        if (pg < gap) gap = pg;
        *g_tie_counter += pties;
        if (g_dlog) {
            uint64_t h = FNV_INIT;
            for (int k = 0; k < x->nnxt; ++k) h = fnv_add(h, (uint64_t)x->nxt[k].canon);
            log_push(2, 0, h, pg, pties);
        }
        if (tr)
            for (int k = 0; k < x->nnxt; ++k)
                if (x->nxt[k].trace_idx >= 0) tr->kept[x->nxt[k].trace_idx] = k;
        if (x->nnxt == 0) break;              /* no path left to expand: keep the last set */
        path_t *tmpp = x->cur; x->cur = x->nxt; x->nxt = tmpp;
        x->ncur = x->nnxt;
    }

    int32_t st;
    if (x->nres > 0) {
        int b = results_best(x, &gap);
        memcpy(out_e, x->results + (size_t)b * N, (size_t)N);
        /* 1 if the returned vector came from the seed BP, else 2 */
        st = (b == 0 && x->res_from_round == 0) ? 1 : 2;
    } else {
        /* R10: nothing converged; the best path of the final set */
        memcpy(out_e, x->cur[0].ehat, (size_t)N);
        st = 4;
    }
    if (x->near_tie) st |= 8;
    *status = st;
    *iters_total = total;
    if (min_gap) *min_gap = gap;
    if (n_ties) *n_ties = ties;
    g_tie_counter = &g_ties_tls_dummy;
}

/* One syndrome with its decision log (see oracle_dlog); the outputs are
   those of oracle_decode.  Returns 0, or 1 if the log ran out of room. */
int oracle_decode_logged(const oracle_graph *g, const oracle_params *prm, const uint8_t *s,
                         uint8_t *ehat, int32_t *status, int64_t *iters, double *min_gap,
                         int32_t *n_ties, oracle_dlog *log)
{
    dec_ctx *x = ctx_new(g, prm);
    log->n = 0;
    g_dlog = log;
    decode_one(x, s, ehat, status, iters, min_gap, n_ties, NULL);
    g_dlog = NULL;
    ctx_free(x);
    return log->n >= log->cap ? 1 : 0;
}

/* ------------------------------------------------------------------------- */
/* exported entry points                                                      */
/* ------------------------------------------------------------------------- */
int oracle_real_bytes(void) { return (int)sizeof(real); }

/* One syndrome, unpacked bytes.  Returns 0. */
int oracle_decode(const oracle_graph *g, const oracle_params *prm, const uint8_t *s,
                  uint8_t *ehat, int32_t *status, int64_t *iters, double *min_gap,
                  int32_t *n_ties, oracle_trace *tr)
{
    dec_ctx *x = ctx_new(g, prm);
    decode_one(x, s, ehat, status, iters, min_gap, n_ties, tr);
    ctx_free(x);
    return 0;
}

typedef struct {
    const oracle_graph *g;
    const oracle_params *prm;
    const uint32_t *synd;
    int64_t b0, b1;
    uint32_t *corr, *obs, *status, *iters;
    double *min_gap;
    int32_t *ties;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *jb = (batch_job *)arg;
    const oracle_graph *g = jb->g;
    const int M = g->M, N = g->N, K = g->K;
    const int WM = (M + 31) / 32, WN = (N + 31) / 32, WK = (K + 31) / 32;
    dec_ctx *x = ctx_new(g, jb->prm);
    uint8_t *s = (uint8_t *)malloc((size_t)(M > 0 ? M : 1));
    uint8_t *e = (uint8_t *)malloc((size_t)(N > 0 ? N : 1));
    for (int64_t b = jb->b0; b < jb->b1; ++b) {
        for (int i = 0; i < M; ++i) s[i] = (uint8_t)((jb->synd[b * WM + i / 32] >> (i % 32)) & 1u);
        int32_t st, nt; int64_t it; double gp;
        decode_one(x, s, e, &st, &it, &gp, &nt, NULL);
        if (jb->corr) {
            uint32_t *o = jb->corr + b * WN;
            for (int k = 0; k < WN; ++k) o[k] = 0;
            for (int j = 0; j < N; ++j) if (e[j]) o[j / 32] |= 1u << (j % 32);
        }
        if (jb->obs) {
            uint32_t *o = jb->obs + b * WK;
            for (int k = 0; k < WK; ++k) o[k] = 0;
            for (int r = 0; r < K; ++r) {
                int par = 0;
                for (int q = g->a_row_ptr[r]; q < g->a_row_ptr[r + 1]; ++q) par ^= e[g->a_col_idx[q]];
                if (par) o[r / 32] |= 1u << (r % 32);
            }
        }
        if (jb->status) jb->status[b] = (uint32_t)st;
        if (jb->iters) jb->iters[b] = (uint32_t)it;
        if (jb->min_gap) jb->min_gap[b] = gp;
        if (jb->ties) jb->ties[b] = nt;
    }
    free(s); free(e);
    ctx_free(x);
    return NULL;
}

/* Decode B bitpacked syndromes (bit i of word i/32), writing bitpacked
   corrections and observable flips A e, status and iteration counts.
   Shots are split into contiguous ranges over nthreads threads; each shot is
   decoded by decode_one exactly as in the single-shot entry point. */
int oracle_decode_batch(const oracle_graph *g, const oracle_params *prm,
                        const uint32_t *synd, int64_t B,
                        uint32_t *corr, uint32_t *obs, uint32_t *status, uint32_t *iters,
                        double *min_gap, int32_t *ties, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > B) nthreads = (int)(B > 0 ? B : 1);
    batch_job *jobs = (batch_job *)calloc((size_t)nthreads, sizeof(batch_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int k = 0; k < nthreads; ++k) {
        jobs[k].g = g; jobs[k].prm = prm; jobs[k].synd = synd;
        jobs[k].b0 = B * k / nthreads; jobs[k].b1 = B * (k + 1) / nthreads;
        jobs[k].corr = corr; jobs[k].obs = obs; jobs[k].status = status; jobs[k].iters = iters;
        jobs[k].min_gap = min_gap;
        jobs[k].ties = ties;
    }
    for (int k = 1; k < nthreads; ++k) pthread_create(&th[k], NULL, batch_worker, &jobs[k]);
    batch_worker(&jobs[0]);
    for (int k = 1; k < nthreads; ++k) pthread_join(th[k], NULL);
    free(jobs); free(th);
    return 0;
}

/* Alg. 2 on its own: masked BP from given edge messages.  masked/val: N
   bytes; s: M bytes.  Outputs as described in bp_call.  llr_traj may be NULL
   (else max_iters * N values).  Returns the number of iterations run. */
int oracle_masked_bp(const oracle_graph *g, const oracle_params *prm,
                     const real *E_in, const uint8_t *masked, const uint8_t *val,
                     const uint8_t *s, int max_iters, int stop_on_success,
                     uint8_t *ehat, real *E_out, real *sum_llr, real *llr_traj,
                     int32_t *success, int32_t *first_success)
{
    dec_ctx *x = ctx_new(g, prm);
    bp_call c;
    memset(&c, 0, sizeof(c));
    c.E_in = E_in; c.masked = masked; c.val = val; c.s = s;
    c.max_iters = max_iters; c.stop_on_success = stop_on_success;
    c.E_out = E_out; c.sum_llr = sum_llr; c.ehat = ehat; c.llr_traj = llr_traj;
    masked_bp(g, prm, &c, &x->w);
    if (success) *success = c.success;
    if (first_success) *first_success = c.first_success;
    ctx_free(x);
    return c.iters;
}

/* Prior LLRs as held by this build (float or double). */
void oracle_prior_llr(const oracle_graph *g, real *out)
{
    for (int j = 0; j < g->N; ++j) out[j] = g->lam[j];
}
