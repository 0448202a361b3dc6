/*
 * walk_oracle.c -- the CPU oracle for node2vec second-order random walks.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this code.  The product library under
 * paper_2110_06196_gb300/ never links, includes or calls it, and this file
 * includes nothing from there.
 *
 * What it computes (GRAPE, "Methods: Implementation of second-order RWs"):
 *   a walk moves from v to a neighbour x with un-normalised probability
 *       pi_vx = alpha_pq(t, x) * w_vx                      (eq. alphaRW)
 *   where t is the previous node and
 *       alpha = 1/p  if x == t          (return bias gamma_p, d(t,x) = 0)
 *       alpha = 1    if x in N(t)       (in-out bias beta_q,  d(t,x) = 1)
 *       alpha = 1/q  otherwise          (d(t,x) = 2)
 *   (eqs. alpha, beta; "Efficient computation of the in-out and return bias").
 *   The first step of a walk has no t and is first-order: pi_vx = w_vx
 *   ("First and second-order RW-based embedding methods").
 *
 * How it samples (exact rejection sampling, one Philox4x32-10 block per trial):
 *   amax = max(1/p, 1, 1/q); the three class thresholds are
 *       T_c = floor((alpha_c / amax) * 2^32)      (IEEE double, round-to-nearest)
 *   trial k at step s of walk w draws (r0,r1,r2,r3) = Philox4x32-10 with
 *       key = (seed lo, seed hi), counter = (w lo, w hi, s, k),
 *   proposes x = row_v[ floor(((r1:r0) * deg_v) / 2^64) ] and accepts iff
 *       unweighted:  r2 < T_c
 *       weighted:    r2 * wmax_v < T_c * w_vx          (exact, over the reals)
 *   where wmax_v is the largest weight in the row of v.  The proposal x is
 *   uniform over the row, so x is accepted with probability (to within
 *   2^-32) (alpha_c / amax) * (w_vx / wmax_v), proportional to pi_vx: the
 *   accepted draw follows eq. alphaRW exactly.  After trial_cap
 *   rejected trials the step is drawn exactly by inverse transform over the
 *   cumulative sum of pi in row order, the paper's own on-the-fly sampler
 *   ("Efficient sampling for Node2Vec RWs"), with u taken from the Philox block
 *   of trial index trial_cap.
 *
 * Written for clarity, not speed: one walk at a time, one trial at a time,
 * plain binary search for membership, no blocking and no reordering.
 * Build with -ffp-contract=off so that no product of the fallback's cumulative
 * sum is fused into another operation.
 */
#include <stdint.h>
#include <stddef.h>
#include <math.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10.  Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC 2011, section on the Philox family: each round maps   */
/* (c0,c1,c2,c3) with key (k0,k1) through two 32x32->64 products by the       */
/* multipliers 0xD2511F53 and 0xCD9E8D57, and the key is advanced between     */
/* rounds by the Weyl increments 0x9E3779B9 and 0xBB67AE85.                   */
/* ------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The Philox block of one trial: key = seed, counter = (walk id, step, trial). */
static void trial_block(uint64_t seed, int64_t walk_id, int32_t step, int64_t trial,
                        uint32_t r[4])
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint64_t w = (uint64_t)walk_id;
    uint32_t ctr[4] = { (uint32_t)w, (uint32_t)(w >> 32), (uint32_t)step, (uint32_t)trial };
    oracle_philox4x32_10(ctr, key, r);
}

/* ------------------------------------------------------------------------ */
/* Acceptance thresholds of the three alpha classes.                         */
/* ------------------------------------------------------------------------ */
enum { CLS_RETURN = 0, CLS_IN = 1, CLS_OUT = 2, CLS_FIRST = 3 };

/* T[0] = return (x == t), T[1] = in (x in N(t)), T[2] = out (otherwise). */
void oracle_thresholds(double p, double q, uint64_t T[3])
{
    double a_ret = 1.0 / p, a_in = 1.0, a_out = 1.0 / q;
    double amax = a_ret;
    if (a_in > amax) amax = a_in;
    if (a_out > amax) amax = a_out;
    double alpha[3] = { a_ret, a_in, a_out };
    for (int c = 0; c < 3; ++c) {
        double ratio = alpha[c] / amax;                 /* in (0, 1] */
        T[c] = (uint64_t)floor(ratio * 4294967296.0);   /* 2^32 when ratio == 1 */
    }
}

/* x = M * 2^E exactly, with M a non-negative integer below 2^24 (frexpf gives
 * x = f * 2^e with f in [0.5, 1), and an fp32 value has at most 24 significant
 * bits, so f * 2^24 is an integer). */
static void split_float(float x, uint64_t* M, int* E)
{
    int e;
    float f = frexpf(x, &e);
    *M = (uint64_t)ldexpf(f, 24);
    *E = e - 24;
}

/* Exact test r2 * wmax < T * w over the reals, for positive finite fp32 weights. */
int oracle_weighted_accept(uint32_t r2, float wmax, uint64_t T, float w)
{
    uint64_t m1, m2;
    int e1, e2;
    split_float(wmax, &m1, &e1);
    split_float(w, &m2, &e2);
    unsigned __int128 lhs = (unsigned __int128)r2 * m1;   /* times 2^e1, below 2^56 */
    unsigned __int128 rhs = (unsigned __int128)T * m2;    /* times 2^e2, at most 2^56 */
    int d = e1 - e2;
    if (d >= 0) {
        if (lhs == 0) return rhs > 0;
        if (d > 60) return 0;                 /* lhs * 2^d >= 2^60 > rhs */
        return (lhs << d) < rhs;
    }
    if (rhs == 0) return 0;
    if (-d > 60) return 1;                    /* rhs * 2^-d >= 2^60 > lhs */
    return lhs < (rhs << (-d));
}

/* Largest weight of every row (0 for an empty row).  Weights are fp32. */
void oracle_node_wmax(const int64_t* offsets, const float* weights, int64_t num_nodes,
                      float* wmax)
{
    for (int64_t v = 0; v < num_nodes; ++v) {
        float m = 0.0f;
        for (int64_t e = offsets[v]; e < offsets[v + 1]; ++e)
            if (weights[e] > m) m = weights[e];
        wmax[v] = m;
    }
}

/* d(t, x) == 1 test: is x in the (sorted, duplicate-free) out-row of t? */
static int in_row(const int64_t* offsets, const int32_t* dsts, int32_t t, int32_t x)
{
    int64_t lo = offsets[t], hi = offsets[t + 1];   /* search [lo, hi) */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (dsts[mid] == x) return 1;
        if (dsts[mid] < x) lo = mid + 1; else hi = mid;
    }
    return 0;
}

static int alpha_class(const int64_t* offsets, const int32_t* dsts, int32_t t, int32_t x)
{
    if (t < 0) return CLS_FIRST;
    if (x == t) return CLS_RETURN;
    if (in_row(offsets, dsts, t, x)) return CLS_IN;
    return CLS_OUT;
}

/* ------------------------------------------------------------------------ */
/* Approximated walks (GRAPE, Methods, "Approximated RWs"): at a node whose   */
/* degree exceeds k, a step considers only k neighbours, one drawn uniformly  */
/* from each of k equal buckets of positions (Sorted Unique Sub-Sampling,     */
/* SUSS), in bucket order.  Bucket b holds positions                          */
/*     [floor(b * deg / k), floor((b + 1) * deg / k))                         */
/* and its member is drawn from the Philox block of trial index 2^31 + b of   */
/* the step, so the sub-sample is fixed for the whole step.                   */
/* ------------------------------------------------------------------------ */
#define SUSS_TRIAL_BASE 0x80000000LL

/* Number of candidates of a step: deg, or k under SUSS. */
static uint64_t cand_count(uint64_t deg, int64_t suss_k)
{
    return (suss_k > 0 && deg > (uint64_t)suss_k) ? (uint64_t)suss_k : deg;
}

/* Position in the row of candidate j (j < cand_count). */
static uint64_t cand_pos(uint64_t deg, int64_t suss_k, uint64_t seed, int64_t walk_id,
                         int32_t step, uint64_t j)
{
    if (!(suss_k > 0 && deg > (uint64_t)suss_k)) return j;
    uint64_t k = (uint64_t)suss_k;
    uint64_t lo = (uint64_t)(((unsigned __int128)j * deg) / k);
    uint64_t hi = (uint64_t)(((unsigned __int128)(j + 1) * deg) / k);
    uint32_t r[4];
    trial_block(seed, walk_id, step, SUSS_TRIAL_BASE + (int64_t)j, r);
    uint64_t r64 = (uint64_t)r[0] | ((uint64_t)r[1] << 32);
    return lo + (uint64_t)(((unsigned __int128)r64 * (hi - lo)) >> 64);
}

/* The SUSS sub-sample of one step, for tests: positions of the k candidates. */
void oracle_suss_positions(int64_t deg, int64_t suss_k, uint64_t seed, int64_t walk_id,
                           int32_t step, int64_t* out)
{
    uint64_t m = cand_count((uint64_t)deg, suss_k);
    for (uint64_t j = 0; j < m; ++j)
        out[j] = (int64_t)cand_pos((uint64_t)deg, suss_k, seed, walk_id, step, j);
}

typedef struct oracle_stats {
    int64_t steps;       /* transitions taken */
    int64_t trials;      /* Philox blocks drawn for rejection trials */
    int64_t fallbacks;   /* steps drawn by the exact inverse-transform fallback */
} oracle_stats;

/*
 * One transition out of v (previous node t, or t = -1 on the first step).
 * Returns the chosen neighbour.  deg(v) must be > 0.  suss_k > 0 samples
 * among the SUSS sub-sample when deg(v) > suss_k (approximated walks); 0 is
 * the exact walk.  trial_cap must stay below 2^31 (SUSS trial indices).
 */
int32_t oracle_next(const int64_t* offsets, const int32_t* dsts, const float* weights,
                    const float* wmax, int32_t t, int32_t v, double p, double q,
                    uint64_t seed, int64_t walk_id, int32_t step, int64_t trial_cap,
                    int64_t suss_k, oracle_stats* st)
{
    uint64_t T[3];
    oracle_thresholds(p, q, T);
    const int64_t off = offsets[v];
    const uint64_t deg = (uint64_t)(offsets[v + 1] - off);
    const uint64_t m = cand_count(deg, suss_k);
    uint32_t r[4];

    for (int64_t k = 0; k < trial_cap; ++k) {
        trial_block(seed, walk_id, step, k, r);
        if (st) st->trials++;
        uint64_t r64 = (uint64_t)r[0] | ((uint64_t)r[1] << 32);
        uint64_t j = (uint64_t)(((unsigned __int128)r64 * m) >> 64);
        uint64_t idx = cand_pos(deg, suss_k, seed, walk_id, step, j);
        int32_t x = dsts[off + (int64_t)idx];
        int cls = alpha_class(offsets, dsts, t, x);
        uint64_t thr = (cls == CLS_FIRST) ? ((uint64_t)1 << 32) : T[cls];
        int accept;
        if (weights == NULL) {
            accept = (uint64_t)r[2] < thr;
        } else {
            accept = oracle_weighted_accept(r[2], wmax[v], thr, weights[off + (int64_t)idx]);
        }
        if (accept) return x;
    }

    /* Exact fallback: inverse transform over the cumulative sum of pi. */
    if (st) st->fallbacks++;
    trial_block(seed, walk_id, step, trial_cap, r);
    double alpha[3] = { 1.0 / p, 1.0, 1.0 / q };
    double total = 0.0;
    for (uint64_t j = 0; j < m; ++j) {
        uint64_t pos = cand_pos(deg, suss_k, seed, walk_id, step, j);
        int32_t x = dsts[off + (int64_t)pos];
        int cls = alpha_class(offsets, dsts, t, x);
        double a = (cls == CLS_FIRST) ? 1.0 : alpha[cls];
        double w = weights ? (double)weights[off + (int64_t)pos] : 1.0;
        total += a * w;
    }
    uint64_t r64 = (uint64_t)r[0] | ((uint64_t)r[1] << 32);
    double u = ((double)(r64 >> 11) * 0x1p-53) * total;
    double run = 0.0;
    for (uint64_t j = 0; j < m; ++j) {
        uint64_t pos = cand_pos(deg, suss_k, seed, walk_id, step, j);
        int32_t x = dsts[off + (int64_t)pos];
        int cls = alpha_class(offsets, dsts, t, x);
        double a = (cls == CLS_FIRST) ? 1.0 : alpha[cls];
        double w = weights ? (double)weights[off + (int64_t)pos] : 1.0;
        run += a * w;
        if (run > u) return x;
    }
    return dsts[off + (int64_t)cand_pos(deg, suss_k, seed, walk_id, step, m - 1)];
}

/*
 * Walks with ids in [walk_begin, walk_end).  Walk w starts at
 * starts[w % num_starts] (or at node w % num_starts when starts is NULL), so
 * walk w = r * num_starts + i is repetition r of start i.  Row w - walk_begin
 * of out holds walk_len node ids: the start, then one node per transition;
 * once the walk reaches a node without out-edges the rest of the row is -1.
 * Returns 0, or -1 when a start id is out of range (its row is then all -1).
 * stats may be NULL.
 */
int oracle_walks(const int64_t* offsets, const int32_t* dsts, const float* weights,
                 const float* wmax, int64_t num_nodes,
                 const int32_t* starts, int64_t num_starts,
                 int32_t walk_len, double p, double q, uint64_t seed, int64_t trial_cap,
                 int64_t suss_k, int64_t walk_begin, int64_t walk_end, int32_t* out,
                 oracle_stats* stats)
{
    int rc = 0;
    for (int64_t w = walk_begin; w < walk_end; ++w) {
        int32_t* row = out + (w - walk_begin) * (int64_t)walk_len;
        int64_t i = w % num_starts;
        int64_t v0 = starts ? (int64_t)starts[i] : i;
        if (v0 < 0 || v0 >= num_nodes) {
            for (int32_t s = 0; s < walk_len; ++s) row[s] = -1;
            rc = -1;
            continue;
        }
        row[0] = (int32_t)v0;
        int32_t t = -1, v = (int32_t)v0;
        int32_t s = 1;
        for (; s < walk_len; ++s) {
            if (offsets[v + 1] == offsets[v]) break;          /* dead end */
            int32_t x = oracle_next(offsets, dsts, weights, wmax, t, v, p, q, seed,
                                    w, s, trial_cap, suss_k, stats);
            row[s] = x;
            if (stats) stats->steps++;
            t = v;
            v = x;
        }
        for (; s < walk_len; ++s) row[s] = -1;
    }
    return rc;
}

/*
 * Distribution probe: the transition out of v (previous node t, -1 for none)
 * at step `step` for every walk id in [walk_begin, walk_begin + n).  Each walk
 * id keys an independent Philox stream, so the n results are independent
 * draws from the transition law of the (t, v) context.
 */
void oracle_next_many(const int64_t* offsets, const int32_t* dsts, const float* weights,
                      const float* wmax, int32_t t, int32_t v, double p, double q,
                      uint64_t seed, int64_t walk_begin, int64_t n, int32_t step,
                      int64_t trial_cap, int64_t suss_k, int32_t* out, oracle_stats* stats)
{
    for (int64_t j = 0; j < n; ++j)
        out[j] = oracle_next(offsets, dsts, weights, wmax, t, v, p, q, seed,
                             walk_begin + j, step, trial_cap, suss_k, stats);
}

/* ------------------------------------------------------------------------ */
/* Context windows of walk rows (GRAPE, "First and second-order RW-based      */
/* embedding methods": SkipGram and CBOW learn from windows of a given size   */
/* sliding over the walks).  For row r and position i, ctx[r][i] lists the    */
/* window around the centre row[r][i]: the `window` positions before it, in   */
/* walk order, then the `window` positions after it:                          */
/*     ctx[r][i][j]          = row[r][i - window + j]     j = 0 .. window-1   */
/*     ctx[r][i][window + j] = row[r][i + 1 + j]          j = 0 .. window-1   */
/* An entry is -1 when its position lies outside the row, when it holds -1    */
/* (after a dead end), or when the centre itself is -1.  SkipGram pairs are   */
/* (centre, entry) over the entries that are not -1; CBOW uses the entries of */
/* a centre together.                                                         */
/* ------------------------------------------------------------------------ */
void oracle_contexts(const int32_t* rows, int64_t num_rows, int32_t walk_len, int32_t window,
                     int32_t* ctx)
{
    const int64_t width = 2 * (int64_t)window;
    for (int64_t r = 0; r < num_rows; ++r) {
        const int32_t* row = rows + r * (int64_t)walk_len;
        for (int32_t i = 0; i < walk_len; ++i) {
            int32_t* out = ctx + (r * (int64_t)walk_len + i) * width;
            for (int32_t j = 0; j < 2 * window; ++j) {
                int64_t pos = (j < window) ? (int64_t)i - window + j : (int64_t)i + 1 + (j - window);
                int32_t val = -1;
                if (row[i] >= 0 && pos >= 0 && pos < walk_len && row[pos] >= 0) val = row[pos];
                out[j] = val;
            }
        }
    }
}
