/*
 * relaybp_oracle.c -- plain, slow, FP64 CPU oracle for the Relay-BP hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file: it exists so that tests, the smoke check and the CPU-baseline leg
 * of the benchmark can check the CUDA path against a direct transcription of
 * the method.  It shares no code, header or table with the CUDA library.
 *
 * What it computes (arXiv 2607.27644, Sec. 6.1 "Quantum circuit-level memory",
 * decoder configuration list; the update rule of Relay-BP itself is cited, not
 * printed, by the paper, so the reading below is the one stated in the design
 * notes):
 *
 *   a1  prior LLRs            L0_j = log((1 - p_j) / p_j)                (FP64)
 *   a2  fault sampler         e_j = [philox word_j < floor(p_j 2^32)],
 *                             s = H e, obs = O e                        (exact)
 *   a3  check update          nu_{i->j} = (-1)^{s_i} prod_{j' != j} sgn(mu_{j'->i})
 *                                                 * min_{j' != j} |mu_{j'->i}|
 *   a4  variable update       L_j(t)  = (1 - g_j) L0_j + g_j M_j(t-1)
 *       (memory strength g)   mu_{j->i} = L_j(t) + sum_{i' != i} nu_{i'->j}(t-1)
 *                             M_j(t)  = L_j(t) + sum_i nu_{i->j}(t)
 *                             e^_j    = [M_j(t) < 0]
 *   a5  residual              converged iff H e^ = s
 *   a6  relay legs            leg 0: pre_iter iterations at g_j = gamma0;
 *                             legs 1..num_sets: max_iterations iterations with
 *                             g_j ~ U[gamma_min, gamma_max] per variable per leg;
 *                             M carries across legs, messages reset (unless
 *                             carry_messages); a leg stops at its first
 *                             convergence; stop after stop_nconv solutions
 *   a7  select                weight w(e^) = sum_j e^_j L0_j in FP64; keep the
 *                             minimum, earliest on ties
 *   a9  accounting            predicted observables O e^
 *
 * Philox4x32-10 follows Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
 * as easy as 1, 2, 3" (SC'11): two 32x32->64 multiplies per round with the
 * published multipliers and Weyl key increments, ten rounds.
 *
 * Bit layouts: bit b of a packed vector lives in word b/32 at position b%32.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (SC'11)                                                      */
/* ------------------------------------------------------------------------- */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Word j of the counter stream (stream id, shot) for a 64-bit seed. */
static uint32_t stream_word(uint64_t seed, uint64_t shot, uint32_t stream, uint64_t j)
{
    uint32_t ctr[4], key[2], out[4];
    ctr[0] = (uint32_t)(j / 4);
    ctr[1] = (uint32_t)(shot & 0xffffffffu);
    ctr[2] = (uint32_t)(shot >> 32);
    ctr[3] = stream;
    key[0] = (uint32_t)(seed & 0xffffffffu);
    key[1] = (uint32_t)(seed >> 32);
    oracle_philox4x32_10(ctr, key, out);
    return out[j % 4];
}

static int get_bit(const uint32_t *v, int64_t b) { return (int)((v[b >> 5] >> (b & 31)) & 1u); }
static void flip_bit(uint32_t *v, int64_t b) { v[b >> 5] ^= (1u << (b & 31)); }

/* ------------------------------------------------------------------------- */
/* a2: Bernoulli fault sampler                                               */
/* ------------------------------------------------------------------------- */
/* Fault j of shot s fires iff word j of stream 0 is below floor(p_j * 2^32).
 * Returns 0, or -1 on a probability outside [0, 1]. */
int oracle_sample(int32_t n_det, int32_t n_loc, int32_t n_obs,
                  const int32_t *H_indptr, const int32_t *H_indices,
                  const int32_t *O_indptr, const int32_t *O_indices,
                  const double *priors, uint64_t seed, uint64_t shot0, int64_t shots,
                  uint32_t *syndromes, uint32_t *obs, uint32_t *errors)
{
    int64_t wd = (n_det + 31) / 32, wo = (n_obs + 31) / 32, wv = (n_loc + 31) / 32;
    /* columns of H and O as lists: plain transposes of the CSR inputs */
    int32_t *hc_ptr = calloc((size_t)n_loc + 1, sizeof(int32_t));
    int32_t *oc_ptr = calloc((size_t)n_loc + 1, sizeof(int32_t));
    int32_t nnz_h = H_indptr[n_det], nnz_o = n_obs ? O_indptr[n_obs] : 0;
    int32_t *hc_rows = malloc(sizeof(int32_t) * (size_t)(nnz_h + 1));
    int32_t *oc_rows = malloc(sizeof(int32_t) * (size_t)(nnz_o + 1));
    uint32_t *thr = malloc(sizeof(uint32_t) * (size_t)(n_loc + 1));
    for (int32_t j = 0; j < n_loc; ++j) {
        double p = priors[j];
        if (!(p >= 0.0 && p <= 1.0)) { free(hc_ptr); free(oc_ptr); free(hc_rows); free(oc_rows); free(thr); return -1; }
        double t = floor(p * 4294967296.0);
        thr[j] = t >= 4294967295.0 ? 0xffffffffu : (uint32_t)t;
    }
    for (int32_t i = 0; i < n_det; ++i)
        for (int32_t e = H_indptr[i]; e < H_indptr[i + 1]; ++e) hc_ptr[H_indices[e] + 1]++;
    for (int32_t i = 0; i < n_obs; ++i)
        for (int32_t e = O_indptr[i]; e < O_indptr[i + 1]; ++e) oc_ptr[O_indices[e] + 1]++;
    for (int32_t j = 0; j < n_loc; ++j) { hc_ptr[j + 1] += hc_ptr[j]; oc_ptr[j + 1] += oc_ptr[j]; }
    {
        int32_t *fh = calloc((size_t)n_loc + 1, sizeof(int32_t));
        int32_t *fo = calloc((size_t)n_loc + 1, sizeof(int32_t));
        for (int32_t i = 0; i < n_det; ++i)
            for (int32_t e = H_indptr[i]; e < H_indptr[i + 1]; ++e) {
                int32_t j = H_indices[e];
                hc_rows[hc_ptr[j] + fh[j]++] = i;
            }
        for (int32_t i = 0; i < n_obs; ++i)
            for (int32_t e = O_indptr[i]; e < O_indptr[i + 1]; ++e) {
                int32_t j = O_indices[e];
                oc_rows[oc_ptr[j] + fo[j]++] = i;
            }
        free(fh); free(fo);
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t s = 0; s < shots; ++s) {
        uint32_t *syn = syndromes + s * wd;
        uint32_t *ob = obs ? obs + s * wo : NULL;
        uint32_t *er = errors ? errors + s * wv : NULL;
        memset(syn, 0, sizeof(uint32_t) * (size_t)wd);
        if (ob) memset(ob, 0, sizeof(uint32_t) * (size_t)wo);
        if (er) memset(er, 0, sizeof(uint32_t) * (size_t)wv);
        for (int32_t j = 0; j < n_loc; ++j) {
            uint32_t w = stream_word(seed, shot0 + (uint64_t)s, 0u, (uint64_t)j);
            if (w < thr[j]) {
                if (er) flip_bit(er, j);
                for (int32_t e = hc_ptr[j]; e < hc_ptr[j + 1]; ++e) flip_bit(syn, hc_rows[e]);
                if (ob)
                    for (int32_t e = oc_ptr[j]; e < oc_ptr[j + 1]; ++e) flip_bit(ob, oc_rows[e]);
            }
        }
    }
    free(hc_ptr); free(oc_ptr); free(hc_rows); free(oc_rows); free(thr);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* a1, a3-a7, a9: Relay-BP                                                    */
/* ------------------------------------------------------------------------- */
typedef struct {
    double gamma0;
    int32_t pre_iter, num_sets, max_iterations, stop_nconv;
    double gamma_min, gamma_max;
    int32_t stop_all;          /* 1: run every leg regardless of solutions */
    int32_t carry_messages;    /* 1: keep check->variable messages across legs */
    uint64_t seed;             /* key of the memory-strength stream */
} oracle_params;

typedef struct {
    int32_t n_det, n_loc;
    const int32_t *rptr, *rcol;   /* CSR of H: edge e = (row i, column rcol[e]) */
    int32_t *cptr, *cedge;        /* per column: the edge ids that touch it */
    const double *L0;
} graph_t;

/* g_j for leg r >= 1: gamma_min + (gamma_max - gamma_min) * u, u = top 24 bits
 * of word (r * ceil(n_loc / 4) * 4 + j) of stream 1, scaled by 2^-24. */
static double draw_gamma(const oracle_params *P, uint64_t shot, int32_t leg, int32_t j, int32_t n_loc)
{
    uint64_t nblk = ((uint64_t)n_loc + 3) / 4;
    uint64_t word_index = (uint64_t)leg * nblk * 4 + (uint64_t)j;
    uint32_t w = stream_word(P->seed, shot, 1u, word_index);
    double u = (double)(w >> 8) * (1.0 / 16777216.0);
    return P->gamma_min + (P->gamma_max - P->gamma_min) * u;
}

static double sgn(double v) { return v < 0.0 ? -1.0 : 1.0; }   /* sgn(0) = +1 */

/* Learned parameters of the decode (the learned form of this library, not the
 * paper's): message weights w[T][E] indexed by the iteration within the leg
 * (iterations past T reuse w[T-1]) and the knot inverse CDF of the memory
 * strengths of legs >= 1.  NULL pointers give the plain method. */
typedef struct {
    int32_t T, K;
    const double *w, *knots;
    int32_t legs;               /* legs < legs use the learned parameters (< 0: every leg) */
} learned_t;

static double knot_gamma_l(const double *knots, int32_t K, double u);

/* Optional record of every solution a decode finds, in the order found: its
 * leg, the shot's iteration count when it was found, its FP64 weight and its
 * bits (packed, ceil(V/32) words each).  Test infrastructure for the
 * minimum-weight select (a7): a test recomputes each weight from the bits and
 * checks that the returned correction is the first record of least weight. */
typedef struct {
    int32_t cap, n;
    int32_t *leg, *iter;
    double *weight;
    uint32_t *bits;
} sol_rec_t;

static void decode_one(const graph_t *g, const oracle_params *P, const learned_t *LP, const uint32_t *syn,
                       uint64_t shot, uint32_t *corr, int32_t *stats, double *weight, int trace_iters,
                       double *trace, double *nu, double *mu, double *M, double *Lam, double *gam, uint8_t *ehat,
                       uint8_t *best, double *final_post, sol_rec_t *rec)
{
    const int32_t V = g->n_loc, C = g->n_det, E = g->rptr[C];
    const double *L0 = g->L0;
    int32_t nsol = 0, legs = 0, iters = 0, have_best = 0;
    double best_w = 0.0;
    for (int32_t j = 0; j < V; ++j) M[j] = L0[j];
    for (int32_t e = 0; e < E; ++e) nu[e] = 0.0;
    memset(ehat, 0, (size_t)V);
    for (int32_t leg = 0; leg <= P->num_sets; ++leg) {
        legs++;
        const int lleg = LP && (LP->legs < 0 || leg < LP->legs);
        for (int32_t j = 0; j < V; ++j) {
            if (leg == 0) gam[j] = P->gamma0;
            else if (lleg && LP->knots) {
                uint64_t nblk = ((uint64_t)V + 3) / 4;
                uint32_t wd = stream_word(P->seed, shot, 1u, (uint64_t)leg * nblk * 4 + (uint64_t)j);
                gam[j] = knot_gamma_l(LP->knots, LP->K, (double)(wd >> 8) * (1.0 / 16777216.0));
            } else gam[j] = draw_gamma(P, shot, leg, j, V);
        }
        if (leg > 0 && !P->carry_messages)
            for (int32_t e = 0; e < E; ++e) nu[e] = 0.0;
        int32_t T = (leg == 0) ? P->pre_iter : P->max_iterations;
        int converged = 0;
        for (int32_t t = 1; t <= T && !converged; ++t) {
            /* a4 (first half): memory-biased prior */
            for (int32_t j = 0; j < V; ++j) Lam[j] = (1.0 - gam[j]) * L0[j] + gam[j] * M[j];
            /* variable-to-check messages: prior plus every other incoming message */
            for (int32_t j = 0; j < V; ++j)
                for (int32_t a = g->cptr[j]; a < g->cptr[j + 1]; ++a) {
                    int32_t e = g->cedge[a];
                    double s = Lam[j];
                    for (int32_t b = g->cptr[j]; b < g->cptr[j + 1]; ++b)
                        if (b != a) s += nu[g->cedge[b]];
                    mu[e] = s;
                }
            /* a3: min-sum check update, leave-one-out by direct loops */
            /* learned weights for the first T iterations of a learned leg, unit weights past them */
            const double *wt = (lleg && LP->w && t - 1 < LP->T) ? LP->w + (int64_t)(t - 1) * E : NULL;
            for (int32_t i = 0; i < C; ++i) {
                double ssign = get_bit(syn, i) ? -1.0 : 1.0;
                for (int32_t e = g->rptr[i]; e < g->rptr[i + 1]; ++e) {
                    double prod = ssign, mn = INFINITY;
                    for (int32_t f = g->rptr[i]; f < g->rptr[i + 1]; ++f) {
                        if (f == e) continue;
                        prod *= sgn(mu[f]);
                        double m = fabs(mu[f]);
                        if (m < mn) mn = m;
                    }
                    nu[e] = wt ? wt[e] * prod * mn : prod * mn;   /* a degree-1 check sends +-inf */
                }
            }
            /* a4 (second half): marginals and hard decisions */
            for (int32_t j = 0; j < V; ++j) {
                double s = Lam[j];
                for (int32_t a = g->cptr[j]; a < g->cptr[j + 1]; ++a) s += nu[g->cedge[a]];
                M[j] = s;
                ehat[j] = (uint8_t)(s < 0.0);
            }
            iters++;
            if (trace && iters <= trace_iters)
                for (int32_t j = 0; j < V; ++j) trace[(int64_t)(iters - 1) * V + j] = M[j];
            /* a5: residual H e^ + s */
            int ok = 1;
            for (int32_t i = 0; i < C && ok; ++i) {
                int par = get_bit(syn, i);
                for (int32_t e = g->rptr[i]; e < g->rptr[i + 1]; ++e) par ^= ehat[g->rcol[e]];
                if (par) ok = 0;
            }
            if (ok) {
                converged = 1;
                double w = 0.0;                                  /* a7: FP64 weight */
                for (int32_t j = 0; j < V; ++j) if (ehat[j]) w += L0[j];
                nsol++;
                if (rec && rec->n < rec->cap) {
                    const int32_t wv = (V + 31) / 32;
                    uint32_t *rb = rec->bits + (int64_t)rec->n * wv;
                    memset(rb, 0, sizeof(uint32_t) * (size_t)wv);
                    for (int32_t j = 0; j < V; ++j) if (ehat[j]) flip_bit(rb, j);
                    rec->leg[rec->n] = leg;
                    rec->iter[rec->n] = iters;
                    rec->weight[rec->n] = w;
                    rec->n++;
                }
                if (!have_best || w < best_w) {
                    have_best = 1;
                    best_w = w;
                    memcpy(best, ehat, (size_t)V);
                }
            }
        }
        if (!P->stop_all && nsol >= P->stop_nconv) break;
    }
    const uint8_t *out = have_best ? best : ehat;
    double w = 0.0;
    for (int32_t j = 0; j < V; ++j) if (out[j]) w += L0[j];
    memset(corr, 0, sizeof(uint32_t) * (size_t)((V + 31) / 32));
    for (int32_t j = 0; j < V; ++j) if (out[j]) flip_bit(corr, j);
    stats[0] = have_best;
    stats[1] = nsol;
    stats[2] = legs;
    stats[3] = iters;
    *weight = w;
    if (final_post) memcpy(final_post, M, sizeof(double) * (size_t)V);     /* marginals after the last iteration */
}

/* Decode `shots` syndromes.  stats: [shots][4] = converged, #solutions, legs,
 * iterations; weights: [shots] FP64 weight of the returned correction; trace
 * (optional): [shots][trace_iters][n_loc] marginals M after each iteration.
 * Returns 0, or -1 on invalid input. */
static int decode_impl(int32_t n_det, int32_t n_loc, int32_t n_obs,
                       const int32_t *H_indptr, const int32_t *H_indices,
                       const int32_t *O_indptr, const int32_t *O_indices,
                       const double *priors, const oracle_params *P, const learned_t *LP,
                       const uint32_t *syndromes, uint64_t shot0, int64_t shots,
                       uint32_t *corrections, uint32_t *pred_obs, int32_t *stats, double *weights,
                       int32_t trace_iters, double *trace, double *final_post, int32_t n_threads,
                       sol_rec_t *rec);

int oracle_relaybp_decode(int32_t n_det, int32_t n_loc, int32_t n_obs,
                          const int32_t *H_indptr, const int32_t *H_indices,
                          const int32_t *O_indptr, const int32_t *O_indices,
                          const double *priors, const oracle_params *P,
                          const uint32_t *syndromes, uint64_t shot0, int64_t shots,
                          uint32_t *corrections, uint32_t *pred_obs, int32_t *stats, double *weights,
                          int32_t trace_iters, double *trace, int32_t n_threads)
{
    return decode_impl(n_det, n_loc, n_obs, H_indptr, H_indices, O_indptr, O_indices, priors, P, NULL, syndromes,
                       shot0, shots, corrections, pred_obs, stats, weights, trace_iters, trace, NULL, n_threads, NULL);
}

/* Same, also writing each shot's marginals M after its last iteration to
 * final_post [shots][n_loc] (the soft output that OSD post-processing of a
 * nonconverged shot orders its columns by). */
int oracle_relaybp_decode_post(int32_t n_det, int32_t n_loc, int32_t n_obs,
                               const int32_t *H_indptr, const int32_t *H_indices,
                               const int32_t *O_indptr, const int32_t *O_indices,
                               const double *priors, const oracle_params *P,
                               const uint32_t *syndromes, uint64_t shot0, int64_t shots,
                               uint32_t *corrections, uint32_t *pred_obs, int32_t *stats, double *weights,
                               double *final_post, int32_t n_threads)
{
    return decode_impl(n_det, n_loc, n_obs, H_indptr, H_indices, O_indptr, O_indices, priors, P, NULL, syndromes,
                       shot0, shots, corrections, pred_obs, stats, weights, 0, NULL, final_post, n_threads, NULL);
}

/* One shot's decode with every solution it finds recorded (sol_rec_t above):
 * up to `cap` records of leg, iteration count, weight and packed bits
 * [cap][ceil(n_loc/32)]; *n_found = solutions found (may exceed cap).
 * Single-threaded.  Returns 0, or -1 on invalid input. */
int oracle_relaybp_solutions(int32_t n_det, int32_t n_loc, const int32_t *H_indptr, const int32_t *H_indices,
                             const double *priors, const oracle_params *P, const uint32_t *syndrome, uint64_t shot,
                             uint32_t *correction, int32_t *stats, double *weight, int32_t cap, int32_t *rec_leg,
                             int32_t *rec_iter, double *rec_weight, uint32_t *rec_bits, int32_t *n_found)
{
    if (cap < 0 || (cap > 0 && (!rec_leg || !rec_iter || !rec_weight || !rec_bits)) || !n_found) return -1;
    sol_rec_t rec = {cap, 0, rec_leg, rec_iter, rec_weight, rec_bits};
    int rc = decode_impl(n_det, n_loc, 0, H_indptr, H_indices, NULL, NULL, priors, P, NULL, syndrome, shot, 1,
                         correction, NULL, stats, weight, 0, NULL, NULL, 1, &rec);
    *n_found = rc == 0 ? stats[1] : 0;
    return rc;
}

/* Relay-BP with learned parameters: w [T][E] (or NULL), knots [K+1] (or NULL). */
int oracle_relaybp_decode_learned(int32_t n_det, int32_t n_loc, int32_t n_obs,
                                  const int32_t *H_indptr, const int32_t *H_indices,
                                  const int32_t *O_indptr, const int32_t *O_indices,
                                  const double *priors, const oracle_params *P,
                                  int32_t T, const double *w, int32_t K, const double *knots, int32_t legs,
                                  const uint32_t *syndromes, uint64_t shot0, int64_t shots,
                                  uint32_t *corrections, uint32_t *pred_obs, int32_t *stats, double *weights,
                                  int32_t trace_iters, double *trace, int32_t n_threads)
{
    if ((w && T < 1) || (knots && K < 1) || (w && P->carry_messages)) return -1;
    learned_t LP = {T, K, w, knots, legs};
    return decode_impl(n_det, n_loc, n_obs, H_indptr, H_indices, O_indptr, O_indices, priors, P, &LP, syndromes,
                       shot0, shots, corrections, pred_obs, stats, weights, trace_iters, trace, NULL, n_threads, NULL);
}

static int decode_impl(int32_t n_det, int32_t n_loc, int32_t n_obs,
                       const int32_t *H_indptr, const int32_t *H_indices,
                       const int32_t *O_indptr, const int32_t *O_indices,
                       const double *priors, const oracle_params *P, const learned_t *LP,
                       const uint32_t *syndromes, uint64_t shot0, int64_t shots,
                       uint32_t *corrections, uint32_t *pred_obs, int32_t *stats, double *weights,
                       int32_t trace_iters, double *trace, double *final_post, int32_t n_threads,
                       sol_rec_t *rec)
{
    if (n_det < 0 || n_loc < 0 || shots < 0 || !P) return -1;
    if (rec && shots != 1) return -1;                         /* a record covers one shot */
    if (P->pre_iter < 0 || P->max_iterations < 0 || P->num_sets < 0 || P->stop_nconv < 1) return -1;
    int64_t wd = (n_det + 31) / 32, wv = (n_loc + 31) / 32, wo = (n_obs + 31) / 32;
    int32_t E = H_indptr[n_det];
    double *L0 = malloc(sizeof(double) * (size_t)(n_loc + 1));
    for (int32_t j = 0; j < n_loc; ++j) {
        double p = priors[j];
        if (!(p > 0.0 && p < 1.0)) { free(L0); return -1; }
        L0[j] = log((1.0 - p) / p);                          /* a1 */
    }
    for (int32_t e = 0; e < E; ++e)
        if (H_indices[e] < 0 || H_indices[e] >= n_loc) { free(L0); return -1; }
    graph_t g;
    g.n_det = n_det; g.n_loc = n_loc; g.rptr = H_indptr; g.rcol = H_indices; g.L0 = L0;
    g.cptr = calloc((size_t)n_loc + 1, sizeof(int32_t));
    g.cedge = malloc(sizeof(int32_t) * (size_t)(E + 1));
    for (int32_t e = 0; e < E; ++e) g.cptr[H_indices[e] + 1]++;
    for (int32_t j = 0; j < n_loc; ++j) g.cptr[j + 1] += g.cptr[j];
    {
        int32_t *fill = calloc((size_t)n_loc + 1, sizeof(int32_t));
        for (int32_t i = 0; i < n_det; ++i)
            for (int32_t e = H_indptr[i]; e < H_indptr[i + 1]; ++e) {
                int32_t j = H_indices[e];
                g.cedge[g.cptr[j] + fill[j]++] = e;
            }
        free(fill);
    }
#ifdef _OPENMP
    omp_set_num_threads(n_threads > 0 ? n_threads : omp_get_num_procs());   /* <= 0: every core */
#else
    (void)n_threads;
#endif
#pragma omp parallel
    {
        double *nu = malloc(sizeof(double) * (size_t)(E + 1));
        double *mu = malloc(sizeof(double) * (size_t)(E + 1));
        double *M = malloc(sizeof(double) * (size_t)(n_loc + 1));
        double *Lam = malloc(sizeof(double) * (size_t)(n_loc + 1));
        double *gam = malloc(sizeof(double) * (size_t)(n_loc + 1));
        uint8_t *ehat = malloc((size_t)n_loc + 1);
        uint8_t *best = malloc((size_t)n_loc + 1);
#pragma omp for schedule(dynamic, 1)
        for (int64_t s = 0; s < shots; ++s) {
            uint32_t *corr = corrections + s * wv;
            decode_one(&g, P, LP, syndromes + s * wd, shot0 + (uint64_t)s, corr, stats + 4 * s, weights + s,
                       trace_iters, trace ? trace + s * (int64_t)trace_iters * n_loc : NULL,
                       nu, mu, M, Lam, gam, ehat, best, final_post ? final_post + s * (int64_t)n_loc : NULL, rec);
            if (pred_obs) {
                uint32_t *po = pred_obs + s * wo;
                memset(po, 0, sizeof(uint32_t) * (size_t)wo);
                for (int32_t i = 0; i < n_obs; ++i) {
                    int par = 0;
                    for (int32_t e = O_indptr[i]; e < O_indptr[i + 1]; ++e) par ^= get_bit(corr, O_indices[e]);
                    if (par) flip_bit(po, i);
                }
            }
        }
        free(nu); free(mu); free(M); free(Lam); free(gam); free(ehat); free(best);
    }
    free(L0); free(g.cptr); free(g.cedge);
    return 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_num_procs();             /* what a call with n_threads <= 0 uses */
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* a10: learned form (not in the paper; the design of this library)          */
/* ------------------------------------------------------------------------- */
/* Learned parameters:
 *   w[t][e]  per-iteration, per-edge weights of the check-to-variable messages,
 *            nu_e(t) = w[t-1][e] * (-1)^{s_i} prod_{f != e} sgn(mu_f) * min_{f != e} |mu_f|,
 *            t = 1..T (iterations past T reuse w[T-1]); e in row-major edge order;
 *   knots[0..K] nondecreasing: the inverse CDF of the memory strengths,
 *            g(u) = knots[k] + (knots[k+1] - knots[k]) * (u*K - k), k = floor(u*K),
 *            u the same 24-bit stream-1 draw as the plain method's legs.
 * Training objective for one shot: T iterations of one memory-BP leg started
 * from M = L0, nu = 0, with g_j = g(u_j) of leg 1, and
 *   loss = sum_t sum_j BCE(M_j(t), e_j),
 *   BCE(M, e) = e * softplus(M) + (1 - e) * softplus(-M)
 * (the error probability of bit j is sigmoid(-M_j)).  Plain loops, FP64. */
static double softplus(double x) { return x > 0 ? x + log1p(exp(-x)) : log1p(exp(x)); }

/* Second training objective (project choice): the soft syndrome.  With the
 * bits independent and bit j in error with probability sigmoid(-M_j), check
 * i holds its syndrome bit s_i with probability
 *   P_i = (1 + (-1)^{s_i} prod_{j in row i} tanh(M_j / 2)) / 2,
 * and the loss of iteration t is -sum_i log(eps + (1 - 2 eps) P_i(t)), summed
 * over the T unrolled iterations: it rewards satisfying every check early,
 * which is what ends a decode.  eps bounds the loss of a confidently violated
 * check. */
#define SOFT_SYN_EPS 1e-6

static double knot_gamma(const double *knots, int32_t K, double u)
{
    double x = u * (double)K;
    int32_t k = (int32_t)floor(x);
    if (k >= K) k = K - 1;
    double f = x - (double)k;
    return knots[k] + (knots[k + 1] - knots[k]) * f;
}

static double draw_u(uint64_t seed, uint64_t shot, int32_t leg, int32_t j, int32_t n_loc)
{
    uint64_t nblk = ((uint64_t)n_loc + 3) / 4;
    uint32_t w = stream_word(seed, shot, 1u, (uint64_t)leg * nblk * 4 + (uint64_t)j);
    return (double)(w >> 8) * (1.0 / 16777216.0);
}

/* Loss of each shot under the learned forward (trace optional: [shots][T][V]). */
int oracle_learned_loss(int32_t n_det, int32_t n_loc, const int32_t *H_indptr, const int32_t *H_indices,
                        const double *priors, int32_t T, const double *w, int32_t K, const double *knots,
                        uint64_t gamma_seed, const uint32_t *syndromes, const uint32_t *errors, uint64_t shot0,
                        int64_t shots, int32_t objective, double *loss, double *trace, int32_t n_threads)
{
    if (n_det < 0 || n_loc < 0 || shots < 0 || T < 1 || K < 1 || objective < 0 || objective > 1) return -1;
    const int32_t E = H_indptr[n_det];
    int64_t wd = (n_det + 31) / 32, wv = (n_loc + 31) / 32;
    double *L0 = malloc(sizeof(double) * (size_t)(n_loc + 1));
    for (int32_t j = 0; j < n_loc; ++j) {
        double p = priors[j];
        if (!(p > 0.0 && p < 1.0)) { free(L0); return -1; }
        L0[j] = log((1.0 - p) / p);
    }
    int32_t *cptr = calloc((size_t)n_loc + 1, sizeof(int32_t));
    int32_t *cedge = malloc(sizeof(int32_t) * (size_t)(E + 1));
    for (int32_t e = 0; e < E; ++e) cptr[H_indices[e] + 1]++;
    for (int32_t j = 0; j < n_loc; ++j) cptr[j + 1] += cptr[j];
    {
        int32_t *fill = calloc((size_t)n_loc + 1, sizeof(int32_t));
        for (int32_t i = 0; i < n_det; ++i)
            for (int32_t e = H_indptr[i]; e < H_indptr[i + 1]; ++e) {
                int32_t j = H_indices[e];
                cedge[cptr[j] + fill[j]++] = e;
            }
        free(fill);
    }
#ifdef _OPENMP
    omp_set_num_threads(n_threads > 0 ? n_threads : omp_get_num_procs());   /* <= 0: every core */
#else
    (void)n_threads;
#endif
#pragma omp parallel
    {
        double *nu = malloc(sizeof(double) * (size_t)(E + 1));
        double *mu = malloc(sizeof(double) * (size_t)(E + 1));
        double *M = malloc(sizeof(double) * (size_t)(n_loc + 1));
        double *Lam = malloc(sizeof(double) * (size_t)(n_loc + 1));
        double *gam = malloc(sizeof(double) * (size_t)(n_loc + 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t s = 0; s < shots; ++s) {
            const uint32_t *syn = syndromes + s * wd;
            const uint32_t *err = errors + s * wv;
            uint64_t shot = shot0 + (uint64_t)s;
            double acc = 0.0;
            for (int32_t j = 0; j < n_loc; ++j) {
                M[j] = L0[j];
                gam[j] = knot_gamma(knots, K, draw_u(gamma_seed, shot, 1, j, n_loc));
            }
            for (int32_t e = 0; e < E; ++e) nu[e] = 0.0;
            for (int32_t t = 1; t <= T; ++t) {
                const double *wt = w + (int64_t)(t - 1) * E;
                for (int32_t j = 0; j < n_loc; ++j) Lam[j] = (1.0 - gam[j]) * L0[j] + gam[j] * M[j];
                for (int32_t j = 0; j < n_loc; ++j)
                    for (int32_t a = cptr[j]; a < cptr[j + 1]; ++a) {
                        double v = Lam[j];
                        for (int32_t b = cptr[j]; b < cptr[j + 1]; ++b)
                            if (b != a) v += nu[cedge[b]];
                        mu[cedge[a]] = v;
                    }
                for (int32_t i = 0; i < n_det; ++i) {
                    double ssign = get_bit(syn, i) ? -1.0 : 1.0;
                    for (int32_t e = H_indptr[i]; e < H_indptr[i + 1]; ++e) {
                        double prod = ssign, mn = INFINITY;
                        for (int32_t f = H_indptr[i]; f < H_indptr[i + 1]; ++f) {
                            if (f == e) continue;
                            prod *= sgn(mu[f]);
                            double m = fabs(mu[f]);
                            if (m < mn) mn = m;
                        }
                        nu[e] = wt[e] * prod * mn;
                    }
                }
                for (int32_t j = 0; j < n_loc; ++j) {
                    double v = Lam[j];
                    for (int32_t a = cptr[j]; a < cptr[j + 1]; ++a) v += nu[cedge[a]];
                    M[j] = v;
                    int e_j = get_bit(err, j);
                    if (objective == 0) acc += e_j ? softplus(v) : softplus(-v);
                    if (trace) trace[((int64_t)s * T + (t - 1)) * n_loc + j] = v;
                }
                if (objective == 1)             /* soft syndrome: -log P(check i satisfied) */
                    for (int32_t i = 0; i < n_det; ++i) {
                        double prod = 1.0;
                        for (int32_t e = H_indptr[i]; e < H_indptr[i + 1]; ++e) prod *= tanh(0.5 * M[H_indices[e]]);
                        const double sat = 0.5 * (1.0 + (get_bit(syn, i) ? -prod : prod));
                        acc -= log(SOFT_SYN_EPS + (1.0 - 2.0 * SOFT_SYN_EPS) * sat);
                    }
            }
            loss[s] = acc;
        }
        free(nu); free(mu); free(M); free(Lam); free(gam);
    }
    free(L0); free(cptr); free(cedge);
    return 0;
}


static double knot_gamma_l(const double *knots, int32_t K, double u) { return knot_gamma(knots, K, u); }


/* Minimum weight of a nonzero codeword of the binary code spanned by k <= 63
 * generator rows of length n <= 64 (row r: bit c of gens[r] = entry c), by
 * Gray-code enumeration of all 2^k - 1 nonzero codewords: consecutive Gray
 * codes differ in one generator, so each step is one XOR and one popcount.
 * Test infrastructure for the code-builder pin of Table 2 (ZSZ-2BGA-64 is a
 * [64, 32, 10] code); the top bits of the message are split over threads.
 * Returns the distance, or -1 on bad sizes. */
int oracle_min_weight(int32_t k, int32_t n, const uint64_t *gens, int32_t n_threads)
{
    if (k < 1 || k > 63 || n < 1 || n > 64) return -1;
    const int top = k > 8 ? 8 : k - 1;             /* message bits fixed per task */
    const int low = k - top;
    const int64_t tasks = (int64_t)1 << top;
    int best = n + 1;
#ifdef _OPENMP
    omp_set_num_threads(n_threads > 0 ? n_threads : omp_get_num_procs());   /* <= 0: every core */
#else
    (void)n_threads;
#endif
#pragma omp parallel for schedule(dynamic, 1) reduction(min : best)
    for (int64_t task = 0; task < tasks; ++task) {
        uint64_t w = 0;                            /* codeword of message (task << low) */
        for (int b = 0; b < top; ++b)
            if ((task >> b) & 1) w ^= gens[low + b];
        int mine = n + 1;
        if (w) mine = __builtin_popcountll(w);
        for (uint64_t g = 1; g < ((uint64_t)1 << low); ++g) {
            w ^= gens[__builtin_ctzll(g)];         /* Gray code g ^ (g >> 1) steps by one bit */
            int c = __builtin_popcountll(w);
            if (c < mine && w) mine = c;
        }
        if (mine < best) best = mine;
    }
    return best;
}
