/*
 * awgn_oracle.c -- plain FP64 CPU oracle for the classical channel-coding
 * workload: BPSK over the additive white Gaussian noise channel, decoded by
 * flooding sum-product belief propagation; and OSD-0 post-processing of
 * decoder outputs (at the end of the file).
 *
 * TEST INFRASTRUCTURE ONLY, like relaybp_oracle.c (compiled into the same
 * library, sharing its Philox4x32-10): nothing on the product path may link,
 * load or call it.
 *
 * What it computes (arXiv 2607.27644, Sec. 6.2, classical channel coding):
 *   codeword bit c_i -> symbol x_i = (-1)^{c_i}; received y_i = x_i + sigma z_i,
 *   z_i ~ N(0, 1); channel LLR L_i = 2 y_i / sigma^2, clipped to +-llr_max;
 *   sum-product BP, flooding schedule, check update in the "boxplus-phi" form
 *     nu_{i->j} = prod_{j' != j} sgn(mu_{j'->i}) * phi(sum_{j' != j} phi(|mu_{j'->i}|)),
 *     phi(x) = -log(tanh(x / 2)) = log1p(2 / expm1(x)),
 *   mu_{j->i} = L_j + sum_{i' != i} nu_{i'->j}, posterior M_j = L_j + sum_i nu_{i->j},
 *   hard decision c^_j = [M_j < 0], at most max_iter iterations.
 * Readings where the text is silent: messages (both directions) are clipped to
 * +-llr_max like the channel LLRs; with early_stop the decoder stops at the
 * first iteration whose hard decision satisfies every check.
 *
 * Gaussian draws: z_i of shot s from the Box-Muller transform of words 2i and
 * 2i+1 of Philox stream 2 (key = seed, counter (word/4, shot lo, shot hi, 2)):
 * u = (w + 0.5) / 2^32, z = sqrt(-2 ln u1) cos(2 pi u2).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]);

static uint32_t awgn_word(uint64_t seed, uint64_t shot, uint64_t j)
{
    uint32_t ctr[4], key[2], out[4];
    ctr[0] = (uint32_t)(j / 4);
    ctr[1] = (uint32_t)(shot & 0xffffffffu);
    ctr[2] = (uint32_t)(shot >> 32);
    ctr[3] = 2u;
    key[0] = (uint32_t)(seed & 0xffffffffu);
    key[1] = (uint32_t)(seed >> 32);
    oracle_philox4x32_10(ctr, key, out);
    return out[j % 4];
}

static double clip(double v, double m) { return v > m ? m : (v < -m ? -m : v); }

/* Channel LLRs of `shots` transmissions of the codewords `codewords`
 * [shots][ceil(n/32)] (NULL: the all-zero codeword) at noise deviation sigma:
 * out_llr [shots][n].  Returns 0, or -1 on bad sizes. */
int oracle_awgn_llr(int32_t n, const uint32_t *codewords, double sigma, double llr_max, uint64_t seed,
                    uint64_t shot0, int64_t shots, double *out_llr)
{
    if (n < 1 || shots < 0 || !(sigma > 0.0)) return -1;
    const int64_t wn = (n + 31) / 32;
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t s = 0; s < shots; ++s) {
        const uint64_t shot = shot0 + (uint64_t)s;
        for (int32_t i = 0; i < n; ++i) {
            const double u1 = ((double)awgn_word(seed, shot, 2 * (uint64_t)i) + 0.5) / 4294967296.0;
            const double u2 = ((double)awgn_word(seed, shot, 2 * (uint64_t)i + 1) + 0.5) / 4294967296.0;
            const double z = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
            const int c = codewords ? (int)((codewords[s * wn + i / 32] >> (i % 32)) & 1u) : 0;
            const double y = (c ? -1.0 : 1.0) + sigma * z;
            out_llr[s * n + i] = clip(2.0 * y / (sigma * sigma), llr_max);
        }
    }
    return 0;
}

static double phi(double x) { return log1p(2.0 / expm1(x)); }   /* phi(0) = inf, phi(inf) = 0 */

/* Flooding sum-product decode of `shots` LLR vectors llr [shots][n] for the
 * m x n parity-check matrix (CSR indptr/indices).  Outputs per shot: the hard
 * decision out_bits [shots][ceil(n/32)], iterations run out_iters[shots],
 * whether the decision satisfies every check out_valid[shots], and (if not
 * NULL) the posteriors out_post [shots][n].  Returns 0, or -1 on bad sizes. */
int oracle_sum_product(int32_t m, int32_t n, const int32_t *indptr, const int32_t *indices, const double *llr,
                       int64_t shots, int32_t max_iter, double llr_max, int32_t early_stop, uint32_t *out_bits,
                       int32_t *out_iters, int32_t *out_valid, double *out_post, int32_t n_threads)
{
    if (m < 0 || n < 1 || shots < 0 || max_iter < 1) return -1;
    const int32_t E = indptr[m];
    const int64_t wn = (n + 31) / 32;
    /* column lists: for each variable the edges (row-major indices) touching it */
    int32_t *cptr = calloc((size_t)n + 1, sizeof(int32_t));
    int32_t *cedge = malloc(sizeof(int32_t) * (size_t)(E + 1));
    for (int32_t e = 0; e < E; ++e) cptr[indices[e] + 1]++;
    for (int32_t j = 0; j < n; ++j) cptr[j + 1] += cptr[j];
    {
        int32_t *fill = calloc((size_t)n + 1, sizeof(int32_t));
        for (int32_t i = 0; i < m; ++i)
            for (int32_t e = indptr[i]; e < indptr[i + 1]; ++e) {
                const int32_t j = indices[e];
                cedge[cptr[j] + fill[j]++] = e;
            }
        free(fill);
    }
#ifdef _OPENMP
    omp_set_num_threads(n_threads > 0 ? n_threads : omp_get_num_procs());
#else
    (void)n_threads;
#endif
#pragma omp parallel
    {
        double *nu = malloc(sizeof(double) * (size_t)(E + 1));
        double *mu = malloc(sizeof(double) * (size_t)(E + 1));
        double *post = malloc(sizeof(double) * (size_t)n);
        int *hard = malloc(sizeof(int) * (size_t)n);
#pragma omp for schedule(dynamic, 1)
        for (int64_t s = 0; s < shots; ++s) {
            const double *L = llr + s * n;
            for (int32_t e = 0; e < E; ++e) nu[e] = 0.0;
            int it = 0, valid = 0;
            for (it = 1; it <= max_iter; ++it) {
                /* variable-to-check: leave-one-out sums, clipped */
                for (int32_t j = 0; j < n; ++j)
                    for (int32_t a = cptr[j]; a < cptr[j + 1]; ++a) {
                        double v = L[j];
                        for (int32_t b = cptr[j]; b < cptr[j + 1]; ++b)
                            if (b != a) v += nu[cedge[b]];
                        mu[cedge[a]] = clip(v, llr_max);
                    }
                /* check-to-variable: sign product and phi of the phi-sum over the others */
                for (int32_t i = 0; i < m; ++i)
                    for (int32_t e = indptr[i]; e < indptr[i + 1]; ++e) {
                        double sg = 1.0, acc = 0.0;
                        for (int32_t f = indptr[i]; f < indptr[i + 1]; ++f) {
                            if (f == e) continue;
                            if (mu[f] < 0.0) sg = -sg;
                            acc += phi(fabs(mu[f]));
                        }
                        nu[e] = clip(sg * phi(acc), llr_max);
                    }
                /* posteriors and hard decision */
                for (int32_t j = 0; j < n; ++j) {
                    double v = L[j];
                    for (int32_t a = cptr[j]; a < cptr[j + 1]; ++a) v += nu[cedge[a]];
                    post[j] = v;
                    hard[j] = v < 0.0;
                }
                valid = 1;
                for (int32_t i = 0; i < m && valid; ++i) {
                    int par = 0;
                    for (int32_t e = indptr[i]; e < indptr[i + 1]; ++e) par ^= hard[indices[e]];
                    if (par) valid = 0;
                }
                if (early_stop && valid) break;
            }
            if (it > max_iter) it = max_iter;
            uint32_t *bits = out_bits + s * wn;
            memset(bits, 0, sizeof(uint32_t) * (size_t)wn);
            for (int32_t j = 0; j < n; ++j)
                if (hard[j]) bits[j / 32] |= 1u << (j % 32);
            out_iters[s] = it;
            out_valid[s] = valid;
            if (out_post) memcpy(out_post + s * n, post, sizeof(double) * (size_t)n);
        }
        free(nu); free(mu); free(post); free(hard);
    }
    free(cptr); free(cedge);
    return 0;
}


/* ------------------------------------------------------------------------- */
/* OSD-0 post-processing (the outlook of Sec. 7, improved decoding, names  */
/* ordered-statistics decoding for the flagged nonconvergences)            */
/* ------------------------------------------------------------------------- */
/* For each shot: order the n columns by the soft value `soft` ascending (the
 * most negative posterior LLR, i.e. the most likely error, first; ties by
 * index), take the first columns that are linearly independent over GF(2)
 * (the information set, rank(H) of them) and solve H e = s on them (OSD-0).
 * With order lambda > 0 (combination sweep): every set T of one or two of the
 * first lambda columns outside the information set, in the same order, is
 * also tried -- e_T = 1 and the information-set bits re-solved -- and the
 * candidate of least weight sum_j e_j w_j (w = col_weights, the prior LLRs)
 * is kept, OSD-0's on ties.  out_valid[s] = 0 when s is not in the column
 * space of H.  Plain dense GF(2) elimination, one byte per entry.  Returns 0,
 * or -1 on bad sizes. */
int oracle_osd(int32_t m, int32_t n, const int32_t *indptr, const int32_t *indices, const uint32_t *syndromes,
               const double *soft, const double *col_weights, int32_t lambda, int64_t shots, uint32_t *out_e,
               int32_t *out_valid, int32_t n_threads)
{
    if (m < 1 || n < 1 || shots < 0 || lambda < 0 || (lambda > 0 && !col_weights)) return -1;
    const int64_t wm = (m + 31) / 32, wn = (n + 31) / 32;
#ifdef _OPENMP
    omp_set_num_threads(n_threads > 0 ? n_threads : omp_get_num_procs());
#else
    (void)n_threads;
#endif
#pragma omp parallel
    {
        unsigned char *A = malloc((size_t)m * (size_t)(n + 1));     /* [H_perm | s], row-major */
        int32_t *order = malloc(sizeof(int32_t) * (size_t)n);
        int32_t *pivcol = malloc(sizeof(int32_t) * (size_t)m);
        unsigned char *ispiv = malloc((size_t)n);
        int32_t *free_cols = malloc(sizeof(int32_t) * (size_t)n);
        unsigned char *x = malloc((size_t)m + 1), *bestx = malloc((size_t)m + 1);
#pragma omp for schedule(dynamic, 1)
        for (int64_t s = 0; s < shots; ++s) {
            const double *q = soft + s * n;
            for (int32_t j = 0; j < n; ++j) order[j] = j;
            /* insertion sort by (q, index): plain and stable */
            for (int32_t a = 1; a < n; ++a) {
                const int32_t v = order[a];
                int32_t b = a - 1;
                while (b >= 0 && (q[order[b]] > q[v])) { order[b + 1] = order[b]; --b; }
                order[b + 1] = v;
            }
            memset(A, 0, (size_t)m * (size_t)(n + 1));
            for (int32_t i = 0; i < m; ++i) {
                for (int32_t e = indptr[i]; e < indptr[i + 1]; ++e) A[(size_t)i * (n + 1) + indices[e]] = 1;
                A[(size_t)i * (n + 1) + n] = (unsigned char)((syndromes[s * wm + i / 32] >> (i % 32)) & 1u);
            }
            /* forward elimination to reduced form over the columns in the chosen order */
            memset(ispiv, 0, (size_t)n);
            int32_t r = 0;
            for (int32_t t = 0; t < n && r < m; ++t) {
                const int32_t c = order[t];
                int32_t p = -1;
                for (int32_t i = r; i < m; ++i)
                    if (A[(size_t)i * (n + 1) + c]) { p = i; break; }
                if (p < 0) continue;
                if (p != r)
                    for (int32_t k = 0; k <= n; ++k) {
                        unsigned char tmp = A[(size_t)p * (n + 1) + k];
                        A[(size_t)p * (n + 1) + k] = A[(size_t)r * (n + 1) + k];
                        A[(size_t)r * (n + 1) + k] = tmp;
                    }
                for (int32_t i = 0; i < m; ++i)
                    if (i != r && A[(size_t)i * (n + 1) + c])
                        for (int32_t k = 0; k <= n; ++k) A[(size_t)i * (n + 1) + k] ^= A[(size_t)r * (n + 1) + k];
                pivcol[r++] = c;
                ispiv[c] = 1;
            }
            int valid = 1;
            for (int32_t i = r; i < m; ++i)
                if (A[(size_t)i * (n + 1) + n]) valid = 0;          /* 0 = 1 row: s outside the column space */
            /* OSD-0: information-set bits = reduced right-hand side */
            for (int32_t i = 0; i < r; ++i) bestx[i] = A[(size_t)i * (n + 1) + n];
            int32_t bt1 = -1, bt2 = -1;                            /* best flipped non-pivot columns */
            if (lambda > 0) {
                int32_t nf = 0;
                for (int32_t t = 0; t < n && nf < lambda; ++t)
                    if (!ispiv[order[t]]) free_cols[nf++] = order[t];
                double bestw = 0.0;
                for (int32_t i = 0; i < r; ++i) if (bestx[i]) bestw += col_weights[pivcol[i]];
                for (int32_t u = 0; u < nf; ++u)
                    for (int32_t v = u; v < nf; ++v) {             /* v == u: the single flip */
                        const int32_t c1 = free_cols[u], c2 = free_cols[v];
                        double w = col_weights[c1] + (v != u ? col_weights[c2] : 0.0);
                        for (int32_t i = 0; i < r; ++i) {
                            unsigned char bit = A[(size_t)i * (n + 1) + n] ^ A[(size_t)i * (n + 1) + c1];
                            if (v != u) bit ^= A[(size_t)i * (n + 1) + c2];
                            x[i] = bit;
                            if (bit) w += col_weights[pivcol[i]];
                        }
                        if (w < bestw) {
                            bestw = w;
                            memcpy(bestx, x, (size_t)r);
                            bt1 = c1;
                            bt2 = (v != u) ? c2 : -1;
                        }
                    }
            }
            uint32_t *e = out_e + s * wn;
            memset(e, 0, sizeof(uint32_t) * (size_t)wn);
            for (int32_t i = 0; i < r; ++i)
                if (bestx[i]) e[pivcol[i] / 32] |= 1u << (pivcol[i] % 32);
            if (bt1 >= 0) e[bt1 / 32] |= 1u << (bt1 % 32);
            if (bt2 >= 0) e[bt2 / 32] |= 1u << (bt2 % 32);
            out_valid[s] = valid;
        }
        free(A); free(order); free(pivcol); free(ispiv); free(free_cols); free(x); free(bestx);
    }
    return 0;
}
