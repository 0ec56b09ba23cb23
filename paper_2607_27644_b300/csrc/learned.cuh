// Learned Relay-BP: training forward (unrolled, with a tape) and backward.
//
// Not in arXiv 2607.27644 (which decodes with plain Relay-BP); this is the
// learned form of this library.  Parameters:
//   w[t][e]   weight of the check-to-variable message of edge e (row-major) in
//             iteration t+1: nu_e(t) = w[t-1][e] * sigma_e * min_{f != e} |mu_f|,
//             sigma_e = (-1)^{s_i} prod_{f != e} sgn(mu_f);
//   knots[k]  k = 0..K, nondecreasing: the inverse CDF of the memory strength,
//             g(u) = knots[k] + (knots[k+1] - knots[k]) (uK - k), k = floor(uK),
//             u the 24-bit Philox stream-1 draw of leg 1.
// Training forward of one shot: T iterations of one memory-BP leg from
// M = L0, nu = 0, with one of two losses summed over the iterations t:
//   objective 0: sum_j BCE(M_j(t), e_j) (bit j in error with probability
//                sigmoid(-M_j)), the sampled error as the label;
//   objective 1: the soft syndrome -sum_i log(eps + (1 - 2 eps) P_i(t)),
//                P_i = (1 + (-1)^{s_i} prod_{j in row i} tanh(M_j / 2)) / 2 the
//                probability that check i holds its syndrome bit; it rewards
//                satisfying every check early, which is what ends a decode.
// Its gradient with respect to M_j(t) is
//   sum_{i in col j} c_i loo_ij (1 - tanh^2(M_j / 2)) / 2,
//   c_i = -(1 - 2 eps) (-1)^{s_i} / (2 (eps + (1 - 2 eps) P_i)),
// loo_ij the product of tanh(M_k / 2) over the row's other variables.
//
// Reverse mode.  With B_j(t) = Mbar_j(t) + sum_{col j} mubar(t+1):
//   Mbar_j(t)   = s (e_j - sigmoid(-M_j(t))) + g_j Lbar_j(t+1)
//   nubar_e(t)  = B_j(t) - mubar_e(t+1)
//   wbar[t-1][e] += nubar_e sigma_e m_e          (m_e = e == a1 ? m2 : m1)
//   mubar_a1(t) = sgn(mu_a1) sum_{e != a1} nubar_e w_e sigma_e,
//   mubar_a2(t) = sgn(mu_a2) nubar_a1 w_a1 sigma_a1, all other mubar_e(t) = 0
//   Lbar_j(t)   = Mbar_j(t) + sum_{col j} mubar(t)
//   gbar_j     += Lbar_j(t) (M_j(t-1) - L0_j)
// (a1, a2: positions of the smallest and second-smallest |mu| of the row,
// ties to the lower position).  Because mubar of a row is nonzero at a1 and a2
// only, the backward keeps two values per row instead of one per edge.
#pragma once
#include "kernels.cuh"

namespace relaybp {

template <typename T> struct TapeRow {
    T m1, m2;
    uint32_t meta;              // a1 | a2 << 12 | parity << 31
};

struct TapePlan {               // byte offsets within one iteration's tape record
    int rows, sgn, M, iter;     // iter: bytes of one iteration
};

constexpr double kSoftSynEps = 1e-6;

struct LearnedDev {
    DevDEM g;
    int T, K;
    int objective;              // 0: cross-entropy against the sampled error, 1: soft syndrome
    const void *w;              // [T][E] of the arithmetic type
    const void *knots;          // [K+1]
    uint64_t gamma_seed;
    const uint32_t *syn, *err;
    uint64_t shot0;
    int64_t shots;
    unsigned char *tape;        // [shots][T][plan.iter]
    TapePlan tp;
    double *loss;               // [shots]
    const uint32_t *cedge_ell;  // row-major edge of each ELL column entry
};

struct LearnedSmem {            // byte offsets of the per-shot shared state
    int a, b, c, d, rows, sgn, syn, srow, total;    // srow: soft-syndrome row terms (objective 1)
};

// Soft-syndrome terms of check row i from the posteriors M: the product of
// tanh(M_j / 2) over the row's nonzero factors, how many factors are zero,
// and the coefficient c_i of the gradient; returns the row's loss.
template <typename T> struct SoftRow {
    T prod, coef;
    int zeros;
};
template <typename T>
__device__ __forceinline__ T soft_row(const DevDEM &g, const T *M, const uint32_t *syn, int i, SoftRow<T> &out)
{
    T prod = (T)1;
    int zeros = 0;
    for (int e = __ldg(g.rptr + i), ee = __ldg(g.rptr + i + 1); e < ee; ++e) {
        const T th = tanh((T)0.5 * M[__ldg(g.rvar + e)]);
        if (th == (T)0) ++zeros;
        else prod *= th;
    }
    const T sgn = ((syn[i >> 5] >> (i & 31)) & 1u) ? (T)-1 : (T)1;
    const T P = (T)0.5 * ((T)1 + sgn * (zeros ? (T)0 : prod));
    const T q = (T)kSoftSynEps + (T)(1.0 - 2.0 * kSoftSynEps) * P;
    out.prod = prod;
    out.zeros = zeros;
    out.coef = -(T)(1.0 - 2.0 * kSoftSynEps) * sgn / ((T)2 * q);
    return -log(q);
}

// d loss / d M_j from the rows' soft-syndrome terms (column j's checks).
template <typename T>
__device__ __forceinline__ T soft_grad(const DevDEM &g, const SoftRow<T> *sr, const T *M, int j)
{
    const T th = tanh((T)0.5 * M[j]);
    T acc = (T)0;
    for (int q = __ldg(g.cptr + j), qe = __ldg(g.cptr + j + 1); q < qe; ++q) {
        const SoftRow<T> r = sr[__ldg(g.cchk + q)];
        T loo;
        if (th != (T)0) loo = r.zeros ? (T)0 : r.prod / th;
        else loo = (r.zeros == 1) ? r.prod : (T)0;
        acc += r.coef * loo;
    }
    return acc * (T)0.5 * ((T)1 - th * th);
}

template <typename T>
__device__ __forceinline__ T knot_gamma(const T *knots, int K, T u)
{
    const T x = u * (T)K;
    int k = (int)floor((double)x);
    if (k >= K) k = K - 1;
    const T f = x - (T)k;
    return knots[k] + (knots[k + 1] - knots[k]) * f;
}

template <typename T>
__device__ __forceinline__ T draw_u(uint64_t seed, uint64_t shot, int j, int V)
{
    const uint32_t nblk = (uint32_t)((V + 3) / 4);
    const uint4 r = philox_block(seed, shot, 1u, 1u * nblk + (uint32_t)(j >> 2));
    return (T)(uint4_word(r, j & 3) >> 8) * (T)(1.0 / 16777216.0);
}

template <typename T>
__device__ __forceinline__ T softplus(T x)
{
    return x > (T)0 ? x + log1p(exp(-x)) : log1p(exp(x));
}

template <typename T>
__device__ __forceinline__ T sigm(T x)
{
    return (T)1 / ((T)1 + exp(-x));
}

// lexicographic (value, position) minimum pair update
template <typename T>
__device__ __forceinline__ void min2_push(T a, uint32_t k, T &b1, uint32_t &i1, T &b2, uint32_t &i2)
{
    if (a < b1 || (a == b1 && k < i1)) { b2 = b1; i2 = i1; b1 = a; i1 = k; }
    else if (a < b2 || (a == b2 && k < i2)) { b2 = a; i2 = k; }
}

// ---------------------------------------------------------------------------
// Training forward: one block per shot, persistent over the batch.
// Shared: A[V], M[V], gam[V] (T), rows[C] (TapeRow<T>), sgnh[C*L], syn bits.
// ---------------------------------------------------------------------------
template <typename T, int L, int NB>
__global__ void __launch_bounds__(512)
learned_forward_kernel(LearnedDev a, LearnedSmem sp, unsigned long long *__restrict__ work)
{
    extern __shared__ __align__(16) unsigned char smem[];
    T *A = reinterpret_cast<T *>(smem + sp.a);
    T *M = reinterpret_cast<T *>(smem + sp.b);
    T *gam = reinterpret_cast<T *>(smem + sp.c);
    TapeRow<T> *rows = reinterpret_cast<TapeRow<T> *>(smem + sp.rows);
    uint16_t *sgnh = reinterpret_cast<uint16_t *>(smem + sp.sgn);
    uint32_t *syn = reinterpret_cast<uint32_t *>(smem + sp.syn);
    __shared__ long long s_shot;
    __shared__ double s_loss[32];

    const DevDEM &g = a.g;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x, nwarp = nthr >> 5;
    const int C = g.C, V = g.V, WC = wordsof(C), WV = wordsof(V);
    const int64_t E = g.E;
    const unsigned FULL = 0xffffffffu;
    const T *W = static_cast<const T *>(a.w);
    const T *knots = static_cast<const T *>(a.knots);
    constexpr int P = 32 / L;
    const int r = lane / L, l = lane % L;

    for (;;) {
        if (tid == 0) s_shot = (long long)atomicAdd(work, 1ull);
        __syncthreads();
        const long long sidx = s_shot;
        if (sidx >= a.shots) break;
        const uint64_t shot = a.shot0 + (uint64_t)sidx;
        unsigned char *tape = a.tape + (size_t)sidx * (size_t)a.T * (size_t)a.tp.iter;
        const uint32_t *err = a.err + sidx * WV;
        for (int j = tid; j < V; j += nthr) {
            const T l0 = (T)__ldg(g.L0d + j);
            const T gj = knot_gamma<T>(knots, a.K, draw_u<T>(a.gamma_seed, shot, j, V));
            gam[j] = gj;
            M[j] = l0;
            A[j] = ((T)1 - gj) * l0 + gj * l0;
        }
        for (int i = tid; i < C; i += nthr) { rows[i].m1 = (T)0; rows[i].m2 = (T)0; rows[i].meta = 0u; }
        for (int w = tid; w < C * L; w += nthr) sgnh[w] = (uint16_t)0;
        for (int w = tid; w < WC; w += nthr) syn[w] = a.syn[sidx * WC + w];
        __syncthreads();
        double acc = 0.0;
        for (int t = 1; t <= a.T; ++t) {
            const T *wprev = W + (int64_t)(t >= 2 ? t - 2 : 0) * E;
            const T *wcur = W + (int64_t)(t - 1) * E;
            TapeRow<T> *trow = reinterpret_cast<TapeRow<T> *>(tape + (size_t)(t - 1) * a.tp.iter + a.tp.rows);
            uint16_t *tsgn = reinterpret_cast<uint16_t *>(tape + (size_t)(t - 1) * a.tp.iter + a.tp.sgn);
            T *tM = reinterpret_cast<T *>(tape + (size_t)(t - 1) * a.tp.iter + a.tp.M);
            // rows: L lanes per row
            for (int base = warp * P; base < C; base += nwarp * P) {
                const int i = base + r;
                const bool rowok = i < C;
                int e0 = 0, deg = 0;
                if (rowok) { e0 = __ldg(g.rptr + i); deg = __ldg(g.rptr + i + 1) - e0; }
                T om1 = (T)0, om2 = (T)0;
                uint32_t ometa = 0u, oldbits = 0u;
                if (rowok) { om1 = rows[i].m1; om2 = rows[i].m2; ometa = rows[i].meta; oldbits = sgnh[i * L + l]; }
                const uint32_t oa1 = ometa & 0xfffu, opar = ometa >> 31;
                T b1 = Num<T>::inf(), b2 = Num<T>::inf();
                uint32_t i1 = 0xfffu, i2 = 0xfffu, newbits = 0u;
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const int k = b * L + l;
                    if (k < deg) {
                        const int e = e0 + k;
                        const T mag = ((uint32_t)k == oa1) ? om2 : om1;
                        const T nu_old = (((oldbits >> b) & 1u) ^ opar) ? -wprev[e] * mag : wprev[e] * mag;
                        const T m = A[__ldg(g.rvar + e)] - nu_old;
                        newbits |= ((m < (T)0) ? 1u : 0u) << b;
                        min2_push<T>(vabs(m), (uint32_t)k, b1, i1, b2, i2);
                    }
                }
#pragma unroll
                for (int off = L / 2; off > 0; off >>= 1) {
                    const T o1 = __shfl_xor_sync(FULL, b1, off), o2 = __shfl_xor_sync(FULL, b2, off);
                    const uint32_t p1 = __shfl_xor_sync(FULL, i1, off), p2 = __shfl_xor_sync(FULL, i2, off);
                    min2_push<T>(o1, p1, b1, i1, b2, i2);
                    min2_push<T>(o2, p2, b1, i1, b2, i2);
                }
                const uint32_t lp = __ballot_sync(FULL, (__popc(newbits) & 1) != 0);
                const uint32_t gm = (L == 32) ? FULL : (((1u << L) - 1u) << (r * L));
                const uint32_t par = (uint32_t)(__popc(lp & gm) & 1);
                if (rowok) {
                    sgnh[i * L + l] = (uint16_t)newbits;
                    tsgn[i * L + l] = (uint16_t)newbits;
                    if (l == 0) {
                        const uint32_t sb = (syn[i >> 5] >> (i & 31)) & 1u;
                        TapeRow<T> n;
                        n.m1 = b1;
                        n.m2 = b2;
                        n.meta = i1 | (i2 << 12) | ((par ^ sb) << 31);
                        rows[i] = n;
                        trow[i] = n;
                    }
                }
            }
            __syncthreads();
            // variables: one lane per variable over the ELL slices
            for (int G = warp; G < WV; G += nwarp) {
                const int j = G * 32 + lane;
                const int D = __ldg(g.gdeg + G);
                const uint32_t *col = g.cinfo + __ldg(g.goff + G) + lane;
                const uint32_t *cel = a.cedge_ell + __ldg(g.goff + G) + lane;
                T S = (T)0;
                for (int k = 0; k < D; ++k) {
                    const uint32_t c = __ldg(col + k * 32);
                    if (c == COL_SENTINEL) continue;
                    const uint32_t i = c >> 12, pos = c & 0xfffu;
                    const TapeRow<T> q = rows[i];
                    const uint32_t hw = sgnh[i * L + (pos % L)];
                    const T mag = (pos == (q.meta & 0xfffu)) ? q.m2 : q.m1;
                    const uint32_t sb = ((hw >> (pos / L)) & 1u) ^ (q.meta >> 31);
                    const T wm = wcur[__ldg(cel + k * 32)] * mag;
                    S += sb ? -wm : wm;
                }
                if (j < V) {
                    const T l0 = (T)__ldg(g.L0d + j), gj = gam[j];
                    const T Mn = ((T)1 - gj) * l0 + gj * M[j] + S;
                    M[j] = Mn;
                    A[j] = ((T)1 - gj) * l0 + gj * Mn + S;
                    tM[j] = Mn;
                    if (a.objective == 0) {
                        const uint32_t ej = (__ldg(err + (j >> 5)) >> (j & 31)) & 1u;
                        acc += (double)(ej ? softplus<T>(Mn) : softplus<T>(-Mn));
                    }
                }
            }
            __syncthreads();
            if (a.objective == 1) {             // soft syndrome of this iteration's posteriors
                for (int i = tid; i < C; i += nthr) {
                    SoftRow<T> sr;
                    acc += (double)soft_row<T>(g, M, syn, i, sr);
                }
            }
        }
        // per-shot loss: block reduction in FP64
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(FULL, acc, off);
        if (lane == 0) s_loss[warp] = acc;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < nwarp; ++w) s += s_loss[w];
            a.loss[sidx] = s;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Backward: one block per shot.  Shared: Lbar[V] (holds Mbar between the two
// variable passes), colbar[V], B[V], gam[V], rec[C] (a1 | a2 << 12, mubar_a1,
// mubar_a2 of the later iteration).  gbar[V] in a per-block global row.
// ---------------------------------------------------------------------------
template <typename T> struct BackRow {
    T mb1, mb2;
    uint32_t meta;
};

template <typename T, int L, int NB>
__global__ void __launch_bounds__(512)
learned_backward_kernel(LearnedDev a, LearnedSmem sp, unsigned long long *__restrict__ work, T scale,
                        T *__restrict__ grad_w, T *__restrict__ grad_knots, T *__restrict__ gbar_scratch)
{
    extern __shared__ __align__(16) unsigned char smem[];
    T *Lbar = reinterpret_cast<T *>(smem + sp.a);
    T *colbar = reinterpret_cast<T *>(smem + sp.b);
    T *B = reinterpret_cast<T *>(smem + sp.c);
    T *gam = reinterpret_cast<T *>(smem + sp.d);
    BackRow<T> *rec = reinterpret_cast<BackRow<T> *>(smem + sp.rows);
    SoftRow<T> *srow = reinterpret_cast<SoftRow<T> *>(smem + sp.srow);
    uint32_t *syn = reinterpret_cast<uint32_t *>(smem + sp.syn);
    __shared__ long long s_shot;
    __shared__ T s_kg[65];

    const DevDEM &g = a.g;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x, nwarp = nthr >> 5;
    const int C = g.C, V = g.V, WV = wordsof(V);
    const int64_t E = g.E;
    const unsigned FULL = 0xffffffffu;
    const T *W = static_cast<const T *>(a.w);
    const T *knots = static_cast<const T *>(a.knots);
    T *gbar = gbar_scratch + (int64_t)blockIdx.x * V;
    constexpr int P = 32 / L;
    const int r = lane / L, l = lane % L;

    for (;;) {
        if (tid == 0) s_shot = (long long)atomicAdd(work, 1ull);
        __syncthreads();
        const long long sidx = s_shot;
        if (sidx >= a.shots) break;
        const uint64_t shot = a.shot0 + (uint64_t)sidx;
        const unsigned char *tape = a.tape + (size_t)sidx * (size_t)a.T * (size_t)a.tp.iter;
        const uint32_t *err = a.err + sidx * WV;
        for (int j = tid; j < V; j += nthr) {
            Lbar[j] = (T)0;
            colbar[j] = (T)0;
            gbar[j] = (T)0;
            gam[j] = knot_gamma<T>(knots, a.K, draw_u<T>(a.gamma_seed, shot, j, V));
        }
        for (int i = tid; i < C; i += nthr) { rec[i].mb1 = (T)0; rec[i].mb2 = (T)0; rec[i].meta = 0xffffffu; }
        for (int k = tid; k <= a.K; k += nthr) s_kg[k] = (T)0;
        if (a.objective == 1)
            for (int w = tid; w < wordsof(C); w += nthr) syn[w] = a.syn[sidx * wordsof(C) + w];
        __syncthreads();
        for (int t = a.T; t >= 1; --t) {
            const unsigned char *it = tape + (size_t)(t - 1) * a.tp.iter;
            const TapeRow<T> *trow = reinterpret_cast<const TapeRow<T> *>(it + a.tp.rows);
            const uint16_t *tsgn = reinterpret_cast<const uint16_t *>(it + a.tp.sgn);
            const T *tM = reinterpret_cast<const T *>(it + a.tp.M);
            const T *wcur = W + (int64_t)(t - 1) * E;
            T *gw = grad_w + (int64_t)(t - 1) * E;
            if (a.objective == 1) {             // the rows' soft-syndrome terms at M(t)
                for (int i = tid; i < C; i += nthr) soft_row<T>(g, tM, syn, i, srow[i]);
                __syncthreads();
            }
            // variable pass A: Mbar(t) and B(t)
            for (int j = tid; j < V; j += nthr) {
                const T Mt = tM[j];
                T src;
                if (a.objective == 0) {
                    const uint32_t ej = (__ldg(err + (j >> 5)) >> (j & 31)) & 1u;
                    src = (T)ej - sigm<T>(-Mt);
                } else {
                    src = soft_grad<T>(g, srow, tM, j);
                }
                const T mbar = scale * src + gam[j] * Lbar[j];
                B[j] = mbar + colbar[j];
                Lbar[j] = mbar;
            }
            __syncthreads();
            // row pass: nubar, weight gradients, mubar at a1 / a2
            for (int base = warp * P; base < C; base += nwarp * P) {
                const int i = base + r;
                const bool rowok = i < C;
                int e0 = 0, deg = 0;
                if (rowok) { e0 = __ldg(g.rptr + i); deg = __ldg(g.rptr + i + 1) - e0; }
                TapeRow<T> q;
                q.m1 = (T)0; q.m2 = (T)0; q.meta = 0u;
                BackRow<T> nx;
                nx.mb1 = (T)0; nx.mb2 = (T)0; nx.meta = 0xffffffu;
                uint32_t bits = 0u;
                if (rowok) { q = trow[i]; nx = rec[i]; bits = tsgn[i * L + l]; }
                const uint32_t a1 = q.meta & 0xfffu, a2 = (q.meta >> 12) & 0xfffu, par = q.meta >> 31;
                const uint32_t na1 = nx.meta & 0xfffu, na2 = (nx.meta >> 12) & 0xfffu;
                T tot = (T)0, ca1 = (T)0;
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const int k = b * L + l;
                    if (k < deg) {
                        const int e = e0 + k;
                        const int j = __ldg(g.rvar + e);
                        const T mub = ((uint32_t)k == na1) ? nx.mb1 : (((uint32_t)k == na2) ? nx.mb2 : (T)0);
                        const T nub = B[j] - mub;
                        const bool neg = (((bits >> b) & 1u) ^ par) != 0u;
                        const T me = ((uint32_t)k == a1) ? q.m2 : q.m1;
                        atomicAdd(gw + e, neg ? -nub * me : nub * me);
                        const T c = neg ? -nub * wcur[e] : nub * wcur[e];
                        tot += c;
                        if ((uint32_t)k == a1) ca1 = c;
                    }
                }
#pragma unroll
                for (int off = L / 2; off > 0; off >>= 1) {
                    tot += __shfl_xor_sync(FULL, tot, off);
                    ca1 += __shfl_xor_sync(FULL, ca1, off);
                }
                if (rowok && l == 0) {
                    // signs of mu at a1 and a2 from the tape's sign words
                    const uint32_t s1 = (tsgn[i * L + (a1 % L)] >> (a1 / L)) & 1u;
                    const uint32_t s2 = (tsgn[i * L + (a2 % L)] >> (a2 / L)) & 1u;
                    BackRow<T> n;
                    n.mb1 = s1 ? -(tot - ca1) : (tot - ca1);
                    n.mb2 = s2 ? -ca1 : ca1;
                    n.meta = a1 | (a2 << 12);
                    rec[i] = n;
                }
            }
            __syncthreads();
            // variable pass B: colbar(t), Lbar(t), memory-strength gradient
            for (int G = warp; G < WV; G += nwarp) {
                const int j = G * 32 + lane;
                const int D = __ldg(g.gdeg + G);
                const uint32_t *col = g.cinfo + __ldg(g.goff + G) + lane;
                T cb = (T)0;
                for (int k = 0; k < D; ++k) {
                    const uint32_t c = __ldg(col + k * 32);
                    if (c == COL_SENTINEL) continue;
                    const uint32_t i = c >> 12, pos = c & 0xfffu;
                    const BackRow<T> n = rec[i];
                    cb += (pos == (n.meta & 0xfffu)) ? n.mb1 : ((pos == ((n.meta >> 12) & 0xfffu)) ? n.mb2 : (T)0);
                }
                if (j < V) {
                    const T lb = Lbar[j] + cb;
                    Lbar[j] = lb;
                    colbar[j] = cb;
                    if (t >= 2) {
                        const T Mprev = reinterpret_cast<const T *>(tape + (size_t)(t - 2) * a.tp.iter + a.tp.M)[j];
                        gbar[j] += lb * (Mprev - (T)__ldg(g.L0d + j));
                    }
                }
            }
            __syncthreads();
        }
        // distribute the memory-strength gradient over the knots
        for (int j = tid; j < V; j += nthr) {
            const T u = draw_u<T>(a.gamma_seed, shot, j, V);
            const T x = u * (T)a.K;
            int k = (int)floor((double)x);
            if (k >= a.K) k = a.K - 1;
            const T f = x - (T)k;
            atomicAdd(&s_kg[k], gbar[j] * ((T)1 - f));
            atomicAdd(&s_kg[k + 1], gbar[j] * f);
        }
        __syncthreads();
        for (int k = tid; k <= a.K; k += nthr) atomicAdd(grad_knots + k, s_kg[k]);
        __syncthreads();
    }
}

}  // namespace relaybp
