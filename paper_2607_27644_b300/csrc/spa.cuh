// Classical channel coding (arXiv 2607.27644, Sec. 6.2): BPSK over AWGN and
// flooding sum-product belief propagation with the "boxplus-phi" check update,
// for the classical seed codes of the ZSZ-LP constructions (Table 2).
//
//   codeword bit c_i -> x_i = (-1)^{c_i}; y_i = x_i + sigma z_i, z_i ~ N(0, 1);
//   channel LLR L_i = clip(2 y_i / sigma^2, +-llr_max);
//   mu_{j->i} = clip(L_j + sum_{i' != i} nu_{i'->j}),
//   nu_{i->j} = clip(prod_{j' != j} sgn(mu_{j'->i}) phi(sum_{j' != j} phi(|mu_{j'->i}|))),
//   phi(x) = -log(tanh(x / 2)) = log1p(2 / expm1(x)),
//   M_j = L_j + sum_i nu_{i->j}, c^_j = [M_j < 0]; stop at the first iteration
//   whose decision satisfies every check (or after max_iter).
// Messages in both directions are clipped to +-llr_max like the channel LLRs.
// Gaussian draws: z_i of frame s is the Box-Muller transform of words 2i and
// 2i+1 of Philox stream 2 under key `seed` (counter (word/4, s lo, s hi, 2)),
// u = (w + 0.5) / 2^32, z = sqrt(-2 ln u1) cos(2 pi u2).
//
// One warp per frame (the seed codes have n <= 310 bits): the warp keeps the
// frame's per-edge messages in shared memory and computes every
// leave-one-out sum and product directly, in the order of the definition.
#pragma once
#include "kernels.cuh"

namespace relaybp {

struct SpaCode {
    int32_t m, n;
    int64_t E;
    const int32_t *rptr, *rvar;     // rows: [m+1], [E]
    const int32_t *cptr, *cedge;    // columns: [n+1], [E] row-major edge of each column entry
};

template <typename T> __device__ __forceinline__ T spa_clip(T v, T m) { return v > m ? m : (v < -m ? -m : v); }
template <typename T> __device__ __forceinline__ T spa_phi(T x) { return log1p((T)2 / expm1(x)); }

// Channel LLRs of `shots` frames: out [shots][n] in precision T.
template <typename T>
__global__ void awgn_llr_kernel(int32_t n, const uint32_t *__restrict__ codewords, double sigma, double llr_max,
                                uint64_t seed, uint64_t shot0, int64_t shots, T *__restrict__ out)
{
    const int64_t total = shots * (int64_t)n;
    const int wn = (n + 31) / 32;
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = q / n;
        const int i = (int)(q % n);
        const uint64_t shot = shot0 + (uint64_t)s;
        const uint32_t w1 = (uint32_t)(2 * i), w2 = w1 + 1u;
        const uint4 r1 = philox_block(seed, shot, 2u, w1 >> 2);
        const uint4 r2 = philox_block(seed, shot, 2u, w2 >> 2);
        const double u1 = ((double)uint4_word(r1, w1 & 3) + 0.5) / 4294967296.0;
        const double u2 = ((double)uint4_word(r2, w2 & 3) + 0.5) / 4294967296.0;
        const double z = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
        const int c = codewords ? (int)((codewords[s * wn + i / 32] >> (i % 32)) & 1u) : 0;
        const double y = (c ? -1.0 : 1.0) + sigma * z;
        out[q] = (T)spa_clip<double>(2.0 * y / (sigma * sigma), llr_max);
    }
}

// Flooding sum-product decode, one warp per frame.  Shared memory per warp:
// nu[E], mu[E] (T) and the decision bits.
template <typename T>
__global__ void __launch_bounds__(256)
spa_kernel(SpaCode h, const T *__restrict__ llr, int64_t shots, int max_iter, T llr_max, int early_stop,
           uint32_t *__restrict__ out_bits, int32_t *__restrict__ out_iters, int32_t *__restrict__ out_valid,
           T *__restrict__ out_post)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int m = h.m, n = h.n, wn = (n + 31) / 32;
    const int64_t E = h.E;
    const size_t per = (2 * (size_t)E * sizeof(T) + 4 * (size_t)wn + 15) & ~(size_t)15;
    T *nu = reinterpret_cast<T *>(smem + per * wib);
    T *mu = nu + E;
    uint32_t *hard = reinterpret_cast<uint32_t *>(mu + E);
    const unsigned FULL = 0xffffffffu;
    for (int64_t s = (int64_t)blockIdx.x * nw + wib; s < shots; s += (int64_t)gridDim.x * nw) {
        const T *L = llr + s * n;
        for (int64_t e = lane; e < E; e += 32) nu[e] = (T)0;
        __syncwarp();
        int it = 0, valid = 0;
        for (it = 1; it <= max_iter; ++it) {
            // variable-to-check: leave-one-out sums in column order, clipped
            for (int j = lane; j < n; j += 32) {
                const int a0 = __ldg(h.cptr + j), a1 = __ldg(h.cptr + j + 1);
                for (int a = a0; a < a1; ++a) {
                    T v = L[j];
                    for (int b = a0; b < a1; ++b)
                        if (b != a) v += nu[__ldg(h.cedge + b)];
                    mu[__ldg(h.cedge + a)] = spa_clip<T>(v, llr_max);
                }
            }
            __syncwarp();
            // check-to-variable: sign product and phi of the phi-sum over the others
            for (int i = lane; i < m; i += 32) {
                const int e0 = __ldg(h.rptr + i), e1 = __ldg(h.rptr + i + 1);
                for (int e = e0; e < e1; ++e) {
                    T sg = (T)1, acc = (T)0;
                    for (int f = e0; f < e1; ++f) {
                        if (f == e) continue;
                        if (mu[f] < (T)0) sg = -sg;
                        acc += spa_phi<T>(fabs(mu[f]));
                    }
                    nu[e] = spa_clip<T>(sg * spa_phi<T>(acc), llr_max);
                }
            }
            __syncwarp();
            // posteriors and hard decisions
            for (int j0 = 0; j0 < n; j0 += 32) {
                const int j = j0 + lane;
                bool d = false;
                if (j < n) {
                    T v = L[j];
                    for (int a = __ldg(h.cptr + j), a1 = __ldg(h.cptr + j + 1); a < a1; ++a) v += nu[__ldg(h.cedge + a)];
                    d = v < (T)0;
                    if (out_post) out_post[s * n + j] = v;
                }
                const uint32_t bw = __ballot_sync(FULL, d);
                if (lane == 0) hard[j0 >> 5] = bw;
            }
            __syncwarp();
            bool bad = false;
            for (int i = lane; i < m; i += 32) {
                uint32_t par = 0u;
                for (int e = __ldg(h.rptr + i), e1 = __ldg(h.rptr + i + 1); e < e1; ++e) {
                    const int j = __ldg(h.rvar + e);
                    par ^= (hard[j >> 5] >> (j & 31)) & 1u;
                }
                bad |= par != 0u;
            }
            valid = !__any_sync(FULL, bad);
            if (early_stop && valid) break;
        }
        if (it > max_iter) it = max_iter;
        for (int w = lane; w < wn; w += 32) out_bits[s * wn + w] = hard[w];
        if (lane == 0) {
            out_iters[s] = it;
            out_valid[s] = valid;
        }
        __syncwarp();
    }
}

}  // namespace relaybp
