// Ordered-statistics decoding (OSD) of the shots Relay-BP leaves unconverged.
//
// The outlook of arXiv 2607.27644 (Sec. 7, improved decoding) names OSD
// post-processing of the flagged nonconvergences, which dominate the
// failures.  For one flagged shot with final posteriors q (M of its last
// iteration):
//   1. order the V columns of H by q ascending (the most likely error first),
//      ties by column index;
//   2. take, in that order, the first columns that are linearly independent
//      over GF(2) -- the information set, rank(H) of them -- and solve
//      H e = s on them (OSD-0); s outside the column space of H is flagged;
//   3. with order lambda > 0, also try every flip of one or two of the first
//      lambda columns outside the information set (their bits set, the
//      information-set bits re-solved) and keep the candidate of least
//      weight sum_j e_j L0_j (prior LLRs, FP64 in the information set's
//      order), OSD-0's on ties and the first candidate among equal ones.
// The result is determined by the order and the reduced syndrome, so it
// equals any correct elimination's bit for bit.
//
// One thread block per flagged shot.  Phase 1 sorts the columns by a bitonic
// network in shared memory.  Phase 2 eliminates column by column without
// storing H: it keeps the row transform Q (C x C bits, rows in shared memory)
// that the elimination so far has applied, so a column's reduced form is
// Q h_c, the XOR of Q's bits at the column's few checks (H is sparse), and a
// pivot costs one row swap and one XOR of row r into the rows where the
// column has a one.  Limits: C <= 1024 checks (a thread per row of Q), V <=
// kOsdSortMax columns, lambda <= kOsdMaxLambda.
#pragma once
#include "kernels.cuh"

namespace relaybp {

constexpr int kOsdSortMax = 16384;
constexpr int kOsdMaxLambda = 64;

struct OsdJob {
    DevDEM g;
    const uint32_t *syn;        // [*][ceil(C/32)] syndromes; flagged shot f uses row idx[f]
    const double *post;         // [n][V] final posteriors of the flagged shots
    const long long *idx;       // [n]
    long long n;
    int lambda, NP;             // NP = sorted length (a power of two >= V)
    uint32_t *out_e;            // [n][ceil(V/32)]
    int32_t *out_valid;         // [n]
    int32_t *order;             // [gridDim.x][V] scratch: each block's column order
};

// Unsigned key with the order of the double (-0 ranks with +0).
__device__ __forceinline__ unsigned long long osd_key(double q)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(q == 0.0 ? 0.0 : q);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void __launch_bounds__(1024, 1) osd_kernel(const __grid_constant__ OsdJob J)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_piv[2], s_sr, s_nf, s_valid;
    __shared__ double s_w0;
    __shared__ double s_bw[32];
    __shared__ int s_bk[32];

    const DevDEM &g = J.g;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x, nwarp = nthr >> 5;
    const unsigned FULL = 0xffffffffu;
    const int C = g.C, V = g.V, WC = wordsof(C), WV = wordsof(V), NP = J.NP;
    int32_t *order = J.order + (size_t)blockIdx.x * V;

    for (long long f = blockIdx.x; f < J.n; f += gridDim.x) {
        // ---- phase 1: columns by (posterior, index), bitonic in shared memory -
        {
            unsigned long long *key = reinterpret_cast<unsigned long long *>(smem);
            uint32_t *id = reinterpret_cast<uint32_t *>(smem + 8 * (size_t)NP);
            const double *q = J.post + f * V;
            for (int i = tid; i < NP; i += nthr) {
                key[i] = i < V ? osd_key(q[i]) : ~0ull;
                id[i] = i < V ? (uint32_t)i : 0xffffffffu;
            }
            __syncthreads();
            for (int k = 2; k <= NP; k <<= 1) {
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int i = tid; i < NP; i += nthr) {
                        const int o = i ^ j;
                        if (o > i) {
                            const bool up = (i & k) == 0;
                            const bool gt = key[i] > key[o] || (key[i] == key[o] && id[i] > id[o]);
                            if (gt == up) {
                                const unsigned long long tk = key[i];
                                key[i] = key[o];
                                key[o] = tk;
                                const uint32_t ti = id[i];
                                id[i] = id[o];
                                id[o] = ti;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            for (int i = tid; i < V; i += nthr) order[i] = (int32_t)id[i];
            __syncthreads();
        }
        // ---- phase 2: elimination in that order ------------------------------
        uint32_t *Q = reinterpret_cast<uint32_t *>(smem);                   // [C][WC]
        uint32_t *sp = Q + (size_t)C * WC;                                  // reduced syndrome [WC]
        uint32_t *x = sp + WC;                                              // reduced column [WC]
        int32_t *pivcol = reinterpret_cast<int32_t *>(x + WC);              // [C]
        uint32_t *ispiv = reinterpret_cast<uint32_t *>(pivcol + C);         // [WV] bits
        int32_t *fc = reinterpret_cast<int32_t *>(ispiv + WV);              // [lambda] free columns
        uint32_t *xf = reinterpret_cast<uint32_t *>(fc + kOsdMaxLambda);    // [lambda][WC]
        const uint32_t *syn = J.syn + (size_t)J.idx[f] * WC;
        for (int i = tid; i < C * WC; i += nthr) {
            const int row = i / WC, w = i % WC;
            Q[i] = (w == (row >> 5)) ? (1u << (row & 31)) : 0u;
        }
        for (int w = tid; w < WC; w += nthr) sp[w] = syn[w];
        for (int w = tid; w < WV; w += nthr) ispiv[w] = 0u;
        if (tid < 2) s_piv[tid] = C;
        __syncthreads();
        // Q h_c into dst (one thread per row; a warp's ballot is one word)
        auto reduce_col = [&](int c, uint32_t *dst) {
            for (int i0 = warp * 32; i0 < C; i0 += nwarp * 32) {
                const int i = i0 + lane;
                uint32_t b = 0u;
                if (i < C) {
                    const uint32_t *qi = Q + (size_t)i * WC;
                    for (int e = __ldg(g.cptr + c), ee = __ldg(g.cptr + c + 1); e < ee; ++e) {
                        const int k = __ldg(g.cchk + e);
                        b ^= (qi[k >> 5] >> (k & 31)) & 1u;
                    }
                }
                const uint32_t word = __ballot_sync(FULL, b != 0u);
                if (lane == 0) dst[i0 >> 5] = word;
            }
        };
        int r = 0;
        for (int t = 0; t < V && r < C; ++t) {
            const int c = order[t];
            const int par = t & 1;
            reduce_col(c, x);
            __syncthreads();
            // pivot: the first row >= r where the reduced column has a one
            for (int w = tid; w < WC; w += nthr) {
                uint32_t m = x[w];
                if (w < (r >> 5)) m = 0u;
                else if (w == (r >> 5)) m &= ~((1u << (r & 31)) - 1u);
                if (m) atomicMin(&s_piv[par], w * 32 + __ffs(m) - 1);
            }
            __syncthreads();
            const int p = s_piv[par];
            if (tid == 0) s_piv[par ^ 1] = C;                  // ready for the next column
            if (p >= C) continue;                              // dependent on the pivots so far
            if (p != r) {                                      // swap rows p and r (Q, syndrome, column)
                for (int w = tid; w < WC; w += nthr) {
                    const uint32_t a = Q[(size_t)p * WC + w];
                    Q[(size_t)p * WC + w] = Q[(size_t)r * WC + w];
                    Q[(size_t)r * WC + w] = a;
                }
                if (tid == 0) {
                    const uint32_t bp = (sp[p >> 5] >> (p & 31)) & 1u, br = (sp[r >> 5] >> (r & 31)) & 1u;
                    if (bp != br) { sp[p >> 5] ^= 1u << (p & 31); sp[r >> 5] ^= 1u << (r & 31); }
                    const uint32_t xp = (x[p >> 5] >> (p & 31)) & 1u, xr = (x[r >> 5] >> (r & 31)) & 1u;
                    if (xp != xr) { x[p >> 5] ^= 1u << (p & 31); x[r >> 5] ^= 1u << (r & 31); }
                }
            }
            if (tid == 0) {
                s_sr = (int)((sp[r >> 5] >> (r & 31)) & 1u);
                pivcol[r] = c;
                ispiv[c >> 5] |= 1u << (c & 31);
            }
            __syncthreads();
            // eliminate the column from every other row
            for (int i = tid; i < C * WC; i += nthr) {
                const int row = i / WC, w = i % WC;
                if (row != r && ((x[row >> 5] >> (row & 31)) & 1u)) Q[i] ^= Q[(size_t)r * WC + w];
            }
            if (s_sr)
                for (int w = tid; w < WC; w += nthr) {
                    uint32_t m = x[w];
                    if (w == (r >> 5)) m &= ~(1u << (r & 31));
                    sp[w] ^= m;
                }
            __syncthreads();
            ++r;
        }
        // s outside the column space: a one left below the pivot rows
        if (tid == 0) s_valid = 1;
        __syncthreads();
        for (int w = tid; w < WC; w += nthr) {
            uint32_t m = sp[w];
            if (w < (r >> 5)) m = 0u;
            else if (w == (r >> 5)) m &= ~((1u << (r & 31)) - 1u);
            if (m) s_valid = 0;
        }
        // order lambda: the first lambda columns outside the information set
        if (warp == 0) {
            int nf = 0;
            for (int t0 = 0; t0 < V && nf < J.lambda; t0 += 32) {
                const int t = t0 + lane;
                int c = -1;
                if (t < V) {
                    c = order[t];
                    if ((ispiv[c >> 5] >> (c & 31)) & 1u) c = -1;
                }
                const uint32_t bal = __ballot_sync(FULL, c >= 0);
                const int pos = nf + __popc(bal & ((1u << lane) - 1u));
                if (c >= 0 && pos < J.lambda) fc[pos] = c;
                nf = min(J.lambda, nf + __popc(bal));
            }
            if (lane == 0) s_nf = nf;
        }
        __syncthreads();
        const int nf = s_nf;
        for (int u = 0; u < nf; ++u) reduce_col(fc[u], xf + (size_t)u * WC);
        if (tid == 0) {                                        // OSD-0 weight, information-set order
            double w0 = 0.0;
            for (int i = 0; i < r; ++i)
                if ((sp[i >> 5] >> (i & 31)) & 1u) w0 = __dadd_rn(w0, __ldg(g.L0d + pivcol[i]));
            s_w0 = w0;
        }
        __syncthreads();
        // candidates (u, v), u <= v < nf, in the enumeration order u-major
        const int ncand = nf * (nf + 1) / 2;
        double bw = s_w0;
        int bk = -1;
        for (int k = tid; k < ncand; k += nthr) {
            int u = 0, rem = k;
            while (rem >= nf - u) { rem -= nf - u; ++u; }
            const int v = u + rem;
            const int c1 = fc[u], c2 = fc[v];
            const uint32_t *x1 = xf + (size_t)u * WC, *x2 = xf + (size_t)v * WC;
            double w = __dadd_rn(__ldg(g.L0d + c1), v != u ? __ldg(g.L0d + c2) : 0.0);
            for (int i = 0; i < r; ++i) {
                uint32_t bit = ((sp[i >> 5] ^ x1[i >> 5]) >> (i & 31)) & 1u;
                if (v != u) bit ^= (x2[i >> 5] >> (i & 31)) & 1u;
                if (bit) w = __dadd_rn(w, __ldg(g.L0d + pivcol[i]));
            }
            if (w < bw) { bw = w; bk = k; }                    // ascending k per thread: first on ties
        }
        // block argmin over (weight, candidate index); -1 = OSD-0
        for (int off = 16; off > 0; off >>= 1) {
            const double ow = __shfl_xor_sync(FULL, bw, off);
            const int ok = __shfl_xor_sync(FULL, bk, off);
            if (ow < bw || (ow == bw && ok >= 0 && (bk < 0 || ok < bk))) { bw = ow; bk = ok; }
        }
        if (lane == 0) { s_bw[warp] = bw; s_bk[warp] = bk; }
        __syncthreads();
        if (tid == 0) {
            double w = s_w0;
            int kbest = -1;
            for (int q = 0; q < nwarp; ++q)
                if (s_bk[q] >= 0 && (s_bw[q] < w || (s_bw[q] == w && kbest >= 0 && s_bk[q] < kbest))) {
                    w = s_bw[q];
                    kbest = s_bk[q];
                }
            s_bk[0] = kbest;
        }
        __syncthreads();
        const int kbest = s_bk[0];
        int u = -1, v = -1;
        if (kbest >= 0) {
            int rem = kbest;
            u = 0;
            while (rem >= nf - u) { rem -= nf - u; ++u; }
            v = u + rem;
        }
        // output: information-set bits (re-solved for the kept flips) and the flips
        uint32_t *e = J.out_e + (size_t)f * WV;
        for (int w = tid; w < WV; w += nthr) e[w] = 0u;
        __syncthreads();
        for (int i = tid; i < r; i += nthr) {
            uint32_t bit = (sp[i >> 5] >> (i & 31)) & 1u;
            if (u >= 0) {
                bit ^= (xf[(size_t)u * WC + (i >> 5)] >> (i & 31)) & 1u;
                if (v != u) bit ^= (xf[(size_t)v * WC + (i >> 5)] >> (i & 31)) & 1u;
            }
            if (bit) atomicOr(e + (pivcol[i] >> 5), 1u << (pivcol[i] & 31));
        }
        if (tid == 0) {
            if (u >= 0) {
                atomicOr(e + (fc[u] >> 5), 1u << (fc[u] & 31));
                if (v != u) atomicOr(e + (fc[v] >> 5), 1u << (fc[v] & 31));
            }
            J.out_valid[f] = s_valid;
        }
        __syncthreads();
    }
}

}  // namespace relaybp
