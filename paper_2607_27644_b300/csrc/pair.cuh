// Relay-BP with two shots per thread block in lockstep (a3-a8, FP32).
//
// The decode of arXiv 2607.27644 (Sec. 6.1: min-sum with memory strengths over
// relay legs, the update rule spelled out in include/relaybp.h) is, per
// iteration, a pass over the check rows and a pass over the variables.  Both
// passes are dominated by per-edge work whose addressing depends only on the
// DEM.  Here every thread processes the same edge slot for two shots at once:
// each gather of the DEM structure (row slots, column codes) and each address
// computed from it serves both shots, the two shots' values sit side by side
// as float2 in shared memory (one 8-byte load fetches both), and the additions
// and products of the variable update run as packed FP32 pairs
// (__fadd2_rn / __ffma2_rn, sm_100 and later).  The arithmetic, its rounding
// and its order are those of relay_decode_kernel<float>: the two kernels give
// identical outputs bit for bit.
//
// Shared memory of one block (byte offsets in PairPlan):
//   bit vectors        e^, best, residual, syndrome, observable accumulator,
//                      per shot (from offset 0)
//   MM[C+1] at X       float4 {m1 shot 0, m1 shot 1, m2 shot 0, m2 shot 1} per
//                      check row: smallest / second-smallest |mu|, signed by
//                      the row parity s_i xor the signs of mu, times the
//                      row-tied learned weight when one applies
//   SG[C+1][4] at 2X   uint2 {shot 0, shot 1}: the sign word of lane l = 0..3
//                      of row i at 2X + 32 i + 8 l
//   A2[V+1], M2[V]     float2 per variable: A_j = L_j(t+1) + sum_i nu_ij(t) and
//                      M_j(t); A2[V] = +inf (the dummy variable of padded slots)
// Row C is an empty dummy check (all zero).  The 16- and 32-byte strides of
// MM and SG spread consecutive rows over all shared-memory banks.
// Sign words: four lanes share a row; lane l owns NB row slots b = 0..NB-1
// (NB <= 27) and keeps the signs of mu for them in bits NB-1-b (shifted in
// one per slot), and in bits 27..31 the code 32 - NB + b of the slot holding
// the row's smallest |mu| (0 when that slot is in another lane).  A column
// entry is coded e = (shared address of its sign word << 5) | (32 - NB + b):
// a funnel shift by e brings its sign bit to bit 31, e << 27 matches the
// argmin code, e >> 5 addresses the sign word, (e >> 6) & ~15 the row's
// minima (MM sits at half SG's offset), and (e >> 10) - X / 16 is its row.
#pragma once
#include "kernels.cuh"

namespace relaybp {

constexpr int kPairLanes = 4;           // lanes per check row

struct PairPlan {
    int ehat, best, res, syn, obsacc, MM, SG, A2, M2, total;    // byte offsets (SG = 2 MM)
};

struct PairJob {
    DevDEM g;
    DecodeParamsDev p;
    PairPlan plan;
    const uint32_t *rslot2;     // [round_up(C, 8)][4][NBP]: shared byte offset of A2[j] per row slot
    const uint32_t *ecode2;     // sliced ELL (goff2 / g.gdeg): column entry codes, padded with row C's;
                                // every group holds max(gdeg, 8) slots
    const int32_t *goff2;       // [ceil(V/32)] offset of each group's slots in ecode2
    const float *L0p;           // [ceil(V/32) * 32] prior LLRs in FP32, padded with 0
    const uint32_t *syn_in;     // [shots][ceil(C/32)]
    uint64_t shot0;
    int64_t shots;
    uint32_t *corr_out, *pobs_out;
    StatsDev *stats_out;
    double *trace;
    int trace_iters;
    uint64_t *times_out;
    FlagOut flag;               // flagged nonconvergences (flag.post NULL: not written)
    TailOut tail;               // shots handed over at a leg boundary (tail.count NULL: never)
};

__device__ __forceinline__ float2 sub2_rn(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

// Memory-biased prior of both shots from P = (1 - g) L0: g M + P in one
// packed fused multiply-add, rounded as memprior<float>().
__device__ __forceinline__ float2 memprior2(float2 P, float2 g, float2 m) { return __ffma2_rn(g, m, P); }

// Row pass over both shots: 4 lanes per row, 8 rows per warp step.
template <int NB>
__device__ __forceinline__ void pair_row_pass(const PairJob &J, unsigned char *smem, const uint32_t *syn0,
                                              const uint32_t *syn1, const float *wrow0, const float *wrow1,
                                              int warp, int nwarp, int lane)
{
    static_assert(NB >= 4 && NB <= 27, "row slots per lane");
    constexpr int NBP = (NB + 3) & ~3;
    constexpr int P = 32 / kPairLanes;
    const unsigned FULL = 0xffffffffu;
    const int r = lane >> 2, l = lane & 3;
    const int Cn = J.g.C;
    const float INF = __int_as_float(0x7f800000);
    constexpr int NQ = NBP / 4;                 // 16-byte vectors of row slots per lane and step
    // Row slots stream two vectors ahead of their use: vector q + 2 of a step
    // loads when vector q starts, and the last two vectors of a step load the
    // next step's first two, so the L2 latency overlaps the slot arithmetic
    // with only a few vectors in registers.
    auto slots = [&](int i) {
        return reinterpret_cast<const uint4 *>(J.rslot2 + ((size_t)i * kPairLanes + l) * NBP);
    };
    uint4 ix[NQ];
    if (warp * P < Cn) {
        ix[0] = __ldg(slots(warp * P + r));
        if constexpr (NQ > 1) ix[1] = __ldg(slots(warp * P + r) + 1);
    }
    for (int base = warp * P; base < Cn; base += nwarp * P) {
        const int i = base + r;                 // rslot2 covers round_up(C, 8) rows
        const int il = min(i, Cn);              // rows past the end read the empty dummy row C
        const bool more = base + nwarp * P < Cn;
        const uint4 *rs = slots(i);
        const uint4 *rsn = slots(more ? i + nwarp * P : i);
        unsigned char *mrow = smem + J.plan.MM + 16 * il;
        unsigned char *srow = smem + J.plan.SG + 32 * il + 8 * l;
        const float4 mm = *reinterpret_cast<const float4 *>(mrow);
        const uint2 sw = *reinterpret_cast<const uint2 *>(srow);
        const uint32_t q0 = sw.x >> 27, q1 = sw.y >> 27;       // argmin code in this lane, or 0
        float b10 = INF, b20 = INF, b11 = INF, b21 = INF;
        int s0 = 0, s1 = 0;
        uint32_t n0 = 0u, n1 = 0u;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if ((b & 3) == 0) {
                const int qn = (b >> 2) + 2;
                if (qn < NQ) ix[qn] = __ldg(rs + qn);
                else if (NQ > 2 && more && qn - NQ < 2) ix[qn - NQ] = __ldg(rsn + (qn - NQ));
            }
            const uint32_t off = uint4_word(ix[b >> 2], b & 3);
            const float2 a = *reinterpret_cast<const float2 *>(smem + off);
            constexpr uint32_t K0 = 32 - NB;
            const uint32_t K = K0 + (uint32_t)b;
            const float mag0 = (q0 == K) ? mm.z : mm.x;
            const float mag1 = (q1 == K) ? mm.w : mm.y;
            const float nu0 = xsign(mag0, (sw.x << K) & 0x80000000u);
            const float nu1 = xsign(mag1, (sw.y << K) & 0x80000000u);
            const float2 mu = sub2_rn(a, make_float2(nu0, nu1));
            n0 = __funnelshift_l(__float_as_uint(mu.x), n0, 1);   // shift in the sign of mu
            n1 = __funnelshift_l(__float_as_uint(mu.y), n1, 1);
            const float a0 = fabsf(mu.x), a1 = fabsf(mu.y);
            b20 = vmin2(b20, vmax2(b10, a0));
            s0 = (a0 < b10) ? b : s0;
            b10 = vmin2(b10, a0);
            b21 = vmin2(b21, vmax2(b11, a1));
            s1 = (a1 < b11) ? b : s1;
            b11 = vmin2(b11, a1);
        }
        if (NQ <= 2 && more) {                  // short rows: the next step's vectors now
#pragma unroll
            for (int q = 0; q < NQ; ++q) ix[q] = __ldg(rsn + q);
        }
        // row minima over the 4 lanes; ties go to the lower position, NaN
        // (an overflowed shot) reaches every lane
        int p0 = (l << 5) | s0, p1 = (l << 5) | s1;
#pragma unroll
        for (int off = 1; off < kPairLanes; off <<= 1) {
            const float o10 = __shfl_xor_sync(FULL, b10, off), o20 = __shfl_xor_sync(FULL, b20, off);
            const int op0 = __shfl_xor_sync(FULL, p0, off);
            if (o10 < b10 || (o10 == b10 && op0 < p0)) { b20 = vmin2(b10, o20); b10 = o10; p0 = op0; }
            else { b20 = vmin2(b20, o10); }
            b10 = vmin2(b10, o10);
            const float o11 = __shfl_xor_sync(FULL, b11, off), o21 = __shfl_xor_sync(FULL, b21, off);
            const int op1 = __shfl_xor_sync(FULL, p1, off);
            if (o11 < b11 || (o11 == b11 && op1 < p1)) { b21 = vmin2(b11, o21); b11 = o11; p1 = op1; }
            else { b21 = vmin2(b21, o11); }
            b11 = vmin2(b11, o11);
        }
        uint32_t c0 = (uint32_t)__popc(n0), c1 = (uint32_t)__popc(n1);
        c0 ^= __shfl_xor_sync(FULL, c0, 1);
        c1 ^= __shfl_xor_sync(FULL, c1, 1);
        c0 ^= __shfl_xor_sync(FULL, c0, 2);
        c1 ^= __shfl_xor_sync(FULL, c1, 2);
        if (i < Cn) {
            const uint32_t w0 = n0 | (((p0 >> 5) == l) ? ((32u - NB + (uint32_t)(p0 & 31)) << 27) : 0u);
            const uint32_t w1 = n1 | (((p1 >> 5) == l) ? ((32u - NB + (uint32_t)(p1 & 31)) << 27) : 0u);
            *reinterpret_cast<uint2 *>(srow) = make_uint2(w0, w1);
            if (l == 0) {
                const bool neg0 = ((c0 ^ (syn0[i >> 5] >> (i & 31))) & 1u) != 0u;
                const bool neg1 = ((c1 ^ (syn1[i >> 5] >> (i & 31))) & 1u) != 0u;
                float v10 = neg0 ? -b10 : b10, v20 = neg0 ? -b20 : b20;
                float v11 = neg1 ? -b11 : b11, v21 = neg1 ? -b21 : b21;
                if (wrow0) {                    // row-tied weight of the messages just formed
                    const float wn = __ldg(wrow0 + i);
                    v10 = mul_rn(v10, wn);
                    v20 = mul_rn(v20, wn);
                }
                if (wrow1) {
                    const float wn = __ldg(wrow1 + i);
                    v11 = mul_rn(v11, wn);
                    v21 = mul_rn(v21, wn);
                }
                *reinterpret_cast<float4 *>(mrow) = make_float4(v10, v11, v20, v21);
            }
        }
    }
}

// One column entry: the message nu_ij of both shots rebuilt from the row state.
__device__ __forceinline__ float2 pair_msg(const unsigned char *smem, uint32_t e)
{
    const uint32_t a = e >> 5;
    const float4 mm = *reinterpret_cast<const float4 *>(smem + ((a >> 1) & ~15u));
    const uint2 sw = *reinterpret_cast<const uint2 *>(smem + a);
    const uint32_t e27 = e << 27;
    const float mag0 = (((sw.x ^ e27) & 0xf8000000u) == 0u) ? mm.z : mm.x;
    const float mag1 = (((sw.y ^ e27) & 0xf8000000u) == 0u) ? mm.w : mm.y;
    return make_float2(xsign(mag0, __funnelshift_l(sw.x, sw.x, e) & 0x80000000u),
                       xsign(mag1, __funnelshift_l(sw.y, sw.y, e) & 0x80000000u));
}

// Launch bound: the longest rows (NB >= 20 slots per lane) keep 96 registers
// per thread (640 threads), the others 80 (768 threads).
__host__ __device__ constexpr int pair_max_threads(int nb) { return nb >= 20 ? 640 : 768; }

// Two slots per block, each running its own shot's relay legs; every
// iteration advances both.  A slot's per-iteration counters (iteration in the
// leg, iterations of the shot) live in registers, identical in every thread;
// what changes only between legs lives in shared memory.
template <int NB, bool TR>
__global__ void __launch_bounds__(pair_max_threads(NB), 1)
relay_pair_kernel(const __grid_constant__ PairJob J, unsigned long long *__restrict__ work,
                  float2 *__restrict__ gamma_scratch)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_sidx[2];     // shot index within the job (< 0: the slot has no shot)
    __shared__ unsigned long long s_t0[2];
    __shared__ int s_leg[2], s_T[2], s_legs[2], s_nsol[2], s_have[2], s_copy[2];
    __shared__ double s_bestw[2], s_w[2];
    __shared__ long long s_fslot[2];
    __shared__ int s_defer[2];          // hand-over slot of a shot leaving at this leg boundary (< 0: none)

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x, nwarp = nthr >> 5;
    const unsigned FULL = 0xffffffffu;
    const int Cn = J.g.C, V = J.g.V;
    const int WC = wordsof(Cn), WV = wordsof(V), WK = wordsof(J.g.K), WKa = max(1, WK);
    const int NG = WV;
    float2 *A2 = reinterpret_cast<float2 *>(smem + J.plan.A2);
    float2 *M2 = reinterpret_cast<float2 *>(smem + J.plan.M2);
    auto ehat = [&](int s) { return reinterpret_cast<uint32_t *>(smem + J.plan.ehat) + s * WV; };
    auto best = [&](int s) { return reinterpret_cast<uint32_t *>(smem + J.plan.best) + s * WV; };
    auto res = [&](int s) { return reinterpret_cast<uint32_t *>(smem + J.plan.res) + s * WC; };
    auto syn = [&](int s) { return reinterpret_cast<uint32_t *>(smem + J.plan.syn) + s * WC; };
    auto obsacc = [&](int s) { return reinterpret_cast<uint32_t *>(smem + J.plan.obsacc) + s * WKa; };
    float2 *gam = gamma_scratch + (size_t)blockIdx.x * (NG * 32);    // rows padded to whole groups

    // the dummy row C and the dummy variable V (never rewritten)
    if (tid < 4) reinterpret_cast<uint32_t *>(smem + J.plan.MM + 16 * Cn)[tid] = 0u;
    if (tid < 8) reinterpret_cast<uint32_t *>(smem + J.plan.SG + 32 * Cn)[tid] = 0u;
    if (tid == 0) A2[V] = make_float2(__int_as_float(0x7f800000), __int_as_float(0x7f800000));

    // Zero the check-to-variable messages of slot s (minima and sign words).
    auto clear_rows = [&](int s) {
        for (int i = tid; i < Cn; i += nthr) {
            float *mm = reinterpret_cast<float *>(smem + J.plan.MM + 16 * i);
            mm[s] = 0.f;
            mm[2 + s] = 0.f;
            uint32_t *sg = reinterpret_cast<uint32_t *>(smem + J.plan.SG + 32 * i);
#pragma unroll
            for (int l = 0; l < kPairLanes; ++l) sg[2 * l + s] = 0u;
        }
    };
    // Start the shot of slot s (block-cooperative): M = L0, leg-0 strengths,
    // zero messages, syndrome and residual.
    auto start_shot = [&](int s, long long sidx) {
        float *A1 = reinterpret_cast<float *>(A2) + s;
        float *M1 = reinterpret_cast<float *>(M2) + s;
        float *g1 = reinterpret_cast<float *>(gam) + s;
        const float g0 = (float)J.p.gamma0;
        for (int j = tid; j < V; j += nthr) {
            const float l0 = __ldg(J.g.L0f + j);
            M1[2 * j] = l0;
            g1[2 * j] = g0;
            A1[2 * j] = memprior<float>(g0, l0, l0);
        }
        clear_rows(s);
        for (int w = tid; w < WV; w += nthr) ehat(s)[w] = 0u;
        for (int w = tid; w < WC; w += nthr) {
            const uint32_t sv = J.syn_in[sidx * WC + w];
            syn(s)[w] = sv;
            res(s)[w] = sv;
        }
    };
    // tid 0: take the next shot for slot s.
    auto grab = [&](int s) {
        const long long q = (long long)atomicAdd(work, 1ull);
        s_sidx[s] = q < J.shots ? q : -1;
        s_leg[s] = 0;
        s_T[s] = J.p.pre_iter;
        s_legs[s] = 1;
        s_nsol[s] = 0;
        s_have[s] = 0;
        s_bestw[s] = 0.0;
        s_t0[s] = globaltimer_ns();
    };

    if (tid == 0) { grab(0); grab(1); }
    __syncthreads();
    bool act[2];
    int t[2], iters[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        act[s] = s_sidx[s] >= 0;
        t[s] = 0;
        iters[s] = 0;
        if (act[s]) start_shot(s, s_sidx[s]);
    }
    __syncthreads();

    while (act[0] || act[1]) {
        // ---- a3: check rows of both shots ----------------------------------
        const float *wrow0 = nullptr, *wrow1 = nullptr;
        if (J.p.lwrow) {                        // first lT iterations of a learned leg; unit past them
            if ((J.p.llegs < 0 || s_leg[0] < J.p.llegs) && t[0] < J.p.lT) wrow0 = J.p.lwrow + (int64_t)t[0] * Cn;
            if ((J.p.llegs < 0 || s_leg[1] < J.p.llegs) && t[1] < J.p.lT) wrow1 = J.p.lwrow + (int64_t)t[1] * Cn;
        }
        pair_row_pass<NB>(J, smem, syn(0), syn(1), wrow0, wrow1, warp, nwarp, lane);
        __syncthreads();
        // ---- a4, a5: variables of both shots, one lane per variable ----------
        // Software pipeline over the warp's column groups: at the top of a
        // group the next group's first eight column codes and the shape of the
        // group after it start loading, with this group's prior and strengths,
        // so the L2 latency of the DEM structure overlaps this group's work.
        auto codes8 = [&](uint32_t (&c)[8], int off) {     // every group holds >= 8 slots
            const uint32_t *p8 = J.ecode2 + off + lane;
#pragma unroll
            for (int u = 0; u < 8; ++u) c[u] = __ldg(p8 + u * 32);
        };
        int G = warp, D = 0, off = 0, D1 = 0, off1 = 0;
        uint32_t c[8];
        if (G < NG) {
            D = __ldg(J.g.gdeg + G);
            off = __ldg(J.goff2 + G);
            codes8(c, off);
        }
        if (G + nwarp < NG) {
            D1 = __ldg(J.g.gdeg + G + nwarp);
            off1 = __ldg(J.goff2 + G + nwarp);
        }
        for (; G < NG; G += nwarp) {
            const int j = G * 32 + lane;
            uint32_t cn[8];
            codes8(cn, off1);                   // past the last group: the padding group at offset 0
            int D2 = 0, off2 = 0;
            if (G + 2 * nwarp < NG) {
                D2 = __ldg(J.g.gdeg + G + 2 * nwarp);
                off2 = __ldg(J.goff2 + G + 2 * nwarp);
            }
            const float l0 = __ldg(J.L0p + j);  // both padded to whole groups
            const float2 gm = gam[j];
            const uint32_t *col = J.ecode2 + off + lane;
            float2 S = make_float2(0.f, 0.f);
            if (D >= 4) {
#pragma unroll
                for (int u = 0; u < 4; ++u) S = __fadd2_rn(S, pair_msg(smem, c[u]));
                if (D >= 8) {
#pragma unroll
                    for (int u = 4; u < 8; ++u) S = __fadd2_rn(S, pair_msg(smem, c[u]));
                } else {
#pragma unroll
                    for (int u = 4; u < 7; ++u)
                        if (u < D) S = __fadd2_rn(S, pair_msg(smem, c[u]));
                }
            } else {
#pragma unroll
                for (int u = 0; u < 3; ++u)
                    if (u < D) S = __fadd2_rn(S, pair_msg(smem, c[u]));
            }
            int k = 8;
            for (; k + 4 <= D; k += 4) {
                uint32_t cc[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) cc[u] = __ldg(col + (k + u) * 32);
#pragma unroll
                for (int u = 0; u < 4; ++u) S = __fadd2_rn(S, pair_msg(smem, cc[u]));
            }
            for (; k < D; ++k) S = __fadd2_rn(S, pair_msg(smem, __ldg(col + k * 32)));
            const int Dc = D;
#pragma unroll
            for (int u = 0; u < 8; ++u) c[u] = cn[u];
            D = D1;
            off = off1;
            D1 = D2;
            off1 = off2;
            bool d0 = false, d1 = false;
            if (j < V) {
                const float2 P2 = __fmul2_rn(__fadd2_rn(make_float2(1.f, 1.f), make_float2(-gm.x, -gm.y)),
                                             make_float2(l0, l0));
                const float2 Mn = __fadd2_rn(memprior2(P2, gm, M2[j]), S);
                M2[j] = Mn;
                A2[j] = __fadd2_rn(memprior2(P2, gm, Mn), S);
                d0 = Mn.x < 0.f;
                d1 = Mn.y < 0.f;
                if (TR) {
                    if (act[0] && iters[0] < J.trace_iters)
                        J.trace[((int64_t)s_sidx[0] * J.trace_iters + iters[0]) * V + j] = (double)Mn.x;
                    if (act[1] && iters[1] < J.trace_iters)
                        J.trace[((int64_t)s_sidx[1] * J.trace_iters + iters[1]) * V + j] = (double)Mn.y;
                }
            }
            const uint32_t nw0 = __ballot_sync(FULL, d0), nw1 = __ballot_sync(FULL, d1);
            uint32_t *e0 = ehat(0), *e1 = ehat(1);
            const uint32_t o0 = e0[G], o1 = e1[G];  // every lane reads, then lane 0 writes
            __syncwarp();
            if (lane == 0) { e0[G] = nw0; e1[G] = nw1; }
            const uint32_t ch0 = o0 ^ nw0, ch1 = o1 ^ nw1;
            if (ch0 | ch1) {                    // warp-uniform: a decision changed (a5, incremental residual)
                // bit s: this lane's decision of shot s changed; its column's
                // checks flip in that shot's residual.  The first eight codes
                // load together (every group holds >= 8 slots), so one L2
                // latency serves both shots; padding codes name the dummy
                // check C and flip nothing.
                const uint32_t mine = ((ch0 >> lane) & 1u) | (((ch1 >> lane) & 1u) << 1);
                if (mine) {
                    const uint32_t r0 = (uint32_t)J.plan.MM >> 4;
                    uint32_t *rs0 = res(0), *rs1 = res(1);
                    auto flip = [&](uint32_t code) {
                        const uint32_t ri = (code >> 10) - r0;
                        if (ri < (uint32_t)Cn) {
                            if (mine & 1u) atomicXor(rs0 + (ri >> 5), 1u << (ri & 31));
                            if (mine & 2u) atomicXor(rs1 + (ri >> 5), 1u << (ri & 31));
                        }
                    };
                    uint32_t cc[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) cc[u] = __ldg(col + u * 32);
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (u < Dc) flip(cc[u]);
                    for (int kk = 8; kk < Dc; ++kk) flip(__ldg(col + kk * 32));
                }
            }
        }
        __syncthreads();
        // ---- convergence and leg bookkeeping (uniform over the block) ---------
        bool conv[2], trans[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            uint32_t acc = 0u;
            const uint32_t *rs = res(s);
            for (int w = lane; w < WC; w += 32) acc |= rs[w];
            conv[s] = act[s] && !__any_sync(FULL, acc != 0u);
            if (act[s]) { iters[s] += 1; t[s] += 1; }
            trans[s] = act[s] && (conv[s] || t[s] == s_T[s]);
        }
        if (!(trans[0] || trans[1])) continue;

        // a7: FP64 weight of each new solution in ascending variable order
        if (tid == 0) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                s_copy[s] = 0;
                s_defer[s] = -1;
                if (!conv[s]) continue;
                const uint32_t *eh = ehat(s);
                double w = 0.0;
                for (int q = 0; q < WV; ++q) {
                    uint32_t x = eh[q];
                    while (x) {
                        const int b = __ffs(x) - 1;
                        x &= x - 1u;
                        w += __ldg(J.g.L0d + q * 32 + b);
                    }
                }
                const int better = (!s_have[s] || w < s_bestw[s]) ? 1 : 0;
                if (better) { s_bestw[s] = w; s_have[s] = 1; }
                s_copy[s] = better;
                s_nsol[s] += 1;
            }
            // tail hand-over: a shot about to start leg >= tail.legs leaves
            // for the cluster kernel while hand-over slots last
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const bool stop = (!J.p.stop_all && s_nsol[s] >= J.p.stop_nconv) || s_leg[s] == J.p.num_sets;
                if (trans[s] && !stop && J.tail.count && s_leg[s] + 1 >= J.tail.legs) {
                    const unsigned q = atomicAdd(J.tail.count, 1u);
                    if ((long long)q < J.tail.max) s_defer[s] = (int)q;
                }
            }
        }
        __syncthreads();
        bool retire[2], newleg[2], defer[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (s_copy[s])
                for (int w = tid; w < WV; w += nthr) best(s)[w] = ehat(s)[w];
            const bool stop = (!J.p.stop_all && s_nsol[s] >= J.p.stop_nconv) || s_leg[s] == J.p.num_sets;
            retire[s] = trans[s] && stop;
            defer[s] = trans[s] && !stop && s_defer[s] >= 0;
            newleg[s] = trans[s] && !stop && !defer[s];
            if (retire[s])
                for (int w = tid; w < WK; w += nthr) obsacc(s)[w] = 0u;
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (defer[s]) {
                // hand the shot over at the leg boundary: its marginals, best
                // solution and counters (messages restart at zero in a new leg)
                const long long q = s_defer[s];
                const float *M1 = reinterpret_cast<const float *>(M2) + s;
                for (int j = tid; j < V; j += nthr) static_cast<float *>(J.tail.M)[q * V + j] = M1[2 * j];
                for (int w = tid; w < WV; w += nthr) J.tail.best[q * WV + w] = best(s)[w];
                if (tid == 0) {
                    TailRec rec;
                    rec.sidx = s_sidx[s];
                    rec.next_leg = s_leg[s] + 1;
                    rec.legs = s_legs[s];
                    rec.iters = iters[s];
                    rec.nsol = s_nsol[s];
                    rec.have = s_have[s];
                    rec.bestw = s_bestw[s];
                    rec.t0 = s_t0[s];
                    J.tail.rec[q] = rec;
                }
            } else if (retire[s]) {
                // outputs: the best solution (or the last decisions), observables
                const long long sidx = s_sidx[s];
                const uint32_t *out = s_have[s] ? best(s) : ehat(s);
                uint32_t *oa = obsacc(s);
                for (int w = tid; w < WV; w += nthr) {
                    const uint32_t x0 = out[w];
                    if (J.corr_out) J.corr_out[sidx * WV + w] = x0;
                    uint32_t x = x0;
                    while (x) {
                        const int b = __ffs(x) - 1;
                        x &= x - 1u;
                        const int j = w * 32 + b;
                        for (int q = __ldg(J.g.optr + j), qe = __ldg(J.g.optr + j + 1); q < qe; ++q) {
                            const int o = __ldg(J.g.oidx + q);
                            atomicXor(oa + (o >> 5), 1u << (o & 31));
                        }
                    }
                }
                if (tid == 0) {
                    double w = s_bestw[s];
                    if (!s_have[s]) {
                        const uint32_t *eh = ehat(s);
                        w = 0.0;
                        for (int q = 0; q < WV; ++q) {
                            uint32_t x = eh[q];
                            while (x) {
                                const int b = __ffs(x) - 1;
                                x &= x - 1u;
                                w += __ldg(J.g.L0d + q * 32 + b);
                            }
                        }
                    }
                    s_w[s] = w;
                    s_fslot[s] = (!s_have[s] && J.flag.post) ? (long long)atomicAdd(J.flag.count, 1u) : -1;
                }
            } else if (newleg[s]) {
                // a6: next leg -- fresh strengths, marginals carried over
                const int leg = s_leg[s] + 1;
                const uint64_t shot = J.shot0 + (uint64_t)s_sidx[s];
                const bool lk = J.p.lknots && (J.p.llegs < 0 || leg < J.p.llegs);
                float *A1 = reinterpret_cast<float *>(A2) + s;
                const float *M1 = reinterpret_cast<const float *>(M2) + s;
                float *g1 = reinterpret_cast<float *>(gam) + s;
                for (int j = tid; j < V; j += nthr) {
                    const float l0 = __ldg(J.g.L0f + j);
                    const float gn = lk ? knot_draw(J.p, shot, leg, j, V) : draw_gamma<float>(J.p, shot, leg, j, V);
                    const float Mj = M1[2 * j];
                    float carry = 0.f;
                    if (J.p.carry_messages) carry = add_rn(A1[2 * j], -memprior<float>(g1[2 * j], l0, Mj));
                    g1[2 * j] = gn;
                    A1[2 * j] = add_rn(memprior<float>(gn, l0, Mj), carry);
                }
                if (!J.p.carry_messages) clear_rows(s);
                t[s] = 0;
            }
        }
        __syncthreads();
        if (tid == 0) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                if (newleg[s]) {
                    s_leg[s] += 1;
                    s_legs[s] += 1;
                    s_T[s] = J.p.max_iterations;
                }
            }
        }
        if (retire[0] || retire[1] || defer[0] || defer[1]) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                if (!retire[s]) continue;
                const long long sidx = s_sidx[s];
                if (J.pobs_out)
                    for (int w = tid; w < WK; w += nthr) J.pobs_out[sidx * WK + w] = obsacc(s)[w];
                const long long fs = s_fslot[s];
                if (fs >= 0 && fs < J.flag.max) {
                    if (tid == 0) J.flag.idx[fs] = sidx;
                    const float *M1 = reinterpret_cast<const float *>(M2) + s;
                    for (int j = tid; j < V; j += nthr) J.flag.post[fs * V + j] = (double)M1[2 * j];
                }
                if (tid == 0) {
                    if (J.stats_out) {
                        StatsDev st;
                        st.converged = s_have[s];
                        st.nsol = s_nsol[s];
                        st.legs = s_legs[s];
                        st.iters = iters[s];
                        st.weight = s_w[s];
                        J.stats_out[sidx] = st;
                    }
                    if (J.times_out) {
                        J.times_out[2 * sidx] = s_t0[s];
                        J.times_out[2 * sidx + 1] = globaltimer_ns();
                    }
                }
            }
            __syncthreads();
            if (tid == 0) {
                if (retire[0] || defer[0]) grab(0);
                if (retire[1] || defer[1]) grab(1);
            }
            __syncthreads();
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                if (!retire[s] && !defer[s]) continue;
                act[s] = s_sidx[s] >= 0;
                t[s] = 0;
                iters[s] = 0;
                if (act[s]) start_shot(s, s_sidx[s]);
            }
        }
        __syncthreads();
    }
}

}  // namespace relaybp
