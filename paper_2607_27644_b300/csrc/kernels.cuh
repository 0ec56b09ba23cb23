// Device kernels of the Relay-BP hot path (sm_103a).
//
//   sample_kernel         a2: Philox Bernoulli fault draws, s = H e, obs = O e
//   relay_decode_kernel   a3-a8: min-sum check update, memory-biased variable
//                         update, residual, relay legs, minimum-weight select,
//                         persistent work queue (early-exit compaction)
//   count_failures_kernel a9: nonconvergences and undetected logical errors
//
// Relay-BP is the decoder arXiv 2607.27644 runs for all circuit-level results
// (Sec. 6.1, decoder configuration list); the update rule is spelled out in
// include/relaybp.h.
//
// Layout of one shot's decoder state in shared memory (per thread block):
//   A[V+1], M[V]      A_j = L_j(t+1) + sum_i nu_ij(t) (A[V] = +inf: the dummy
//                     variable of padded row slots) and the marginal M_j(t)
//   cs[C+1]           per check row: +-smallest and +-second-smallest |mu|
//                     (signed by the row parity = s_i xor the row's mu sign
//                     bits) and the argmin's column code; row C is an empty
//                     dummy check that padded column slots name
//   sgw[(C+1)*rw]     sign bit of mu for every edge, by position in the row
//   ehat[WV], best[WV], res[WC], syn[WC], obsacc[WK]   bit vectors
// With this compressed check state a message is rebuilt on demand:
//   nu_ij = (-1)^sign_e * (e == argmin_i ? m2_i : m1_i),
// which equals the leave-one-out product of signs and minimum of magnitudes.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "philox.cuh"

namespace relaybp {

struct DevDEM {
    int32_t C, V, K;
    int64_t E;
    const int32_t *rptr;        // [C+1] row pointers into rvar
    const int32_t *rvar;        // [E] variable of each edge, row-major
    const int32_t *cptr;        // [V+1] column pointers into cchk / cbit
    const int32_t *cchk;        // [E] check of each column entry
    const int32_t *cedge;       // [E] row-major edge index of each column entry
    const uint32_t *cinfo;      // sliced ELL: per 32-variable group, slot-major entries
    const int32_t *goff;        // [ceil(V/32)] offset of each group's slots in cinfo
    const int32_t *gdeg;        // [ceil(V/32)] slots (largest column degree) of each group
    const uint32_t *cedge_ell;  // same slots as cinfo: row-major edge index of each entry
    const int32_t *optr;        // [V+1] column pointers into oidx
    const int32_t *oidx;        // observables flipped by each fault
    const double *L0d;          // [V] prior LLRs, FP64
    const float *L0f;           // [V] prior LLRs rounded to FP32
    const uint32_t *thr;        // [V] floor(p_j 2^32)
    // branch-free layout of the decode kernel
    const int32_t *rslot;       // [round_up(C, 32)][kRowStride] row variables, padded with V
    const uint32_t *ecode;      // sliced ELL (goff / gdeg): column code i << lg_rsp | position, padded
                                // with the empty dummy check C (code C << lg_rsp)
    int32_t lg_rsp;             // log2 of the positions per row in the sign words (>= 5)
    int32_t rw;                 // sign words per row, 2^lg_rsp / 32
};

constexpr int kRowStride = 512;     // row slots in rslot (the widest row geometry)
// Column entry of the learned kernels: check index << 12 | position of the
// entry within its row; padding is COL_SENTINEL.
constexpr uint32_t COL_SENTINEL = 0xffffffffu;

struct DecodeParamsDev {
    double gamma0, gamma_min, gamma_max;
    int32_t pre_iter, num_sets, max_iterations, stop_nconv;
    int32_t stop_all, carry_messages;
    uint64_t seed;
    // learned form (NULL: plain method): message weights [lT][E] indexed by
    // the iteration within the leg (past lT: the last), memory-strength
    // inverse-CDF knots [lK+1] for legs >= 1
    const float *lw;
    const float *lknots;
    int32_t lT, lK;
    const float *lwrow;         // learned weights tied per check row: [lT][C] (NULL: none)
    int32_t llegs;              // legs < llegs use the learned parameters (< 0: every leg)
    float qscale;               // int8 storage: value of one step
};

// Flagged nonconvergences (optional output): a shot that ends without a
// solution takes the next slot of *count and, if slot < max, writes its shot
// index and its final posteriors M (FP64) -- the soft input of OSD
// post-processing of exactly the shots Relay-BP leaves unresolved.
struct FlagOut {
    long long *idx;             // [max] shot index within the batch
    double *post;               // [max][V]
    unsigned int *count;        // shots flagged (may exceed max)
    long long max;
};

// Tail hand-over (optional output of the two-shot kernel, input of the
// cluster kernel): a shot that is about to start relay leg >= legs leaves the
// kernel at that leg boundary and takes the next slot of *count; if slot <
// max, rec[slot] keeps what the next legs need -- the shot, the leg to start,
// the counters and the best solution so far -- with its marginals M in
// M[slot][V] and the best solution's bits in best[slot][ceil(V/32)].  A new
// leg restarts the messages at zero (without message carry-over), so nothing
// else is needed; the cluster kernel continues from there with the same
// operations.  Past max, shots stay in the two-shot kernel.
struct TailRec {
    long long sidx;             // shot index within the batch
    int next_leg, legs, iters, nsol, have, pad;
    double bestw;
    unsigned long long t0;
};
struct TailOut {
    TailRec *rec;
    void *M;                    // [max][V] marginals in the storage precision
    uint32_t *best;
    unsigned int *count;        // NULL: no hand-over
    long long max;
    int legs;                   // first leg that hands a shot over
};

struct StatsDev {               // mirrors relaybp_shot_stats
    int32_t converged, nsol, legs, iters;
    double weight;
};

__device__ __forceinline__ int wordsof(int64_t bits) { return (int)((bits + 31) >> 5); }

// Device-wide clock in nanoseconds (the %globaltimer register).
__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------
// a2: fault sampler.  One warp per shot; the warp's syndrome / observable /
// error words are accumulated in shared memory and written out coalesced.
// ---------------------------------------------------------------------------
__global__ void sample_kernel(DevDEM g, uint64_t seed, uint64_t shot0, int64_t shots,
                              uint32_t *__restrict__ syn_out, uint32_t *__restrict__ obs_out,
                              uint32_t *__restrict__ err_out)
{
    extern __shared__ uint32_t sbuf[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int WC = wordsof(g.C), WK = wordsof(g.K), WV = wordsof(g.V);
    const int per_warp = WC + WK + (err_out ? WV : 0);
    uint32_t *s_syn = sbuf + wib * per_warp;
    uint32_t *s_obs = s_syn + WC;
    uint32_t *s_err = s_obs + WK;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const uint32_t nblk = (uint32_t)((g.V + 3) / 4);
    for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; s < shots; s += warps) {
        for (int w = lane; w < per_warp; w += 32) s_syn[w] = 0u;
        __syncwarp();
        const uint64_t shot = shot0 + (uint64_t)s;
        for (uint32_t b = lane; b < nblk; b += 32) {
            const uint4 r = philox_block(seed, shot, 0u, b);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int j = (int)(4 * b) + t;
                if (j < g.V && uint4_word(r, t) < __ldg(g.thr + j)) {
                    if (err_out) atomicOr(s_err + (j >> 5), 1u << (j & 31));
                    for (int q = __ldg(g.cptr + j), qe = __ldg(g.cptr + j + 1); q < qe; ++q) {
                        const int i = __ldg(g.cchk + q);
                        atomicXor(s_syn + (i >> 5), 1u << (i & 31));
                    }
                    for (int q = __ldg(g.optr + j), qe = __ldg(g.optr + j + 1); q < qe; ++q) {
                        const int o = __ldg(g.oidx + q);
                        atomicXor(s_obs + (o >> 5), 1u << (o & 31));
                    }
                }
            }
        }
        __syncwarp();
        for (int w = lane; w < WC; w += 32) syn_out[s * WC + w] = s_syn[w];
        if (obs_out)
            for (int w = lane; w < WK; w += 32) obs_out[s * WK + w] = s_obs[w];
        if (err_out)
            for (int w = lane; w < WV; w += 32) err_out[s * WV + w] = s_err[w];
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// a3-a8: Relay-BP, one thread block per shot, persistent over the batch.
// ---------------------------------------------------------------------------
// Explicitly rounded products and sums: no FMA contraction, so every kernel
// variant (plain or learned, shared or global state, any launch) evaluates
// the memory term and the weighted messages with identical rounding.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
// memory-biased prior (1 - g) L0 + g M: in FP64 two rounded products and a
// rounded sum (the oracle's evaluation); in FP32 the product (1 - g) L0
// rounded, then g M added to it in one fused multiply-add -- the form the
// two-shot kernel's packed FP32 pairs evaluate (a packed multiply followed by
// a packed add is always fused), so every FP32 kernel rounds alike.
template <typename C> __device__ __forceinline__ C memprior(C g, C l0, C m);
template <> __device__ __forceinline__ double memprior<double>(double g, double l0, double m)
{
    return add_rn(mul_rn(add_rn(1.0, -g), l0), mul_rn(g, m));
}
template <> __device__ __forceinline__ float memprior<float>(float g, float l0, float m)
{
    return __fmaf_rn(g, m, mul_rn(add_rn(1.f, -g), l0));
}

template <typename T> __device__ __forceinline__ T vmin(T a, T b) { return b < a ? b : a; }
template <typename T> __device__ __forceinline__ T vabs(T a) { return a < (T)0 ? -a : a; }

template <typename T> struct Num;
template <> struct Num<float> {
    static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
    static __device__ __forceinline__ float l0(const DevDEM &g, int j) { return __ldg(g.L0f + j); }
};
template <> struct Num<double> {
    static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000LL); }
    static __device__ __forceinline__ double l0(const DevDEM &g, int j) { return __ldg(g.L0d + j); }
};

// Memory strength of variable j in leg `leg` >= 1: the top 24 bits of Philox
// stream 1 word (leg * 4 * ceil(V/4) + j), scaled to [0, 1) exactly, mapped
// to gamma_min + (gamma_max - gamma_min) u with explicitly rounded FP64
// operations (the FP64 value of the definition, never contracted into an
// FMA) and rounded once to T: every kernel draws the same strengths.
template <typename T>
__device__ __forceinline__ T draw_gamma(const DecodeParamsDev &p, uint64_t shot, int leg, int j, int V)
{
    const uint32_t nblk = (uint32_t)((V + 3) / 4);
    const uint4 r = philox_block(p.seed, shot, 1u, (uint32_t)leg * nblk + (uint32_t)(j >> 2));
    const uint32_t w = uint4_word(r, j & 3);
    const double u = __dmul_rn((double)(w >> 8), 1.0 / 16777216.0);
    return (T)__dadd_rn(p.gamma_min, __dmul_rn(__dadd_rn(p.gamma_max, -p.gamma_min), u));
}

// Memory strength of variable j in leg `leg` from the learned inverse CDF of
// K+1 knots at the same stream-1 draw u: knots[k] + (knots[k+1] - knots[k])
// (uK - k), k = floor(uK), in explicitly rounded FP32 operations.
__device__ __forceinline__ float knot_draw(const DecodeParamsDev &p, uint64_t shot, int leg, int j, int V)
{
    const uint32_t nblk = (uint32_t)((V + 3) / 4);
    const uint4 rr = philox_block(p.seed, shot, 1u, (uint32_t)leg * nblk + (uint32_t)(j >> 2));
    const float u = __fmul_rn((float)(uint4_word(rr, j & 3) >> 8), (float)(1.0 / 16777216.0));
    const float x = __fmul_rn(u, (float)p.lK);
    int kk = (int)floorf(x);
    if (kk >= p.lK) kk = p.lK - 1;
    const float lo = __ldg(p.lknots + kk), hi = __ldg(p.lknots + kk + 1);
    return __fadd_rn(lo, __fmul_rn(__fadd_rn(hi, -lo), __fadd_rn(x, -(float)kk)));
}

// Byte offsets of one shot's state, A first (at 0) and the rest in falling
// order of access intensity.  Bytes [0, split) live in shared memory, the rest
// in the block's region of global memory at (offset - split); split == total
// when everything fits on chip.
struct SmemPlan {
    int A, cs, ehat, res, syn, obsacc, sgn, M, best, total, split;
};

// Scale of the int8 storage form: value = q * s, q = clamp(rne(value / s),
// -127, 127); code -128 stands for +inf.  Unused by the other forms.
struct QScale {
    float s;
};

// Storage precision S of the per-shot state (M, A and the check minima) and
// the arithmetic precision C it is computed in: FP64 and FP32 store what they
// compute; FP16, BF16 and int8 store rounded values and compute in FP32.  FP16
// stores saturate at +-65504 (the largest finite half), int8 at +-127 steps.
template <typename S> struct Prec;
template <> struct Prec<float> {
    using C = float;
    static __device__ __forceinline__ C ld(float v, const QScale &) { return v; }
    static __device__ __forceinline__ float st(C v, const QScale &) { return v; }
    static __device__ __forceinline__ float pinf() { return __int_as_float(0x7f800000); }
};
template <> struct Prec<double> {
    using C = double;
    static __device__ __forceinline__ C ld(double v, const QScale &) { return v; }
    static __device__ __forceinline__ double st(C v, const QScale &) { return v; }
    static __device__ __forceinline__ double pinf() { return __longlong_as_double(0x7ff0000000000000LL); }
};
template <> struct Prec<__half> {
    using C = float;
    static __device__ __forceinline__ C ld(__half v, const QScale &) { return __half2float(v); }
    static __device__ __forceinline__ __half st(C v, const QScale &)
    {
        return __float2half_rn(fminf(fmaxf(v, -65504.f), 65504.f));
    }
    static __device__ __forceinline__ __half pinf() { return __ushort_as_half((unsigned short)0x7c00u); }
};
template <> struct Prec<__nv_bfloat16> {
    using C = float;
    static __device__ __forceinline__ C ld(__nv_bfloat16 v, const QScale &) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 st(C v, const QScale &) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ __nv_bfloat16 pinf() { return __ushort_as_bfloat16((unsigned short)0x7f80u); }
};
template <> struct Prec<int8_t> {
    using C = float;
    static __device__ __forceinline__ C ld(int8_t q, const QScale &qs)
    {
        return q == (int8_t)-128 ? __int_as_float(0x7f800000) : __fmul_rn((float)q, qs.s);
    }
    static __device__ __forceinline__ int8_t st(C v, const QScale &qs)
    {
        const int q = __float2int_rn(__fdiv_rn(v, qs.s));          // round half to even
        return (int8_t)max(-127, min(127, q));
    }
    static __device__ __forceinline__ int8_t pinf() { return (int8_t)-128; }
};

// Compressed state of one check row.  m1 / m2 carry the row's parity as their
// sign (parity = s_i xor the row's mu sign bits) and, in the learned form with
// row-tied weights, the weight of the messages they stand for; meta is the
// column code (i << lg_rsp | position) of the argmin, so a column entry is the
// argmin iff its code equals meta.  16 bytes for FP32 (one 16-byte load), 32
// for FP64, 8 for FP16 / BF16 / int8.
template <typename S> struct alignas(sizeof(S) >= 4 ? 16 : 8) CheckState {
    S m1, m2;                   // +-(w) smallest / +-(w) second-smallest |mu| over the row
    uint32_t meta;              // column code of the argmin
};

// Flip the sign of v when bit 31 of s is set (exact: sign-magnitude).
__device__ __forceinline__ float xsign(float v, uint32_t s) { return __int_as_float(__float_as_int(v) ^ (int)s); }
__device__ __forceinline__ double xsign(double v, uint32_t s)
{
    return __hiloint2double(__double2hiint(v) ^ (int)s, __double2loint(v));
}
// Minimum and maximum that propagate NaN (any NaN operand gives NaN).  A
// shot whose values overflow the arithmetic's range meets inf - inf = NaN in
// mu; with NaN-ignoring min/max the row minima would then depend on the
// order the slots are reduced in (the launch shape).  Propagating it makes
// the overflowed shot's state NaN in every kernel and shape alike: it never
// converges and is reported as a nonconvergence.
__device__ __forceinline__ float vmin2(float a, float b)
{
    float r;
    asm("min.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float vmax2(float a, float b)
{
    float r;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ double vmin2(double a, double b) { return (a != a || b != b) ? a + b : fmin(a, b); }
__device__ __forceinline__ double vmax2(double a, double b) { return (a != a || b != b) ? a + b : fmax(a, b); }
__device__ __forceinline__ float vabs2(float a) { return fabsf(a); }
__device__ __forceinline__ double vabs2(double a) { return fabs(a); }

// Sign word w of row r of a warp step from the step's slot ballots: slots
// wP .. wP + P - 1 (P = 32 / L), L bits each, bit t*L + l = lane l of slot
// wP + t.  Positional order; the caller reverses it.
template <int L, int NB>
__device__ __forceinline__ uint32_t sign_word(const uint32_t (&bal)[NB], int w, int r)
{
    constexpr int P = 32 / L;
    auto at = [&](int b) -> uint32_t { return b < NB ? bal[b] : 0u; };
    if (L == 32) return at(w);
    if (L == 16) return __byte_perm(at(2 * w), at(2 * w + 1), r ? 0x7632u : 0x5410u);
    if (L == 8) {
        const uint32_t sel = (uint32_t)r | ((uint32_t)(r + 4) << 4);
        const uint32_t lo = __byte_perm(at(4 * w), at(4 * w + 1), sel);
        const uint32_t hi = __byte_perm(at(4 * w + 2), at(4 * w + 3), sel);
        return __byte_perm(lo, hi, 0x5410u);
    }
    constexpr uint32_t GM = (L >= 32) ? 0xffffffffu : ((1u << (L & 31)) - 1u);
    uint32_t word = 0u;
#pragma unroll
    for (int t = 0; t < P; ++t) word |= ((at(w * P + t) >> (r * L)) & GM) << (t * L);
    return word;
}

// Row pass geometry: L lanes share a row (P = 32 / L rows per warp step); lane
// l of a row handles positions l, l + L, l + 2L, ... (NB of them).  Padded
// row slots (rslot, stride kRowStride) name the dummy variable V, whose A is
// +inf: such a slot yields |mu| = +inf and a clear sign bit, so it changes
// neither minimum nor parity and needs no test.
// Sign words: one row's signs of mu are rw = 2^lg_rsp / 32 words, the sign at
// position p in bit 31 - p % 32 of word p / 32 (reversed, so that a funnel
// shift by the column code brings it to bit 31).  The P rows of a warp step
// gather their bits from one ballot per slot.
// The check states and sign words are read from (csr, sgr) and written to
// (cs, sgw); the one-shot kernels pass the same arrays, the cluster kernel
// two buffers.
template <typename S, int L, int NB, bool LW>
__device__ __forceinline__ void row_pass(const DevDEM &g, const S *A, const CheckState<S> *csr, const uint32_t *sgr,
                                         CheckState<S> *cs, uint32_t *sgw, const uint32_t *syn, int warp, int nwarp,
                                         int lane, const float *wprev, const float *wrow_new, const QScale &qs)
{
    static_assert(32 % L == 0 && NB <= 16, "row geometry");
    using C = typename Prec<S>::C;
    constexpr int P = 32 / L;                   // rows per warp step = slots per sign word
    constexpr int NW = (NB + P - 1) / P;        // sign words spanned by the L * NB positions
    constexpr uint32_t GM = (L == 32) ? 0xffffffffu : ((1u << L) - 1u);
    const unsigned FULL = 0xffffffffu;
    const int r = lane / L, l = lane % L;
    const int Cn = g.C, RW = g.rw, lg = g.lg_rsp;
    // the next warp step's row slots load while this one computes
    const int stride = nwarp * P;
    int nidx[NB];
    if (warp * P < Cn) {
        const int32_t *rs = g.rslot + (size_t)(warp * P + r) * kRowStride + l;
#pragma unroll
        for (int b = 0; b < NB; ++b) nidx[b] = __ldg(rs + b * L);
    }
    for (int base = warp * P; base < Cn; base += stride) {
        const int i = base + r;
        const int il = min(i, Cn);              // rows past the end read the empty dummy row C
        int idx[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) idx[b] = nidx[b];
        if (base + stride < Cn) {
            const int32_t *rs = g.rslot + (size_t)(i + stride) * kRowStride + l;
#pragma unroll
            for (int b = 0; b < NB; ++b) nidx[b] = __ldg(rs + b * L);
        }
        const CheckState<S> o = csr[il];
        const C om1 = Prec<S>::ld(o.m1, qs), om2 = Prec<S>::ld(o.m2, qs);     // weighted when learned
        // slot b holds the argmin iff q == b * L
        const int q = (int)o.meta - (il << lg) - l;
        uint32_t W[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const uint32_t x = (w < RW) ? sgr[il * RW + w] : 0u;
            W[w] = __funnelshift_l(x, x, l);
        }
        int e0 = 0, deg = 0;
        if (LW && wprev) {
            e0 = __ldg(g.rptr + il);
            deg = (i < Cn) ? __ldg(g.rptr + il + 1) - e0 : 0;
        }
        C b1 = Num<C>::inf(), b2 = Num<C>::inf();
        int bs = 0;                             // slot of the lane's smallest |mu|
        uint32_t bal[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            C mag = (q == b * L) ? om2 : om1;
            if (LW && wprev) {
                const int pos = b * L + l;
                mag = mul_rn(mag, (C)((pos < deg) ? __ldg(wprev + e0 + pos) : 1.0f));
            }
            const uint32_t sb = (W[b / P] << ((b % P) * L)) & 0x80000000u;
            const C m = add_rn(Prec<S>::ld(A[idx[b]], qs), -xsign(mag, sb));
            bal[b] = __ballot_sync(FULL, m < (C)0);
            const C a = vabs2(m);
            b2 = vmin2(b2, vmax2(b1, a));
            bs = (a < b1) ? b : bs;
            b1 = vmin2(b1, a);
        }
        int bi = bs * L + l;
#pragma unroll
        for (int off = L / 2; off > 0; off >>= 1) {
            const C o1 = __shfl_xor_sync(FULL, b1, off);
            const C o2 = __shfl_xor_sync(FULL, b2, off);
            const int oi = __shfl_xor_sync(FULL, bi, off);
            if (o1 < b1 || (o1 == b1 && oi < bi)) { b2 = vmin2(b1, o2); b1 = o1; bi = oi; }
            else { b2 = vmin2(b2, o1); }
            b1 = vmin2(b1, o1);                 // NaN from either side reaches every lane
        }
        uint32_t X = 0u;
#pragma unroll
        for (int b = 0; b < NB; ++b) X ^= bal[b];
        const uint32_t par = (uint32_t)(__popc((X >> (r * L)) & GM) & 1);
        uint32_t mine = 0u;                     // lane l of the row stores sign word l
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const uint32_t word = sign_word<L, NB>(bal, w, r);
            mine = (l == w) ? word : mine;
        }
        if (i < Cn) {
            if (l < NW && l < RW) sgw[i * RW + l] = __brev(mine);
            if (l == 0) {
                const uint32_t sb = (syn[i >> 5] >> (i & 31)) & 1u;
                const bool neg = (par ^ sb) != 0u;
                C v1 = neg ? -b1 : b1, v2 = neg ? -b2 : b2;
                if (wrow_new) {                 // row-tied weight of the messages just formed
                    const C wn = (C)__ldg(wrow_new + i);
                    v1 = mul_rn(v1, wn);
                    v2 = mul_rn(v2, wn);
                }
                CheckState<S> n;
                n.m1 = Prec<S>::st(v1, qs);
                n.m2 = Prec<S>::st(v2, qs);
                n.meta = ((uint32_t)i << lg) + (uint32_t)bi;
                cs[i] = n;
            }
        }
    }
}

// One DEM of a launch: its structure, decoder parameters, shared-state plan
// and the batch of shots to decode with its outputs.
struct DecodeJob {
    DevDEM g;
    DecodeParamsDev p;
    SmemPlan plan;
    const uint32_t *syn_in;     // [shots][ceil(C/32)]
    uint64_t shot0;             // global index of the first shot (keys the draws)
    int64_t shots;
    uint32_t *corr_out, *pobs_out;
    StatsDev *stats_out;
    double *trace;
    int trace_iters;
    uint64_t *times_out;        // [shots][2] device clock (ns) at shot start and retire, or NULL
    FlagOut flag;               // flagged nonconvergences (flag.post NULL: not written)
    TailOut tail;               // shots handed over at a leg boundary (tail.count NULL: never)
};

constexpr int kMaxJobs = 16;
// Jobs of one launch; start[d] = first work index of job d (prefix sums of
// the shot counts), start[n] = total.
struct JobTable {
    DecodeJob job[kMaxJobs];
    int64_t start[kMaxJobs + 1];
    int n;
};

// Compressed-row Relay-BP over a table of jobs (one DEM each) in one
// persistent launch: every block takes the next work index from one device
// counter, finds its job and decodes that shot with the job's DEM, so shots of
// all DEMs share the SMs and a block whose shot ends early moves on at once.
// S: storage precision; L, NB: row geometry (for the longest row of any job);
// GS: the per-shot state does not fit in shared memory: the plan's hottest
// prefix stays there and the rest goes to a per-block region of global memory
// (gstate, state_stride bytes per block, L2-resident).
template <typename S, int L, int NB, bool GS, bool LW>
__global__ void __launch_bounds__(512, GS ? 1 : 2)
relay_decode_kernel(const __grid_constant__ JobTable tab, unsigned long long *__restrict__ work,
                    typename Prec<S>::C *__restrict__ gamma_scratch, int vmax,
                    unsigned char *__restrict__ gstate, size_t state_stride)
{
    using C = typename Prec<S>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *gblk = GS ? gstate + (size_t)blockIdx.x * state_stride : nullptr;

    __shared__ long long s_shot, s_fslot, s_defer;
    __shared__ unsigned long long s_t0;
    __shared__ int s_job, s_nsol, s_have_best, s_copy;
    __shared__ double s_best_w, s_w;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x, nwarp = nthr >> 5;
    const unsigned FULL = 0xffffffffu;
    C *gam = gamma_scratch + (int64_t)blockIdx.x * vmax;
    const int64_t total = tab.start[tab.n];

    for (;;) {
        if (tid == 0) {
            const long long q = (long long)atomicAdd(work, 1ull);
            int d = 0;
            while (d + 1 < tab.n && q >= tab.start[d + 1]) ++d;
            s_job = d;
            s_shot = q;
            s_nsol = 0;
            s_have_best = 0;
            s_best_w = 0.0;
            s_t0 = globaltimer_ns();
        }
        __syncthreads();
        if (s_shot >= total) break;
        const DecodeJob &J = tab.job[s_job];
        const DevDEM &g = J.g;
        const DecodeParamsDev &p = J.p;
        const SmemPlan &plan = J.plan;
        const long long sidx = s_shot - tab.start[s_job];
        const uint64_t shot = J.shot0 + (uint64_t)sidx;
        const uint32_t *syn_in = J.syn_in;
        uint32_t *corr_out = J.corr_out;
        uint32_t *pobs_out = J.pobs_out;
        StatsDev *stats_out = J.stats_out;
        double *trace = J.trace;
        const int trace_iters = J.trace_iters;
        // on chip: everything in shared memory, A at its start (gathers need
        // no base offset); off chip: the plan's prefix in shared memory
        auto place = [&](int off) -> unsigned char * {
            if (!GS) return smem + off;
            return off < plan.split ? smem + off : gblk + (off - plan.split);
        };
        S *M = reinterpret_cast<S *>(place(plan.M));
        S *A = reinterpret_cast<S *>(GS ? place(plan.A) : smem);
        CheckState<S> *cs = reinterpret_cast<CheckState<S> *>(place(plan.cs));
        uint32_t *sgw = reinterpret_cast<uint32_t *>(place(plan.sgn));
        uint32_t *ehat = reinterpret_cast<uint32_t *>(place(plan.ehat));
        uint32_t *best = reinterpret_cast<uint32_t *>(place(plan.best));
        uint32_t *res = reinterpret_cast<uint32_t *>(place(plan.res));
        uint32_t *syn = reinterpret_cast<uint32_t *>(place(plan.syn));
        uint32_t *obsacc = reinterpret_cast<uint32_t *>(place(plan.obsacc));
        const int Cn = g.C, V = g.V;
        const int WC = wordsof(Cn), WV = wordsof(V), WK = wordsof(g.K);
        const int NG = WV;      // variable groups of 32 (one ELL slice each)
        const int lg = g.lg_rsp, NSW = (Cn + 1) * g.rw;
        const QScale qs{p.qscale};

        // ---- shot start: M = L0, leg-0 strengths, zero messages ------------
        for (int j = tid; j < V; j += nthr) {
            const C l0 = Num<C>::l0(g, j);
            const C gm = (C)p.gamma0;
            M[j] = Prec<S>::st(l0, qs);
            gam[j] = gm;
            A[j] = Prec<S>::st(memprior<C>(gm, l0, l0), qs);
        }
        if (tid == 0) A[V] = Prec<S>::pinf();               // the dummy variable of padded row slots (+inf)
        for (int i = tid; i <= Cn; i += nthr) {             // row C: the empty dummy check
            CheckState<S> z;
            z.m1 = Prec<S>::st((C)0, qs); z.m2 = Prec<S>::st((C)0, qs); z.meta = 0u;
            cs[i] = z;
        }
        for (int w = tid; w < NSW; w += nthr) sgw[w] = 0u;
        for (int w = tid; w < WV; w += nthr) ehat[w] = 0u;
        for (int w = tid; w < WC; w += nthr) {
            const uint32_t sv = syn_in[sidx * WC + w];
            syn[w] = sv;
            res[w] = sv;                        // residual of e^ = 0
        }
        __syncthreads();

        int legs = 0, iters = 0;
        bool handed = false;
        for (int leg = 0; leg <= p.num_sets; ++leg) {
            ++legs;
            // learned parameters in this leg (row-tied weights and knots act
            // outside the inner loops; LW kernels add per-edge weights)
            const bool lleg = (p.lw || p.lwrow || p.lknots) && (p.llegs < 0 || leg < p.llegs);
            if (leg > 0) {
                // a6: new leg -- fresh strengths, marginals carried over
                for (int j = tid; j < V; j += nthr) {
                    const C l0 = Num<C>::l0(g, j);
                    C gn;
                    if (lleg && p.lknots) {
                        gn = (C)knot_draw(p, shot, leg, j, V);
                    } else {
                        gn = draw_gamma<C>(p, shot, leg, j, V);
                    }
                    const C Mj = Prec<S>::ld(M[j], qs);
                    C carry = (C)0;
                    if (p.carry_messages) {
                        const C go = gam[j];
                        carry = add_rn(Prec<S>::ld(A[j], qs), -memprior<C>(go, l0, Mj));
                    }
                    gam[j] = gn;
                    A[j] = Prec<S>::st(add_rn(memprior<C>(gn, l0, Mj), carry), qs);
                }
                if (!p.carry_messages) {
                    for (int i = tid; i < Cn; i += nthr) {
                        CheckState<S> z;
                        z.m1 = Prec<S>::st((C)0, qs); z.m2 = Prec<S>::st((C)0, qs); z.meta = 0u;
                        cs[i] = z;
                    }
                    for (int w = tid; w < Cn * g.rw; w += nthr) sgw[w] = 0u;
                }
                __syncthreads();
            }
            const int T_leg = (leg == 0) ? p.pre_iter : p.max_iterations;
            bool conv = false;
            for (int t = 0; t < T_leg; ++t) {
                // ---- a3: check rows, L lanes per row ---------------------------
                // learned weights for the first lT iterations of a learned leg,
                // unit weights (NULL) past them
                const float *wprev = nullptr, *wcur = nullptr, *wrow = nullptr;
                if (LW && lleg && p.lw) {
                    if (t > 0 && t - 1 < p.lT) wprev = p.lw + (int64_t)(t - 1) * g.E;
                    if (t < p.lT) wcur = p.lw + (int64_t)t * g.E;
                }
                if (lleg && p.lwrow && t < p.lT) wrow = p.lwrow + (int64_t)t * g.C;
                if (LW) row_pass<S, L, NB, true>(g, A, cs, sgw, cs, sgw, syn, warp, nwarp, lane, wprev, wrow, qs);
                else row_pass<S, L, NB, false>(g, A, cs, sgw, cs, sgw, syn, warp, nwarp, lane, nullptr, wrow, qs);
                __syncthreads();
                // ---- a4: variables, one lane per variable, ELL slices --------
                for (int G = warp; G < NG; G += nwarp) {
                    const int j = G * 32 + lane;
                    const bool act = j < V;
                    const C l0 = act ? Num<C>::l0(g, j) : (C)0;
                    const C gm = act ? gam[j] : (C)0;
                    const int D = __ldg(g.gdeg + G);
                    const int go = __ldg(g.goff + G);
                    const uint32_t *col = g.ecode + go + lane;
                    const uint32_t *cel = g.cedge_ell + go + lane;
                    C Ssum = (C)0;
                    // column messages nu_ij rebuilt from the check states; padded
                    // slots name the dummy check C, whose message is +0.  Four
                    // independent slots per step, the remainder one by one (D is
                    // uniform over the warp, so the split does not diverge)
                    auto msg = [&](uint32_t e, int slot) -> C {
                        const CheckState<S> q = cs[e >> lg];
                        const uint32_t hw = sgw[e >> 5];
                        C mag = Prec<S>::ld((e == q.meta) ? q.m2 : q.m1, qs);
                        if (LW && wcur) mag = mul_rn(mag, (C)__ldg(wcur + __ldg(cel + slot * 32)));
                        return xsign(mag, __funnelshift_l(hw, hw, e) & 0x80000000u);
                    };
                    int k = 0;
                    for (; k + 4 <= D; k += 4) {
                        uint32_t c[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) c[u] = __ldg(col + (k + u) * 32);
#pragma unroll
                        for (int u = 0; u < 4; ++u) Ssum = add_rn(Ssum, msg(c[u], k + u));
                    }
                    for (; k < D; ++k) Ssum = add_rn(Ssum, msg(__ldg(col + k * 32), k));
                    uint32_t dec = 0u;
                    if (act) {
                        const C Mn = add_rn(memprior<C>(gm, l0, Prec<S>::ld(M[j], qs)), Ssum);
                        M[j] = Prec<S>::st(Mn, qs);
                        A[j] = Prec<S>::st(add_rn(memprior<C>(gm, l0, Mn), Ssum), qs);
                        dec = (Mn < (C)0) ? 1u : 0u;
                        if (trace && iters < trace_iters)
                            trace[((int64_t)sidx * trace_iters + iters) * V + j] = (double)Mn;
                    }
                    const uint32_t nw = __ballot_sync(FULL, dec);
                    const uint32_t old = ehat[G];       // every lane reads, then lane 0 writes
                    __syncwarp();
                    if (lane == 0) ehat[G] = nw;
                    // a5: residual r = s + H e^ kept incrementally
                    if (((old ^ nw) >> lane) & 1u) {
                        for (int k = 0; k < D; ++k) {
                            const uint32_t i = __ldg(col + k * 32) >> lg;
                            if (i >= (uint32_t)Cn) break;          // padding (the dummy check)
                            atomicXor(res + (i >> 5), 1u << (i & 31));
                        }
                    }
                }
                __syncthreads();
                ++iters;
                uint32_t acc = 0u;
                for (int w = lane; w < WC; w += 32) acc |= res[w];
                conv = !__any_sync(FULL, acc != 0u);
                if (conv) break;
            }
            if (conv) {
                // a7: FP64 weight in ascending variable order; keep the minimum
                if (tid == 0) {
                    double w = 0.0;
                    for (int q = 0; q < WV; ++q) {
                        uint32_t x = ehat[q];
                        while (x) {
                            const int b = __ffs(x) - 1;
                            x &= x - 1u;
                            w += __ldg(g.L0d + q * 32 + b);
                        }
                    }
                    const int better = (!s_have_best || w < s_best_w) ? 1 : 0;
                    if (better) { s_best_w = w; s_have_best = 1; }
                    s_copy = better;
                    s_nsol += 1;
                }
                __syncthreads();
                if (s_copy)
                    for (int w = tid; w < WV; w += nthr) best[w] = ehat[w];
                __syncthreads();
            }
            if (!p.stop_all && s_nsol >= p.stop_nconv) break;
            // tail hand-over: a shot about to start leg >= tail.legs leaves
            // for the cluster kernel while hand-over slots last (its marginals
            // as stored, best solution and counters; a new leg restarts the
            // messages at zero)
            if (J.tail.count && leg + 1 <= p.num_sets && leg + 1 >= J.tail.legs) {
                if (tid == 0) {
                    const unsigned q = atomicAdd(J.tail.count, 1u);
                    s_defer = ((long long)q < J.tail.max) ? (long long)q : -1;
                }
                __syncthreads();
                const long long q = s_defer;
                if (q >= 0) {
                    for (int j = tid; j < V; j += nthr) reinterpret_cast<S *>(J.tail.M)[q * V + j] = M[j];
                    for (int w = tid; w < WV; w += nthr) J.tail.best[q * WV + w] = best[w];
                    if (tid == 0) {
                        TailRec rec;
                        rec.sidx = sidx;
                        rec.next_leg = leg + 1;
                        rec.legs = legs;
                        rec.iters = iters;
                        rec.nsol = s_nsol;
                        rec.have = s_have_best;
                        rec.pad = 0;
                        rec.bestw = s_best_w;
                        rec.t0 = s_t0;
                        J.tail.rec[q] = rec;
                    }
                    handed = true;
                    break;
                }
            }
        }
        if (handed) {                           // the cluster kernel writes this shot's outputs
            __syncthreads();
            continue;
        }

        // ---- outputs --------------------------------------------------------
        const int have = s_have_best;
        const uint32_t *out = have ? best : ehat;
        for (int w = tid; w < WK; w += nthr) obsacc[w] = 0u;
        __syncthreads();
        for (int w = tid; w < WV; w += nthr) {
            const uint32_t x0 = out[w];
            if (corr_out) corr_out[sidx * WV + w] = x0;
            uint32_t x = x0;
            while (x) {
                const int b = __ffs(x) - 1;
                x &= x - 1u;
                const int j = w * 32 + b;
                for (int q = __ldg(g.optr + j), qe = __ldg(g.optr + j + 1); q < qe; ++q) {
                    const int o = __ldg(g.oidx + q);
                    atomicXor(obsacc + (o >> 5), 1u << (o & 31));
                }
            }
        }
        if (tid == 0) {
            double w = s_best_w;
            if (!have) {
                w = 0.0;
                for (int q = 0; q < WV; ++q) {
                    uint32_t x = ehat[q];
                    while (x) {
                        const int b = __ffs(x) - 1;
                        x &= x - 1u;
                        w += __ldg(g.L0d + q * 32 + b);
                    }
                }
            }
            s_w = w;
            s_fslot = (!have && J.flag.post) ? (long long)atomicAdd(J.flag.count, 1u) : -1;
        }
        __syncthreads();
        if (s_fslot >= 0 && s_fslot < J.flag.max) {
            if (tid == 0) J.flag.idx[s_fslot] = sidx;
            for (int j = tid; j < V; j += nthr) J.flag.post[s_fslot * V + j] = (double)Prec<S>::ld(M[j], qs);
        }
        if (pobs_out)
            for (int w = tid; w < WK; w += nthr) pobs_out[sidx * WK + w] = obsacc[w];
        if (stats_out && tid == 0) {
            StatsDev st;
            st.converged = have;
            st.nsol = s_nsol;
            st.legs = legs;
            st.iters = iters;
            st.weight = s_w;
            stats_out[sidx] = st;
        }
        if (J.times_out && tid == 0) {
            J.times_out[2 * sidx] = s_t0;
            J.times_out[2 * sidx + 1] = globaltimer_ns();
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// FP64 decode in the literal evaluation order, for DEMs whose per-edge
// messages fit in shared memory.  Every floating-point operation is an
// explicitly rounded __dadd_rn / __dmul_rn (never contracted into an FMA) and
// sums run in the order of the definition:
//   L_j      = (1 - g_j) * L0_j + g_j * M_j
//   mu_e     = L_j + nu_b + nu_b' + ...   over the column's other entries, in
//              ascending check order
//   nu_e     = +-(minimum over the row's other |mu|)   (exact: a min and a sign)
//   M_j      = L_j + nu_b + ...           over all column entries, ascending
// so the decisions reproduce any FP64 evaluation of the same sums bit for bit.
// Shared memory: mu[E], nu[E], M[V], L[V], g[V] (FP64) and the bit vectors.
// ---------------------------------------------------------------------------
struct ExactPlan {
    int mu, nu, M, L, g, ehat, best, res, syn, obsacc, total;
};

__device__ __forceinline__ double exact_gamma(const DecodeParamsDev &p, uint64_t shot, int leg, int j, int V)
{
    const uint32_t nblk = (uint32_t)((V + 3) / 4);
    const uint4 r = philox_block(p.seed, shot, 1u, (uint32_t)leg * nblk + (uint32_t)(j >> 2));
    const double u = __dmul_rn((double)(uint4_word(r, j & 3) >> 8), 1.0 / 16777216.0);
    return __dadd_rn(p.gamma_min, __dmul_rn(__dadd_rn(p.gamma_max, -p.gamma_min), u));
}

__global__ void __launch_bounds__(256)
relay_decode_exact_kernel(DevDEM g, DecodeParamsDev p, ExactPlan plan,
                          const uint32_t *__restrict__ syn_in, uint64_t shot0, int64_t shots,
                          uint32_t *__restrict__ corr_out, uint32_t *__restrict__ pobs_out,
                          StatsDev *__restrict__ stats_out, unsigned long long *__restrict__ work,
                          double *__restrict__ trace, int trace_iters, FlagOut flag)
{
    extern __shared__ __align__(16) unsigned char smem[];
    double *mu = reinterpret_cast<double *>(smem + plan.mu);
    double *nu = reinterpret_cast<double *>(smem + plan.nu);
    double *M = reinterpret_cast<double *>(smem + plan.M);
    double *L = reinterpret_cast<double *>(smem + plan.L);
    double *gm = reinterpret_cast<double *>(smem + plan.g);
    uint32_t *ehat = reinterpret_cast<uint32_t *>(smem + plan.ehat);
    uint32_t *best = reinterpret_cast<uint32_t *>(smem + plan.best);
    uint32_t *res = reinterpret_cast<uint32_t *>(smem + plan.res);
    uint32_t *syn = reinterpret_cast<uint32_t *>(smem + plan.syn);
    uint32_t *obsacc = reinterpret_cast<uint32_t *>(smem + plan.obsacc);

    __shared__ long long s_shot, s_fslot;
    __shared__ int s_nsol, s_have_best, s_copy;
    __shared__ double s_best_w, s_w;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x, nwarp = nthr >> 5;
    const int C = g.C, V = g.V;
    const int WC = wordsof(C), WV = wordsof(V), WK = wordsof(g.K);
    const unsigned FULL = 0xffffffffu;
    const double INF = __longlong_as_double(0x7ff0000000000000LL);

    for (;;) {
        if (tid == 0) {
            s_shot = (long long)atomicAdd(work, 1ull);
            s_nsol = 0;
            s_have_best = 0;
            s_best_w = 0.0;
        }
        __syncthreads();
        const long long sidx = s_shot;
        if (sidx >= shots) break;
        const uint64_t shot = shot0 + (uint64_t)sidx;
        for (int j = tid; j < V; j += nthr) { M[j] = __ldg(g.L0d + j); gm[j] = p.gamma0; }
        for (int e = tid; e < g.E; e += nthr) nu[e] = 0.0;
        for (int w = tid; w < WV; w += nthr) ehat[w] = 0u;
        for (int w = tid; w < WC; w += nthr) {
            const uint32_t sv = syn_in[sidx * WC + w];
            syn[w] = sv;
            res[w] = sv;
        }
        __syncthreads();
        int legs = 0, iters = 0;
        for (int leg = 0; leg <= p.num_sets; ++leg) {
            ++legs;
            if (leg > 0) {
                for (int j = tid; j < V; j += nthr) gm[j] = exact_gamma(p, shot, leg, j, V);
                if (!p.carry_messages)
                    for (int e = tid; e < g.E; e += nthr) nu[e] = 0.0;
                __syncthreads();
            }
            const int T_leg = (leg == 0) ? p.pre_iter : p.max_iterations;
            bool conv = false;
            for (int t = 0; t < T_leg; ++t) {
                // memory-biased prior and variable-to-check messages
                for (int j = tid; j < V; j += nthr) {
                    const double l0 = __ldg(g.L0d + j), gj = gm[j];
                    const double Lj = __dadd_rn(__dmul_rn(__dadd_rn(1.0, -gj), l0), __dmul_rn(gj, M[j]));
                    L[j] = Lj;
                    const int q0 = __ldg(g.cptr + j), q1 = __ldg(g.cptr + j + 1);
                    for (int a = q0; a < q1; ++a) {
                        double sacc = Lj;
                        for (int b = q0; b < q1; ++b)
                            if (b != a) sacc = __dadd_rn(sacc, nu[__ldg(g.cedge + b)]);
                        mu[__ldg(g.cedge + a)] = sacc;
                    }
                }
                __syncthreads();
                // check rows: leave-one-out sign product and minimum (exact)
                for (int i = warp; i < C; i += nwarp) {
                    const int e0 = __ldg(g.rptr + i), deg = __ldg(g.rptr + i + 1) - e0;
                    if (deg == 0) continue;
                    double b1 = INF, b2 = INF;
                    int bi = 0x7fffffff;
                    uint32_t par = 0u;
                    for (int k0 = 0; k0 < deg; k0 += 32) {
                        const int k = k0 + lane;
                        uint32_t nb = 0u;
                        if (k < deg) {
                            const double m = mu[e0 + k];
                            nb = (m < 0.0) ? 1u : 0u;
                            const double a = nb ? -m : m;
                            if (a < b1) { b2 = b1; b1 = a; bi = k; }
                            else if (a < b2) { b2 = a; }
                        }
                        par ^= (uint32_t)(__popc(__ballot_sync(FULL, nb)) & 1);
                    }
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
                        const double o1 = __shfl_xor_sync(FULL, b1, off);
                        const double o2 = __shfl_xor_sync(FULL, b2, off);
                        const int oi = __shfl_xor_sync(FULL, bi, off);
                        if (o1 < b1 || (o1 == b1 && oi < bi)) { b2 = vmin(b1, o2); b1 = o1; bi = oi; }
                        else { b2 = vmin(b2, o1); }
                    }
                    const uint32_t sb = ((syn[i >> 5] >> (i & 31)) & 1u) ^ par;
                    for (int k = lane; k < deg; k += 32) {
                        const double m = mu[e0 + k];
                        const uint32_t neg = sb ^ ((m < 0.0) ? 1u : 0u);
                        const double mag = (k == bi) ? b2 : b1;
                        nu[e0 + k] = neg ? -mag : mag;
                    }
                }
                __syncthreads();
                // marginals, decisions, incremental residual
                for (int j0 = warp * 32; j0 < V; j0 += nwarp * 32) {
                    const int j = j0 + lane;
                    uint32_t dec = 0u;
                    if (j < V) {
                        double sacc = L[j];
                        const int q0 = __ldg(g.cptr + j), q1 = __ldg(g.cptr + j + 1);
                        for (int a = q0; a < q1; ++a) sacc = __dadd_rn(sacc, nu[__ldg(g.cedge + a)]);
                        M[j] = sacc;
                        dec = (sacc < 0.0) ? 1u : 0u;
                        if (trace && iters < trace_iters)
                            trace[((int64_t)sidx * trace_iters + iters) * V + j] = sacc;
                    }
                    const uint32_t nw = __ballot_sync(FULL, dec);
                    uint32_t old = 0u;
                    if (lane == 0) { old = ehat[j0 >> 5]; ehat[j0 >> 5] = nw; }
                    old = __shfl_sync(FULL, old, 0);
                    if (((old ^ nw) >> lane) & 1u) {
                        const int q0 = __ldg(g.cptr + j), q1 = __ldg(g.cptr + j + 1);
                        for (int q = q0; q < q1; ++q) {
                            const int i = __ldg(g.cchk + q);
                            atomicXor(res + (i >> 5), 1u << (i & 31));
                        }
                    }
                }
                __syncthreads();
                ++iters;
                uint32_t acc = 0u;
                for (int w = lane; w < WC; w += 32) acc |= res[w];
                conv = !__any_sync(FULL, acc != 0u);
                if (conv) break;
            }
            if (conv) {
                if (tid == 0) {
                    double w = 0.0;
                    for (int q = 0; q < WV; ++q) {
                        uint32_t x = ehat[q];
                        while (x) {
                            const int b = __ffs(x) - 1;
                            x &= x - 1u;
                            w = __dadd_rn(w, __ldg(g.L0d + q * 32 + b));
                        }
                    }
                    const int better = (!s_have_best || w < s_best_w) ? 1 : 0;
                    if (better) { s_best_w = w; s_have_best = 1; }
                    s_copy = better;
                    s_nsol += 1;
                }
                __syncthreads();
                if (s_copy)
                    for (int w = tid; w < WV; w += nthr) best[w] = ehat[w];
                __syncthreads();
            }
            if (!p.stop_all && s_nsol >= p.stop_nconv) break;
        }
        const int have = s_have_best;
        const uint32_t *out = have ? best : ehat;
        for (int w = tid; w < WK; w += nthr) obsacc[w] = 0u;
        __syncthreads();
        for (int w = tid; w < WV; w += nthr) {
            const uint32_t x0 = out[w];
            if (corr_out) corr_out[sidx * WV + w] = x0;
            uint32_t x = x0;
            while (x) {
                const int b = __ffs(x) - 1;
                x &= x - 1u;
                const int j = w * 32 + b;
                for (int q = __ldg(g.optr + j), qe = __ldg(g.optr + j + 1); q < qe; ++q) {
                    const int o = __ldg(g.oidx + q);
                    atomicXor(obsacc + (o >> 5), 1u << (o & 31));
                }
            }
        }
        if (tid == 0) {
            double w = s_best_w;
            if (!have) {
                w = 0.0;
                for (int q = 0; q < WV; ++q) {
                    uint32_t x = ehat[q];
                    while (x) {
                        const int b = __ffs(x) - 1;
                        x &= x - 1u;
                        w = __dadd_rn(w, __ldg(g.L0d + q * 32 + b));
                    }
                }
            }
            s_w = w;
            s_fslot = (!have && flag.post) ? (long long)atomicAdd(flag.count, 1u) : -1;
        }
        __syncthreads();
        if (s_fslot >= 0 && s_fslot < flag.max) {
            if (tid == 0) flag.idx[s_fslot] = sidx;
            for (int j = tid; j < V; j += nthr) flag.post[s_fslot * V + j] = M[j];
        }
        if (pobs_out)
            for (int w = tid; w < WK; w += nthr) pobs_out[sidx * WK + w] = obsacc[w];
        if (stats_out && tid == 0) {
            StatsDev st;
            st.converged = have;
            st.nsol = s_nsol;
            st.legs = legs;
            st.iters = iters;
            st.weight = s_w;
            stats_out[sidx] = st;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// a9: failure accounting, one thread per shot, warp-aggregated atomics.
// ---------------------------------------------------------------------------
__global__ void count_failures_kernel(const uint32_t *__restrict__ pobs, const uint32_t *__restrict__ tobs,
                                      const StatsDev *__restrict__ stats, int64_t shots, int WK,
                                      unsigned long long *__restrict__ counters)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t nonconv = 0u, logical = 0u, valid = 0u;
    if (s < shots) {
        valid = 1u;
        if (!stats[s].converged) {
            nonconv = 1u;
        } else {
            for (int w = 0; w < WK; ++w)
                if (pobs[s * WK + w] != tobs[s * WK + w]) { logical = 1u; break; }
        }
    }
    const unsigned FULL = 0xffffffffu;
    const int nv = __popc(__ballot_sync(FULL, valid));
    const int nn = __popc(__ballot_sync(FULL, nonconv));
    const int nl = __popc(__ballot_sync(FULL, logical));
    if ((threadIdx.x & 31) == 0) {
        if (nv) atomicAdd(counters + 0, (unsigned long long)nv);
        if (nn) atomicAdd(counters + 1, (unsigned long long)nn);
        if (nl) atomicAdd(counters + 2, (unsigned long long)nl);
        if (nn + nl) atomicAdd(counters + 3, (unsigned long long)(nn + nl));
    }
}

// ---------------------------------------------------------------------------
// Shared-memory read bandwidth probe: every thread streams 16-byte loads over
// a 32 KiB shared buffer in a bank-conflict-free pattern.  The denominator of
// the decode kernel's roofline when its messages are shared-memory resident.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) smem_read_probe(float *__restrict__ sink, int reps)
{
    __shared__ float4 buf[2048];
    for (int i = threadIdx.x; i < 2048; i += blockDim.x) buf[i] = make_float4((float)i, 1.f, 2.f, 3.f);
    __syncthreads();
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int r = 0; r < reps; ++r) {
        const float4 v = buf[(threadIdx.x + r * 32) & 2047];
        acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
    if (acc.x + acc.y + acc.z + acc.w == -1.f) sink[blockIdx.x] = acc.x;
}

}  // namespace relaybp
