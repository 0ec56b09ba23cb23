// Relay-BP with one shot spread over a thread-block cluster (latency mode).
//
// The paper measures decoding latency one shot at a time (Sec. 6.1, Table 5;
// App. F, Table 12): a single shot must then use more of the GPU than one
// SM.  Here a cluster of NC CTAs (NC <= 16, one per SM) decodes one shot: CTA
// c owns a contiguous range of check rows and of 32-variable groups and keeps
// their state in its shared memory -- A and M (FP32), the memory strengths,
// the compressed check states and sign words.  Remote state is never read per
// edge: each CTA keeps local halo copies of exactly what its passes read --
// A of every variable its rows touch, the check state and sign words of every
// row its variables touch -- and refreshes them once per pass with coalesced
// reads of the owners' shared memory (mapa + ld.shared::cluster; the halo
// lists are sorted by owner and index, so a warp reads contiguous runs).  The
// iteration is the one of the one-shot-per-block FP32 kernel, operation for
// operation and in the same order (same row minima and argmin rule, column
// sums over the same sliced-ELL slots, FP64 weights summed in ascending
// variable order), so both return the same bits.
//
// Per iteration: row pass (own rows, from the A halo), cluster barrier, pull
// the row halo, column pass (own variables, from the row halo; residual flips
// sent to the row owners with remote atomics), cluster barrier, pull the A
// halo.  The convergence test of iteration t is folded into the next barrier:
// each CTA posts "my rows are satisfied" to every CTA after the column pass
// and the next row pass runs speculatively into the other of two check-state
// buffers; if iteration t converged, that buffer is dropped.
//
// Codes (built on the host for one NC, per CTA):
//   row slot   index into the A halo (padding: the halo's dummy entry, +inf);
//              the row pass is the one-block kernels' (16 lanes per row) on
//              the CTA's rows, numbered locally, with a zero dummy row after
//              the last
//   column     (row-halo index << lg) | position (padding: the row halo's
//              dummy entry, all zero)
//   argmin     compared by position alone (the row is known from where its
//              state is kept)
//   halo src   (owner << lgv) | owner-local variable, (owner << lgcs) | row
#pragma once
#include "kernels.cuh"

namespace relaybp {

struct ClusterPlan {
    int A, M, gam, Ah, cs0, cs1, sg0, sg1, csh, sgh, ahs, rhs, ehat, best, res, syn, lst, obsacc, flags, total;
};

struct ClusterJob {
    DevDEM g;
    DecodeParamsDev p;
    ClusterPlan plan;
    const int32_t *rslot;       // [NC][CPc][kRowStride] row slots: A-halo indices (padding: the dummy)
    const uint32_t *ecode;      // sliced ELL (g.goff / g.gdeg): (row-halo index << lg) | position
    const uint32_t *ahs, *rhs;  // halo source lists of all CTAs (at ha_off / hr_off)
    int nc, Cc, CPc, lgcs, NGc, Vc, lgv;
    int ha_off[16], ha_cnt[16], hr_off[16], hr_cnt[16];
    const uint32_t *syn_in;
    uint64_t shot0;
    int64_t shots;
    uint32_t *corr_out, *pobs_out;
    StatsDev *stats_out;
    uint64_t *times_out;
    TailOut tail;               // resume: decode the shots the two-shot kernel handed over (rec != NULL)
};

__device__ __forceinline__ uint32_t cl_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_map(uint32_t saddr, uint32_t rank)
{
    uint32_t r;
    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ float cl_ld_f32(uint32_t a)
{
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t cl_ld_u32(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ uint4 cl_ld_v4(uint32_t a)
{
    uint4 v;
    asm volatile("ld.shared::cluster.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ uint2 cl_ld_v2(uint32_t a)
{
    uint2 v;
    asm volatile("ld.shared::cluster.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t cl_ld_u16(uint32_t a)
{
    unsigned short v;
    asm volatile("ld.shared::cluster.u16 %0, [%1];" : "=h"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t cl_ld_u8(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared::cluster.u8 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
// One stored value of type S / one check state from another CTA's shared memory.
template <typename S> __device__ __forceinline__ S cl_ld_val(uint32_t a);
template <> __device__ __forceinline__ float cl_ld_val<float>(uint32_t a) { return cl_ld_f32(a); }
template <> __device__ __forceinline__ __half cl_ld_val<__half>(uint32_t a)
{
    return __ushort_as_half((unsigned short)cl_ld_u16(a));
}
template <> __device__ __forceinline__ __nv_bfloat16 cl_ld_val<__nv_bfloat16>(uint32_t a)
{
    return __ushort_as_bfloat16((unsigned short)cl_ld_u16(a));
}
template <> __device__ __forceinline__ int8_t cl_ld_val<int8_t>(uint32_t a) { return (int8_t)cl_ld_u8(a); }
template <typename S> __device__ __forceinline__ CheckState<S> cl_ld_cs(uint32_t a)
{
    CheckState<S> c;
    if constexpr (sizeof(CheckState<S>) == 16) {
        const uint4 v = cl_ld_v4(a);
        memcpy(&c, &v, 16);
    } else {
        const uint2 v = cl_ld_v2(a);
        memcpy(&c, &v, 8);
    }
    return c;
}

__device__ __forceinline__ void cl_st_u32(uint32_t a, uint32_t v)
{
    asm volatile("st.shared::cluster.u32 [%0], %1;" :: "r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void cl_xor(uint32_t a, uint32_t v)
{
    asm volatile("red.shared::cluster.xor.b32 [%0], %1;" :: "r"(a), "r"(v) : "memory");
}
// Every thread of every CTA of the cluster; release / acquire orders the
// shared-memory writes before it against the reads after it, cluster-wide.
__device__ __forceinline__ void cl_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Ordered FP64 weight sum_j e_j L0_j over the cluster's bit vector `bits`
// (own words in each CTA), summed in ascending j like the one-block kernels.
// Every CTA calls it; the result is valid in CTA 0, thread 0.  Uses lst and
// s_cnt; contains one cluster barrier.
__device__ __forceinline__ double cl_weight(const ClusterJob &J, uint32_t rank, const uint32_t *bits, int nwords,
                                            int g0, int32_t *lst, int *s_cnt, uint32_t lstS, uint32_t cntS, int tid,
                                            int lane)
{
    const unsigned FULL = 0xffffffffu;
    if (tid < 32) {
        int base_cnt = 0;
        for (int w0 = 0; w0 < nwords; w0 += 32) {
            const int w = w0 + lane;
            uint32_t x = (w < nwords) ? bits[w] : 0u;
            const int c = __popc(x);
            int pre = c;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(FULL, pre, off);
                if (lane >= off) pre += y;
            }
            int at = base_cnt + pre - c;
            while (x) {
                const int b = __ffs(x) - 1;
                x &= x - 1u;
                lst[at++] = (g0 + w) * 32 + b;
            }
            base_cnt += __shfl_sync(FULL, pre, 31);
        }
        if (lane == 0) *s_cnt = base_cnt;
    }
    cl_sync();
    double wsum = 0.0;
    if (rank == 0 && tid < 32) {
        const int n_k = (lane < J.nc) ? (int)cl_ld_u32(cl_map(cntS, (uint32_t)lane)) : 0;
        int pre = n_k;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(FULL, pre, off);
            if (lane >= off) pre += y;
        }
        const int total = __shfl_sync(FULL, pre, 31);
        const int start = pre - n_k;                    // exclusive prefix of CTA `lane`
        for (int base = 0; base < total; base += 32) {
            const int idx = base + lane;
            // owner CTA of list entry idx: the last k whose start <= idx (CTAs
            // with empty lists share their successor's start)
            int kk = 0, sk = 0;
            for (int k = 0; k < J.nc; ++k) {
                const int sk2 = __shfl_sync(FULL, start, k);
                if (sk2 <= idx) { kk = k; sk = sk2; }
            }
            double v = 0.0;
            if (idx < total) {
                const int j = (int)cl_ld_u32(cl_map(lstS + 4u * (uint32_t)(idx - sk), (uint32_t)kk));
                v = __ldg(J.g.L0d + j);
            }
            const int m = min(32, total - base);
            for (int i = 0; i < m; ++i) wsum += __shfl_sync(FULL, v, i);
        }
    }
    return wsum;
}

// S: storage precision of A, M and the check minima (FP32, FP16, BF16 or
// scaled int8; arithmetic in FP32), loaded and stored exactly as the
// one-block kernels do.
template <typename S, int NB>
__global__ void __launch_bounds__(1024, 1)
relay_cluster_kernel(const __grid_constant__ ClusterJob J, unsigned long long *__restrict__ work)
{
    constexpr int L = 16;                               // lanes per row in the row pass
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_shot;
    __shared__ unsigned long long s_t0;
    __shared__ int s_cnt, s_copy;
    __shared__ double s_best_w;
    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nthr = blockDim.x, nwarp = nthr >> 5;
    const uint32_t rank = cl_rank();
    const DevDEM &g = J.g;
    const DecodeParamsDev &p = J.p;
    const ClusterPlan &pl = J.plan;
    const int V = g.V, Cn = g.C, NG = wordsof(V), WC = wordsof(Cn), WV = NG, WK = wordsof(g.K);
    const int lg = g.lg_rsp, RW = g.rw;
    const uint32_t pmask = (1u << lg) - 1u;
    // own rows [r0, r0 + nrow), own groups [g0, g1), halo sizes
    const int r0 = (int)rank * J.Cc, nrow = max(0, min(Cn - r0, J.Cc));
    const int g0 = (int)rank * J.NGc, g1 = min(NG, g0 + J.NGc), ngr = max(0, g1 - g0);
    const int HA = J.ha_cnt[rank], HR = J.hr_cnt[rank];
    DevDEM gl = g;                                      // the row pass's view: own rows, local numbering
    gl.C = nrow;
    gl.rslot = J.rslot + (size_t)rank * J.CPc * kRowStride;
    using C = float;
    constexpr uint32_t SZ = sizeof(S);
    const QScale qs{p.qscale};
    S *A = reinterpret_cast<S *>(smem + pl.A);                  // own variables (read by the others)
    S *M = reinterpret_cast<S *>(smem + pl.M);
    float *gam = reinterpret_cast<float *>(smem + pl.gam);
    S *Ah = reinterpret_cast<S *>(smem + pl.Ah);                // A halo [HA + 1]
    // the two check-state / sign-word buffers of the own rows (selected by
    // `cur`, not indexed: a register select keeps them out of local memory)
    CheckState<S> *const cs0 = reinterpret_cast<CheckState<S> *>(smem + pl.cs0);
    CheckState<S> *const cs1 = reinterpret_cast<CheckState<S> *>(smem + pl.cs1);
    uint32_t *const sg0 = reinterpret_cast<uint32_t *>(smem + pl.sg0);
    uint32_t *const sg1 = reinterpret_cast<uint32_t *>(smem + pl.sg1);
    auto CS = [&](int b) { return b ? cs1 : cs0; };
    auto SG = [&](int b) { return b ? sg1 : sg0; };
    CheckState<S> *csh = reinterpret_cast<CheckState<S> *>(smem + pl.csh);   // row halo [HR + 1]
    uint32_t *sgh = reinterpret_cast<uint32_t *>(smem + pl.sgh);
    uint32_t *ahs = reinterpret_cast<uint32_t *>(smem + pl.ahs);
    uint32_t *rhs = reinterpret_cast<uint32_t *>(smem + pl.rhs);
    uint32_t *ehat = reinterpret_cast<uint32_t *>(smem + pl.ehat);
    uint32_t *best = reinterpret_cast<uint32_t *>(smem + pl.best);
    uint32_t *res = reinterpret_cast<uint32_t *>(smem + pl.res);
    uint32_t *syn = reinterpret_cast<uint32_t *>(smem + pl.syn);
    int32_t *lst = reinterpret_cast<int32_t *>(smem + pl.lst);
    uint32_t *obsacc = reinterpret_cast<uint32_t *>(smem + pl.obsacc);
    uint32_t *flags = reinterpret_cast<uint32_t *>(smem + pl.flags);   // [2][16]
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t aS = sbase + pl.A, resS = sbase + pl.res, lstS = sbase + pl.lst, obsS = sbase + pl.obsacc;
    const uint32_t flagS = sbase + pl.flags, cntS = (uint32_t)__cvta_generic_to_shared(&s_cnt);
    const uint32_t copyS = (uint32_t)__cvta_generic_to_shared(&s_copy);
    const uint32_t shotS = (uint32_t)__cvta_generic_to_shared(&s_shot);
    const uint32_t vmask = (1u << J.lgv) - 1u, rmask = (1u << J.lgcs) - 1u;
    constexpr uint32_t CSZ = sizeof(CheckState<S>);

    // halo source lists (fixed for the launch) and the halos' dummy entries
    for (int k = tid; k < HA; k += nthr) ahs[k] = __ldg(J.ahs + J.ha_off[rank] + k);
    for (int k = tid; k < HR; k += nthr) rhs[k] = __ldg(J.rhs + J.hr_off[rank] + k);
    if (tid == 0) {
        Ah[HA] = Prec<S>::pinf();                       // padded row slots: |mu| = inf, no sign
        CheckState<S> z;
        z.m1 = Prec<S>::st(0.f, qs); z.m2 = z.m1; z.meta = 0u;
        csh[HR] = z;                                    // padded column slots: message +0
    }
    for (int w = tid; w < RW; w += nthr) sgh[HR * RW + w] = 0u;
    // refresh the A halo from the owners (coalesced: the list is sorted)
    auto pull_A = [&]() {
        for (int k = tid; k < HA; k += nthr) {
            const uint32_t c = ahs[k];
            Ah[k] = cl_ld_val<S>(cl_map(aS + SZ * (c & vmask), c >> J.lgv));
        }
    };
    // refresh the row halo (check states and sign words of buffer b)
    auto pull_rows = [&](int b) {
        const uint32_t csS = sbase + (b ? pl.cs1 : pl.cs0), sgS = sbase + (b ? pl.sg1 : pl.sg0);
        for (int k = tid; k < HR; k += nthr) {
            const uint32_t c = rhs[k], own = c >> J.lgcs, lr = c & rmask;
            csh[k] = cl_ld_cs<S>(cl_map(csS + CSZ * lr, own));
        }
        for (int x = tid; x < HR * RW; x += nthr) {
            const int k = x >> (lg - 5), w = x & (RW - 1);
            const uint32_t c = rhs[k], own = c >> J.lgcs, lr = c & rmask;
            sgh[x] = cl_ld_u32(cl_map(sgS + 4u * (lr * RW + w), own));
        }
    };

    cl_sync();                                          // every CTA runs before any remote access
    for (;;) {
        // ---- next shot: CTA 0 takes it from the counter and posts it --------
        if (rank == 0 && tid == 0) {
            const long long q = (long long)atomicAdd(work, 1ull);
            for (int k = 0; k < J.nc; ++k) {
                cl_st_u32(cl_map(shotS, (uint32_t)k), (uint32_t)(unsigned long long)q);
                cl_st_u32(cl_map(shotS + 4u, (uint32_t)k), (uint32_t)((unsigned long long)q >> 32));
            }
            s_t0 = globaltimer_ns();
        }
        cl_sync();
        // resume mode: work index -> hand-over record (its count was written
        // by the kernel before this one on the stream)
        const bool rsm = J.tail.rec != nullptr;
        const long long nwork = rsm ? min((long long)*J.tail.count, J.tail.max) : J.shots;
        if (s_shot >= nwork) break;
        const long long qrec = s_shot;
        const long long sidx = rsm ? J.tail.rec[qrec].sidx : s_shot;
        const uint64_t shot = J.shot0 + (uint64_t)sidx;

        // ---- shot start -------------------------------------------------------
        for (int jl = tid; jl < ngr * 32; jl += nthr) {
            const int j = g0 * 32 + jl;
            if (j < V) {
                const C l0 = __ldg(g.L0f + j), gm = (C)p.gamma0;
                M[jl] = rsm ? reinterpret_cast<const S *>(J.tail.M)[qrec * V + j] : Prec<S>::st(l0, qs);
                gam[jl] = gm;                           // resumed shots: redrawn at their leg start
                A[jl] = Prec<S>::st(memprior<C>(gm, l0, l0), qs);
            } else {
                A[jl] = Prec<S>::pinf();
            }
        }
        for (int i = tid; i <= nrow; i += nthr) {      // row nrow: the row pass's dummy
            CheckState<S> z;
            z.m1 = Prec<S>::st(0.f, qs); z.m2 = z.m1; z.meta = 0u;
            cs0[i] = z;
            cs1[i] = z;
        }
        for (int w = tid; w < (nrow + 1) * RW; w += nthr) { sg0[w] = 0u; sg1[w] = 0u; }
        for (int w = tid; w < ngr; w += nthr) {
            ehat[w] = 0u;                               // e^ = 0 with residual s: consistent for the incremental residual
            best[w] = rsm ? J.tail.best[qrec * WV + g0 + w] : 0u;
        }
        for (int w = warp; w < (J.Cc + 31) / 32; w += nwarp) {
            const int r = w * 32 + lane, i = r0 + r;
            const uint32_t bit = (r < nrow) ? (J.syn_in[(size_t)sidx * WC + (i >> 5)] >> (i & 31)) & 1u : 0u;
            const uint32_t word = __ballot_sync(FULL, bit != 0u);
            if (lane == 0) { syn[w] = word; res[w] = word; }
        }
        if (rank == 0) for (int w = tid; w < WK; w += nthr) obsacc[w] = 0u;
        int nsol = 0, have = 0, legs = 0, iters = 0, cur = 0, leg0 = 0;
        if (rsm) {
            const TailRec rec = J.tail.rec[qrec];
            nsol = rec.nsol;
            have = rec.have;
            legs = rec.legs;
            iters = rec.iters;
            leg0 = rec.next_leg;
        }
        if (tid == 0) s_best_w = rsm ? J.tail.rec[qrec].bestw : 0.0;
        if (rsm && tid == 0) s_t0 = J.tail.rec[qrec].t0;
        cl_sync();
        pull_A();
        __syncthreads();

        for (int leg = leg0; leg <= p.num_sets; ++leg) {
            ++legs;
            if (leg > 0) {
                for (int jl = tid; jl < ngr * 32; jl += nthr) {
                    const int j = g0 * 32 + jl;
                    if (j >= V) continue;
                    const C l0 = __ldg(g.L0f + j);
                    const C gn = draw_gamma<C>(p, shot, leg, j, V);
                    const C Mj = Prec<S>::ld(M[jl], qs);
                    C carry = 0.f;
                    if (p.carry_messages) carry = add_rn(Prec<S>::ld(A[jl], qs), -memprior<C>(gam[jl], l0, Mj));
                    gam[jl] = gn;
                    A[jl] = Prec<S>::st(add_rn(memprior<C>(gn, l0, Mj), carry), qs);
                }
                if (!p.carry_messages) {
                    for (int r = tid; r < nrow; r += nthr) {
                        CheckState<S> z;
                        z.m1 = Prec<S>::st(0.f, qs); z.m2 = z.m1; z.meta = 0u;
                        CS(cur)[r] = z;
                    }
                    for (int w = tid; w < nrow * RW; w += nthr) SG(cur)[w] = 0u;
                }
                cl_sync();
                pull_A();
                __syncthreads();
            }
            const int T_leg = (leg == 0) ? p.pre_iter : p.max_iterations;
            bool conv = false;
            for (int t = 0; t < T_leg; ++t) {
                // ---- a3: own rows; for t > 0 also speculative past iteration t-1
                row_pass<S, L, NB, false>(gl, Ah, CS(cur), SG(cur), CS(cur ^ 1), SG(cur ^ 1), syn, warp, nwarp, lane,
                                          nullptr, nullptr, qs);
                cl_sync();
                if (t > 0) {
                    const uint32_t f = (lane < J.nc) ? flags[((t - 1) & 1) * 16 + lane] : 0u;
                    if (!__any_sync(FULL, f != 0u)) { conv = true; break; }   // iteration t-1 solved H e = s
                }
                cur ^= 1;
                pull_rows(cur);
                __syncthreads();
                // ---- a4: own variables, from the row halo ------------------------
                for (int G = g0 + warp; G < g1; G += nwarp) {
                    const int j = G * 32 + lane, jl = (G - g0) * 32 + lane;
                    const bool act = j < V;
                    const float l0 = act ? __ldg(g.L0f + j) : 0.f;
                    const float gm = act ? gam[jl] : 0.f;
                    const int D = __ldg(g.gdeg + G);
                    const uint32_t *col = J.ecode + __ldg(g.goff + G) + lane;
                    float Ssum = 0.f;
                    int k = 0;
                    for (; k + 4 <= D; k += 4) {
                        uint32_t c[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) c[u] = __ldg(col + (k + u) * 32);
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const uint32_t hr = c[u] >> lg;
                            const CheckState<S> q = csh[hr];
                            const uint32_t hw = sgh[hr * RW + ((c[u] & pmask) >> 5)];
                            const C mag = Prec<S>::ld(((c[u] & pmask) == (q.meta & pmask)) ? q.m2 : q.m1, qs);
                            Ssum = add_rn(Ssum, xsign(mag, __funnelshift_l(hw, hw, c[u]) & 0x80000000u));
                        }
                    }
                    for (; k < D; ++k) {
                        const uint32_t c = __ldg(col + k * 32), hr = c >> lg;
                        const CheckState<S> q = csh[hr];
                        const uint32_t hw = sgh[hr * RW + ((c & pmask) >> 5)];
                        const C mag = Prec<S>::ld(((c & pmask) == (q.meta & pmask)) ? q.m2 : q.m1, qs);
                        Ssum = add_rn(Ssum, xsign(mag, __funnelshift_l(hw, hw, c) & 0x80000000u));
                    }
                    uint32_t dec = 0u;
                    if (act) {
                        const C Mn = add_rn(memprior<C>(gm, l0, Prec<S>::ld(M[jl], qs)), Ssum);
                        M[jl] = Prec<S>::st(Mn, qs);
                        A[jl] = Prec<S>::st(add_rn(memprior<C>(gm, l0, Mn), Ssum), qs);
                        dec = (Mn < 0.f) ? 1u : 0u;
                    }
                    const uint32_t nw = __ballot_sync(FULL, dec);
                    const uint32_t old = ehat[G - g0];
                    __syncwarp();
                    if (lane == 0) ehat[G - g0] = nw;
                    if (((old ^ nw) >> lane) & 1u) {        // a5: flip this variable's checks at their owners
                        // the first eight codes load together; padding codes
                        // (the dummy row, at the end of a column) flip nothing
                        auto flip = [&](uint32_t hr) {
                            const uint32_t c = rhs[hr], lr = c & rmask;
                            cl_xor(cl_map(resS + 4u * (lr >> 5), c >> J.lgcs), 1u << (lr & 31));
                        };
                        uint32_t cc[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) cc[u] = (u < D) ? __ldg(col + u * 32) : 0u;
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const uint32_t hr = cc[u] >> lg;
                            if (u < D && hr < (uint32_t)HR) flip(hr);
                        }
                        for (int kk = 8; kk < D; ++kk) {
                            const uint32_t hr = __ldg(col + kk * 32) >> lg;
                            if (hr >= (uint32_t)HR) break;               // padding (the dummy row)
                            flip(hr);
                        }
                    }
                }
                cl_sync();
                ++iters;
                // post "my rows are satisfied" to every CTA
                if (warp == 0) {
                    uint32_t acc = 0u;
                    for (int w = lane; w < ((nrow + 31) >> 5); w += 32) acc |= res[w];
                    const uint32_t bad = __any_sync(FULL, acc != 0u) ? 1u : 0u;
                    if (lane < J.nc) cl_st_u32(cl_map(flagS + 4u * ((t & 1) * 16 + rank), (uint32_t)lane), bad);
                }
                pull_A();
                __syncthreads();
                if (t + 1 == T_leg) {                       // no next iteration to overlap with
                    cl_sync();
                    const uint32_t f = (lane < J.nc) ? flags[(t & 1) * 16 + lane] : 0u;
                    conv = !__any_sync(FULL, f != 0u);
                }
            }
            if (conv) {
                // a7: ordered FP64 weight; keep the lowest (earliest on ties)
                const double w = cl_weight(J, rank, ehat, ngr, g0, lst, &s_cnt, lstS, cntS, tid, lane);
                if (rank == 0 && tid == 0) {
                    const int better = (!have || w < s_best_w) ? 1 : 0;
                    if (better) s_best_w = w;
                    for (int k = 0; k < J.nc; ++k) cl_st_u32(cl_map(copyS, (uint32_t)k), (uint32_t)better);
                }
                cl_sync();
                if (s_copy)
                    for (int w2 = tid; w2 < ngr; w2 += nthr) best[w2] = ehat[w2];
                have = 1;
                nsol += 1;
                __syncthreads();
            }
            if (!p.stop_all && nsol >= p.stop_nconv) break;
        }

        // ---- outputs ----------------------------------------------------------
        const uint32_t *out = have ? best : ehat;
        double wfin = 0.0;
        if (!have) wfin = cl_weight(J, rank, ehat, ngr, g0, lst, &s_cnt, lstS, cntS, tid, lane);
        for (int w = tid; w < ngr; w += nthr) {
            const uint32_t x0 = out[w];
            if (J.corr_out) J.corr_out[(size_t)sidx * WV + g0 + w] = x0;
            uint32_t x = x0;
            while (x) {
                const int b = __ffs(x) - 1;
                x &= x - 1u;
                const int j = (g0 + w) * 32 + b;
                for (int q = __ldg(g.optr + j), qe = __ldg(g.optr + j + 1); q < qe; ++q) {
                    const int o = __ldg(g.oidx + q);
                    cl_xor(cl_map(obsS + 4u * (uint32_t)(o >> 5), 0u), 1u << (o & 31));
                }
            }
        }
        cl_sync();
        if (rank == 0) {
            if (J.pobs_out)
                for (int w = tid; w < WK; w += nthr) J.pobs_out[(size_t)sidx * WK + w] = obsacc[w];
            if (tid == 0) {
                if (J.stats_out) {
                    StatsDev st;
                    st.converged = have;
                    st.nsol = nsol;
                    st.legs = legs;
                    st.iters = iters;
                    st.weight = have ? s_best_w : wfin;
                    J.stats_out[sidx] = st;
                }
                if (J.times_out) {
                    J.times_out[2 * sidx] = s_t0;
                    J.times_out[2 * sidx + 1] = globaltimer_ns();
                }
            }
        }
        cl_sync();                                      // no CTA still reads this shot's state
    }
}

}  // namespace relaybp
