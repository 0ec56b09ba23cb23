// Host side of the C ABI declared in include/relaybp.h.
//
// relaybp_build lays the DEM out for the kernels: the check matrix in row
// order, in column order (check and row-major edge of each entry) and as
// sliced-ELL column groups of 32 variables (check << 12 | position in row),
// prior LLRs in FP64 and FP32, and the sampler thresholds floor(p_j 2^32).  The handle owns every device
// allocation and a small scratch area: the persistent kernel's work counter,
// failure counters and a per-block buffer for the leg's memory strengths.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/relaybp.h"
#include "kernels.cuh"
#include "learned.cuh"
#include "pair.cuh"
#include "osd.cuh"
#include "spa.cuh"
#include "windows.cuh"
#include "cluster.cuh"

using namespace relaybp;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(expr)                                                                    \
    do {                                                                                  \
        cudaError_t e__ = (expr);                                                         \
        if (e__ != cudaSuccess)                                                           \
            return fail(RELAYBP_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e__), \
                        __FILE__, __LINE__);                                              \
    } while (0)

int words(int64_t bits) { return (int)((bits + 31) / 32); }

}  // namespace

struct relaybp_handle;
namespace {
int check_device(const relaybp_handle *h);
}

// Device scratch of a launch owner (a handle or a group): the persistent
// kernel's work counter, one row of memory strengths per resident block and,
// for DEMs too large for shared memory, one state region per resident block.
struct Scratch {
    unsigned long long *work = nullptr;
    void *gamma = nullptr;
    size_t gamma_bytes = 0;
    unsigned char *gstate = nullptr;
    size_t gstate_bytes = 0;
    bool fixed = false;             // true: never (re)allocate (allocation-free entry point)
};

struct relaybp_handle {
    int device = 0;
    int num_sms = 0;
    relaybp_params params{};
    DevDEM dem{};
    std::vector<void *> allocs;
    Scratch scratch;
    // host-buffer staging (relaybp_decode_host)
    uint32_t *d_stage_syn = nullptr, *d_stage_pobs = nullptr;
    StatsDev *d_stage_stats = nullptr;
    int64_t stage_shots = 0;
    int64_t launches = 0;
    int max_row_deg = 0;
    double l0max = 0.0;             // largest |prior LLR| (automatic int8 scale)
    // learned-form training scratch: work counter and one gradient row per block
    int tuned_L = 0, tuned_NB = 0, tuned_threads = 0; // autotuned launch shape (0: heuristic)
    // two-shot lockstep kernel (FP32): row slots and column codes, or NULL
    const uint32_t *rslot2 = nullptr, *ecode2 = nullptr;
    const int32_t *goff2 = nullptr;                   // group offsets of ecode2 (>= 8 slots per group)
    const float *L0p = nullptr;                       // FP32 priors padded to whole groups
    int pair_nb = 0;                                  // row slots per lane (template NB)
    int pair_warps = 0;                               // warps per block (0: heuristic)
    int pair_off = 1;                                 // 1: never use it (relaybp_set_kernel)
    const float *lw = nullptr, *lknots = nullptr;     // learned inference parameters (caller-owned)
    const float *lwrow = nullptr;                     // row-tied learned weights [lT][C]
    int lT = 0, lK = 0;
    int llegs = -1;                                   // legs using the learned parameters (< 0: all)
    unsigned long long *d_lwork = nullptr;
    void *d_lgbar = nullptr;
    size_t lgbar_bytes = 0;
    int32_t *d_osd_order = nullptr;                   // OSD: per-block column order scratch
    size_t osd_order_bytes = 0;
    // cluster kernel: codes for cl_nc CTAs per shot (cl_nc == 0: none);
    // cl_mode 1 decodes every shot with it, 2 only the shots the two-shot
    // kernel hands over at leg tail_legs (tail offload)
    int cl_nc = 0, cl_nb = 0, cl_clusters = 0, cl_mode = 0;
    int tail_legs = 0;
    long long tail_max = 0;
    TailRec *tail_rec = nullptr;
    float *tail_M = nullptr;
    uint32_t *tail_best = nullptr;
    unsigned int *tail_count = nullptr;
    ClusterJob cl{};                                  // layout part (codes, sizes, plan)
    int32_t *cl_rslot = nullptr;
    uint32_t *cl_ecode = nullptr;
    uint32_t *cl_halo[2] = {nullptr, nullptr};        // A-halo and row-halo source lists
};

struct relaybp_group {
    int device = 0;
    std::vector<relaybp_handle *> handles;
    Scratch scratch;
    int64_t launches = 0;
};

namespace {
// Launching entry points work on the handle's own device only: its arrays
// live there, and a launch on another device would read them across devices.
int check_device(const relaybp_handle *h)
{
    int cur = -1;
    CUDA_TRY(cudaGetDevice(&cur));
    if (cur != h->device)
        return fail(RELAYBP_ERR_INVALID, "the handle's device %d is not current (device %d is)", h->device, cur);
    return 0;
}
}  // namespace

namespace {

template <typename T>
int upload(relaybp_handle *h, const std::vector<T> &v, const T **dst)
{
    void *p = nullptr;
    size_t n = std::max<size_t>(1, v.size()) * sizeof(T);
    CUDA_TRY(cudaMalloc(&p, n));
    h->allocs.push_back(p);
    if (!v.empty()) CUDA_TRY(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    *dst = static_cast<const T *>(p);
    return 0;
}

int check_csr(const relaybp_csr *m, const char *name)
{
    if (!m || !m->indptr || (m->indptr[m->rows] > 0 && !m->indices))
        return fail(RELAYBP_ERR_INVALID, "%s: null pointer", name);
    if (m->rows < 0 || m->cols < 0) return fail(RELAYBP_ERR_INVALID, "%s: negative size", name);
    if (m->indptr[0] != 0) return fail(RELAYBP_ERR_INVALID, "%s: indptr[0] != 0", name);
    for (int32_t i = 0; i < m->rows; ++i) {
        if (m->indptr[i + 1] < m->indptr[i]) return fail(RELAYBP_ERR_INVALID, "%s: indptr decreases at row %d", name, i);
        for (int32_t e = m->indptr[i]; e < m->indptr[i + 1]; ++e) {
            int32_t c = m->indices[e];
            if (c < 0 || c >= m->cols)
                return fail(RELAYBP_ERR_INVALID, "%s: column %d out of range at row %d", name, c, i);
            if (e > m->indptr[i] && c <= m->indices[e - 1])
                return fail(RELAYBP_ERR_INVALID, "%s: row %d not strictly increasing", name, i);
        }
    }
    return 0;
}

int check_params(const relaybp_params *p)
{
    if (!p) return fail(RELAYBP_ERR_INVALID, "params is NULL");
    if (p->pre_iter < 1 || p->max_iterations < 1 || p->num_sets < 0 || p->stop_nconv < 1)
        return fail(RELAYBP_ERR_INVALID, "iteration/leg/solution counts out of range");
    if (!std::isfinite(p->gamma0) || !std::isfinite(p->gamma_min) || !std::isfinite(p->gamma_max) ||
        p->gamma_min > p->gamma_max)
        return fail(RELAYBP_ERR_INVALID, "memory strengths must be finite with gamma_min <= gamma_max");
    if (p->msg_dtype != RELAYBP_MSG_F64 && p->msg_dtype != RELAYBP_MSG_F32 && p->msg_dtype != RELAYBP_MSG_F16 &&
        p->msg_dtype != RELAYBP_MSG_BF16 && p->msg_dtype != RELAYBP_MSG_I8)
        return fail(RELAYBP_ERR_UNSUPPORTED, "msg_dtype %d not supported", p->msg_dtype);
    if (p->msg_dtype == RELAYBP_MSG_I8 ? !(p->int8_scale >= 0.0f && p->int8_scale < 1e30f) : p->int8_scale != 0.0f)
        return fail(RELAYBP_ERR_INVALID, "int8_scale must be finite and >= 0 for int8 storage, 0 otherwise");
    return 0;
}

// The memory-strength counter block (leg * ceil(V/4) + j/4) must fit 32 bits.
int check_legs(const relaybp_params *p, int32_t V)
{
    if ((uint64_t)(p->num_sets + 1) * (uint64_t)((V + 3) / 4) > 0xffffffffull)
        return fail(RELAYBP_ERR_INVALID, "num_sets * ceil(V/4) exceeds the 32-bit draw counter");
    return 0;
}

// The automatic int8 step is the largest |prior LLR| / 24; it is 0 only when
// every prior is exactly 1/2, and a zero step cannot scale anything.
int check_int8_step(const relaybp_params &p, double l0max)
{
    if (p.msg_dtype == RELAYBP_MSG_I8 && p.int8_scale == 0.0f && !((float)(l0max / 24.0) > 0.0f))
        return fail(RELAYBP_ERR_INVALID, "automatic int8 step is 0 (every prior LLR is 0): give int8_scale > 0");
    return 0;
}

// Row-pass geometry (lanes per row L, positions per lane NB) for the longest row.
struct RowGeom { int L, NB; };
RowGeom row_geom(int maxdeg)
{
    const RowGeom opts[] = {{4, 4}, {8, 4}, {8, 8}, {8, 12}, {8, 16}, {16, 16}, {32, 16}};
    for (const RowGeom &o : opts)
        if (maxdeg <= o.L * o.NB) return o;
    return {0, 0};
}

// One shot's state in falling order of access intensity: A (gathered per edge
// by the row pass), the check states and the bit vectors (per column entry /
// per variable group), the sign words, M (streamed once per variable), best
// (per solution).  `budget` = shared-memory bytes available: split = the end
// of the longest prefix of whole arrays that fits (everything when it all
// fits).
SmemPlan make_plan(const DevDEM &g, size_t esz, size_t csz, size_t budget)
{
    SmemPlan s{};
    size_t off = 0, split = 0;
    auto take = [&](size_t bytes) {
        off = (off + 15) & ~size_t(15);
        size_t at = off;
        off += bytes;
        if (((split + 15) & ~size_t(15)) == at && off <= budget) split = off;
        return (int)at;
    };
    s.A = take(esz * ((size_t)g.V + 1));            // first: the row pass gathers A[j] at offset 0
    s.cs = take(csz * ((size_t)g.C + 1));           // + the empty dummy check
    s.ehat = take(4 * (size_t)words(g.V));
    s.res = take(4 * (size_t)words(g.C));
    s.syn = take(4 * (size_t)words(g.C));
    s.obsacc = take(4 * (size_t)std::max(1, words(g.K)));
    s.sgn = take(4 * ((size_t)g.C + 1) * (size_t)g.rw);
    s.M = take(esz * g.V);
    s.best = take(4 * (size_t)words(g.V));
    s.total = (int)((off + 15) & ~size_t(15));
    s.split = (size_t)s.total <= budget ? s.total : (int)((split + 15) & ~size_t(15));
    return s;
}

ExactPlan make_exact_plan(const DevDEM &g)
{
    ExactPlan s{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 15) & ~size_t(15);
        size_t at = off;
        off += bytes;
        return (int)at;
    };
    s.mu = take(8 * (size_t)g.E);
    s.nu = take(8 * (size_t)g.E);
    s.M = take(8 * (size_t)g.V);
    s.L = take(8 * (size_t)g.V);
    s.g = take(8 * (size_t)g.V);
    s.ehat = take(4 * (size_t)words(g.V));
    s.best = take(4 * (size_t)words(g.V));
    s.res = take(4 * (size_t)words(g.C));
    s.syn = take(4 * (size_t)words(g.C));
    s.obsacc = take(4 * (size_t)std::max(1, words(g.K)));
    s.total = (int)((off + 15) & ~size_t(15));
    return s;
}

DecodeParamsDev dev_params(const relaybp_params &p)
{
    DecodeParamsDev d{};
    d.gamma0 = p.gamma0;
    d.gamma_min = p.gamma_min;
    d.gamma_max = p.gamma_max;
    d.pre_iter = p.pre_iter;
    d.num_sets = p.num_sets;
    d.max_iterations = p.max_iterations;
    d.stop_nconv = p.stop_nconv;
    d.stop_all = p.stop_all;
    d.carry_messages = p.carry_messages;
    d.seed = p.seed;
    return d;
}

int block_threads(const DevDEM &g)
{
    if (g.E <= 2048) return 64;
    if (g.E <= 16384) return 256;
    return 512;
}

int scratch_reserve(Scratch &sc, size_t gamma_bytes, size_t gstate_bytes)
{
    if (!sc.work) {
        if (sc.fixed) return fail(RELAYBP_ERR_UNSUPPORTED, "scratch has no work counter");
        CUDA_TRY(cudaMalloc(&sc.work, 256));
    }
    if (sc.gamma_bytes < gamma_bytes) {
        if (sc.fixed)
            return fail(RELAYBP_ERR_UNSUPPORTED, "needs %zu bytes of memory-strength scratch, %zu available",
                        gamma_bytes, sc.gamma_bytes);
        if (sc.gamma) { cudaFree(sc.gamma); sc.gamma = nullptr; }
        sc.gamma_bytes = 0;
        CUDA_TRY(cudaMalloc(&sc.gamma, gamma_bytes));
        sc.gamma_bytes = gamma_bytes;
    }
    if (sc.gstate_bytes < gstate_bytes) {
        if (sc.fixed)
            return fail(RELAYBP_ERR_UNSUPPORTED, "needs %zu bytes of off-chip decoder state, %zu available",
                        gstate_bytes, sc.gstate_bytes);
        if (sc.gstate) { cudaFree(sc.gstate); sc.gstate = nullptr; }
        sc.gstate_bytes = 0;
        CUDA_TRY(cudaMalloc(&sc.gstate, gstate_bytes));
        sc.gstate_bytes = gstate_bytes;
    }
    return 0;
}

void scratch_free(Scratch &sc)
{
    if (sc.fixed) return;
    cudaFree(sc.work);
    cudaFree(sc.gamma);
    cudaFree(sc.gstate);
    sc = Scratch{};
}

// Inputs and outputs of one DEM in a launch.
struct JobIO {
    const uint32_t *syn;
    uint64_t shot0;
    int64_t shots;
    uint32_t *corr, *pobs;
    StatsDev *stats;
    double *trace;
    int trace_iters;
    uint64_t *times = nullptr;
    FlagOut flag{};
    TailOut tail{};             // two-shot kernel: hand long shots over (count NULL: no)
};

// FP64 in the literal evaluation order whenever one shot's per-edge messages
// fit in one block's shared memory (FP64 is the parity form: evaluation order
// before occupancy); returns 1 if the DEM is too large for this kernel.
int launch_decode_exact(relaybp_handle *h, Scratch &sc, const JobIO &io, cudaStream_t st)
{
    const DevDEM &g = h->dem;
    ExactPlan plan = make_exact_plan(g);
    int maxsm = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    if (plan.total > maxsm) return 1;
    CUDA_TRY(cudaFuncSetAttribute(relay_decode_exact_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, plan.total));
    const int threads = g.E <= 4096 ? 128 : 256;
    int per_sm = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, relay_decode_exact_kernel, threads, plan.total));
    if (per_sm < 1) return 1;
    int64_t blocks = (int64_t)per_sm * h->num_sms;
    if (blocks > io.shots) blocks = io.shots;
    if (int rc = scratch_reserve(sc, 0, 0)) return rc;
    CUDA_TRY(cudaMemsetAsync(sc.work, 0, sizeof(unsigned long long), st));
    relay_decode_exact_kernel<<<(unsigned)blocks, threads, plan.total, st>>>(
        g, dev_params(h->params), plan, io.syn, io.shot0, io.shots, io.corr, io.pobs, io.stats, sc.work, io.trace,
        io.trace_iters, io.flag);
    CUDA_TRY(cudaGetLastError());
    h->launches += 1;
    return 0;
}

// One persistent launch of the compressed kernel over n jobs (DEMs).
template <typename S, int L, int NB>
int launch_jobs(relaybp_handle *const *hs, const JobIO *io, int n, Scratch &sc, cudaStream_t st, bool on_chip_only)
{
    using C = typename Prec<S>::C;
    if (n < 1 || n > kMaxJobs) return fail(RELAYBP_ERR_INVALID, "%d DEMs in one launch (1..%d)", n, kMaxJobs);
    const int device = hs[0]->device, num_sms = hs[0]->num_sms;
    JobTable tab{};
    bool learned = false;
    int plan_max = 0, vmax = 0, threads = 64;
    int64_t total = 0;
    for (int d = 0; d < n; ++d) {
        const relaybp_handle *h = hs[d];
        if (!h->dem.rslot)
            return fail(RELAYBP_ERR_UNSUPPORTED, "DEM %d: rows of %d entries exceed the decode kernel's %d", d,
                        h->max_row_deg, kRowStride);
        DecodeJob &J = tab.job[d];
        J.g = h->dem;
        J.p = dev_params(h->params);
        J.p.lw = h->lw;
        J.p.lknots = h->lknots;
        J.p.lT = h->lT;
        J.p.lK = h->lK;
        J.p.lwrow = h->lwrow;
        J.p.llegs = h->llegs;
        J.p.qscale = h->params.int8_scale > 0.0f ? h->params.int8_scale : (float)(h->l0max / 24.0);
        if (h->lw) learned = true;      // per-edge weights; row-tied weights and knots run in the plain kernel
        J.plan = make_plan(h->dem, sizeof(S), sizeof(CheckState<S>), (size_t)-1);
        J.syn_in = io[d].syn;
        J.tail = io[d].tail;
        J.shot0 = io[d].shot0;
        J.shots = io[d].shots;
        J.corr_out = io[d].corr;
        J.pobs_out = io[d].pobs;
        J.stats_out = io[d].stats;
        J.trace = io[d].trace;
        J.trace_iters = io[d].trace_iters;
        J.times_out = io[d].times;
        J.flag = io[d].flag;
        tab.start[d] = total;
        total += io[d].shots;
        plan_max = std::max(plan_max, J.plan.total);
        vmax = std::max(vmax, h->dem.V);
        threads = std::max(threads, h->tuned_threads > 0 ? h->tuned_threads : block_threads(h->dem));
    }
    tab.start[n] = total;
    tab.n = n;
    if (total == 0) return 0;
    int maxsm = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    // shared-memory state when one shot's state fits, else a per-block region
    // of global memory (one block per SM keeps the regions L2-resident)
    const bool gs = plan_max + 1024 > maxsm;
    // off chip: each job keeps its plan's hottest prefix in shared memory
    int smem_gs = 0, gbytes = 0;
    if (gs) {
        for (int d = 0; d < n; ++d) {
            DecodeJob &J = tab.job[d];
            J.plan = make_plan(hs[d]->dem, sizeof(S), sizeof(CheckState<S>), (size_t)(maxsm - 1024));
            smem_gs = std::max(smem_gs, J.plan.split);
            gbytes = std::max(gbytes, J.plan.total - J.plan.split);
        }
    }
    if (gs && on_chip_only)
        return fail(RELAYBP_ERR_UNSUPPORTED, "one shot's decoder state (%d bytes) exceeds shared memory (%d bytes); "
                    "the allocation-free entry point keeps it on chip only: use relaybp_decode_batch",
                    plan_max, maxsm);
    int64_t resident = num_sms;
    {
        auto kern = gs ? (learned ? relay_decode_kernel<S, L, NB, true, true> : relay_decode_kernel<S, L, NB, true, false>)
                       : (learned ? relay_decode_kernel<S, L, NB, false, true> : relay_decode_kernel<S, L, NB, false, false>);
        const int dyn = gs ? smem_gs : plan_max;
        CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
        int per_sm = 0;
        CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, dyn));
        if (per_sm < 1)
            return fail(RELAYBP_ERR_UNSUPPORTED, "decode kernel cannot be resident with %d bytes", dyn);
        resident = (int64_t)per_sm * num_sms;
    }
    int64_t blocks = std::min<int64_t>(resident, total);
    const size_t stride = ((size_t)std::max(gbytes, 16) + 255) & ~(size_t)255;
    const size_t gamma_need = (size_t)(sc.fixed ? blocks : resident) * vmax * sizeof(C);
    if (int rc = scratch_reserve(sc, gamma_need, gs ? (size_t)resident * stride : 0)) return rc;
    CUDA_TRY(cudaMemsetAsync(sc.work, 0, sizeof(unsigned long long), st));
    if (!gs && !learned)
        relay_decode_kernel<S, L, NB, false, false><<<(unsigned)blocks, threads, plan_max, st>>>(
            tab, sc.work, static_cast<C *>(sc.gamma), vmax, nullptr, 0);
    else if (!gs)
        relay_decode_kernel<S, L, NB, false, true><<<(unsigned)blocks, threads, plan_max, st>>>(
            tab, sc.work, static_cast<C *>(sc.gamma), vmax, nullptr, 0);
    else if (!learned)
        relay_decode_kernel<S, L, NB, true, false><<<(unsigned)blocks, threads, smem_gs, st>>>(
            tab, sc.work, static_cast<C *>(sc.gamma), vmax, sc.gstate, stride);
    else
        relay_decode_kernel<S, L, NB, true, true><<<(unsigned)blocks, threads, smem_gs, st>>>(
            tab, sc.work, static_cast<C *>(sc.gamma), vmax, sc.gstate, stride);
    CUDA_TRY(cudaGetLastError());
    return 0;
}

template <typename S>
int launch_jobs_geom(relaybp_handle *const *hs, const JobIO *io, int n, Scratch &sc, cudaStream_t st,
                     bool on_chip_only)
{
    int maxdeg = 0;
    for (int d = 0; d < n; ++d) maxdeg = std::max(maxdeg, hs[d]->max_row_deg);
    RowGeom rg = row_geom(maxdeg);
    if (n == 1 && hs[0]->tuned_L > 0 && hs[0]->tuned_L * hs[0]->tuned_NB >= maxdeg)
        rg = RowGeom{hs[0]->tuned_L, hs[0]->tuned_NB};
#define RELAYBP_GEOM(LL, NN)                                                                                   \
    if (rg.L == LL && rg.NB == NN) return launch_jobs<S, LL, NN>(hs, io, n, sc, st, on_chip_only);
    RELAYBP_GEOM(4, 4)
    RELAYBP_GEOM(8, 4)
    RELAYBP_GEOM(8, 8)
    RELAYBP_GEOM(8, 12)
    RELAYBP_GEOM(8, 16)
    RELAYBP_GEOM(16, 16)
    RELAYBP_GEOM(32, 16)
#undef RELAYBP_GEOM
    return fail(RELAYBP_ERR_UNSUPPORTED, "a detector touches %d faults; the decode kernel handles at most 512", maxdeg);
}

// Storage-precision dispatch of the compressed kernel (all jobs share it).
int launch_jobs_dtype(relaybp_handle *const *hs, const JobIO *io, int n, Scratch &sc, cudaStream_t st,
                      bool on_chip_only = false)
{
    switch (hs[0]->params.msg_dtype) {
    case RELAYBP_MSG_F64: return launch_jobs_geom<double>(hs, io, n, sc, st, on_chip_only);
    case RELAYBP_MSG_F16: return launch_jobs_geom<__half>(hs, io, n, sc, st, on_chip_only);
    case RELAYBP_MSG_BF16: return launch_jobs_geom<__nv_bfloat16>(hs, io, n, sc, st, on_chip_only);
    case RELAYBP_MSG_I8: return launch_jobs_geom<int8_t>(hs, io, n, sc, st, on_chip_only);
    default: return launch_jobs_geom<float>(hs, io, n, sc, st, on_chip_only);
    }
}

// ---- two-shot lockstep kernel (FP32) -----------------------------------------
// Row slots per lane of the instantiated kernels; a DEM uses the smallest that
// covers its longest row (4 lanes per row).
constexpr int kPairNB[] = {4, 8, 12, 16, 23, 27};

PairPlan make_pair_plan(const DevDEM &g)
{
    PairPlan s{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 15) & ~size_t(15);
        size_t at = off;
        off += bytes;
        return (int)at;
    };
    s.ehat = take(2 * 4 * (size_t)words(g.V));
    s.best = take(2 * 4 * (size_t)words(g.V));
    s.res = take(2 * 4 * (size_t)words(g.C));
    s.syn = take(2 * 4 * (size_t)words(g.C));
    s.obsacc = take(2 * 4 * (size_t)std::max(1, words(g.K)));
    // MM at X, SG at 2X (X >= the minima's size, a multiple of 16)
    const size_t X = (std::max(off, (size_t)(g.C + 1) * 16) + 15) & ~size_t(15);
    s.MM = (int)X;
    s.SG = (int)(2 * X);
    off = 2 * X + (size_t)(g.C + 1) * 32;
    s.A2 = take(8 * ((size_t)g.V + 1));
    s.M2 = take(8 * (size_t)g.V);
    s.total = (int)((off + 15) & ~size_t(15));
    return s;
}

// Warps per block: the count in [16, the kernel's limit] with the least work
// on the busiest warp (row steps of 8 rows at NB slot pairs, column groups at
// their slots).
int pair_warps_heuristic(const relaybp_handle *h)
{
    const int steps = (h->dem.C + 7) / 8, groups = words(h->dem.V);
    const double grp_cost = 30.0 + 15.0 * (double)h->dem.E / std::max(1, h->dem.V);
    const int wmax = pair_max_threads(h->pair_nb) / 32;
    int best = wmax;
    double bw = 1e300;
    for (int w = wmax; w >= 16; --w) {
        const double work = ((steps + w - 1) / w) * 22.0 * h->pair_nb + ((groups + w - 1) / w) * grp_cost;
        if (work < bw * 0.999) { bw = work; best = w; }
    }
    return best;
}

// The pair kernel decodes single-DEM FP32 launches without per-edge learned
// weights whose two-shot state fits in shared memory; returns 1 otherwise.
template <int NB>
int launch_pair_nb(relaybp_handle *h, Scratch &sc, const JobIO &io, cudaStream_t st, int dyn)
{
    const DevDEM &g = h->dem;
    PairJob J{};
    J.g = g;
    J.p = dev_params(h->params);
    J.p.lknots = h->lknots;
    J.p.lK = h->lK;
    J.p.lwrow = h->lwrow;
    J.p.lT = h->lT;
    J.p.llegs = h->llegs;
    J.plan = make_pair_plan(g);
    J.rslot2 = h->rslot2;
    J.ecode2 = h->ecode2;
    J.goff2 = h->goff2;
    J.L0p = h->L0p;
    J.syn_in = io.syn;
    J.shot0 = io.shot0;
    J.shots = io.shots;
    J.corr_out = io.corr;
    J.pobs_out = io.pobs;
    J.stats_out = io.stats;
    J.trace = io.trace;
    J.trace_iters = io.trace_iters;
    J.times_out = io.times;
    J.flag = io.flag;
    J.tail = io.tail;
    const int warps = std::min(h->pair_warps > 0 ? h->pair_warps : pair_warps_heuristic(h),
                               pair_max_threads(NB) / 32);
    const int threads = 32 * warps;
    auto kern = io.trace ? relay_pair_kernel<NB, true> : relay_pair_kernel<NB, false>;
    CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    int per_sm = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, dyn));
    if (per_sm < 1) return 1;
    const int64_t blocks = std::min<int64_t>((int64_t)per_sm * h->num_sms, (io.shots + 1) / 2);
    const size_t gamma_need = (size_t)blocks * words(g.V) * 32 * sizeof(float2);
    if (int rc = scratch_reserve(sc, gamma_need, 0)) return rc;
    CUDA_TRY(cudaMemsetAsync(sc.work, 0, sizeof(unsigned long long), st));
    if (io.trace)
        relay_pair_kernel<NB, true><<<(unsigned)blocks, threads, dyn, st>>>(J, sc.work,
                                                                           static_cast<float2 *>(sc.gamma));
    else
        relay_pair_kernel<NB, false><<<(unsigned)blocks, threads, dyn, st>>>(J, sc.work,
                                                                            static_cast<float2 *>(sc.gamma));
    CUDA_TRY(cudaGetLastError());
    return 0;
}

int launch_pair(relaybp_handle *h, Scratch &sc, const JobIO &io, cudaStream_t st)
{
    if (h->pair_off || !h->rslot2 || h->params.msg_dtype != RELAYBP_MSG_F32 || h->lw) return 1;
    int maxsm = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    const PairPlan pl = make_pair_plan(h->dem);
    if (pl.total + 1024 > maxsm) return 1;
    switch (h->pair_nb) {
    case 4: return launch_pair_nb<4>(h, sc, io, st, pl.total);
    case 8: return launch_pair_nb<8>(h, sc, io, st, pl.total);
    case 12: return launch_pair_nb<12>(h, sc, io, st, pl.total);
    case 16: return launch_pair_nb<16>(h, sc, io, st, pl.total);
    case 23: return launch_pair_nb<23>(h, sc, io, st, pl.total);
    case 27: return launch_pair_nb<27>(h, sc, io, st, pl.total);
    default: return 1;
    }
}

// Single-DEM decode: the literal-order FP64 kernel when it applies, the
// two-shot FP32 kernel when it applies, else one job of the general kernel.
// Cluster (latency) kernel: NB = row slots per lane (32 lanes per row).
constexpr int kClusterNB[] = {2, 4, 6, 8, 12, 16};     // slots per lane, 16 lanes per row

template <typename S, int NB>
int launch_cluster_nb(relaybp_handle *h, Scratch &sc, const ClusterJob &job, cudaStream_t st)
{
    auto kern = relay_cluster_kernel<S, NB>;
    CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, job.plan.total));
    if (job.nc > 8) CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)job.nc;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = (size_t)job.plan.total;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (h->cl_clusters == 0) {
        cfg.gridDim = dim3((unsigned)job.nc);
        int n = 0;
        CUDA_TRY(cudaOccupancyMaxActiveClusters(&n, kern, &cfg));
        if (n < 1) return fail(RELAYBP_ERR_UNSUPPORTED, "no cluster of %d CTAs with %d bytes of shared memory fits",
                               job.nc, job.plan.total);
        h->cl_clusters = n;
    }
    const int64_t clusters = std::min<int64_t>(h->cl_clusters, job.shots);
    cfg.gridDim = dim3((unsigned)(clusters * job.nc));
    if (int rc = scratch_reserve(sc, 0, 0)) return rc;
    CUDA_TRY(cudaMemsetAsync(sc.work, 0, sizeof(unsigned long long), st));
    CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, job, sc.work));
    CUDA_TRY(cudaGetLastError());
    return 0;
}

template <typename S>
int launch_cluster_s(relaybp_handle *h, Scratch &sc, const ClusterJob &job, cudaStream_t st)
{
    switch (h->cl_nb) {
    case 2: return launch_cluster_nb<S, 2>(h, sc, job, st);
    case 4: return launch_cluster_nb<S, 4>(h, sc, job, st);
    case 6: return launch_cluster_nb<S, 6>(h, sc, job, st);
    case 8: return launch_cluster_nb<S, 8>(h, sc, job, st);
    case 12: return launch_cluster_nb<S, 12>(h, sc, job, st);
    case 16: return launch_cluster_nb<S, 16>(h, sc, job, st);
    default: return fail(RELAYBP_ERR_UNSUPPORTED, "cluster kernel: %d row slots per lane", h->cl_nb);
    }
}

int launch_cluster(relaybp_handle *h, Scratch &sc, const JobIO &io, cudaStream_t st)
{
    ClusterJob job = h->cl;
    job.g = h->dem;
    job.p = dev_params(h->params);
    job.syn_in = io.syn;
    job.shot0 = io.shot0;
    job.shots = io.shots;
    job.corr_out = io.corr;
    job.pobs_out = io.pobs;
    job.stats_out = io.stats;
    job.times_out = io.times;
    if (io.tail.count) {                                // resume the handed-over shots
        job.tail = io.tail;
        job.shots = io.tail.max;
    }
    job.p.qscale = h->params.int8_scale > 0.0f ? h->params.int8_scale : (float)(h->l0max / 24.0);
    int rc;
    switch (h->params.msg_dtype) {
    case RELAYBP_MSG_F32: rc = launch_cluster_s<float>(h, sc, job, st); break;
    case RELAYBP_MSG_F16: rc = launch_cluster_s<__half>(h, sc, job, st); break;
    case RELAYBP_MSG_BF16: rc = launch_cluster_s<__nv_bfloat16>(h, sc, job, st); break;
    case RELAYBP_MSG_I8: rc = launch_cluster_s<int8_t>(h, sc, job, st); break;
    default: return fail(RELAYBP_ERR_UNSUPPORTED, "cluster kernel: storage form %d", h->params.msg_dtype);
    }
    if (rc == 0) h->launches += 1;
    return rc;
}

// Tail offload applies to plain legs of decodes without traces, flagged
// posteriors or message carry-over (a handed-over shot keeps its start time:
// the cluster kernel writes both times of a timed decode).
bool tail_applies(const relaybp_handle *h, const JobIO &io)
{
    if (h->cl_mode != 2 || io.trace || io.flag.post || h->params.carry_messages || h->lw ||
        h->params.msg_dtype == RELAYBP_MSG_F64)
        return false;
    if ((h->lknots || h->lwrow) && (h->llegs < 0 || h->tail_legs < h->llegs)) return false;
    return true;
}

int decode_single(relaybp_handle *h, Scratch &sc, const JobIO &io, cudaStream_t st, bool on_chip_only)
{
    if (h->cl_mode == 1 && !h->lw && !h->lknots && !h->lwrow && !io.trace && !io.flag.post)
        return launch_cluster(h, sc, io, st);
    if (h->params.msg_dtype == RELAYBP_MSG_F64 && !h->lw && !h->lknots && !h->lwrow && !io.times) {
        int rc = launch_decode_exact(h, sc, io, st);
        if (rc <= 0) return rc;
    }
    {
        JobIO io2 = io;
        const bool tail = tail_applies(h, io);
        if (tail) {
            CUDA_TRY(cudaMemsetAsync(h->tail_count, 0, sizeof(unsigned int), st));
            io2.tail = TailOut{h->tail_rec, h->tail_M, h->tail_best, h->tail_count, h->tail_max, h->tail_legs};
        }
        int rc = launch_pair(h, sc, io2, st);
        if (rc > 0) {
            rc = launch_jobs_dtype(&h, &io2, 1, sc, st, on_chip_only);
            if (rc > 0) rc = fail(RELAYBP_ERR_UNSUPPORTED, "no decode kernel for this handle");
        }
        if (rc == 0) {
            h->launches += 1;
            if (tail) rc = launch_cluster(h, sc, io2, st);         // the handed-over shots, same stream
        }
        return rc;
    }
}

// ---- learned form ----------------------------------------------------------
template <typename T>
TapePlan tape_plan(const DevDEM &g, int L)
{
    TapePlan tp{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 15) & ~size_t(15);
        size_t at = off;
        off += bytes;
        return (int)at;
    };
    tp.rows = take(sizeof(TapeRow<T>) * (size_t)g.C);
    tp.sgn = take(2 * (size_t)g.C * (size_t)L);
    tp.M = take(sizeof(T) * (size_t)g.V);
    tp.iter = (int)((off + 15) & ~size_t(15));
    return tp;
}

template <typename T>
LearnedSmem learned_smem(const DevDEM &g, int L, bool backward)
{
    LearnedSmem sp{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 15) & ~size_t(15);
        size_t at = off;
        off += bytes;
        return (int)at;
    };
    sp.a = take(sizeof(T) * (size_t)g.V);
    sp.b = take(sizeof(T) * (size_t)g.V);
    sp.c = take(sizeof(T) * (size_t)g.V);
    sp.d = backward ? take(sizeof(T) * (size_t)g.V) : 0;
    sp.rows = take((backward ? sizeof(BackRow<T>) : sizeof(TapeRow<T>)) * (size_t)g.C);
    sp.sgn = backward ? 0 : take(2 * (size_t)g.C * (size_t)L);
    sp.syn = take(4 * (size_t)words(g.C));
    sp.srow = backward ? take(sizeof(SoftRow<T>) * (size_t)g.C) : 0;
    sp.total = (int)((off + 15) & ~size_t(15));
    return sp;
}

struct LearnedCall {
    int precision, T, K, objective;
    const void *w, *knots;
    uint64_t gamma_seed;
    const uint32_t *syn, *err;
    uint64_t shot0;
    int64_t shots;
    void *tape;
    double *loss;
    double scale;
    void *grad_w, *grad_knots;
};

template <typename T, int L, int NB>
int learned_launch(relaybp_handle *h, const LearnedCall &c, bool backward, cudaStream_t st)
{
    const DevDEM &g = h->dem;
    LearnedSmem sp = learned_smem<T>(g, L, backward);
    int maxsm = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    if (sp.total + 1024 > maxsm)
        return fail(RELAYBP_ERR_UNSUPPORTED, "learned %s state (%d bytes) exceeds shared memory (%d bytes)",
                    backward ? "backward" : "forward", sp.total, maxsm);
    LearnedDev a{};
    a.g = g;
    a.T = c.T;
    a.K = c.K;
    a.objective = c.objective;
    a.w = c.w;
    a.knots = c.knots;
    a.gamma_seed = c.gamma_seed;
    a.syn = c.syn;
    a.err = c.err;
    a.shot0 = c.shot0;
    a.shots = c.shots;
    a.tape = static_cast<unsigned char *>(c.tape);
    a.tp = tape_plan<T>(g, L);
    a.loss = c.loss;
    a.cedge_ell = g.cedge_ell;
    const int threads = 512;
    int per_sm = 0;
    if (!backward) {
        auto kern = learned_forward_kernel<T, L, NB>;
        CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sp.total));
        CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, sp.total));
    } else {
        auto kern = learned_backward_kernel<T, L, NB>;
        CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sp.total));
        CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, sp.total));
    }
    if (per_sm < 1) return fail(RELAYBP_ERR_UNSUPPORTED, "learned kernel cannot be resident");
    const int64_t blocks = std::min<int64_t>((int64_t)per_sm * h->num_sms, c.shots);
    if (!h->d_lwork) CUDA_TRY(cudaMalloc(&h->d_lwork, 256));
    CUDA_TRY(cudaMemsetAsync(h->d_lwork, 0, sizeof(unsigned long long), st));
    if (!backward) {
        learned_forward_kernel<T, L, NB><<<(unsigned)blocks, threads, sp.total, st>>>(a, sp, h->d_lwork);
    } else {
        const size_t need = (size_t)blocks * g.V * sizeof(T);
        if (h->lgbar_bytes < need) {
            cudaFree(h->d_lgbar);
            h->d_lgbar = nullptr;
            h->lgbar_bytes = 0;
            CUDA_TRY(cudaMalloc(&h->d_lgbar, need));
            h->lgbar_bytes = need;
        }
        learned_backward_kernel<T, L, NB><<<(unsigned)blocks, threads, sp.total, st>>>(
            a, sp, h->d_lwork, (T)c.scale, static_cast<T *>(c.grad_w), static_cast<T *>(c.grad_knots),
            static_cast<T *>(h->d_lgbar));
    }
    CUDA_TRY(cudaGetLastError());
    h->launches += 1;
    return 0;
}

template <typename T>
int learned_dispatch(relaybp_handle *h, const LearnedCall &c, bool backward, cudaStream_t st)
{
    const RowGeom rg = row_geom(h->max_row_deg);
#define RELAYBP_LGEOM(LL, NN) \
    if (rg.L == LL && rg.NB == NN) return learned_launch<T, LL, NN>(h, c, backward, st);
    RELAYBP_LGEOM(4, 4)
    RELAYBP_LGEOM(8, 4)
    RELAYBP_LGEOM(8, 8)
    RELAYBP_LGEOM(8, 12)
    RELAYBP_LGEOM(8, 16)
    RELAYBP_LGEOM(16, 16)
    RELAYBP_LGEOM(32, 16)
#undef RELAYBP_LGEOM
    return fail(RELAYBP_ERR_UNSUPPORTED, "a detector touches %d faults (limit 512)", h->max_row_deg);
}

int learned_check(relaybp_handle *h, const LearnedCall &c, bool backward)
{
    if (!h) return fail(RELAYBP_ERR_INVALID, "handle is NULL");
    if (int rc = check_device(h)) return rc;
    if (c.precision != RELAYBP_MSG_F32 && c.precision != RELAYBP_MSG_F64)
        return fail(RELAYBP_ERR_UNSUPPORTED, "learned training runs in FP32 or FP64");
    if (c.T < 1 || c.K < 1 || c.K > 64) return fail(RELAYBP_ERR_INVALID, "need T >= 1 and 1 <= K <= 64");
    if (c.objective != 0 && c.objective != 1) return fail(RELAYBP_ERR_INVALID, "objective must be 0 or 1");
    if (backward && c.objective == 1 && !c.syn)
        return fail(RELAYBP_ERR_INVALID, "the soft-syndrome objective needs the syndromes");
    if (c.shots < 0) return fail(RELAYBP_ERR_INVALID, "negative shot count");
    if (!c.w || !c.knots || !c.err || !c.tape) return fail(RELAYBP_ERR_INVALID, "null pointer");
    if (!backward && (!c.syn || !c.loss)) return fail(RELAYBP_ERR_INVALID, "null pointer");
    if (backward && (!c.grad_w || !c.grad_knots)) return fail(RELAYBP_ERR_INVALID, "null pointer");
    return 0;
}

}  // namespace

extern "C" {

int64_t relaybp_learned_tape_bytes(const relaybp_handle *h, int32_t precision, int32_t T, int64_t shots)
{
    if (!h || T < 1 || shots < 0) return -1;
    const RowGeom rg = row_geom(h->max_row_deg);
    if (rg.L == 0) return -1;
    const TapePlan tp = precision == RELAYBP_MSG_F64 ? tape_plan<double>(h->dem, rg.L) : tape_plan<float>(h->dem, rg.L);
    return (int64_t)tp.iter * T * shots;
}

int relaybp_learned_forward(relaybp_handle *h, int32_t precision, int32_t T, const void *d_w, int32_t K,
                            const void *d_knots, uint64_t gamma_seed, int32_t objective,
                            const uint32_t *d_syndromes, const uint32_t *d_errors, uint64_t shot0, int64_t shots,
                            void *d_tape, double *d_loss, void *cuda_stream)
{
    g_err.clear();
    LearnedCall c{precision, T, K, objective, d_w, d_knots, gamma_seed, d_syndromes, d_errors, shot0, shots, d_tape,
                  d_loss, 0.0, nullptr, nullptr};
    if (int rc = learned_check(h, c, false)) return rc;
    if (shots == 0) return 0;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    return precision == RELAYBP_MSG_F64 ? learned_dispatch<double>(h, c, false, st)
                                        : learned_dispatch<float>(h, c, false, st);
}

int relaybp_learned_backward(relaybp_handle *h, int32_t precision, int32_t T, const void *d_w, int32_t K,
                             const void *d_knots, uint64_t gamma_seed, int32_t objective,
                             const uint32_t *d_syndromes, const uint32_t *d_errors, uint64_t shot0, int64_t shots,
                             const void *d_tape, double scale, void *d_grad_w, void *d_grad_knots,
                             void *cuda_stream)
{
    g_err.clear();
    LearnedCall c{precision, T, K, objective, d_w, d_knots, gamma_seed, d_syndromes, d_errors, shot0, shots,
                  const_cast<void *>(d_tape), nullptr, scale, d_grad_w, d_grad_knots};
    if (int rc = learned_check(h, c, true)) return rc;
    if (shots == 0) return 0;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    return precision == RELAYBP_MSG_F64 ? learned_dispatch<double>(h, c, true, st)
                                        : learned_dispatch<float>(h, c, true, st);
}


const char *relaybp_last_error(void) { return g_err.c_str(); }

int relaybp_build(const relaybp_csr *H, const double *priors, const relaybp_csr *obs, const relaybp_params *params,
                  relaybp_handle **out)
{
    g_err.clear();
    if (!out) return fail(RELAYBP_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (int rc = check_csr(H, "H")) return rc;
    if (!priors) return fail(RELAYBP_ERR_INVALID, "priors is NULL");
    if (obs) {
        if (int rc = check_csr(obs, "obs")) return rc;
        if (obs->cols != H->cols) return fail(RELAYBP_ERR_INVALID, "obs has %d columns, H has %d", obs->cols, H->cols);
    }
    if (int rc = check_params(params)) return rc;
    if (int rc = check_legs(params, H->cols)) return rc;
    const int32_t C = H->rows, V = H->cols, K = obs ? obs->rows : 0;
    const int64_t E = H->indptr[C];
    if (C >= (1 << 20) || E >= (int64_t)1 << 30) return fail(RELAYBP_ERR_UNSUPPORTED, "DEM too large");
    double l0max = 0.0;                                 // largest |prior LLR| (automatic int8 step)
    for (int32_t j = 0; j < V; ++j) {
        if (!(priors[j] > 0.0 && priors[j] < 1.0))
            return fail(RELAYBP_ERR_INVALID, "prior %d = %g is not in (0, 1)", j, priors[j]);
        l0max = std::max(l0max, std::fabs(std::log((1.0 - priors[j]) / priors[j])));
    }
    if (int rc = check_int8_step(*params, l0max)) return rc;
    for (int32_t i = 0; i < C; ++i) {
        const int32_t deg = H->indptr[i + 1] - H->indptr[i];
        if (deg == 1)
            return fail(RELAYBP_ERR_INVALID, "detector %d is touched by a single fault; rows need 0 or >= 2 entries", i);
        if (deg > 4095) return fail(RELAYBP_ERR_UNSUPPORTED, "detector %d has %d entries (limit 4095)", i, deg);
    }

    relaybp_handle *h = new relaybp_handle();
    h->params = *params;
    auto bail = [&](int rc) {
        relaybp_destroy(h);
        return rc;
    };
    cudaError_t ce = cudaGetDevice(&h->device);
    if (ce != cudaSuccess) { delete h; return fail(RELAYBP_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(ce)); }
    ce = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (ce != cudaSuccess) { delete h; return fail(RELAYBP_ERR_CUDA, "SM count: %s", cudaGetErrorString(ce)); }

    // row order
    std::vector<int32_t> rptr(H->indptr, H->indptr + C + 1), rvar(H->indices, H->indices + E);
    // column order (ascending check within each column)
    std::vector<int32_t> cptr(V + 1, 0), cchk(E), cedge(E), fill(V, 0);
    for (int64_t e = 0; e < E; ++e) cptr[rvar[e] + 1]++;
    for (int32_t j = 0; j < V; ++j) cptr[j + 1] += cptr[j];
    for (int32_t i = 0; i < C; ++i)
        for (int32_t e = rptr[i]; e < rptr[i + 1]; ++e) {
            int32_t j = rvar[e];
            int32_t at = cptr[j] + fill[j]++;
            cchk[at] = i;
            cedge[at] = e;
        }
    // sliced ELL of the columns: groups of 32 variables, slot-major, each entry
    // (check << 12 | position in row), padded with sentinels
    const int32_t NG = (V + 31) / 32;
    std::vector<int32_t> goff(NG + 1, 0), gdeg(NG, 0);
    for (int32_t G = 0; G < NG; ++G) {
        int32_t D = 0;
        for (int32_t j = G * 32; j < std::min(V, G * 32 + 32); ++j) D = std::max(D, cptr[j + 1] - cptr[j]);
        gdeg[G] = D;
        goff[G + 1] = goff[G] + D * 32;
    }
    std::vector<uint32_t> cinfo((size_t)goff[NG], COL_SENTINEL), cedge_ell((size_t)goff[NG], 0u);
    for (int32_t j = 0; j < V; ++j) {
        const int32_t G = j / 32, l = j % 32;
        for (int32_t k = 0; k < cptr[j + 1] - cptr[j]; ++k) {
            const int32_t i = cchk[cptr[j] + k];
            const int32_t pos = cedge[cptr[j] + k] - rptr[i];
            cinfo[(size_t)goff[G] + (size_t)k * 32 + l] = ((uint32_t)i << 12) | (uint32_t)pos;
            cedge_ell[(size_t)goff[G] + (size_t)k * 32 + l] = (uint32_t)cedge[cptr[j] + k];
        }
    }
    // branch-free layout of the decode kernel: padded rows (dummy variable V)
    // and column codes i << lg_rsp | position (dummy check C)
    int32_t maxdeg = 0;
    for (int32_t i = 0; i < C; ++i) maxdeg = std::max(maxdeg, rptr[i + 1] - rptr[i]);
    int32_t lg_rsp = 5;
    while ((1 << lg_rsp) < maxdeg) ++lg_rsp;
    std::vector<int32_t> rslot;
    std::vector<uint32_t> ecode((size_t)goff[NG], (uint32_t)C << lg_rsp);
    if (maxdeg <= kRowStride && ((uint64_t)C + 1) << lg_rsp <= 0xffffffffull) {
        const int32_t CP = (C + 31) / 32 * 32;
        rslot.assign((size_t)std::max(CP, 32) * kRowStride, V);
        for (int32_t i = 0; i < C; ++i)
            for (int32_t e = rptr[i]; e < rptr[i + 1]; ++e) rslot[(size_t)i * kRowStride + (e - rptr[i])] = rvar[e];
        for (int32_t j = 0; j < V; ++j) {
            const int32_t G = j / 32, l = j % 32;
            for (int32_t k = 0; k < cptr[j + 1] - cptr[j]; ++k) {
                const int32_t i = cchk[cptr[j] + k];
                const int32_t pos = cedge[cptr[j] + k] - rptr[i];
                ecode[(size_t)goff[G] + (size_t)k * 32 + l] = ((uint32_t)i << lg_rsp) | (uint32_t)pos;
            }
        }
    }
    // two-shot kernel: row slots (lane k % 4, slot k / 4 of row entry k) as
    // shared byte offsets of A2[j], and column codes (sign-word offset << 5 |
    // 32 - NB + slot); rows padded with the dummy variable V, columns with the
    // dummy row C
    int32_t pair_nb = 0;
    for (int nb : kPairNB)
        if (4 * nb >= maxdeg) { pair_nb = nb; break; }
    std::vector<uint32_t> rslot2, ecode2;
    std::vector<int32_t> goff2;
    std::vector<float> L0p;
    if (pair_nb > 0) {
        DevDEM tmp{};
        tmp.C = C; tmp.V = V; tmp.K = K; tmp.E = E;
        const PairPlan pl = make_pair_plan(tmp);
        const int32_t nbp = (pair_nb + 3) & ~3, CP8 = (C + 7) / 8 * 8;
        rslot2.assign((size_t)CP8 * kPairLanes * nbp, (uint32_t)pl.A2 + 8u * (uint32_t)V);
        for (int32_t i = 0; i < C; ++i)
            for (int32_t k = 0; k < rptr[i + 1] - rptr[i]; ++k)
                rslot2[((size_t)i * kPairLanes + k % kPairLanes) * nbp + k / kPairLanes] =
                    (uint32_t)pl.A2 + 8u * (uint32_t)rvar[rptr[i] + k];
        const uint32_t dummy = ((uint32_t)pl.SG + 32u * (uint32_t)C) << 5;
        goff2.assign(NG + 1, 0);
        for (int32_t G = 0; G < NG; ++G) goff2[G + 1] = goff2[G] + std::max(gdeg[G], 8) * 32;
        ecode2.assign((size_t)goff2[NG], dummy);
        L0p.assign((size_t)NG * 32, 0.f);
        for (int32_t j = 0; j < V; ++j) L0p[j] = (float)std::log((1.0 - priors[j]) / priors[j]);
        for (int32_t j = 0; j < V; ++j) {
            const int32_t G = j / 32, l = j % 32;
            for (int32_t k = 0; k < cptr[j + 1] - cptr[j]; ++k) {
                const int32_t i = cchk[cptr[j] + k];
                const int32_t pos = cedge[cptr[j] + k] - rptr[i];
                const uint32_t sg = (uint32_t)pl.SG + 32u * (uint32_t)i + 8u * (uint32_t)(pos % kPairLanes);
                ecode2[(size_t)goff2[G] + (size_t)k * 32 + l] = (sg << 5) | (uint32_t)(32 - pair_nb + pos / kPairLanes);
            }
        }
    }
    // observables per column
    std::vector<int32_t> optr(V + 1, 0), oidx;
    if (obs) {
        const int64_t nnzo = obs->indptr[K];
        oidx.resize(nnzo);
        std::vector<int32_t> of(V, 0);
        for (int64_t e = 0; e < nnzo; ++e) optr[obs->indices[e] + 1]++;
        for (int32_t j = 0; j < V; ++j) optr[j + 1] += optr[j];
        for (int32_t i = 0; i < K; ++i)
            for (int32_t e = obs->indptr[i]; e < obs->indptr[i + 1]; ++e) {
                int32_t j = obs->indices[e];
                oidx[optr[j] + of[j]++] = i;
            }
    }
    // a1: prior LLRs in FP64 on the host; sampler thresholds
    std::vector<double> L0d(V);
    std::vector<float> L0f(V);
    std::vector<uint32_t> thr(V);
    for (int32_t j = 0; j < V; ++j) {
        L0d[j] = std::log((1.0 - priors[j]) / priors[j]);
        L0f[j] = (float)L0d[j];
        double t = std::floor(priors[j] * 4294967296.0);
        thr[j] = t >= 4294967295.0 ? 0xffffffffu : (uint32_t)t;
    }
    for (int32_t i = 0; i < C; ++i) h->max_row_deg = std::max(h->max_row_deg, rptr[i + 1] - rptr[i]);
    h->l0max = l0max;
    DevDEM &g = h->dem;
    g.C = C; g.V = V; g.K = K; g.E = E;
    g.lg_rsp = lg_rsp;
    g.rw = 1 << (lg_rsp - 5);
    int rc = 0;
    if ((rc = upload(h, rptr, &g.rptr)) || (rc = upload(h, rvar, &g.rvar)) || 
        (rc = upload(h, cptr, &g.cptr)) || (rc = upload(h, cchk, &g.cchk)) || 
        (rc = upload(h, cedge, &g.cedge)) || (rc = upload(h, cinfo, &g.cinfo)) || (rc = upload(h, cedge_ell, &g.cedge_ell)) || (rc = upload(h, goff, &g.goff)) ||
        (rc = upload(h, gdeg, &g.gdeg)) || (rc = upload(h, ecode, &g.ecode)) ||
        (!rslot.empty() && (rc = upload(h, rslot, &g.rslot))) ||
        (rc = upload(h, optr, &g.optr)) || (rc = upload(h, oidx, &g.oidx)) || (rc = upload(h, L0d, &g.L0d)) ||
        (rc = upload(h, L0f, &g.L0f)) || (rc = upload(h, thr, &g.thr)))
        return bail(rc);
    if (pair_nb > 0) {
        if ((rc = upload(h, rslot2, &h->rslot2)) || (rc = upload(h, ecode2, &h->ecode2)) ||
            (rc = upload(h, goff2, &h->goff2)) || (rc = upload(h, L0p, &h->L0p)))
            return bail(rc);
        h->pair_nb = pair_nb;
        h->pair_off = 0;
    }
    if ((rc = scratch_reserve(h->scratch, 0, 0))) return bail(rc);
    *out = h;
    return 0;
}

int relaybp_set_params(relaybp_handle *h, const relaybp_params *params)
{
    g_err.clear();
    if (!h) return fail(RELAYBP_ERR_INVALID, "handle is NULL");
    if (int rc = check_params(params)) return rc;
    if (int rc = check_legs(params, h->dem.V)) return rc;
    if (int rc = check_int8_step(*params, h->l0max)) return rc;
    h->params = *params;
    return 0;
}

int relaybp_set_learned(relaybp_handle *h, const float *d_w, int32_t T, const float *d_knots, int32_t K)
{
    g_err.clear();
    if (!h) return fail(RELAYBP_ERR_INVALID, "handle is NULL");
    if ((d_w && T < 1) || (d_knots && (K < 1 || K > 64)))
        return fail(RELAYBP_ERR_INVALID, "need T >= 1 with weights and 1 <= K <= 64 with knots");
    if ((d_w || d_knots) && h->params.msg_dtype == RELAYBP_MSG_F64)
        return fail(RELAYBP_ERR_UNSUPPORTED, "learned decoding runs with FP32 arithmetic (msg_dtype F32/F16/BF16/I8)");
    if (d_w && h->params.carry_messages)
        return fail(RELAYBP_ERR_UNSUPPORTED, "learned weights with carry_messages are not supported");
    h->lw = d_w;
    h->lwrow = nullptr;
    h->lT = d_w ? T : 0;
    h->lknots = d_knots;
    h->lK = d_knots ? K : 0;
    return 0;
}

int relaybp_set_learned_rows(relaybp_handle *h, const float *d_wrow, int32_t T, const float *d_knots, int32_t K)
{
    g_err.clear();
    if (!h) return fail(RELAYBP_ERR_INVALID, "handle is NULL");
    if ((d_wrow && T < 1) || (d_knots && (K < 1 || K > 64)))
        return fail(RELAYBP_ERR_INVALID, "need T >= 1 with weights and 1 <= K <= 64 with knots");
    if ((d_wrow || d_knots) && h->params.msg_dtype == RELAYBP_MSG_F64)
        return fail(RELAYBP_ERR_UNSUPPORTED, "learned decoding runs with FP32 arithmetic (msg_dtype F32/F16/BF16/I8)");
    if (d_wrow && h->params.carry_messages)
        return fail(RELAYBP_ERR_UNSUPPORTED, "learned weights with carry_messages are not supported");
    h->lw = nullptr;
    h->lwrow = d_wrow;
    h->lT = d_wrow ? T : 0;
    h->lknots = d_knots;
    h->lK = d_knots ? K : 0;
    return 0;
}

int relaybp_set_cluster_kernel(relaybp_handle *h, int32_t cluster)
{
    g_err.clear();
    if (!h) return fail(RELAYBP_ERR_INVALID, "handle is NULL");
    if (cluster < 0 || cluster > 16) return fail(RELAYBP_ERR_INVALID, "cluster = %d; need 0 (off) or 1..16", cluster);
    if (int rc = check_device(h)) return rc;
    cudaFree(h->cl_rslot);
    cudaFree(h->cl_ecode);
    cudaFree(h->cl_halo[0]);
    cudaFree(h->cl_halo[1]);
    h->cl_rslot = nullptr;
    h->cl_ecode = h->cl_halo[0] = h->cl_halo[1] = nullptr;
    h->cl_nc = h->cl_nb = h->cl_clusters = h->cl_mode = 0;
    if (cluster == 0) return 0;
    if (h->params.msg_dtype == RELAYBP_MSG_F64)
        return fail(RELAYBP_ERR_UNSUPPORTED, "the cluster kernel stores FP32, FP16, BF16 or int8 (not FP64)");
    const int es = h->params.msg_dtype == RELAYBP_MSG_F32 ? 4 : (h->params.msg_dtype == RELAYBP_MSG_I8 ? 1 : 2);
    const int css = h->params.msg_dtype == RELAYBP_MSG_F32 ? 16 : 8;     // sizeof(CheckState<S>)
    const DevDEM &g = h->dem;
    const int32_t C = g.C, V = g.V, NG = (V + 31) / 32, lg = g.lg_rsp;
    int nb = 0;
    for (int x : kClusterNB)
        if (16 * x >= h->max_row_deg) { nb = x; break; }
    if (!nb) return fail(RELAYBP_ERR_UNSUPPORTED, "rows of %d entries exceed the cluster kernel's 256", h->max_row_deg);
    if (!g.rslot) return fail(RELAYBP_ERR_UNSUPPORTED, "the DEM has no row-slot layout");
    const int32_t nc = cluster;
    const int32_t Cc = (C + nc - 1) / nc;
    int32_t lgcs = 1;
    while ((1 << lgcs) < Cc) ++lgcs;
    const int32_t NGc = (NG + nc - 1) / nc, Vc = NGc * 32;
    int32_t lgv = 1;
    while ((1 << lgv) < Vc) ++lgv;
    if (lgv + 4 > 32 || lgcs + 4 > 32) return fail(RELAYBP_ERR_UNSUPPORTED, "cluster codes do not fit 32 bits");
    // host copies of the row lists and the sliced-ELL column codes
    std::vector<int32_t> rptr(C + 1), rvar(g.E), goff(NG), gdeg(NG);
    CUDA_TRY(cudaMemcpy(rptr.data(), g.rptr, (C + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(rvar.data(), g.rvar, g.E * sizeof(int32_t), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(goff.data(), g.goff, NG * sizeof(int32_t), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(gdeg.data(), g.gdeg, NG * sizeof(int32_t), cudaMemcpyDeviceToHost));
    const size_t nell = (size_t)goff[NG - 1] + (size_t)gdeg[NG - 1] * 32;
    std::vector<uint32_t> ecode(nell);
    CUDA_TRY(cudaMemcpy(ecode.data(), g.ecode, nell * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    const int32_t CPc = (Cc + 1 + 31) / 32 * 32;      // rows per CTA in the row-slot table (dummy rows after)
    const uint32_t pmask = (1u << lg) - 1u;
    // per CTA: the A halo (variables its rows touch) and the row halo (rows
    // its variables touch), both ascending -- hence sorted by owner, then by
    // the owner's local index
    std::vector<int32_t> rs((size_t)nc * CPc * kRowStride, 0);
    std::vector<uint32_t> ec(nell, 0), ahs, rhs;
    ClusterJob &J = h->cl;
    J = ClusterJob{};
    int HAmax = 0, HRmax = 0;
    std::vector<int32_t> hidx(std::max(V, C), -1);
    for (int32_t c = 0; c < nc; ++c) {
        const int32_t i0 = std::min(C, c * Cc), i1 = std::min(C, (c + 1) * Cc);
        std::vector<int32_t> cols;
        for (int32_t i = i0; i < i1; ++i) cols.insert(cols.end(), rvar.begin() + rptr[i], rvar.begin() + rptr[i + 1]);
        std::sort(cols.begin(), cols.end());
        cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
        const int HA = (int)cols.size();
        J.ha_off[c] = (int)ahs.size();
        J.ha_cnt[c] = HA;
        for (int k = 0; k < HA; ++k) {
            const int32_t j = cols[k], oc = (j / 32) / NGc;
            hidx[j] = k;
            ahs.push_back(((uint32_t)oc << lgv) | (uint32_t)(j - oc * Vc));
        }
        for (int32_t r = 0; r < CPc; ++r) {
            const int32_t i = i0 + r;
            const int32_t deg = (i < i1) ? rptr[i + 1] - rptr[i] : 0;
            for (int32_t k = 0; k < kRowStride; ++k)
                rs[((size_t)c * CPc + r) * kRowStride + k] = (k < deg) ? hidx[rvar[rptr[i] + k]] : HA;
        }
        for (int32_t j : cols) hidx[j] = -1;
        const int32_t G0 = std::min(NG, c * NGc), G1 = std::min(NG, (c + 1) * NGc);
        std::vector<int32_t> rows;
        for (int32_t G = G0; G < G1; ++G)
            for (size_t x = (size_t)goff[G]; x < (size_t)goff[G] + (size_t)gdeg[G] * 32; ++x)
                if ((ecode[x] >> lg) < (uint32_t)C) rows.push_back((int32_t)(ecode[x] >> lg));
        std::sort(rows.begin(), rows.end());
        rows.erase(std::unique(rows.begin(), rows.end()), rows.end());
        const int HR = (int)rows.size();
        J.hr_off[c] = (int)rhs.size();
        J.hr_cnt[c] = HR;
        for (int k = 0; k < HR; ++k) {
            hidx[rows[k]] = k;
            rhs.push_back(((uint32_t)(rows[k] / Cc) << lgcs) | (uint32_t)(rows[k] % Cc));
        }
        for (int32_t G = G0; G < G1; ++G)
            for (size_t x = (size_t)goff[G]; x < (size_t)goff[G] + (size_t)gdeg[G] * 32; ++x) {
                const uint32_t i = ecode[x] >> lg;
                ec[x] = (i < (uint32_t)C) ? ((uint32_t)hidx[i] << lg) | (ecode[x] & pmask) : (uint32_t)HR << lg;
            }
        for (int32_t i : rows) hidx[i] = -1;
        if (((uint64_t)HR + 1) << lg > 0xffffffffull)
            return fail(RELAYBP_ERR_UNSUPPORTED, "cluster codes do not fit 32 bits");
        HAmax = std::max(HAmax, HA);
        HRmax = std::max(HRmax, HR);
    }
    const int RWd = g.rw;
    ClusterPlan pl{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 15) & ~size_t(15);
        const size_t at = off;
        off += bytes;
        return (int)at;
    };
    pl.A = take(es * (size_t)Vc);
    pl.M = take(es * (size_t)Vc);
    pl.gam = take(4 * (size_t)Vc);
    pl.Ah = take(es * (size_t)(HAmax + 1));
    pl.cs0 = take(css * (size_t)(Cc + 1));
    pl.cs1 = take(css * (size_t)(Cc + 1));
    pl.sg0 = take(4 * (size_t)(Cc + 1) * RWd);
    pl.sg1 = take(4 * (size_t)(Cc + 1) * RWd);
    pl.csh = take(css * (size_t)(HRmax + 1));
    pl.sgh = take(4 * (size_t)(HRmax + 1) * RWd);
    pl.ahs = take(4 * (size_t)HAmax);
    pl.rhs = take(4 * (size_t)HRmax);
    pl.ehat = take(4 * (size_t)NGc);
    pl.best = take(4 * (size_t)NGc);
    pl.res = take(4 * (size_t)((Cc + 31) / 32));
    pl.syn = take(4 * (size_t)((Cc + 31) / 32));
    pl.lst = take(4 * (size_t)Vc);
    pl.obsacc = take(4 * (size_t)std::max(1, (g.K + 31) / 32));
    pl.flags = take(4 * 32);
    pl.total = (int)((off + 15) & ~size_t(15));
    int maxsm = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    if (pl.total + 64 > maxsm)
        return fail(RELAYBP_ERR_UNSUPPORTED, "cluster of %d: %d bytes of shared memory per CTA (limit %d)", nc,
                    pl.total, maxsm);
    uint32_t *d_ahs = nullptr, *d_rhs = nullptr;
    CUDA_TRY(cudaMalloc(&h->cl_rslot, rs.size() * 4));
    CUDA_TRY(cudaMemcpy(h->cl_rslot, rs.data(), rs.size() * 4, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMalloc(&h->cl_ecode, ec.size() * 4));
    CUDA_TRY(cudaMemcpy(h->cl_ecode, ec.data(), ec.size() * 4, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMalloc(&d_ahs, std::max<size_t>(1, ahs.size()) * 4));
    h->cl_halo[0] = d_ahs;
    CUDA_TRY(cudaMemcpy(d_ahs, ahs.data(), ahs.size() * 4, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMalloc(&d_rhs, std::max<size_t>(1, rhs.size()) * 4));
    h->cl_halo[1] = d_rhs;
    CUDA_TRY(cudaMemcpy(d_rhs, rhs.data(), rhs.size() * 4, cudaMemcpyHostToDevice));
    J.plan = pl;
    J.rslot = h->cl_rslot;
    J.ecode = h->cl_ecode;
    J.ahs = d_ahs;
    J.rhs = d_rhs;
    J.nc = nc; J.Cc = Cc; J.CPc = CPc; J.lgcs = lgcs; J.NGc = NGc; J.Vc = Vc; J.lgv = lgv;
    h->cl_nc = nc;
    h->cl_nb = nb;
    h->cl_mode = 1;
    return 0;
}

int relaybp_set_tail_offload(relaybp_handle *h, int32_t legs, int32_t cluster, int64_t max_shots)
{
    g_err.clear();
    if (!h) return fail(RELAYBP_ERR_INVALID, "handle is NULL");
    if (legs < 0 || max_shots < 0) return fail(RELAYBP_ERR_INVALID, "legs and max_shots must be >= 0");
    if (int rc = check_device(h)) return rc;
    if (legs == 0) {                                    // off; the cluster layout stays for later use
        if (h->cl_mode == 2) h->cl_mode = 0;
        return 0;
    }
    if (h->params.carry_messages)
        return fail(RELAYBP_ERR_UNSUPPORTED, "tail offload restarts messages at a leg boundary (no carry-over)");
    if (h->params.msg_dtype == RELAYBP_MSG_F64)
        return fail(RELAYBP_ERR_UNSUPPORTED, "tail offload continues shots in the cluster kernel (not FP64)");
    if (h->cl_nc != cluster || h->cl_mode == 0) {
        if (int rc = relaybp_set_cluster_kernel(h, cluster)) return rc;
    }
    const long long mx = max_shots > 0 ? max_shots : 256;
    if (mx != h->tail_max) {
        cudaFree(h->tail_rec);
        cudaFree(h->tail_M);
        cudaFree(h->tail_best);
        h->tail_rec = nullptr;
        h->tail_M = nullptr;
        h->tail_best = nullptr;
        h->tail_max = 0;
        CUDA_TRY(cudaMalloc(&h->tail_rec, (size_t)mx * sizeof(TailRec)));
        CUDA_TRY(cudaMalloc(&h->tail_M, (size_t)mx * h->dem.V * sizeof(float)));
        CUDA_TRY(cudaMalloc(&h->tail_best, (size_t)mx * words(h->dem.V) * sizeof(uint32_t)));
        h->tail_max = mx;
    }
    if (!h->tail_count) CUDA_TRY(cudaMalloc(&h->tail_count, sizeof(unsigned int)));
    h->tail_legs = legs;
    h->cl_mode = 2;
    return 0;
}

int relaybp_set_pair_kernel(relaybp_handle *h, int32_t enable, int32_t warps)
{
    g_err.clear();
    if (!h) return fail(RELAYBP_ERR_INVALID, "handle is NULL");
    if (warps != 0 && (warps < 1 || warps > 32)) return fail(RELAYBP_ERR_INVALID, "warps must be 0 or 1..32");
    if (enable && !h->rslot2)
        return fail(RELAYBP_ERR_UNSUPPORTED, "rows of %d entries exceed the two-shot kernel's %d", h->max_row_deg,
                    kPairLanes * kPairNB[sizeof(kPairNB) / sizeof(kPairNB[0]) - 1]);
    h->pair_off = enable ? 0 : 1;
    h->pair_warps = warps;
    return 0;
}

int relaybp_set_learned_legs(relaybp_handle *h, int32_t legs)
{
    g_err.clear();
    if (!h) return fail(RELAYBP_ERR_INVALID, "handle is NULL");
    if (legs < -1) return fail(RELAYBP_ERR_INVALID, "learned legs must be >= -1");
    h->llegs = legs;
    return 0;
}

int relaybp_sizes(const relaybp_handle *h, int32_t *n_det, int32_t *n_loc, int32_t *n_obs, int64_t *n_edges)
{
    if (!h) return fail(RELAYBP_ERR_INVALID, "handle is NULL");
    if (n_det) *n_det = h->dem.C;
    if (n_loc) *n_loc = h->dem.V;
    if (n_obs) *n_obs = h->dem.K;
    if (n_edges) *n_edges = h->dem.E;
    return 0;
}

int relaybp_sample(relaybp_handle *h, uint64_t seed, uint64_t shot0, int64_t shots, uint32_t *d_syndromes,
                   uint32_t *d_obs, uint32_t *d_errors, void *cuda_stream)
{
    g_err.clear();
    if (!h) return fail(RELAYBP_ERR_INVALID, "handle is NULL");
    if (int rc = check_device(h)) return rc;
    if (shots < 0) return fail(RELAYBP_ERR_INVALID, "negative shot count");
    if (shots == 0) return 0;
    if (!d_syndromes) return fail(RELAYBP_ERR_INVALID, "d_syndromes is NULL");
    const DevDEM &g = h->dem;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int per_warp = words(g.C) + words(g.K) + (d_errors ? words(g.V) : 0);
    int maxsm = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    int warps = 8;
    while (warps > 1 && (size_t)warps * per_warp * 4 > (size_t)maxsm) warps /= 2;
    const size_t smem = (size_t)warps * per_warp * 4;
    if (smem > (size_t)maxsm) return fail(RELAYBP_ERR_UNSUPPORTED, "sampler state exceeds shared memory");
    CUDA_TRY(cudaFuncSetAttribute(sample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sample_kernel, warps * 32, smem));
    int64_t blocks = (int64_t)std::max(1, per_sm) * h->num_sms;
    const int64_t need = (shots + warps - 1) / warps;
    if (blocks > need) blocks = need;
    sample_kernel<<<(unsigned)blocks, warps * 32, smem, st>>>(g, seed, shot0, shots, d_syndromes, d_obs, d_errors);
    CUDA_TRY(cudaGetLastError());
    h->launches += 1;
    return 0;
}

int relaybp_decode_batch(relaybp_handle *h, const uint32_t *d_syndromes, uint64_t shot0, int64_t shots,
                         uint32_t *d_corrections, uint32_t *d_pred_obs, relaybp_shot_stats *d_stats,
                         void *cuda_stream)
{
    g_err.clear();
    if (!h) return fail(RELAYBP_ERR_INVALID, "handle is NULL");
    if (int rc = check_device(h)) return rc;
    if (shots < 0) return fail(RELAYBP_ERR_INVALID, "negative shot count");
    if (shots == 0) return 0;
    if (!d_syndromes) return fail(RELAYBP_ERR_INVALID, "d_syndromes is NULL");
    static_assert(sizeof(StatsDev) == sizeof(relaybp_shot_stats), "stats layout");
    const JobIO io{d_syndromes, shot0, shots, d_corrections, d_pred_obs, reinterpret_cast<StatsDev *>(d_stats),
                   nullptr, 0};
    return decode_single(h, h->scratch, io, static_cast<cudaStream_t>(cuda_stream), false);
}

int relaybp_decode_timed(relaybp_handle *h, const uint32_t *d_syndromes, uint64_t shot0, int64_t shots,
                         uint32_t *d_corrections, uint32_t *d_pred_obs, relaybp_shot_stats *d_stats,
                         uint64_t *d_times, void *cuda_stream)
{
    g_err.clear();
    if (!h) return fail(RELAYBP_ERR_INVALID, "handle is NULL");
    if (int rc = check_device(h)) return rc;
    if (shots < 0) return fail(RELAYBP_ERR_INVALID, "negative shot count");
    if (shots == 0) return 0;
    if (!d_syndromes || !d_times) return fail(RELAYBP_ERR_INVALID, "null pointer");
    JobIO io{d_syndromes, shot0, shots, d_corrections, d_pred_obs, reinterpret_cast<StatsDev *>(d_stats), nullptr, 0};
    io.times = d_times;
    return decode_single(h, h->scratch, io, static_cast<cudaStream_t>(cuda_stream), false);
}

int relaybp_decode_trace(relaybp_handle *h, const uint32_t *d_syndromes, uint64_t shot0, int64_t shots,
                         int32_t trace_iters, double *d_trace, relaybp_shot_stats *d_stats, void *cuda_stream)
{
    g_err.clear();
    if (!h) return fail(RELAYBP_ERR_INVALID, "handle is NULL");
    if (int rc = check_device(h)) return rc;
    if (shots < 0 || trace_iters < 0) return fail(RELAYBP_ERR_INVALID, "negative size");
    if (shots == 0) return 0;
    if (!d_syndromes || (trace_iters > 0 && !d_trace)) return fail(RELAYBP_ERR_INVALID, "null pointer");
    const JobIO io{d_syndromes, shot0, shots, nullptr, nullptr, reinterpret_cast<StatsDev *>(d_stats), d_trace,
                   trace_iters};
    return decode_single(h, h->scratch, io, static_cast<cudaStream_t>(cuda_stream), false);
}

int relaybp_decode_flagged(relaybp_handle *h, const uint32_t *d_syndromes, uint64_t shot0, int64_t shots,
                           uint32_t *d_corrections, uint32_t *d_pred_obs, relaybp_shot_stats *d_stats,
                           int64_t max_flagged, int64_t *d_flag_idx, double *d_flag_post, uint32_t *d_flag_count,
                           void *cuda_stream)
{
    g_err.clear();
    if (!h) return fail(RELAYBP_ERR_INVALID, "handle is NULL");
    if (int rc = check_device(h)) return rc;
    if (shots < 0 || max_flagged < 0) return fail(RELAYBP_ERR_INVALID, "negative size");
    if (shots == 0) return 0;
    if (!d_syndromes || !d_flag_count || (max_flagged > 0 && (!d_flag_idx || !d_flag_post)))
        return fail(RELAYBP_ERR_INVALID, "null pointer");
    JobIO io{d_syndromes, shot0, shots, d_corrections, d_pred_obs, reinterpret_cast<StatsDev *>(d_stats), nullptr, 0};
    io.flag = FlagOut{reinterpret_cast<long long *>(d_flag_idx), d_flag_post, d_flag_count, max_flagged};
    return decode_single(h, h->scratch, io, static_cast<cudaStream_t>(cuda_stream), false);
}

int relaybp_osd(relaybp_handle *h, const uint32_t *d_syndromes, const double *d_post, const int64_t *d_idx, int64_t n,
                int32_t lambda, uint32_t *d_out_e, int32_t *d_out_valid, void *cuda_stream)
{
    g_err.clear();
    if (!h) return fail(RELAYBP_ERR_INVALID, "handle is NULL");
    if (int rc = check_device(h)) return rc;
    if (n < 0) return fail(RELAYBP_ERR_INVALID, "negative shot count");
    if (lambda < 0 || lambda > kOsdMaxLambda) return fail(RELAYBP_ERR_INVALID, "lambda must be in 0..%d", kOsdMaxLambda);
    if (n == 0) return 0;
    if (!d_syndromes || !d_post || !d_idx || !d_out_e || !d_out_valid) return fail(RELAYBP_ERR_INVALID, "null pointer");
    const DevDEM &g = h->dem;
    if (g.V > kOsdSortMax)
        return fail(RELAYBP_ERR_UNSUPPORTED, "OSD sorts at most %d columns in shared memory (DEM has %d)", kOsdSortMax,
                    g.V);
    int NP = 1;
    while (NP < g.V) NP <<= 1;
    const size_t WC = (size_t)words(g.C), WV = (size_t)words(g.V);
    const size_t sort_bytes = 12 * (size_t)NP;
    const size_t elim_bytes = 4 * ((size_t)g.C * WC + 2 * WC + (size_t)g.C + WV + kOsdMaxLambda +
                                   (size_t)kOsdMaxLambda * WC);
    const size_t dyn = std::max(sort_bytes, elim_bytes);
    int maxsm = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    if (dyn + 1024 > (size_t)maxsm)
        return fail(RELAYBP_ERR_UNSUPPORTED, "OSD state (%zu bytes for %d checks) exceeds shared memory", dyn, g.C);
    const int64_t blocks = std::min<int64_t>(n, h->num_sms);
    const size_t need = (size_t)blocks * g.V * sizeof(int32_t);
    if (h->osd_order_bytes < need) {
        cudaFree(h->d_osd_order);
        h->d_osd_order = nullptr;
        h->osd_order_bytes = 0;
        CUDA_TRY(cudaMalloc(&h->d_osd_order, need));
        h->osd_order_bytes = need;
    }
    OsdJob J{};
    J.g = g;
    J.syn = d_syndromes;
    J.post = d_post;
    J.idx = reinterpret_cast<const long long *>(d_idx);
    J.n = n;
    J.lambda = lambda;
    J.NP = NP;
    J.out_e = d_out_e;
    J.out_valid = d_out_valid;
    J.order = h->d_osd_order;
    CUDA_TRY(cudaFuncSetAttribute(osd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    const int threads = 1024;
    osd_kernel<<<(unsigned)blocks, threads, dyn, static_cast<cudaStream_t>(cuda_stream)>>>(J);
    CUDA_TRY(cudaGetLastError());
    h->launches += 1;
    return 0;
}

}  // extern "C"

struct relaybp_spa {
    int device = 0, num_sms = 0;
    SpaCode code{};
    std::vector<void *> allocs;
};

namespace {
template <typename T>
int spa_upload(relaybp_spa *h, const std::vector<T> &v, const T **dst)
{
    void *p = nullptr;
    CUDA_TRY(cudaMalloc(&p, std::max<size_t>(1, v.size()) * sizeof(T)));
    h->allocs.push_back(p);
    if (!v.empty()) CUDA_TRY(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    *dst = static_cast<const T *>(p);
    return 0;
}
int spa_check(const relaybp_spa *h, int32_t precision)
{
    if (!h) return fail(RELAYBP_ERR_INVALID, "handle is NULL");
    int cur = -1;
    CUDA_TRY(cudaGetDevice(&cur));
    if (cur != h->device) return fail(RELAYBP_ERR_INVALID, "the handle's device %d is not current", h->device);
    if (precision != RELAYBP_MSG_F64 && precision != RELAYBP_MSG_F32)
        return fail(RELAYBP_ERR_UNSUPPORTED, "sum-product runs in FP64 or FP32");
    return 0;
}
}  // namespace

extern "C" {

int relaybp_spa_create(const relaybp_csr *H, relaybp_spa **out)
{
    g_err.clear();
    if (!out) return fail(RELAYBP_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (int rc = check_csr(H, "H")) return rc;
    const int32_t m = H->rows, n = H->cols;
    const int64_t E = H->indptr[m];
    if (n < 1 || n > 4096 || E > (int64_t)1 << 20)
        return fail(RELAYBP_ERR_UNSUPPORTED, "sum-product codes of 1..4096 bits (one warp per frame)");
    relaybp_spa *h = new relaybp_spa();
    cudaError_t ce = cudaGetDevice(&h->device);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (ce != cudaSuccess) { delete h; return fail(RELAYBP_ERR_CUDA, "device query: %s", cudaGetErrorString(ce)); }
    std::vector<int32_t> rptr(H->indptr, H->indptr + m + 1), rvar(H->indices, H->indices + E);
    std::vector<int32_t> cptr(n + 1, 0), cedge(E), fillc(n, 0);
    for (int64_t e = 0; e < E; ++e) cptr[rvar[e] + 1]++;
    for (int32_t j = 0; j < n; ++j) cptr[j + 1] += cptr[j];
    for (int32_t i = 0; i < m; ++i)
        for (int32_t e = rptr[i]; e < rptr[i + 1]; ++e) cedge[cptr[rvar[e]] + fillc[rvar[e]]++] = e;
    h->code.m = m;
    h->code.n = n;
    h->code.E = E;
    int rc = 0;
    if ((rc = spa_upload(h, rptr, &h->code.rptr)) || (rc = spa_upload(h, rvar, &h->code.rvar)) ||
        (rc = spa_upload(h, cptr, &h->code.cptr)) || (rc = spa_upload(h, cedge, &h->code.cedge))) {
        relaybp_spa_destroy(h);
        return rc;
    }
    *out = h;
    return 0;
}

int relaybp_spa_llr(relaybp_spa *h, int32_t precision, const uint32_t *d_codewords, double sigma, double llr_max,
                    uint64_t seed, uint64_t shot0, int64_t shots, void *d_llr, void *cuda_stream)
{
    g_err.clear();
    if (int rc = spa_check(h, precision)) return rc;
    if (shots < 0 || !(sigma > 0.0) || !(llr_max > 0.0)) return fail(RELAYBP_ERR_INVALID, "bad size or noise level");
    if (shots == 0) return 0;
    if (!d_llr) return fail(RELAYBP_ERR_INVALID, "d_llr is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int threads = 256;
    const int64_t total = shots * (int64_t)h->code.n;
    const int64_t blocks = std::min<int64_t>((total + threads - 1) / threads, (int64_t)h->num_sms * 16);
    if (precision == RELAYBP_MSG_F64)
        awgn_llr_kernel<double><<<(unsigned)blocks, threads, 0, st>>>(h->code.n, d_codewords, sigma, llr_max, seed,
                                                                       shot0, shots, static_cast<double *>(d_llr));
    else
        awgn_llr_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(h->code.n, d_codewords, sigma, llr_max, seed,
                                                                      shot0, shots, static_cast<float *>(d_llr));
    CUDA_TRY(cudaGetLastError());
    return 0;
}

int relaybp_spa_decode(relaybp_spa *h, int32_t precision, const void *d_llr, int64_t shots, int32_t max_iter,
                       double llr_max, int32_t early_stop, uint32_t *d_bits, int32_t *d_iters, int32_t *d_valid,
                       void *d_post, void *cuda_stream)
{
    g_err.clear();
    if (int rc = spa_check(h, precision)) return rc;
    if (shots < 0 || max_iter < 1 || !(llr_max > 0.0)) return fail(RELAYBP_ERR_INVALID, "bad size or limit");
    if (shots == 0) return 0;
    if (!d_llr || !d_bits || !d_iters || !d_valid) return fail(RELAYBP_ERR_INVALID, "null pointer");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t tsz = precision == RELAYBP_MSG_F64 ? 8 : 4;
    const size_t per = (2 * (size_t)h->code.E * tsz + 4 * (size_t)words(h->code.n) + 15) & ~(size_t)15;
    int maxsm = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    int warps = 8;
    while (warps > 1 && per * warps > (size_t)maxsm) warps >>= 1;
    if (per * warps > (size_t)maxsm) return fail(RELAYBP_ERR_UNSUPPORTED, "one frame's messages exceed shared memory");
    const size_t dyn = per * warps;
    const int64_t blocks = std::min<int64_t>((shots + warps - 1) / warps, (int64_t)h->num_sms * 8);
    if (precision == RELAYBP_MSG_F64) {
        CUDA_TRY(cudaFuncSetAttribute(spa_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
        spa_kernel<double><<<(unsigned)blocks, 32 * warps, dyn, st>>>(h->code, static_cast<const double *>(d_llr), shots,
                                                                      max_iter, llr_max, early_stop, d_bits, d_iters,
                                                                      d_valid, static_cast<double *>(d_post));
    } else {
        CUDA_TRY(cudaFuncSetAttribute(spa_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
        spa_kernel<float><<<(unsigned)blocks, 32 * warps, dyn, st>>>(h->code, static_cast<const float *>(d_llr), shots,
                                                                     max_iter, (float)llr_max, early_stop, d_bits,
                                                                     d_iters, d_valid, static_cast<float *>(d_post));
    }
    CUDA_TRY(cudaGetLastError());
    return 0;
}

int relaybp_spa_destroy(relaybp_spa *h)
{
    if (!h) return 0;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    for (void *p : h->allocs) cudaFree(p);
    if (prev >= 0) cudaSetDevice(prev);
    delete h;
    return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Sliding-window decoding (relaybp_windows_*): one ordinary handle per window,
// built from the DEM restricted to the window's rows and columns, and the
// gather / commit / observable kernels of windows.cuh between them.
// ---------------------------------------------------------------------------
struct relaybp_windows {
    int device = 0, num_sms = 0;
    int32_t C = 0, V = 0, K = 0, R = 0, w = 0;
    std::vector<relaybp_handle *> hs;                  // window t's decoder
    std::vector<int32_t> nrows, ncommit;               // per window
    std::vector<const int32_t *> rows, clocal, cfull;  // device: window rows, committed columns
    const int32_t *cptr = nullptr, *crow = nullptr;    // device: H by columns
    const int32_t *optr = nullptr, *oidx = nullptr;    // device: O by columns
    std::vector<void *> allocs;
    // scratch grown on demand
    uint32_t *wsyn = nullptr, *wcorr = nullptr, *resid = nullptr, *corr = nullptr;
    StatsDev *wstats = nullptr;
    int64_t cap = 0;
    int wcw_max = 0, wvw_max = 0;
};

namespace {
template <typename T>
int win_upload(relaybp_windows *W, const std::vector<T> &v, const T **dst)
{
    void *p = nullptr;
    CUDA_TRY(cudaMalloc(&p, std::max<size_t>(1, v.size()) * sizeof(T)));
    W->allocs.push_back(p);
    if (!v.empty()) CUDA_TRY(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    *dst = static_cast<const T *>(p);
    return 0;
}

int win_build(relaybp_windows *W, const relaybp_csr *H, const double *priors, const relaybp_csr *obs,
              const int32_t *det_round, const relaybp_params *params)
{
    const int32_t C = W->C, V = W->V, R = W->R, w = W->w;
    const int64_t E = H->indptr[C];
    // column rounds: the least round of the column's detectors (R + 1: none)
    std::vector<int32_t> col_round(V, R + 1), cptr(V + 1, 0), crow(E), fill(V, 0);
    for (int32_t i = 0; i < C; ++i)
        for (int32_t e = H->indptr[i]; e < H->indptr[i + 1]; ++e) {
            const int32_t j = H->indices[e];
            col_round[j] = std::min(col_round[j], det_round[i]);
            cptr[j + 1]++;
        }
    for (int32_t j = 0; j < V; ++j) cptr[j + 1] += cptr[j];
    for (int32_t i = 0; i < C; ++i)
        for (int32_t e = H->indptr[i]; e < H->indptr[i + 1]; ++e) {
            const int32_t j = H->indices[e];
            crow[cptr[j] + fill[j]++] = i;
        }
    std::vector<int32_t> optr(V + 1, 0), oidx;
    if (obs) {
        const int64_t EO = obs->indptr[obs->rows];
        oidx.resize(EO);
        std::vector<int32_t> of(V, 0);
        for (int64_t e = 0; e < EO; ++e) optr[obs->indices[e] + 1]++;
        for (int32_t j = 0; j < V; ++j) optr[j + 1] += optr[j];
        for (int32_t k = 0; k < obs->rows; ++k)
            for (int32_t e = obs->indptr[k]; e < obs->indptr[k + 1]; ++e) {
                const int32_t j = obs->indices[e];
                oidx[optr[j] + of[j]++] = k;
            }
    }
    int rc = 0;
    if ((rc = win_upload(W, cptr, &W->cptr)) || (rc = win_upload(W, crow, &W->crow)) ||
        (rc = win_upload(W, optr, &W->optr)) || (rc = win_upload(W, oidx, &W->oidx)))
        return rc;
    std::vector<int32_t> local(V, -1);
    for (int32_t t = 0;; ++t) {
        const bool last = t + w >= R;
        std::vector<int32_t> rows, cols;
        for (int32_t i = 0; i < C; ++i)
            if (det_round[i] >= t && det_round[i] < t + w) rows.push_back(i);
        for (int32_t j = 0; j < V; ++j)
            if (col_round[j] >= t && col_round[j] < t + w) cols.push_back(j);
        if (rows.empty() || cols.empty())
            return fail(RELAYBP_ERR_INVALID, "window %d (rounds %d..%d) has no %s", t, t, t + w - 1,
                        rows.empty() ? "detector" : "fault column");
        std::fill(local.begin(), local.end(), -1);
        for (size_t k = 0; k < cols.size(); ++k) local[cols[k]] = (int32_t)k;
        // the restriction: the window's rows, in order, over its columns, in order
        std::vector<int32_t> sp(1, 0), si;
        for (int32_t i : rows) {
            for (int32_t e = H->indptr[i]; e < H->indptr[i + 1]; ++e)
                if (local[H->indices[e]] >= 0) si.push_back(local[H->indices[e]]);
            sp.push_back((int32_t)si.size());
        }
        std::vector<double> sprior(cols.size());
        for (size_t k = 0; k < cols.size(); ++k) sprior[k] = priors[cols[k]];
        relaybp_csr sub{(int32_t)rows.size(), (int32_t)cols.size(), sp.data(), si.data()};
        relaybp_handle *h = nullptr;
        if ((rc = relaybp_build(&sub, sprior.data(), nullptr, params, &h))) {
            const std::string msg = g_err;
            return fail(rc, "window %d (rounds %d..%d): %s", t, t, t + w - 1, msg.c_str());
        }
        W->hs.push_back(h);
        std::vector<int32_t> cl, cf;
        for (size_t k = 0; k < cols.size(); ++k)
            if (last || col_round[cols[k]] == t) {
                cl.push_back((int32_t)k);
                cf.push_back(cols[k]);
            }
        const int32_t *drows = nullptr, *dcl = nullptr, *dcf = nullptr;
        if ((rc = win_upload(W, rows, &drows)) || (rc = win_upload(W, cl, &dcl)) || (rc = win_upload(W, cf, &dcf)))
            return rc;
        W->rows.push_back(drows);
        W->clocal.push_back(dcl);
        W->cfull.push_back(dcf);
        W->nrows.push_back((int32_t)rows.size());
        W->ncommit.push_back((int32_t)cl.size());
        W->wcw_max = std::max(W->wcw_max, words((int64_t)rows.size()));
        W->wvw_max = std::max(W->wvw_max, words((int64_t)cols.size()));
        if (last) break;
    }
    return 0;
}

int win_check(const relaybp_windows *W)
{
    if (!W) return fail(RELAYBP_ERR_INVALID, "windows handle is NULL");
    int cur = -1;
    CUDA_TRY(cudaGetDevice(&cur));
    if (cur != W->device) return fail(RELAYBP_ERR_INVALID, "the windows' device %d is not current", W->device);
    return 0;
}
}  // namespace

extern "C" {

int relaybp_windows_create(const relaybp_csr *H, const double *priors, const relaybp_csr *obs,
                           const int32_t *det_round, int32_t window, const relaybp_params *params,
                           relaybp_windows **out)
{
    g_err.clear();
    if (!out) return fail(RELAYBP_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (int rc = check_csr(H, "H")) return rc;
    if (obs) {
        if (int rc = check_csr(obs, "obs")) return rc;
        if (obs->cols != H->cols) return fail(RELAYBP_ERR_INVALID, "obs has %d columns, H has %d", obs->cols, H->cols);
    }
    if (!priors || !det_round) return fail(RELAYBP_ERR_INVALID, "priors or det_round is NULL");
    if (window < 1) return fail(RELAYBP_ERR_INVALID, "window = %d rounds; need >= 1", window);
    if (int rc = check_params(params)) return rc;
    int32_t R = 0;
    for (int32_t i = 0; i < H->rows; ++i) {
        if (det_round[i] < 0) return fail(RELAYBP_ERR_INVALID, "detector %d has round %d < 0", i, det_round[i]);
        R = std::max(R, det_round[i] + 1);
    }
    if (R == 0) return fail(RELAYBP_ERR_INVALID, "no detectors");
    relaybp_windows *W = new relaybp_windows();
    W->C = H->rows;
    W->V = H->cols;
    W->K = obs ? obs->rows : 0;
    W->R = R;
    W->w = window;
    cudaError_t ce = cudaGetDevice(&W->device);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&W->num_sms, cudaDevAttrMultiProcessorCount, W->device);
    if (ce != cudaSuccess) { delete W; return fail(RELAYBP_ERR_CUDA, "device query: %s", cudaGetErrorString(ce)); }
    if (int rc = win_build(W, H, priors, obs, det_round, params)) {
        const std::string msg = g_err;
        relaybp_windows_destroy(W);
        return fail(rc, "%s", msg.c_str());
    }
    *out = W;
    return 0;
}

int relaybp_windows_info(const relaybp_windows *W, int32_t *n_windows, int32_t *n_rounds)
{
    if (!W) return fail(RELAYBP_ERR_INVALID, "windows handle is NULL");
    if (n_windows) *n_windows = (int32_t)W->hs.size();
    if (n_rounds) *n_rounds = W->R;
    return 0;
}

int relaybp_windows_handle(relaybp_windows *W, int32_t t, relaybp_handle **out)
{
    if (!W || !out) return fail(RELAYBP_ERR_INVALID, "NULL argument");
    if (t < 0 || t >= (int32_t)W->hs.size())
        return fail(RELAYBP_ERR_INVALID, "window %d of %d", t, (int)W->hs.size());
    *out = W->hs[t];
    return 0;
}

int relaybp_windows_decode(relaybp_windows *W, const uint32_t *d_syndromes, uint64_t shot0, int64_t shots,
                           uint32_t *d_corrections, uint32_t *d_pred_obs, uint32_t *d_residual,
                           int32_t *d_converged, void *cuda_stream)
{
    g_err.clear();
    if (int rc = win_check(W)) return rc;
    if (shots < 0) return fail(RELAYBP_ERR_INVALID, "shots < 0");
    if (shots == 0) return 0;
    if (!d_syndromes) return fail(RELAYBP_ERR_INVALID, "d_syndromes is NULL");
    if (d_pred_obs && W->K == 0) return fail(RELAYBP_ERR_INVALID, "d_pred_obs given but the DEM has no observables");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int wcf = words(W->C), wvf = words(W->V), wk = words(W->K);
    if (shots > W->cap) {
        CUDA_TRY(cudaStreamSynchronize(st));
        cudaFree(W->wsyn);
        cudaFree(W->wcorr);
        cudaFree(W->wstats);
        cudaFree(W->resid);
        cudaFree(W->corr);
        W->wsyn = W->wcorr = W->resid = W->corr = nullptr;
        W->wstats = nullptr;
        W->cap = 0;
        CUDA_TRY(cudaMalloc(&W->wsyn, (size_t)shots * W->wcw_max * 4));
        CUDA_TRY(cudaMalloc(&W->wcorr, (size_t)shots * W->wvw_max * 4));
        CUDA_TRY(cudaMalloc(&W->wstats, (size_t)shots * sizeof(StatsDev)));
        CUDA_TRY(cudaMalloc(&W->resid, (size_t)shots * wcf * 4));
        CUDA_TRY(cudaMalloc(&W->corr, (size_t)shots * wvf * 4));
        W->cap = shots;
    }
    uint32_t *resid = d_residual ? d_residual : W->resid;
    uint32_t *corr = d_corrections ? d_corrections : W->corr;
    CUDA_TRY(cudaMemcpyAsync(resid, d_syndromes, (size_t)shots * wcf * 4, cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(cudaMemsetAsync(corr, 0, (size_t)shots * wvf * 4, st));
    if (d_converged) {
        // every shot starts converged; each window ANDs its own flag in
        fill_i32_kernel<<<std::max(1, std::min<int>(W->num_sms * 4, (int)((shots + 255) / 256))), 256, 0, st>>>(
            d_converged, 1, shots);
        CUDA_TRY(cudaGetLastError());
    }
    const int g_blocks = W->num_sms * 8;
    for (size_t t = 0; t < W->hs.size(); ++t) {
        relaybp_handle *h = W->hs[t];
        const int wcw = words(W->nrows[t]), wvw = words(h->dem.V);
        win_gather_kernel<<<g_blocks, 256, 0, st>>>(resid, wcf, W->rows[t], W->nrows[t], W->wsyn, wcw, shots);
        CUDA_TRY(cudaGetLastError());
        if (int rc = relaybp_decode_batch(h, W->wsyn, shot0, shots, W->wcorr, nullptr,
                                          reinterpret_cast<relaybp_shot_stats *>(W->wstats), st)) {
            const std::string msg = g_err;
            return fail(rc, "window %d: %s", (int)t, msg.c_str());
        }
        win_commit_kernel<<<g_blocks, 256, 0, st>>>(W->wcorr, wvw, W->clocal[t], W->cfull[t], W->ncommit[t], W->cptr,
                                                     W->crow, corr, wvf, resid, wcf, W->wstats, d_converged, shots);
        CUDA_TRY(cudaGetLastError());
    }
    if (d_pred_obs) {
        CUDA_TRY(cudaMemsetAsync(d_pred_obs, 0, (size_t)shots * wk * 4, st));
        win_obs_kernel<<<g_blocks, 256, 0, st>>>(corr, wvf, W->V, W->optr, W->oidx, d_pred_obs, wk, shots);
        CUDA_TRY(cudaGetLastError());
    }
    return 0;
}

int relaybp_windows_destroy(relaybp_windows *W)
{
    if (!W) return 0;
    for (relaybp_handle *h : W->hs) relaybp_destroy(h);
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(W->device);
    cudaDeviceSynchronize();
    for (void *p : W->allocs) cudaFree(p);
    cudaFree(W->wsyn);
    cudaFree(W->wcorr);
    cudaFree(W->wstats);
    cudaFree(W->resid);
    cudaFree(W->corr);
    if (prev >= 0) cudaSetDevice(prev);
    delete W;
    return 0;
}

}  // extern "C"

extern "C" {

int relaybp_decode_host(relaybp_handle *h, const uint32_t *h_syndromes, uint64_t shot0, int64_t shots,
                        uint32_t *h_pred_obs, relaybp_shot_stats *h_stats, void *cuda_stream)
{
    g_err.clear();
    if (!h) return fail(RELAYBP_ERR_INVALID, "handle is NULL");
    if (int rc = check_device(h)) return rc;
    if (shots < 0) return fail(RELAYBP_ERR_INVALID, "negative shot count");
    if (shots == 0) return 0;
    if (!h_syndromes) return fail(RELAYBP_ERR_INVALID, "h_syndromes is NULL");
    const DevDEM &g = h->dem;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int WC = words(g.C), WK = std::max(1, words(g.K));
    if (h->stage_shots < shots) {
        cudaFree(h->d_stage_syn);
        cudaFree(h->d_stage_pobs);
        cudaFree(h->d_stage_stats);
        h->d_stage_syn = nullptr; h->d_stage_pobs = nullptr; h->d_stage_stats = nullptr;
        h->stage_shots = 0;
        CUDA_TRY(cudaMalloc(&h->d_stage_syn, (size_t)shots * WC * 4));
        CUDA_TRY(cudaMalloc(&h->d_stage_pobs, (size_t)shots * WK * 4));
        CUDA_TRY(cudaMalloc(&h->d_stage_stats, (size_t)shots * sizeof(StatsDev)));
        h->stage_shots = shots;
    }
    CUDA_TRY(cudaMemcpyAsync(h->d_stage_syn, h_syndromes, (size_t)shots * WC * 4, cudaMemcpyHostToDevice, st));
    int rc = relaybp_decode_batch(h, h->d_stage_syn, shot0, shots, nullptr, h_pred_obs ? h->d_stage_pobs : nullptr,
                                  h_stats ? reinterpret_cast<relaybp_shot_stats *>(h->d_stage_stats) : nullptr,
                                  cuda_stream);
    if (rc) return rc;
    if (h_pred_obs)
        CUDA_TRY(cudaMemcpyAsync(h_pred_obs, h->d_stage_pobs, (size_t)shots * words(g.K) * 4, cudaMemcpyDeviceToHost, st));
    if (h_stats)
        CUDA_TRY(cudaMemcpyAsync(h_stats, h->d_stage_stats, (size_t)shots * sizeof(StatsDev), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return 0;
}

int relaybp_count_failures(relaybp_handle *h, const uint32_t *d_pred_obs, const uint32_t *d_true_obs,
                           const relaybp_shot_stats *d_stats, int64_t shots, unsigned long long *d_counters,
                           void *cuda_stream)
{
    g_err.clear();
    if (!h) return fail(RELAYBP_ERR_INVALID, "handle is NULL");
    if (int rc = check_device(h)) return rc;
    if (shots < 0) return fail(RELAYBP_ERR_INVALID, "negative shot count");
    if (shots == 0) return 0;
    if (!d_stats || !d_counters || (h->dem.K > 0 && (!d_pred_obs || !d_true_obs)))
        return fail(RELAYBP_ERR_INVALID, "null pointer");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int threads = 256;
    const int64_t blocks = (shots + threads - 1) / threads;
    count_failures_kernel<<<(unsigned)blocks, threads, 0, st>>>(d_pred_obs, d_true_obs,
                                                                reinterpret_cast<const StatsDev *>(d_stats), shots,
                                                                words(h->dem.K), d_counters);
    CUDA_TRY(cudaGetLastError());
    h->launches += 1;
    return 0;
}

int relaybp_autotune(relaybp_handle *h, const uint32_t *d_syndromes, uint64_t shot0, int64_t shots, int32_t *out_L,
                     int32_t *out_NB, int32_t *out_threads, float *out_ms, void *cuda_stream)
{
    g_err.clear();
    if (!h) return fail(RELAYBP_ERR_INVALID, "handle is NULL");
    if (int rc = check_device(h)) return rc;
    if (shots < 1 || !d_syndromes) return fail(RELAYBP_ERR_INVALID, "need at least one syndrome");
    if (h->params.msg_dtype == RELAYBP_MSG_F64 && !h->lw && !h->lknots) {
        ExactPlan ep = make_exact_plan(h->dem);
        int maxsm = 0;
        CUDA_TRY(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
        if (ep.total <= maxsm) return fail(RELAYBP_ERR_UNSUPPORTED, "the literal-order FP64 kernel has no shape to tune");
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const RowGeom opts[] = {{4, 4}, {8, 4}, {8, 8}, {8, 12}, {8, 16}, {16, 16}, {32, 16}};
    const int thr[] = {256, 512};
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    if (!h->pair_off && h->rslot2 && h->params.msg_dtype == RELAYBP_MSG_F32 && !h->lw) {
        // the two-shot kernel: warps per block
        const int sw = h->pair_warps;
        const JobIO io{d_syndromes, shot0, shots, nullptr, nullptr, nullptr, nullptr, 0};
        float best = 0.f;
        int bw = 0;
        for (int w = 16; w <= pair_max_threads(h->pair_nb) / 32; w += 2) {
            h->pair_warps = w;
            int rc = launch_pair(h, h->scratch, io, st);
            if (rc == 0) {
                cudaEventRecord(e0, st);
                rc = launch_pair(h, h->scratch, io, st);
                cudaEventRecord(e1, st);
            }
            if (rc != 0) continue;
            CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (bw == 0 || ms < best) { best = ms; bw = w; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (bw == 0) {
            h->pair_warps = sw;
            return fail(RELAYBP_ERR_UNSUPPORTED, "no launch shape ran");
        }
        h->pair_warps = bw;
        g_err.clear();
        if (out_L) *out_L = kPairLanes;
        if (out_NB) *out_NB = h->pair_nb;
        if (out_threads) *out_threads = 32 * bw;
        if (out_ms) *out_ms = best;
        return 0;
    }
    const int sL = h->tuned_L, sNB = h->tuned_NB, sT = h->tuned_threads;
    float best = 0.f;
    int bL = 0, bNB = 0, bT = 0;
    const JobIO io{d_syndromes, shot0, shots, nullptr, nullptr, nullptr, nullptr, 0};
    for (const RowGeom &o : opts) {
        if (o.L * o.NB < h->max_row_deg || o.L * o.NB > 4 * std::max(32, h->max_row_deg)) continue;
        for (int tc : thr) {
            h->tuned_L = o.L;
            h->tuned_NB = o.NB;
            h->tuned_threads = tc;
            int rc = launch_jobs_dtype(&h, &io, 1, h->scratch, st);             // warm-up (also sizes scratch)
            if (rc == 0) {
                cudaEventRecord(e0, st);
                rc = launch_jobs_dtype(&h, &io, 1, h->scratch, st);
                cudaEventRecord(e1, st);
            }
            if (rc != 0) continue;
            CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (bL == 0 || ms < best) { best = ms; bL = o.L; bNB = o.NB; bT = tc; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (bL == 0) {
        h->tuned_L = sL; h->tuned_NB = sNB; h->tuned_threads = sT;
        return fail(RELAYBP_ERR_UNSUPPORTED, "no launch shape ran");
    }
    h->tuned_L = bL;
    h->tuned_NB = bNB;
    h->tuned_threads = bT;
    g_err.clear();
    if (out_L) *out_L = bL;
    if (out_NB) *out_NB = bNB;
    if (out_threads) *out_threads = bT;
    if (out_ms) *out_ms = best;
    return 0;
}

int relaybp_group_create(relaybp_handle *const *handles, int32_t n, relaybp_group **out)
{
    g_err.clear();
    if (!out) return fail(RELAYBP_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!handles || n < 1 || n > kMaxJobs) return fail(RELAYBP_ERR_INVALID, "a group holds 1..%d handles", kMaxJobs);
    for (int32_t d = 0; d < n; ++d) {
        if (!handles[d]) return fail(RELAYBP_ERR_INVALID, "handle %d is NULL", d);
        if (handles[d]->device != handles[0]->device)
            return fail(RELAYBP_ERR_INVALID, "handles of a group must share one device");
        if (handles[d]->params.msg_dtype != handles[0]->params.msg_dtype)
            return fail(RELAYBP_ERR_INVALID, "handles of a group must share one message precision");
    }
    relaybp_group *grp = new relaybp_group();
    grp->device = handles[0]->device;
    grp->handles.assign(handles, handles + n);
    *out = grp;
    return 0;
}

int relaybp_group_decode(relaybp_group *grp, const uint32_t *const *d_syndromes, const uint64_t *shot0,
                         const int64_t *shots, uint32_t *const *d_corrections, uint32_t *const *d_pred_obs,
                         relaybp_shot_stats *const *d_stats, void *cuda_stream)
{
    g_err.clear();
    if (!grp) return fail(RELAYBP_ERR_INVALID, "group is NULL");
    if (!d_syndromes || !shot0 || !shots) return fail(RELAYBP_ERR_INVALID, "null array");
    const int n = (int)grp->handles.size();
    if (int rc = check_device(grp->handles[0])) return rc;
    std::vector<JobIO> io(n);
    for (int d = 0; d < n; ++d) {
        if (shots[d] < 0) return fail(RELAYBP_ERR_INVALID, "negative shot count for DEM %d", d);
        if (shots[d] > 0 && !d_syndromes[d]) return fail(RELAYBP_ERR_INVALID, "syndromes of DEM %d are NULL", d);
        io[d] = JobIO{d_syndromes[d], shot0[d], shots[d], d_corrections ? d_corrections[d] : nullptr,
                      d_pred_obs ? d_pred_obs[d] : nullptr,
                      d_stats ? reinterpret_cast<StatsDev *>(d_stats[d]) : nullptr, nullptr, 0};
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // DEMs with tail offload hand their long shots to one cluster launch each
    std::vector<int> tails;
    for (int d = 0; d < n; ++d) {
        relaybp_handle *h = grp->handles[d];
        if (io[d].shots > 0 && tail_applies(h, io[d])) {
            CUDA_TRY(cudaMemsetAsync(h->tail_count, 0, sizeof(unsigned int), st));
            io[d].tail = TailOut{h->tail_rec, h->tail_M, h->tail_best, h->tail_count, h->tail_max, h->tail_legs};
            tails.push_back(d);
        }
    }
    int rc = launch_jobs_dtype(grp->handles.data(), io.data(), n, grp->scratch, st);
    if (rc == 0) grp->launches += 1;
    for (size_t k = 0; k < tails.size() && rc == 0; ++k) {
        const int d = tails[k];
        rc = launch_cluster(grp->handles[d], grp->scratch, io[d], st);
        if (rc == 0) grp->launches += 1;
    }
    return rc;
}

int relaybp_group_destroy(relaybp_group *grp)
{
    if (!grp) return 0;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(grp->device);
    cudaDeviceSynchronize();
    scratch_free(grp->scratch);
    if (prev >= 0) cudaSetDevice(prev);
    delete grp;
    return 0;
}

int64_t relaybp_group_launch_count(const relaybp_group *grp) { return grp ? grp->launches : -1; }

int64_t relaybp_launch_count(const relaybp_handle *h) { return h ? h->launches : -1; }

int relaybp_sync(relaybp_handle *h, void *cuda_stream)
{
    g_err.clear();
    if (!h) return fail(RELAYBP_ERR_INVALID, "handle is NULL");
    if (int rc = check_device(h)) return rc;
    CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream)));
    CUDA_TRY(cudaGetLastError());
    return 0;
}

int relaybp_probe_smem_read(int32_t reps, float *d_sink, double *bytes_read, void *cuda_stream)
{
    g_err.clear();
    if (reps < 1 || !d_sink || !bytes_read) return fail(RELAYBP_ERR_INVALID, "bad probe arguments");
    int dev = 0, sms = 0, per_sm = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, smem_read_probe, 1024, 0));
    const int blocks = sms * std::max(1, per_sm);
    smem_read_probe<<<blocks, 1024, 0, static_cast<cudaStream_t>(cuda_stream)>>>(d_sink, reps);
    CUDA_TRY(cudaGetLastError());
    *bytes_read = (double)blocks * 1024.0 * (double)reps * 16.0;
    return 0;
}

int relaybp_destroy(relaybp_handle *h)
{
    if (!h) return 0;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    for (void *p : h->allocs) cudaFree(p);
    scratch_free(h->scratch);
    cudaFree(h->d_lwork);
    cudaFree(h->d_lgbar);
    cudaFree(h->d_osd_order);
    cudaFree(h->cl_rslot);
    cudaFree(h->cl_ecode);
    cudaFree(h->cl_halo[0]);
    cudaFree(h->cl_halo[1]);
    cudaFree(h->tail_rec);
    cudaFree(h->tail_M);
    cudaFree(h->tail_best);
    cudaFree(h->tail_count);
    cudaFree(h->d_stage_syn);
    cudaFree(h->d_stage_pobs);
    cudaFree(h->d_stage_stats);
    if (prev >= 0) cudaSetDevice(prev);
    delete h;
    return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free decode (relaybp_decode_batch_noalloc).
//
// relaybp_decode_batch keeps its scratch (the persistent kernel's work counter
// and one row of memory strengths per thread block) in handle-owned device
// memory that it allocates, and grows, with cudaMalloc on first use.  This
// variant instead uses one fixed array compiled into the library, so a call
// never allocates or frees device memory.  Every GPU that loads the library
// reserves the array until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;     // 16 MiB
constexpr size_t kNoAllocCounterBytes = 256;                   // work counter, padded
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// In host code `g_noalloc_scratch` only names a host-side stand-in; its device
// address comes from cudaGetSymbolAddress, looked up once per device with that
// device current and cached here.
constexpr int kNoAllocMaxDevices = 64;
unsigned char *g_noalloc_addr[kNoAllocMaxDevices] = {};
std::mutex g_noalloc_mutex;

int noalloc_scratch(int device, unsigned char **out)
{
    if (device < 0 || device >= kNoAllocMaxDevices)
        return fail(RELAYBP_ERR_UNSUPPORTED, "device ordinal %d beyond %d", device, kNoAllocMaxDevices);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[device]) {
        int cur = -1;
        CUDA_TRY(cudaGetDevice(&cur));
        if (cur != device)
            return fail(RELAYBP_ERR_INVALID, "the handle's device %d is not current (device %d is)", device, cur);
        void *p = nullptr;
        CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_addr[device] = static_cast<unsigned char *>(p);
    }
    *out = g_noalloc_addr[device];
    return 0;
}

}  // namespace

extern "C" int relaybp_decode_batch_noalloc(relaybp_handle *h, const uint32_t *d_syndromes, uint64_t shot0,
                                            int64_t shots, uint32_t *d_corrections, uint32_t *d_pred_obs,
                                            relaybp_shot_stats *d_stats, void *cuda_stream)
{
    g_err.clear();
    if (!h) return fail(RELAYBP_ERR_INVALID, "handle is NULL");
    if (shots < 0) return fail(RELAYBP_ERR_INVALID, "negative shot count");
    if (shots == 0) return 0;
    if (!d_syndromes) return fail(RELAYBP_ERR_INVALID, "d_syndromes is NULL");
    if (int rc = check_device(h)) return rc;           // every call, not only the first on a device
    unsigned char *scratch = nullptr;
    if (int rc = noalloc_scratch(h->device, &scratch)) return rc;
    // a fixed scratch view of the static array: counter first, then the rows;
    // it never grows, so a launch that needs more is rejected
    Scratch sc;
    sc.fixed = true;
    sc.work = reinterpret_cast<unsigned long long *>(scratch);
    sc.gamma = scratch + kNoAllocCounterBytes;
    sc.gamma_bytes = kNoAllocScratchBytes - kNoAllocCounterBytes;
    const JobIO io{d_syndromes, shot0, shots, d_corrections, d_pred_obs, reinterpret_cast<StatsDev *>(d_stats),
                   nullptr, 0};
    return decode_single(h, sc, io, static_cast<cudaStream_t>(cuda_stream), true);
}
