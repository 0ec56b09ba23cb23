/*
 * relaybp.h -- C ABI of the B300 (sm_103a) Relay-BP decoding library.
 *
 * The library samples syndromes from a detector error model (DEM) and decodes
 * them with Relay-BP: min-sum belief propagation with disordered memory
 * strengths, run as a chain of relay legs that keeps the lowest-weight of up to
 * stop_nconv valid solutions.  arXiv 2607.27644 uses this decoder for every
 * circuit-level result (Sec. 6.1, decoder configuration list: gamma0 = 0.125,
 * pre_iter = 80, num_sets = 1000, max_iterations = 60, stop_nconv = 5, fp32
 * messages, flooding schedule; gamma intervals in Table 9; DEM sizes in
 * Table 5).  The paper cites Relay-BP without printing its update rule; the
 * rule implemented here is:
 *
 *   L0_j    = log((1 - p_j) / p_j)                                 (host, FP64)
 *   L_j(t)  = (1 - g_j) L0_j + g_j M_j(t-1)                       memory term
 *   mu_ji   = L_j(t) + sum_{i' != i} nu_i'j(t-1)
 *   nu_ij   = (-1)^{s_i} prod_{j' != j} sgn(mu_j'i) min_{j' != j} |mu_j'i|
 *   M_j(t)  = L_j(t) + sum_i nu_ij(t),   e^_j = [M_j(t) < 0]
 *   a leg stops at its first t with H e^ = s; leg 0 runs pre_iter iterations
 *   at g_j = gamma0, legs 1..num_sets run max_iterations at
 *   g_j ~ U[gamma_min, gamma_max]; M carries across legs, messages reset.
 *
 * Conventions shared by every call:
 *   - Status: 0 on success, a negative RELAYBP_ERR_* code otherwise;
 *     relaybp_last_error() returns a message for the calling thread.  No call
 *     aborts the process or traps the device.
 *   - Bit vectors are packed little-endian into uint32 words: bit b lives in
 *     word b / 32 at position b % 32.  A batch of vectors is row-major, one row
 *     of ceil(nbits / 32) words per shot.
 *   - "d_" pointers are device memory owned by the caller; "h_" pointers are
 *     host memory owned by the caller.  Structures passed to relaybp_build are
 *     copied; the caller may free them on return.
 *   - A handle belongs to the device that was current when it was built:
 *     every call that launches work checks that this device is current and
 *     returns RELAYBP_ERR_INVALID otherwise.
 *   - Calls taking a stream are asynchronous on that stream (NULL = the legacy
 *     default stream); the caller synchronises before reading results.  A
 *     handle is not thread-safe: use one handle per host thread and stream.
 *   - Random draws are counter-based (Philox4x32-10, Salmon et al. SC'11):
 *     fault j of shot s uses word j of stream 0 under key `seed`; the memory
 *     strength of variable j in leg r uses word r*4*ceil(V/4) + j of stream 1
 *     under key params.seed.  Results therefore depend only on (seed, global
 *     shot index), never on batching or sharding.
 */
#ifndef RELAYBP_H
#define RELAYBP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    RELAYBP_OK = 0,
    RELAYBP_ERR_INVALID = -1,   /* bad argument: null pointer, size, index or value out of range */
    RELAYBP_ERR_CUDA = -2,      /* a CUDA runtime call failed; message has the CUDA error string */
    RELAYBP_ERR_UNSUPPORTED = -3/* valid input the library does not handle (e.g. too large for a kernel) */
};

enum {                           /* message storage precision */
    RELAYBP_MSG_F64 = 0,         /* FP64 storage and arithmetic */
    RELAYBP_MSG_F32 = 1,         /* FP32 storage and arithmetic (the paper's proc_float = fp32) */
    RELAYBP_MSG_F16 = 2,         /* FP16 storage (saturating at +-65504), FP32 arithmetic */
    RELAYBP_MSG_BF16 = 3,        /* BF16 storage, FP32 arithmetic */
    RELAYBP_MSG_I8 = 4           /* scaled int8 storage, FP32 arithmetic: q = clamp(rne(v / int8_scale),
                                    -127, 127), v = q * int8_scale */
};

/* Compressed sparse rows of a binary matrix, host memory.
 * indptr[rows + 1] nondecreasing with indptr[0] = 0; indices[indptr[rows]]
 * column indices in [0, cols), strictly increasing within each row. */
typedef struct {
    int32_t rows, cols;
    const int32_t *indptr;
    const int32_t *indices;
} relaybp_csr;

/* Decoder parameters; names follow the paper's decoder configuration list. */
typedef struct {
    double gamma0;              /* memory strength of leg 0 (paper: 0.125) */
    int32_t pre_iter;           /* iteration cap of leg 0 (paper: 80), >= 1 */
    int32_t num_sets;           /* number of relay legs after leg 0 (paper: 1000), >= 0 */
    int32_t max_iterations;     /* iteration cap of each later leg (paper: 60), >= 1 */
    int32_t stop_nconv;         /* stop after this many solutions (paper: 5), >= 1 */
    double gamma_min, gamma_max;/* memory-strength interval of legs >= 1 (Table 9) */
    int32_t msg_dtype;          /* RELAYBP_MSG_* */
    int32_t stop_all;           /* 1: run every leg regardless of solutions (the paper's 'All') */
    int32_t carry_messages;     /* 1: keep check-to-variable messages across legs */
    float int8_scale;           /* RELAYBP_MSG_I8: value of one int8 step, > 0, or 0 for the automatic
                                   scale (largest |prior LLR| / 24, per DEM; rejected with
                                   RELAYBP_ERR_INVALID when every prior is 1/2, which makes it 0);
                                   must be 0 for the other forms */
    uint64_t seed;              /* key of the memory-strength draws */
} relaybp_params;

/* Per-shot decoding statistics (24 bytes). */
typedef struct {
    int32_t converged;          /* 1 if at least one leg reached H e^ = s */
    int32_t nsol;               /* number of solutions found (<= stop_nconv unless stop_all) */
    int32_t legs;               /* legs run, leg 0 included */
    int32_t iters;              /* BP iterations run over all legs */
    double weight;              /* sum_j e^_j L0_j of the returned correction, FP64 */
} relaybp_shot_stats;

typedef struct relaybp_handle relaybp_handle;
typedef struct relaybp_group relaybp_group;
typedef struct relaybp_spa relaybp_spa;
typedef struct relaybp_windows relaybp_windows;

/* Build a decoder for one DEM on the current CUDA device.
 * H: detector x fault check matrix (C rows, V columns); every row has 0 or at
 *    least 2 entries, C < 2^20, nnz < 2^30.
 * priors: V fault probabilities, each in (0, 1).
 * obs: observable x fault matrix (K rows, V columns), or NULL for K = 0.
 * params: decoder parameters (validated here; copied into the handle).
 * out: receives the handle, which owns all device memory it allocates.
 * The DEM is copied to the device synchronously; the handle records the
 * current device and must be used with that device current. */
int relaybp_build(const relaybp_csr *H, const double *priors, const relaybp_csr *obs,
                  const relaybp_params *params, relaybp_handle **out);

/* Replace the decoder parameters of an existing handle (validated as above). */
int relaybp_set_params(relaybp_handle *h, const relaybp_params *params);

/* Attach learned parameters to a handle for decoding (the learned form of
 * this library; no counterpart in the paper).  d_w [T][E] FP32 message weights
 * indexed by the iteration within each leg (iterations past T of a leg use
 * unit weights: the trained horizon ends there),
 * d_knots [K+1] FP32 nondecreasing memory-strength inverse CDF for legs >= 1
 * (same meaning as in relaybp_learned_forward; u from stream 1 of the leg).
 * Either may be NULL (NULL and NULL restore the plain method).  Device
 * pointers stay owned by the caller and must outlive the decodes that use
 * them.  Needs msg_dtype F32, F16, BF16 or I8 and carry_messages = 0. */
int relaybp_set_learned(relaybp_handle *h, const float *d_w, int32_t T, const float *d_knots, int32_t K);

/* Same with weights tied per check row: d_wrow [T][C], the weight of every
 * message check i sends in iteration t+1 of a leg (the per-edge weights with
 * w[t][e] = d_wrow[t][row of e]).  The weight is applied once per row when
 * the row's compressed state is formed, so decoding costs no extra loads and
 * no per-message multiply.  With FP16/BF16/int8 storage the weighted minima
 * are what is rounded (per-edge weights multiply after the rounding).
 * Replaces any per-edge weights. */
int relaybp_set_learned_rows(relaybp_handle *h, const float *d_wrow, int32_t T, const float *d_knots, int32_t K);

/* Learned parameters apply to legs 0 .. legs-1 only; later legs run the plain
 * method (unit weights, gamma ~ U[gamma_min, gamma_max]) in the same launch --
 * the plain fallback for shots the learned legs do not settle.  legs = -1: all
 * legs (the default); below -1: RELAYBP_ERR_INVALID, setting unchanged. */
int relaybp_set_learned_legs(relaybp_handle *h, int32_t legs);

/* Query sizes: n_det (C), n_loc (V), n_obs (K), n_edges (nnz of H). */
int relaybp_sizes(const relaybp_handle *h, int32_t *n_det, int32_t *n_loc, int32_t *n_obs, int64_t *n_edges);

/* Draw `shots` shots with global indices shot0 .. shot0 + shots - 1.
 * Fault j of a shot fires iff its Philox word is below floor(p_j * 2^32).
 * d_syndromes: [shots][ceil(C/32)] words = H e;  d_obs: [shots][ceil(K/32)]
 * words = O e (may be NULL); d_errors: [shots][ceil(V/32)] fired faults (may
 * be NULL).  Exact integer work: bit-identical to any other implementation of
 * the same definition. */
int relaybp_sample(relaybp_handle *h, uint64_t seed, uint64_t shot0, int64_t shots,
                   uint32_t *d_syndromes, uint32_t *d_obs, uint32_t *d_errors, void *cuda_stream);

/* Decode `shots` syndromes d_syndromes [shots][ceil(C/32)] whose global shot
 * indices start at shot0 (they key the memory-strength draws).
 * d_corrections: [shots][ceil(V/32)] the returned e^ (lowest-weight solution,
 *   earliest on ties; the last iterate if no leg converged), or NULL.
 * d_pred_obs: [shots][ceil(K/32)] O e^, or NULL.
 * d_stats: [shots] per-shot statistics, or NULL.
 * One persistent kernel decodes the whole batch: each thread block takes the
 * next undecoded shot from a device work counter owned by the handle, so
 * blocks whose shots finish early move on at once. */
int relaybp_decode_batch(relaybp_handle *h, const uint32_t *d_syndromes, uint64_t shot0, int64_t shots,
                         uint32_t *d_corrections, uint32_t *d_pred_obs, relaybp_shot_stats *d_stats,
                         void *cuda_stream);

/* Allocation-free variant of relaybp_decode_batch (no counterpart in the
 * paper; the decoding it performs is identical, shot for shot).
 *
 * relaybp_decode_batch allocates its scratch -- the persistent kernel's work
 * counter and one row of memory strengths per thread block -- with cudaMalloc
 * the first time it needs it and whenever a larger launch needs more.  Some
 * callers must not allocate device memory while they decode: a real-time
 * decoding loop cannot absorb the implicit device-wide synchronisation and
 * latency of cudaMalloc/cudaFree, and a host program whose device memory is
 * carved up by another allocator (a framework's caching allocator or a fixed
 * per-process budget) must not have a library allocate behind its back or
 * fail when that budget is exhausted.  This entry point allocates nothing:
 * its scratch is one 16 MiB array compiled into the library
 * (kNoAllocScratchBytes), reserved on every GPU that loads the library until
 * the process exits.  The caller still passes the inputs and outputs exactly
 * as for relaybp_decode_batch; the handle must come from relaybp_build, done
 * beforehand at set-up time.
 *
 * - The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with the handle's device current and caches it;
 *   make that first call before any stream capture.  Every call checks that
 *   the handle's device is current (RELAYBP_ERR_INVALID otherwise).
 * - The call zeroes the work counter in the array before its launch; the
 *   memory-strength rows are rewritten before use, so nothing else needs
 *   clearing.  The array keeps the last call's contents.
 * - All calls on a device share the one array: calls whose kernels overlap on
 *   the GPU (other streams, other handles, other host threads) race and give
 *   wrong results.  Serialise them, e.g. by issuing them on one stream.
 * - A launch whose scratch (256 bytes + one row of V memory strengths, FP32
 *   or FP64, per thread block) exceeds 16 MiB, or a DEM whose per-shot state
 *   does not fit in shared memory, is rejected with RELAYBP_ERR_UNSUPPORTED
 *   and a message giving the sizes; use relaybp_decode_batch for it.  (The
 *   ZSZ-LP-160 circuit DEM in FP32 needs 12.3 MB.) */
int relaybp_decode_batch_noalloc(relaybp_handle *h, const uint32_t *d_syndromes, uint64_t shot0, int64_t shots,
                                 uint32_t *d_corrections, uint32_t *d_pred_obs, relaybp_shot_stats *d_stats,
                                 void *cuda_stream);

/* relaybp_decode_batch that also records, per shot, the device clock
 * (%globaltimer, nanoseconds) when a thread block starts decoding it and when
 * it retires: d_times [shots][2] = {start, retire}, device memory, required.
 * retire - start is the shot's decoding latency; retire minus the launch
 * time adds its wait in the batch.  Outputs otherwise equal those of
 * relaybp_decode_batch, except that FP64 handles always take the compressed
 * FP64 kernel here (the literal-order kernel records no times).  The paper
 * reports per-shot decoding latency (Sec. 6.1, App. F, Table 12); this call
 * measures the same quantity for a batched decoder. */
int relaybp_decode_timed(relaybp_handle *h, const uint32_t *d_syndromes, uint64_t shot0, int64_t shots,
                         uint32_t *d_corrections, uint32_t *d_pred_obs, relaybp_shot_stats *d_stats,
                         uint64_t *d_times, void *cuda_stream);

/* Diagnostic variant of relaybp_decode_batch for parity checks: also writes
 * the marginals M_j after each of the first trace_iters iterations (counted
 * over all legs) to d_trace [shots][trace_iters][V] as FP64 (entries past a
 * shot's last iteration are left untouched).  d_stats may be NULL. */
int relaybp_decode_trace(relaybp_handle *h, const uint32_t *d_syndromes, uint64_t shot0, int64_t shots,
                         int32_t trace_iters, double *d_trace, relaybp_shot_stats *d_stats, void *cuda_stream);

/* Same as relaybp_decode_batch with host buffers: copies h_syndromes to the
 * device, decodes, copies the results back, and synchronises the stream before
 * returning.  Staging buffers are owned by the handle and grow on demand.
 * h_pred_obs and h_stats may be NULL.  The whole batch is one persistent
 * launch: a synchronous call lasts as long as its slowest shot (a shot that
 * runs every relay leg), and one launch keeps every other shot decoding in
 * that shot's shadow; cutting the batch into chunks on several streams made
 * the call slower (measured), the copies being small beside the decode.
 * Callers that stream many batches overlap their tails by issuing
 * relaybp_decode_batch on several streams with one handle each. */
int relaybp_decode_host(relaybp_handle *h, const uint32_t *h_syndromes, uint64_t shot0, int64_t shots,
                        uint32_t *h_pred_obs, relaybp_shot_stats *h_stats, void *cuda_stream);

/* relaybp_decode_batch that also hands over the shots it leaves unresolved
 * (no solution in any leg; the paper's outlook, Sec. 7, names them as the
 * failures that dominate and OSD as their post-processing): each such shot
 * takes the next slot of *d_flag_count (uint32, caller-zeroed, device
 * memory; it counts every flagged shot even past max_flagged) and, if the
 * slot is below max_flagged, writes its index within this batch to
 * d_flag_idx[slot] (int64) and its final posteriors M (the marginals after
 * its last iteration, FP64 whatever the storage precision) to
 * d_flag_post[slot][V].  Slots are taken in completion order, which varies
 * between runs; their contents do not.  Other arguments as for
 * relaybp_decode_batch. */
int relaybp_decode_flagged(relaybp_handle *h, const uint32_t *d_syndromes, uint64_t shot0, int64_t shots,
                           uint32_t *d_corrections, uint32_t *d_pred_obs, relaybp_shot_stats *d_stats,
                           int64_t max_flagged, int64_t *d_flag_idx, double *d_flag_post, uint32_t *d_flag_count,
                           void *cuda_stream);

/* Ordered-statistics decoding (the paper's outlook, Sec. 7) of n shots from
 * their posteriors: for shot f, the syndrome row d_idx[f] of d_syndromes and
 * the posteriors d_post[f][V] (as relaybp_decode_flagged writes them).  The
 * columns of H are ordered by posterior ascending (the most likely error
 * first; ties by column index); the first rank(H) linearly independent ones
 * over GF(2) form the information set, on which H e = s is solved (OSD-0).
 * With lambda > 0 every flip of one or two of the first lambda columns
 * outside the information set is also tried, keeping the candidate of least
 * FP64 weight sum_j e_j L0_j (OSD-0 on ties, else the first candidate in
 * u-major order).  Outputs: d_out_e [n][ceil(V/32)] and d_out_valid[n] = 0
 * when s is not in the column space of H.  Limits: V <= 16,384 columns,
 * lambda <= 64, and the C x C elimination state in shared memory (C up to
 * about 1,300 checks); beyond them RELAYBP_ERR_UNSUPPORTED.  One thread
 * block per shot; the handle keeps a column-order scratch (allocated on
 * first use). */
int relaybp_osd(relaybp_handle *h, const uint32_t *d_syndromes, const double *d_post, const int64_t *d_idx, int64_t n,
                int32_t lambda, uint32_t *d_out_e, int32_t *d_out_valid, void *cuda_stream);

/* Failure accounting (paper Sec. 7, Outlook, "Improved decoding": failures
 * are either flagged nonconvergences or undetected logical errors).  Adds to
 * d_counters[0] the shots counted, [1] shots that did not converge, [2]
 * converged shots whose predicted observables differ from d_true_obs, [3]
 * all failures ([1] + [2]).  d_counters: 4 x uint64, caller-zeroed. */
int relaybp_count_failures(relaybp_handle *h, const uint32_t *d_pred_obs, const uint32_t *d_true_obs,
                           const relaybp_shot_stats *d_stats, int64_t shots, unsigned long long *d_counters,
                           void *cuda_stream);

/* Autotuner (launch shape only; no counterpart in the paper): times the
 * decode kernel the handle uses on d_syndromes and keeps the fastest launch
 * shape in the handle for later single-DEM decodes.  For the two-shot FP32
 * kernel (relaybp_set_pair_kernel) that is the warps per block (16..32,
 * L = 4 lanes per row, NB its row slots per lane); for the general kernel
 * every valid row geometry (L lanes per check row x NB positions per lane,
 * L*NB >= the longest row) and block size (256, 512 threads).  Synchronises
 * the stream.  Results of a decode do not depend on the launch shape
 * (per-shot arithmetic is identical), only its speed.  Outputs (each may be
 * NULL): the chosen L, NB, threads and its time in ms.
 * RELAYBP_ERR_UNSUPPORTED for DEMs decoded by the literal-order FP64 kernel,
 * which has no shape to tune. */
int relaybp_autotune(relaybp_handle *h, const uint32_t *d_syndromes, uint64_t shot0, int64_t shots, int32_t *out_L,
                     int32_t *out_NB, int32_t *out_threads, float *out_ms, void *cuda_stream);

/* Batched decoding of several DEMs in one persistent launch (no counterpart
 * in the paper, which decodes one shot at a time; its App. F notes that
 * batched decoding is bound by device memory capacity and bandwidth).
 *
 * relaybp_group_create: a group of 1..16 handles built on one device with one
 * message precision (their other parameters may differ: each DEM decodes with
 * its own).  The group owns its own scratch; the handles must outlive it.
 * relaybp_group_decode: decode, in ONE kernel launch, shots[d] syndromes of
 * DEM d from d_syndromes[d] (global shot indices shot0[d]...) for every d,
 * writing d_corrections[d], d_pred_obs[d], d_stats[d] (each array, or any of
 * its entries, may be NULL).  Every thread block takes the next shot of any
 * DEM from one work counter, so uneven shot counts and shots that finish
 * early leave no SM idle until the whole batch is done.  Results equal those
 * of relaybp_decode_batch on each DEM alone (except for FP64 DEMs small enough
 * for its literal-order kernel, which a group decodes with the compressed
 * FP64 kernel).  Asynchronous on the stream; one group per stream. */
int relaybp_group_create(relaybp_handle *const *handles, int32_t n, relaybp_group **out);
int relaybp_group_decode(relaybp_group *grp, const uint32_t *const *d_syndromes, const uint64_t *shot0,
                         const int64_t *shots, uint32_t *const *d_corrections, uint32_t *const *d_pred_obs,
                         relaybp_shot_stats *const *d_stats, void *cuda_stream);
int64_t relaybp_group_launch_count(const relaybp_group *grp);
int relaybp_group_destroy(relaybp_group *grp);

/* Learned Relay-BP training (no counterpart in the paper: the learned form
 * of this library).  Parameters, both in the precision `precision`
 * (RELAYBP_MSG_F32 or RELAYBP_MSG_F64), device memory:
 *   d_w [T][E]   weight of the check-to-variable message of edge e (row-major
 *                order of H) in iteration t+1;
 *   d_knots [K+1], nondecreasing, 1 <= K <= 64: the memory-strength inverse
 *                CDF g(u) = knots[k] + (knots[k+1] - knots[k]) (uK - k),
 *                k = floor(uK), u = the leg-1 Philox stream-1 draw (key
 *                gamma_seed) of each variable.
 * relaybp_learned_forward runs, for each shot, T iterations of one memory-BP
 * leg from M = L0, nu = 0 with weighted messages and these strengths, writes
 * the shot's loss d_loss[s], summed over the T iterations, and a tape of
 * relaybp_learned_tape_bytes bytes.  objective 0: sum_j BCE(M_j(t), e_j)
 * (e = d_errors, bit j in error with probability sigmoid(-M_j)); objective 1:
 * the soft syndrome -sum_i log(eps + (1 - 2 eps) P_i(t)), eps = 1e-6,
 * P_i = (1 + (-1)^{s_i} prod_{j in row i} tanh(M_j / 2)) / 2 the probability
 * that check i holds its syndrome bit (s = d_syndromes): it rewards
 * satisfying every check early, which is what ends a decode.
 * relaybp_learned_backward reads the tape and ADDS scale * dLoss/dw and
 * scale * dLoss/dknots (Loss = sum of the shots' losses) into the
 * caller-zeroed d_grad_w [T][E] and d_grad_knots [K+1]; it needs d_errors for
 * objective 0 and d_syndromes for objective 1.  Gradients flow through the
 * argmin and second-argmin of every check (sign products are piecewise
 * constant); the summation order of the atomics is not fixed.  Objectives
 * other than 0 and 1: RELAYBP_ERR_INVALID. */
int64_t relaybp_learned_tape_bytes(const relaybp_handle *h, int32_t precision, int32_t T, int64_t shots);
int relaybp_learned_forward(relaybp_handle *h, int32_t precision, int32_t T, const void *d_w, int32_t K,
                            const void *d_knots, uint64_t gamma_seed, int32_t objective,
                            const uint32_t *d_syndromes, const uint32_t *d_errors, uint64_t shot0, int64_t shots,
                            void *d_tape, double *d_loss, void *cuda_stream);
int relaybp_learned_backward(relaybp_handle *h, int32_t precision, int32_t T, const void *d_w, int32_t K,
                             const void *d_knots, uint64_t gamma_seed, int32_t objective,
                             const uint32_t *d_syndromes, const uint32_t *d_errors, uint64_t shot0, int64_t shots,
                             const void *d_tape, double scale, void *d_grad_w, void *d_grad_knots,
                             void *cuda_stream);

/* Wait until the work queued on cuda_stream (NULL = the legacy default
 * stream) has finished and report an asynchronous failure there: 0, or
 * RELAYBP_ERR_CUDA with the CUDA error text in relaybp_last_error() (a launch
 * that failed after its call returned, a kernel that faulted).  The handle's
 * device must be current (RELAYBP_ERR_INVALID otherwise).  The paper has no
 * counterpart: it is the boundary's synchronisation point.  No kernel of this
 * library waits on a flag, a peer or a timeout, so CUDA's own status is the
 * only device-side error there is to report. */
int relaybp_sync(relaybp_handle *h, void *cuda_stream);

/* Number of kernel launches this handle has issued since it was built. */
int64_t relaybp_launch_count(const relaybp_handle *h);

/* Measurement utility (no paper counterpart): launch a kernel on the current
 * device that streams conflict-free 16-byte shared-memory loads, `reps` per
 * thread, over every SM.  *bytes_read receives the bytes the launch reads;
 * dividing by its event-timed duration gives the shared-memory bandwidth that
 * bounds the decode kernel.  d_sink: one float per block, device memory. */
int relaybp_probe_smem_read(int32_t reps, float *d_sink, double *bytes_read, void *cuda_stream);

/* Kernel choice for FP32 single-DEM decodes (no counterpart in the paper;
 * results are identical either way, bit for bit).  By default a DEM whose
 * rows have at most 108 entries and whose two-shot state fits in shared
 * memory (ZSZ-LP-160 circuit DEMs: 217 KB) is decoded by the two-shot
 * kernel: each thread block decodes two shots in lockstep, sharing every
 * load of the DEM structure between them and adding their messages as packed
 * FP32 pairs.  enable = 0 selects the general one-shot-per-block kernel
 * (relaybp_autotune tunes whichever is selected); warps = warps per block of
 * the two-shot kernel, 0 for the built-in choice.  Per-edge learned weights
 * (relaybp_set_learned) and the other storage precisions always use the
 * general kernel.  RELAYBP_ERR_UNSUPPORTED when enable = 1 and the DEM's
 * rows are too long; RELAYBP_ERR_INVALID for warps outside 0..32. */
int relaybp_set_pair_kernel(relaybp_handle *h, int32_t enable, int32_t warps);

/* Latency mode (Sec. 6.1, Table 5; App. F, Table 12 measure decoding latency
 * one shot at a time): decode each shot with a thread-block cluster of
 * `cluster` CTAs (1..16; 0 turns it off) instead of one block.  CTA c of a
 * cluster owns a contiguous 1/cluster of the check rows and of the 32-variable
 * groups and keeps their state in its shared memory; the other CTAs read it
 * through distributed shared memory.  The iteration is the one-block FP32
 * kernel's, operation for operation, so outputs are equal bit for bit.
 * Applies to FP32 handles without learned parameters, in relaybp_decode_batch,
 * relaybp_decode_batch_noalloc, relaybp_decode_timed and relaybp_decode_host
 * (trace and flagged decodes keep the one-block kernels).  A launch runs as
 * many clusters as fit on the GPU, each taking the next shot from the work
 * counter.  Builds the cluster's row-slot and column-code layout now (device
 * memory ~ 4 * (cluster * rows_per_cta_rounded * 32 * ceil(max row degree / 32)
 * + nnz) bytes).  RELAYBP_ERR_UNSUPPORTED if the handle is not FP32, a row has
 * more than 256 entries, or a CTA's share of the state does not fit in shared
 * memory. */
int relaybp_set_cluster_kernel(relaybp_handle *h, int32_t cluster);

/* Tail offload: shots that need many relay legs finish on thread-block
 * clusters.  The decode kernel (the two-shot FP32 kernel or the one-shot
 * kernel for every storage form but FP64) hands a shot over when it is about
 * to start leg `legs` (>= 1; 0 turns offload off) -- its marginals M as
 * stored, best solution with its FP64 weight, and solution / leg / iteration
 * counts -- and one launch of the cluster kernel (clusters of `cluster` CTAs,
 * 1..16, as in relaybp_set_cluster_kernel, same storage form) on the same
 * stream continues those shots from that leg.  A new leg restarts the
 * messages at zero, the residual restarts consistent with e^ = 0, and the
 * kernels evaluate the same operations in the same order, so every output
 * equals that of a decode without offload, bit for bit.  Up to `max_shots`
 * shots per launch are handed over (0: 256; device memory ~ max_shots * 4 *
 * (V + V / 32) bytes); later ones stay where they are.  A shot that runs every
 * leg takes about 60,000 iterations: seconds on one SM, a fraction of that on
 * a cluster, so a batch no longer waits on its slowest shot.  Applies to
 * relaybp_decode_batch, relaybp_decode_batch_noalloc, relaybp_decode_host
 * and relaybp_group_decode (one cluster launch per offloading DEM after the
 * group launch) and relaybp_decode_timed (a handed-over shot keeps its start
 * time); not to traced or flagged decodes, message carry-over,
 * per-edge learned weights, or row-tied learned weights and knots in the legs
 * being handed over (legs must be >= the learned legs).  Turning the cluster
 * kernel on for every shot (relaybp_set_cluster_kernel) turns offload off. */
int relaybp_set_tail_offload(relaybp_handle *h, int32_t legs, int32_t cluster, int64_t max_shots);

/* Classical channel coding (paper Sec. 6.2): BPSK over AWGN and flooding
 * sum-product belief propagation for classical codes such as the ZSZ-2BGA
 * seed codes of Table 2.
 *   relaybp_spa_create: copy a parity-check matrix H (CSR, host memory,
 *     1..4096 columns) to the current device.
 *   relaybp_spa_llr: channel LLRs d_llr [shots][n] (FP64 or FP32 per
 *     `precision`, RELAYBP_MSG_F64 / _F32) of frames shot0.. at noise
 *     deviation sigma: bit c_i is sent as (-1)^{c_i} (d_codewords
 *     [shots][ceil(n/32)], or NULL for the all-zero codeword), y_i = x_i +
 *     sigma z_i with z_i the Box-Muller transform of words 2i, 2i+1 of Philox
 *     stream 2 under key `seed` (u = (w + 0.5) / 2^32, z = sqrt(-2 ln u1)
 *     cos(2 pi u2)), L_i = clip(2 y_i / sigma^2, +-llr_max).  The Gaussian
 *     is computed in FP64 and rounded to `precision`.
 *   relaybp_spa_decode: at most max_iter flooding iterations per frame, the
 *     check update nu = prod sgn(mu) * phi(sum phi(|mu|)) over the row's other
 *     entries, phi(x) = -log tanh(x / 2), every message clipped to
 *     +-llr_max; with early_stop a frame stops at the first iteration whose
 *     hard decision [M < 0] satisfies every check.  Outputs: d_bits
 *     [shots][ceil(n/32)] hard decisions, d_iters[shots], d_valid[shots]
 *     (1 if the decision satisfies every check), d_post [shots][n] final
 *     posteriors (may be NULL).  One warp per frame.
 * Errors as elsewhere; sizes beyond the limits: RELAYBP_ERR_UNSUPPORTED. */
int relaybp_spa_create(const relaybp_csr *H, relaybp_spa **out);
int relaybp_spa_llr(relaybp_spa *h, int32_t precision, const uint32_t *d_codewords, double sigma, double llr_max,
                    uint64_t seed, uint64_t shot0, int64_t shots, void *d_llr, void *cuda_stream);
int relaybp_spa_decode(relaybp_spa *h, int32_t precision, const void *d_llr, int64_t shots, int32_t max_iter,
                       double llr_max, int32_t early_stop, uint32_t *d_bits, int32_t *d_iters, int32_t *d_valid,
                       void *d_post, void *cuda_stream);
int relaybp_spa_destroy(relaybp_spa *h);

/* Sliding-window decoding with a commit region of one round (Sec. 6.1,
 * decoding-latency paragraph: a real-time decoder decodes about d rounds of
 * syndromes once per syndrome-extraction round; the paper names the scheme
 * and does not spell the steps out).  The reading implemented:
 *   - each detector i has a round det_round[i] >= 0 (R = 1 + the largest; a
 *     memory experiment's final data-readout detectors form the last round),
 *     each fault column the least round of its detectors (a column with no
 *     detector is never decoded: its bit of e^ stays 0);
 *   - window t = 0, 1, ... holds the rows of rounds [t, t + window) and the
 *     columns of those rounds; it decodes the residual syndrome r restricted
 *     to its rows with an ordinary handle built from that restriction of H
 *     (same priors, same parameters, same global shot indices -- so each
 *     window draws the memory strengths a whole-DEM decode of that
 *     restriction would);
 *   - the columns of round t are committed (all of the window's columns in
 *     the last window, the first with t + window >= R): their bits join e^
 *     and their detector sets are XORed into r, which clears round t whenever
 *     the window converged.
 * max(R - window, 0) + 1 windows; window >= R is one whole-DEM decode.
 *
 * relaybp_windows_create: H, priors, obs, params as relaybp_build (the whole
 *   DEM, host memory); det_round [C] host.  Builds every window's handle now
 *   (RELAYBP_ERR_INVALID naming the window if a window has no row or no
 *   column, or if a row of a window keeps a single entry).
 * relaybp_windows_decode: d_syndromes [shots][ceil(C/32)] device; shot indices
 *   shot0 .. shot0 + shots - 1.  Outputs (device, each may be NULL):
 *   d_corrections [shots][ceil(V/32)] the committed e^; d_pred_obs
 *   [shots][ceil(K/32)] O e^; d_residual [shots][ceil(C/32)] H e^ + s (zero
 *   when every window converged); d_converged [shots] 1 iff every window
 *   converged.  Per window: one gather launch, the window's decode launch(es)
 *   and one commit launch, all on cuda_stream; scratch grows on demand.
 * relaybp_windows_handle: borrow window t's handle (owned by the windows
 *   object), e.g. to choose its kernel; relaybp_windows_info: window and
 *   round counts. */
int relaybp_windows_create(const relaybp_csr *H, const double *priors, const relaybp_csr *obs,
                           const int32_t *det_round, int32_t window, const relaybp_params *params,
                           relaybp_windows **out);
int relaybp_windows_info(const relaybp_windows *w, int32_t *n_windows, int32_t *n_rounds);
int relaybp_windows_handle(relaybp_windows *w, int32_t t, relaybp_handle **out);
int relaybp_windows_decode(relaybp_windows *w, const uint32_t *d_syndromes, uint64_t shot0, int64_t shots,
                           uint32_t *d_corrections, uint32_t *d_pred_obs, uint32_t *d_residual,
                           int32_t *d_converged, void *cuda_stream);
int relaybp_windows_destroy(relaybp_windows *w);

/* Free the handle and every device allocation it owns (synchronises its
 * device first).  NULL is accepted. */
int relaybp_destroy(relaybp_handle *h);

/* Message describing the last error on the calling thread ("" if none). */
const char *relaybp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RELAYBP_H */
