/*
 * pt.h -- C ABI of the GB300 (sm_103a) Parallel-Tempering engine for the smoothed-cubic
 * 4-body random-laser model of arXiv 2511.13508.
 *
 * The model (paper Sec. II): N complex mode amplitudes a_k on the complete mode-locked comb
 * graph (omega_k = k), quadruplets a<b<c<d with a+d = b+c (frequency matching condition,
 * Eq. (1)), real Gaussian couplings J_q, Hamiltonian Eq. (4)
 *     H = -cc * sum_q J_q Re( conj(a_a) a_b a_c conj(a_d) ),   cc = 2 ("+ c.c."),
 * sampled from P[a] ~ exp(-beta H) delta(N - sum_k |a_k|^4) (Eq. (8)) with the
 * constraint-preserving pair Metropolis move (Sec. III.A.1) and exchange Monte Carlo between
 * neighbouring temperatures (Sec. III.A.2, Eq. (15)).  Observables: energy moments for the
 * specific heat (Eq. (21)), the replica overlap q and its 201-bin histogram (Sec. IV.C), the
 * inverse participation ratios Y2, Y4 (Sec. IV.D).
 *
 * Conventions shared by every call:
 *  - S disorder samples, sample s has N[s] modes (even, 4 <= N <= 512), R replicas and n_T
 *    temperatures (ascending, index 0 = coldest).  A "chain" is one (sample, replica,
 *    temperature) configuration; canonical chain order is (s, r, t), t fastest.
 *  - Complex arrays are interleaved (re, im) doubles; a state array holds, in canonical chain
 *    order, N[s] complex amplitudes per chain (total sum_s N[s]*R*n_T complex numbers).
 *  - Every call returns an int status: PT_OK (0) or a negative PT_E* code.  No call aborts or
 *    throws.  pt_last_error() gives a static, human-readable message for the last failure.
 *  - Random numbers come from Philox4x32-10 (Salmon et al., SC'11) with key = seed and
 *    counters (stream, sweep, update, tag); the streams are documented in the design notes and
 *    make a run reproducible bit-for-bit for a given precision, seed and kernel configuration.
 *  - Device work runs asynchronously on the stream given to pt_create; calls that return host
 *    data (pt_measure, pt_get_state, pt_fields, pt_energy, pt_save) synchronise that stream.
 */
#ifndef PT_H
#define PT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define PT_OK 0
#define PT_EINVAL (-1)       /* bad argument: N odd or out of range, temps not ascending/positive, ... */
#define PT_ENOMEM (-2)       /* device or host allocation failed */
#define PT_ECUDA (-3)        /* a CUDA runtime call failed (message in pt_last_error) */
#define PT_ETIMEOUT (-4)     /* a bounded device wait or the host watchdog ran out */
#define PT_ENAN (-5)         /* non-finite coupling, or non-finite state found at resync */
#define PT_ESTATE (-6)       /* checkpoint bytes do not match this context */
#define PT_EUNSUPPORTED (-7) /* valid request the library does not implement */

/* ---------------------------------------------------------------- precision */
#define PT_PREC_FP32 0       /* FP32 fields/moves, FP64 running energy, resync, swap log-ratio */
#define PT_PREC_FP64 1       /* the same J-sharing kernels in FP64 throughout */
#define PT_PREC_FP64_PLAIN 2 /* the paper's GPU design restated: one thread per quadruplet term of
                                Delta E, tree reduction, one chain per thread block, no J sharing, FP64 */

#define PT_QBINS 201 /* overlap histogram: bins centred at -1, -0.99, ..., 1 */
#define PT_NSTAT 7   /* per (sample, T): n, sumE, sumE^2, sumY2, sumY4, sumI, sumI^2  (I = sum |a|^2) */
#define PT_NQSTAT 5  /* per (sample, T): n, sum q, sum q^2, sum q^3, sum q^4 over replica pairs */

/* Optional device allocator (e.g. PyTorch's caching allocator).  alloc returns NULL on failure. */
typedef void *(*pt_alloc_fn)(size_t bytes, void *user);
typedef void (*pt_free_fn)(void *ptr, void *user);

typedef struct pt_config {
    int precision;        /* PT_PREC_*; default PT_PREC_FP32 */
    double cc_factor;     /* multiplier of the quadruplet sum in H; default 2 ("+ c.c." of Eq. (4)) */
    int swap_every;       /* sweeps between swap passes (paper: 64); 0 = only on pt_swap() */
    int measure_every;    /* sweeps between measurements; 0 = never */
    int resync_every;     /* sweeps between renormalisation + full FP64-accumulated H; 0 = never */
    int chains_per_block; /* chains sharing one J stream inside a thread block: 0 = tuned, or 8/16/32 */
    int sweeps_per_unit;  /* sweeps in one scheduling unit of the persistent kernel; 0 = tuned */
    int blocks_per_sm;    /* persistent thread blocks per SM; 0 = tuned */
    int consumer_warps;   /* field-computing warps per thread block (plus one copy warp); 0 = tuned.  FP32:
                           * 7, 11 or 15 with 8 or 16 chains per block, 3, 7, 9 or 11 with 32; FP64: 7 with 8
                           * chains, 3 with 16 (PT_EINVAL otherwise) */
    int use_graphs;       /* replay each sweep segment as a captured CUDA graph (default 1) */
    int watchdog_ms;      /* host watchdog on synchronising calls; 0 = wait forever (default 600000) */
} pt_config;

/* Fills *cfg with the defaults above.  Cannot fail. */
void pt_config_default(pt_config *cfg);

typedef struct pt_ctx pt_ctx; /* opaque; owned by the library */

/* Observable accumulators, copied out by pt_measure into caller-owned buffers (any may be NULL).
 * Layouts (C order):  stat [S][n_T][PT_NSTAT]   qstat [S][n_T][PT_NQSTAT]   qhist [S][n_T][PT_QBINS]
 *                     swap_acc, swap_att [S][R][n_T-1]    mc_acc, mc_att [S][n_T]
 * stat and qstat count one entry per chain (stat) or replica pair (qstat) per measurement. */
typedef struct pt_observables {
    double *stat;
    double *qstat;
    uint64_t *qhist;
    uint64_t *swap_acc;
    uint64_t *swap_att;
    uint64_t *mc_acc;
    uint64_t *mc_att;
    uint64_t *gm_acc;   /* [S][n_T] learned global moves accepted / attempted (zero without them) */
    uint64_t *gm_att;
} pt_observables;

/* Canonical quadruplet list of the N-mode comb (paper Sec. II.C "Graph generation"; Eq. (1) with
 * omega_k = k): every a<b<c<d with a+d = b+c, lexicographic in (a,b,c).  Writes 4*count int32 to
 * abcd when abcd != NULL; *count receives the count.  This is the order of J in pt_create.
 * PT_EINVAL if N < 4 or N > 512 or count == NULL. */
int pt_enumerate_quads(int N, int32_t *abcd, int64_t *count);

/* Creates a context and uploads everything; the host->device boundary is crossed here.
 *  cfg        NULL = defaults.
 *  S, N[S]    samples and their mode counts (each even, 4..512).
 *  J          couplings of all samples back to back, each in canonical quadruplet order;
 *  J_offsets  [S+1] start of each sample in J (J_offsets[s+1]-J_offsets[s] must equal the count).
 *  n_T, temps temperatures (positive, strictly ascending).
 *  replicas   R >= 1 (overlaps need R >= 2).
 *  seed       Philox key.  Initial chains are exact draws of the beta = 0 law (uniform on the
 *             constraint surface), then E = H(a) is computed on the device.
 *  alloc/free optional device allocator (both or neither); alloc_user is passed through.
 *  stream     cudaStream_t to run on; NULL = a non-blocking stream owned by the context (the legacy
 *             default stream cannot be captured into CUDA graphs).
 * Caller keeps ownership of every input array; they are copied.  On failure *out is NULL. */
int pt_create(pt_ctx **out, const pt_config *cfg, int S, const int32_t *N, const double *J,
              const int64_t *J_offsets, int n_T, const double *temps, int replicas, uint64_t seed,
              pt_alloc_fn alloc, pt_free_fn free_, void *alloc_user, void *stream);

/* Random-frequency mode-locked graph (paper Sec. II.C "Quenched random frequencies" and "Graph generation",
 * Eq. (1) with the linewidth of Eq. (gamma_scaling), gamma = 1/(2(N-1)) for frequencies in [0,1]).
 *  omega  [N] mode frequencies, strictly ascending (the modes are indexed in frequency order).
 *  gamma  linewidth of the matching condition, > 0.
 * For every 4-subset a<b<c<d, each of its three splittings into a conjugated pair {p,q} and a plain
 * pair {u,v} with |omega_p + omega_q - omega_u - omega_v| < gamma is one interaction with its own
 * coupling; it is written as (p, u, v, q) so that its term of H is -cc J Re(conj(a_p) a_u a_v conj(a_q)).
 * Order: by (a, b, c, d), then splitting {a,d}|{b,c}, {a,b}|{c,d}, {a,c}|{b,d}.  With omega_k = k/(N-1)
 * the list is exactly that of pt_enumerate_quads.  Writes 4*count int32 to quads when quads != NULL.
 * PT_EINVAL for N outside 4..512, a non-ascending omega, gamma <= 0 or count == NULL.  Host code. */
int pt_fmc_graph(int N, const double *omega, double gamma, int32_t *quads, int64_t *count);

/* As pt_create, on explicit interaction lists instead of the comb: sample s has the quadruplets
 * quads[4 q_offsets[s] .. 4 q_offsets[s+1]) in term order (term -cc J Re(conj(a_q0) a_q1 a_q2 conj(a_q3)),
 * the four modes distinct and < N[s]) and the couplings J[q_offsets[s] .. q_offsets[s+1]) (q_offsets[0] = 0);
 * every N[s] even, 4..2048.
 * Runs on the quadruplet-list paths: PT_PREC_FP64_PLAIN (one thread block per chain, FP64) or PT_PREC_FP32
 * (one thread block per 8 chains of a sample, which read each quadruplet once for all 8; FP32 products,
 * FP64 energies); PT_EUNSUPPORTED for PT_PREC_FP64.  pt_fields and pt_autotune are unsupported on these
 * paths.  PT_EINVAL for a bad index or offsets.  The caller keeps ownership of the arrays. */
int pt_create_graph(pt_ctx **out, const pt_config *cfg, int S, const int32_t *N, const int32_t *quads,
                    const double *J, const int64_t *q_offsets, int n_T, const double *temps, int replicas,
                    uint64_t seed, pt_alloc_fn alloc, pt_free_fn free_, void *alloc_user, void *stream);

/* Runs n_sweeps Monte Carlo sweeps (one sweep = N/2 pair updates per chain, Sec. III.A.1) on every
 * chain, asynchronously.  After each completed sweep t (counted from creation) the schedule is:
 * resync if t % resync_every == 0, measure if t % measure_every == 0, swap pass if
 * t % swap_every == 0.  All chains of one sample update the same (j,k) pair sequence. */
int pt_sweep(pt_ctx *ctx, int64_t n_sweeps);

/* One sequential swap pass over every (sample, replica) temperature ladder, ascending in T
 * (Sec. III.A.2, Eq. (15)); exchanges temperature labels, asynchronously. */
int pt_swap(pt_ctx *ctx);

/* Renormalises every chain onto sum|a|^4 = N and recomputes E = H(a) in full (asynchronous). */
int pt_resync(pt_ctx *ctx);

/* Measures every chain now (same accumulators as the schedule), asynchronously. */
int pt_measure_now(pt_ctx *ctx);

/* Copies the accumulated observables into *out (synchronous). */
int pt_measure(pt_ctx *ctx, pt_observables *out);

/* Zeroes all accumulators (e.g. after burn-in; paper Sec. III.B uses the last half of the run). */
int pt_reset_observables(pt_ctx *ctx);

/* State in canonical chain order: a (interleaved complex doubles) and/or E (doubles); NULL skips. */
int pt_get_state(pt_ctx *ctx, double *a, double *E);

/* Replaces every chain's amplitudes (canonical order, as pt_get_state) and recomputes E on the
 * device.  The state is taken as given (not renormalised). */
int pt_set_state(pt_ctx *ctx, const double *a);

/* Full recompute of H for every chain of the current state, canonical order, without changing it. */
int pt_energy(pt_ctx *ctx, double *E);

/* Per-step local fields (the sweep kernel's field phase, Sec. III.A.3): for the pair (j,k) and every
 * chain of sample s, writes 8 doubles per chain in canonical (r, t) order:
 *   h_j, h_k   (complex) local fields, H = -cc Re(conj(a_l) h_l) + terms without a_l;
 *   B_jk       (complex) sum over quadruplets {j,m,k,y}, j+m = k+y, of J conj(a_m) a_y;
 *   A_jk       (complex) sum over quadruplets {j,k,x,y}, x+y = j+k, of J a_x a_y;
 * so that Delta H = -cc Re[ conj(dj) h_j + conj(dk) h_k + conj(dj) dk B_jk + conj(dj) conj(dk) A_jk ]
 * for a_j += dj, a_k += dk.  Not available for PT_PREC_FP64_PLAIN (PT_EUNSUPPORTED). */
int pt_fields(pt_ctx *ctx, int sample, int j, int k, double *out);

/* Update trace of the sweep kernel itself (Sec. III.A.1 pair move, Sec. III.A.3 parallel Delta E): runs
 * the next sweep exactly as pt_sweep(ctx, 1) would (same kernel, block shape and graph, then the schedule
 * due after it) while the production kernel records pair update `update` (0 <= update < N/2) of that
 * sweep for every chain of every sample with N[s]/2 > update.  Outputs, canonical (s, r, t) order:
 *   rec [n_chains][PT_TRACE_REC] doubles: j, k, h_j (re, im), h_k (re, im), B_jk (re, im), A_jk (re, im)
 *       as the kernel reduced them (definitions as in pt_fields), the proposed a_j', a_k' (re, im each),
 *       the Metropolis uniform U, the kernel's Delta H, accepted (0/1), beta, the running energy before the
 *       update, and 1.0 for a written record (0.0 everywhere for chains that were not traced);
 *   a   optional (NULL = not wanted), state layout of pt_get_state: every traced chain's amplitudes just
 *       before the update, in the kernel's precision widened to double.
 * Contexts of pt_create_graph (the FP32 quadruplet-list kernels) reduce the j-k cross term for the kernel's
 * own proposal instead of B_jk and A_jk: there fields 6..9 hold Re sum_{q holding j and k} J_q (product of
 * the other two factors) dx_j dx_k (dx = conj(d) at positions 0 and 3, d at 1 and 2; the energy change is
 * then -cc Re[conj(dj) h_j + conj(dk) h_k] - cc * field 6) and three zeros.
 * Caller-owned host buffers; the call synchronises the context's stream.  The first call allocates the device
 * buffer of the trace (n_chains * PT_TRACE_REC + 2 * (state size) doubles) and re-captures the sweep graphs.
 * PT_EINVAL for an update outside [0, max N/2); PT_ENOMEM if that buffer cannot be allocated;
 * PT_EUNSUPPORTED for PT_PREC_FP64_PLAIN. */
#define PT_TRACE_REC 20
int pt_trace_update(pt_ctx *ctx, int update, double *rec, double *a);

/* Checkpoint.  pt_save with buf == NULL stores the needed size in *len; otherwise writes *len bytes
 * (PT_EINVAL if *len is too small).  pt_load restores a checkpoint of a context created with the
 * same arguments (PT_ESTATE otherwise); resuming is bit-identical to an uninterrupted run. */
int pt_save(pt_ctx *ctx, void *buf, size_t *len);
int pt_load(pt_ctx *ctx, const void *buf, size_t len);

/* Autotuner of the sweep blocks (chains per block, field warps, sweeps per scheduling unit): times
 * every supported shape for trial_sweeps sweeps on the live ensemble, keeps the fastest and restores
 * the ensemble (state, counters, accumulators) exactly as before the call.  chosen (optional, 3 ints)
 * receives {chains_per_block, consumer_warps, sweeps_per_unit}.  PT_EUNSUPPORTED for the plain path. */
int pt_autotune(pt_ctx *ctx, int trial_sweeps, int *chosen);

/* The sweep-block shape pt_create picks when pt_config.chains_per_block and consumer_warps are 0, for a batch of
 * n_samples samples whose largest mode count is max_n (even, 4..512), chains_per_sample = replicas x
 * temperatures, on a device with sm_count multiprocessors (0: unknown).  Host-only, no device call: writes
 * *chains_per_block (8, 16 or 32) and *consumer_warps.  The rule (measured on GB300): 8 chains from N = 160 on;
 * for 48 <= N < 160 the most chains per block (32 below N = 96, else 16, then 8) that still give at least 0.8 x
 * sm_count groups; 16 chains below N = 48; 8 when a sample has at most 8 chains; 11 field warps from N = 48 on,
 * else 7.  FP64: 8 x 7 from N = 128 on, else 16 x 3.  precision: PT_PREC_FP32 or PT_PREC_FP64 (PT_EINVAL
 * otherwise, and for out-of-range arguments or NULL outputs). */
int pt_default_shape(int precision, int max_n, int n_samples, int chains_per_sample, int sm_count,
                     int *chains_per_block, int *consumer_warps);

/* ---- Learned global-move proposal (built for this engine; the paper has none).  A per-sample masked,
 * block-autoregressive MLP (two hidden layers of 256, BF16 weights on the tensor cores, FP32 accumulate
 * and FP32 master weights with Adam) gives a normalised density q over gauge-fixed coordinates: global
 * phase and comb gauge removed (phi~_0 = phi~_1 = 0), intensity fractions s_k = |a_k|^4/N stick-broken into
 * logit-normal v_k, phases phi~_k wrapped Cauchy, conditioned on the temperature index among the n_cold
 * coldest.  A global move replaces a cold chain's configuration by a draw from q with a fresh uniform
 * gauge and accepts it with the exact Metropolis-Hastings ratio
 *   log A = -beta (H' - H) + [log q(x) + extra(x)] - [log q(x') + extra(x')],
 * where log q is the log density of (v_k, phi~_k) and extra = -sum_{k<=N-2} log r_k + 1/2 sum_k log s_k
 * (r_k = sum_{i>=k} s_i) turns it into the density on the constraint surface relative to the beta = 0 law
 * of Eq. (8), prod_k s_k^(-1/2) ds dphi; so the tempered target stays invariant whatever the network has
 * learned.  All samples must share one N in {16, 32, 48, 64}.
 *
 * pt_learn_init: allocates the networks and buffers.  n_cold: temperatures 0..n_cold-1 are conditioned
 *   and moved; batch: training rows per sample and step (multiple of 128); data_per_sample: capacity of
 *   the training set; seed: initial weights.  PT_EUNSUPPORTED for other N. */
int pt_learn_init(pt_ctx *ctx, int n_cold, int batch, int data_per_sample, uint64_t seed);

/* Runs `rounds` times: `every` sweeps (full schedule), then appends the configurations of the chains at the
 * n_cold coldest temperatures (n_cold * R per sample) to the training set, until it is full. */
int pt_collect(pt_ctx *ctx, int64_t every, int rounds);

/* `steps` Adam steps (learning rate lr) on the mean negative log-likelihood of random minibatches of the
 * training set.  losses (optional, steps doubles): mean -log q on the constraint surface per step. */
int pt_train(pt_ctx *ctx, int steps, double lr, double *losses);

/* One round of global moves on the n_cold coldest temperatures of every ladder (asynchronous). */
int pt_global_move(pt_ctx *ctx);

/* Schedules a round of global moves every `every` sweeps inside pt_sweep (0 = off); it runs after the
 * resync and before the measurement of the same sweep. */
int pt_set_global_every(pt_ctx *ctx, int every);

/* Range of the move's first resampled block of modes (8 blocks of N/8 modes): every proposal draws it
 * uniformly from {lo, ..., hi} (from its own random stream, independently of the state).  Block 0 draws a
 * whole new configuration under a fresh gauge; block b > 0 keeps modes < b N/8, the gauge and the tail
 * mass r_{bN/8} of the current configuration and redraws the tail from q's conditionals, with the same
 * exact acceptance ratio (the kept modes' terms cancel).  Default {0, ..., 7}.  PT_EINVAL outside 0..7. */
int pt_set_global_blocks(pt_ctx *ctx, int lo, int hi);

/* How a move's autoregressive sampling runs: one_launch != 0 (the default) runs the network passes of all mode
 * blocks and the draws in one launch with the network's weights held on chip, when the proposal rows per
 * sample (n_cold x replicas) are at most 64; one_launch == 0 (or more rows) launches a network pass and a
 * sampling kernel per block.  Both draw identical proposals (same random streams, same arithmetic).
 * PT_EINVAL before pt_learn_init. */
int pt_set_global_sampler(pt_ctx *ctx, int one_launch);

/* FP32 master parameters of all samples, [S][psize] (layout from pt_learn_shape): set != 0 uploads them
 * (and refreshes the BF16 copies), set == 0 downloads them. */
int pt_learn_params(pt_ctx *ctx, float *params, int set);

/* 14 int64: N, H, Din, Dout, n_cold, psize, offsets of W1 [H][Din], b1 [H], C1 [n_cold][H], W2 [H][H], b2,
 * W3 [Dout][H], b3 [Dout] within one sample's parameters, and the number of collected configurations. */
int pt_learn_shape(pt_ctx *ctx, int64_t *out);

/* Evaluates the proposal on given configurations: a = [S][rows][N] interleaved complex doubles, cond =
 * [S][rows] temperature indices (< n_cold).  logq [S][rows] receives log q (network part), extra (optional)
 * [S][rows] the coordinate terms -sum log r_k + 1/2 sum log s_k (log q + extra = log density on the
 * constraint surface), grad (optional, [S][psize] floats, rows % 8 == 0) the gradient of the mean over the
 * rows of -log q with respect to the parameters.  rows <= max(batch, n_cold * R rounded up to 128). */
int pt_learn_eval(pt_ctx *ctx, const double *a, const int *cond, int rows, double *logq, double *extra,
                  float *grad);

/* Health check of the failure detection: launches a one-thread kernel that waits, bounded by limit_ms
 * (1..60000), on a device flag that no kernel sets, so the wait always runs out and records the timeout
 * status the engine's own bounded waits record.  Returns what the synchronising calls then report,
 * PT_ETIMEOUT, and clears the status afterwards, so the context stays usable with its state untouched.
 * PT_EINVAL for a bad limit; another code if the context already carried an error. */
int pt_check_wait(pt_ctx *ctx, int limit_ms);

/* Counters: sweeps done since creation, swap passes done. */
int pt_counters(pt_ctx *ctx, int64_t *sweeps_done, int64_t *swap_passes);

/* Waits for the context's stream under the watchdog; reports device-side errors. */
int pt_sync(pt_ctx *ctx);

/* Frees everything; NULL-safe. */
int pt_destroy(pt_ctx *ctx);

/* Message of the last failing call on ctx (or of the last failing pt_create when ctx is NULL). */
const char *pt_last_error(const pt_ctx *ctx);

/* Batched tensor-core GEMM used by the learned global-move proposal (the paper has none): for every
 * b < batch, D[b] = A[b] * B[b]^T with A[b] an M x K and B[b] an N x K row-major BF16 matrix
 * (device pointers, batches back to back) and D[b] an M x N row-major FP32 matrix, accumulated in FP32
 * on the sm_100-class tensor cores (tcgen05.mma, accumulator in tensor memory).  Constraints:
 * 16 <= N <= 256, N % 16 == 0, K % 8 == 0, K >= 16.  Asynchronous on stream.  PT_EINVAL / PT_ECUDA;
 * message in pt_last_error(NULL). */
int pt_gemm_bf16(int batch, int M, int N, int K, const void *A, const void *B, float *D, void *stream);

/* Allocation-free FP64 energies of a batch of chains.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory (a program whose device memory belongs to
 * another runtime's pool, a real-time loop where cudaMalloc/cudaFree would synchronise the device, a
 * plug-in limited to the buffers its host hands it).  It computes the same H as pt_energy of a
 * PT_PREC_FP64_PLAIN context, one thread block per chain.
 *  N         modes, 4 <= N <= 64 (PT_EINVAL otherwise: the working table has room for the 20336
 *            quadruplets of the 64-mode comb).
 *  n_chains  chains (0 returns PT_OK at once).
 *  J         device pointer: the N-mode couplings in canonical quadruplet order (pt_enumerate_quads).
 *  a         device pointer: n_chains * N complex amplitudes, interleaved (re, im) doubles, chain-major.
 *  E         device pointer: n_chains doubles receive H of each chain.
 *  cc        multiplier of the quadruplet sum (2 for the paper's "+ c.c.").
 *  stream    cudaStream_t (NULL = legacy default stream); the call is asynchronous on it.
 * Caller owns J, a and E.  The call allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine): its working table is a static device array of 20336 int4 (325 KB) that every GPU loading
 * the library holds until exit.  Every call rewrites the part of the table it uses, so a call never
 * sees stale contents, but all calls share the one table: calls that overlap on the GPU (other streams
 * or threads, same device) race and must be serialised by the caller.  The table's device address is
 * only valid in the CUDA context in which it was looked up (cudaGetSymbolAddress): a call made while
 * `stream` is not capturing looks it up again in the context current on the calling thread and records it
 * for that context; a call made during stream capture uses the address an earlier call recorded for the
 * current context, so make the first call in each context before any stream capture (PT_EINVAL
 * otherwise).  Errors: PT_EINVAL (arguments), PT_ECUDA (a CUDA error left pending by earlier work on the
 * thread, no context, lookup or launch failure, each with the CUDA error string); the message is in
 * pt_last_error(NULL). */
int pt_energy_fp64_static(int N, int n_chains, const double *J, const double *a, double *E, double cc,
                          void *stream);

/* Incidence records of the FP32 quadruplet-list kernels (the sweep of pt_create_graph contexts), built on the
 * host exactly as pt_create_graph builds them, for inspection and tests; no device work.  For a list of nq
 * quadruplets of N modes (term order: the term of quadruplet (q0, q1, q2, q3) is J conj(a_q0) a_q1 a_q2
 * conj(a_q3), Sec. II.C with Eq. (4)):
 *   offsets [N+1]    records of mode l are rec[offsets[l] .. offsets[l+1]), one per quadruplet holding l, in
 *                    list order;
 *   rec [4 nq][4]    int32 (A, B, C, w): the three other modes as row offsets mode * 8 of the kernels'
 *                    amplitude table, ordered so that the record's contribution to the local field of l
 *                    (Sec. III.A.3, H = -cc Re(conj(a_l) h_l) + terms without l) is J a_A a_B conj(a_C);
 *                    w = position of l | positions of A, B, C << 2, 4, 6;
 *   recJ [4 nq]      J of the record's quadruplet in FP32.
 * Caller-owned host buffers.  PT_EINVAL for N outside [4, 2048], nq < 0 or above 2^28, a mode index out of
 * range or a NULL buffer. */
int pt_graph_records(int N, int64_t nq, const int32_t *quads, const double *J, int32_t *offsets, int32_t *rec,
                     float *recJ);

/* ---- Measurement probe (not part of the paper's method).  The sweep is bound by FP32 arithmetic, so its
 * roofline is the FP32 fused multiply-add throughput of the GPU it runs on, measured here instead of derived
 * from unit counts and a nominal clock.  Launches `blocks` x `threads` threads, each running 8 independent
 * fused multiply-add chains for `iters` iterations: packed != 0 issues them as paired FP32 FMAs (two per
 * instruction), packed == 0 as scalar FMAs; either way 32 flops per thread and iteration, so one launch
 * does blocks * threads * iters * 32 flops.  sink: caller-owned device buffer of blocks * threads floats
 * (written only in a case that cannot occur; it keeps the arithmetic alive).  Asynchronous on `stream`
 * (cudaStream_t, NULL = legacy default stream): time it with events on that stream.  Errors: PT_EINVAL
 * (threads not a multiple of 32 in [32, 1024], blocks or iters < 1, NULL sink), PT_ECUDA (launch);
 * message in pt_last_error(NULL). */
int pt_fma_probe(int packed, int blocks, int threads, int iters, float *sink, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PT_H */
