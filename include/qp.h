/*
 * qp.h - C ABI of the GB300 MACGIC-iQUAPI path-update library (libqp.so).
 *
 * The library propagates the reduced density matrix rho(t) of an M-state
 * system linearly coupled to a harmonic bath (paper Sec. 2, Eq. tot_ham) by
 * the iterative quasi-adiabatic path integral with the MACGIC mask and the
 * pre-merging order of Sec. 3.1.  One call of qp_step advances the stored
 * path set Omega(t-1) -> Omega(t):
 *
 *   1. pre-merge: paths identical on the shifted mask P' are merged; the
 *      group keeps its largest-weight path and the summed weight
 *      (Sec. 3.1 "Pre-merging", routine premerging());
 *   2. extension by all M^2 new forward/backward points, each child weighted
 *      by the bare propagator (Eqs. SysP0, SysP) and the influence factor of
 *      the new point (Eq. inf_fun with Toeplitz coefficients eta_d);
 *   3. filter: children with |amplitude| < theta are dropped (Sec. 2.1);
 *   4. rho(t): surviving children summed by end point (Eq. quapi_red_rho).
 *
 * Conventions
 *   - hbar = 1.  Every function returns qp_status and never aborts, throws or
 *     prints; qp_last_error(ctx) gives a one-line reason for the last failure.
 *   - Host arrays passed in are caller-owned and copied before the call
 *     returns; host arrays passed out are written before the call returns.
 *   - Device memory: the library performs no device allocation.  The caller
 *     provides one device workspace (size from qp_workspace_size, 256-byte
 *     aligned), which must outlive the context.  All device work is ordered
 *     on the CUDA stream given to qp_create (a cudaStream_t passed as void*;
 *     NULL = the legacy default stream).
 *   - Calls that read results back (qp_read_*, qp_sync, qp_export_paths)
 *     synchronise the stream and report device-side errors (capacity
 *     overflow of the path buffers or of the merge table).  After such an
 *     error the context refuses qp_step with QP_ERR_STATE until qp_set_rho0
 *     restarts the propagation.
 *   - Packed path key: a stored path is the window of its newest
 *     min(t+1, dkmax) points.  With bs = max(1, ceil(log2 M)) bits per state
 *     and b = 2*bs bits per point, window position p (0 = newest point)
 *     occupies bits [b*p, b*p + b) of a uint64: s+ in the low bs bits, s- in
 *     the high bs bits.  Requires b * dkmax <= 64.
 *   - Supported system sizes: 2 <= M <= 4.
 *   - Not thread-safe per context; distinct contexts are independent.
 */
#ifndef QP_H
#define QP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QP_OK = 0,
    QP_ERR_ARG = 1,       /* invalid argument or configuration            */
    QP_ERR_OOM = 2,       /* workspace too small / host allocation failed */
    QP_ERR_CUDA = 3,      /* a CUDA runtime call failed                   */
    QP_ERR_CAPACITY = 4,  /* path buffer or merge table overflowed        */
    QP_ERR_TIMEOUT = 5,   /* a bounded device-side wait gave up           */
    QP_ERR_STATE = 6      /* call not valid in the context's state        */
} qp_status;

enum { QP_FP64 = 0,       /* complex128 amplitudes, FP64 everywhere */
       QP_C64 = 1 };      /* complex64 amplitudes, FP32 influence exponent
                             with compensated (Kahan) sums; FP64 eta and rho.
                             Group sums of the pre-merge: FP64 in the merge
                             table; in the stream engine the FP32 members are
                             added in FP32 with every rounding error kept in
                             a second word (TwoSum) and the pair is rounded
                             once to FP32, the precision of the children   */

enum { QP_ENGINE_AUTO = 0,    /* library picks: the stream engine where the
                                 mask allows it, else the merge table; the
                                 workspace holds both                         */
       QP_ENGINE_HASH = 1,    /* device open-addressing table keyed by the
                                 masked key (any mask, batches)                 */
       QP_ENGINE_STREAM = 2   /* order-preserving stream: groups stay
                                 contiguous, merge = segmented reduction
                                 (masks whose P' is a prefix {0..k-1}; single
                                 problems with M = 2 also allow one more
                                 position).  Stored paths live in n_inst * M*M
                                 regions of max_paths / (n_inst * M*M)
                                 entries, by (instance, newest point).  The
                                 workspace holds no merge table: about
                                 2 * (8 + amplitude bytes) per path.          */ };

typedef struct {
    int M;                 /* number of system states (DVR points), 2..4            */
    int dkmax;             /* memory length Delta k_max (window points), >= 1       */
    double dt;             /* Trotter time step                                     */
    const double *q;       /* [M] coupling eigenvalues q_i of Eq. tot_ham           */
    const double *hs_re;   /* [M*M] row-major real part of H_S (Hermitian)          */
    const double *hs_im;   /* [M*M] row-major imaginary part of H_S (NULL = 0)      */
    int precision;         /* QP_FP64 or QP_C64                                     */
    int engine;            /* QP_ENGINE_*                                            */
    double theta;          /* filter threshold on |amplitude| (0 = keep all)        */
    int64_t max_paths;     /* capacity of each stored-path buffer, entries,
                              1 .. 2^40 (post-merging: below 2^32)           */
    int64_t max_groups;    /* capacity of the merge table, groups (0 = max_paths),
                              at most 2^30: with max_paths > 2^30 it must be
                              set unless engine is QP_ENGINE_STREAM (which has
                              no merge table)                                */
    int rho_history;       /* rho(t) slots kept on the device, ring (0 = 4096),
                              at most 2^24                                   */
    int n_inst;            /* independent instances propagated together (0 or 1 =
                              one problem; at most 128).  All instances share M,
                              q, H_S, dt, dkmax, mask and theta; each has its own
                              eta (qp_set_eta_instance).  The instance index is
                              stored above the path bits of the key (the stream
                              engine keeps it in the region and adds it on
                              export), so b*dkmax + ceil(log2 n_inst) <= 64.   */
    int scheme;            /* QP_PREMERGE (0) or QP_POSTMERGE: the order of merging
                              and propagation (see below)                      */
} qp_config;

/* Order of merging and propagation.
 *   QP_PREMERGE  the pre-merging order of Sec. 3.1: the stored set is merged on
 *                the shifted mask P' before it is extended (the engines of
 *                qp_config.engine).
 *   QP_POSTMERGE the original order of Sec. 2.1 (Scheme macgic): every stored
 *                path is extended by its M^2 children with its own history, the
 *                survivors of the filter form the unmerged set Omega(t,
 *                unmerged), which is sorted by its masked key (stable radix sort
 *                on the device) and merged on the mask P itself once the window
 *                is full: every run of equal masked keys becomes one stored path,
 *                the child of largest weight with the run's summed amplitude.
 *                max_paths is then the capacity of the unmerged set (M^2 times
 *                the stored set at most); single problems only (n_inst <= 1);
 *                qp_config.engine is ignored; graph launches only.            */
enum { QP_PREMERGE = 0, QP_POSTMERGE = 1 };

/* Spectral density J(w) = (pi/2) ohmic_alpha w exp(-w/ohmic_wc)
 *                       + the resonance of Eq. sharpSD with Omega = res_w0,
 *                         width 2 pi kappa Omega = res_gamma and amplitude
 *                         fixed by lambda = int J/w dw = res_lambda.
 * A part is off when its strength (ohmic_alpha, res_lambda) is 0.          */
typedef struct {
    double beta;           /* inverse temperature 1/kT                              */
    double ohmic_alpha, ohmic_wc;
    double res_w0, res_gamma, res_lambda;
} qp_bath;

typedef struct {
    int64_t t;             /* time step index of the stored set              */
    int64_t groups;        /* parents of the step (entries after pre-merge;
                              post-merging: the stored paths extended)       */
    int64_t extended;      /* children generated, groups * M^2               */
    int64_t kept;          /* stored paths after the step (pre-merging: the
                              children surviving the filter; post-merging:
                              the merged set)                                */
    int64_t intermediate;  /* largest set of the step: pre-merging = kept;
                              post-merging: the unmerged survivors           */
} qp_step_stats;

/* Launch shape and table size of the step (qp_set_tuning / qp_autotune). */
enum { QP_LAUNCH_GRAPH = 0,        /* CUDA graphs of the step's kernels          */
       QP_LAUNCH_PERSISTENT = 1 }; /* one cooperative kernel for all steps of a
                                      qp_step call, bounded grid barriers between
                                      phases (merge-table engine) or steps
                                      (batches on the stream engine); single
                                      problems on the stream engine run graphs  */
typedef struct {
    int mode;                  /* QP_LAUNCH_*                                     */
    int insert_blocks_per_sm;  /* pre-merge kernels (graph mode)                 */
    int expand_blocks_per_sm;  /* extension kernel (graph mode)                  */
    int persistent_blocks;     /* grid of the persistent kernel                  */
    int graph_steps;           /* steps captured per CUDA graph launch           */
    int table_log2;            /* active merge-table slots = 2^table_log2        */
    int engine;                /* engine of the running propagation (QP_ENGINE_HASH
                                  or QP_ENGINE_STREAM; read-only, set at
                                  qp_set_rho0 from qp_config.engine and the mask) */
    int stream_tile;           /* stream engine: stored paths per tile, 256, 512
                                  or 1024 (0 in qp_set_tuning: unchanged;
                                  batches take 512 for 256); its grid is
                                  min(expand_blocks_per_sm, co-resident blocks
                                  per SM) blocks per SM                      */
} qp_tuning;

typedef struct qp_ctx qp_ctx;

/* Library version (major*10000 + minor*100 + patch). */
int qp_version(void);

/* Static string for a status code. */
const char *qp_status_string(qp_status s);

/* Device bytes the caller must provide to qp_create for this configuration.
 * Validates cfg against the limits stated on the fields of qp_config
 * (QP_ERR_ARG on an invalid one; no context exists yet to hold the reason).
 * Host only, no GPU needed.                                                 */
qp_status qp_workspace_size(const qp_config *cfg, size_t *bytes);

/* Create a context on the current CUDA device.  d_workspace: device pointer,
 * 256-byte aligned, at least qp_workspace_size bytes, owned by the caller.
 * cuda_stream: cudaStream_t or NULL.  On success *out is a new context in
 * the "no initial state" phase (call qp_set_eta, optionally qp_set_mask,
 * then qp_set_rho0 before stepping).                                       */
qp_status qp_create(const qp_config *cfg, void *d_workspace, size_t bytes,
                    void *cuda_stream, qp_ctx **out);

/* Release the host side of the context (the workspace stays the caller's).
 * Does not wait for work already queued on the context's stream: synchronise
 * that stream before the workspace is freed or reused.  Safe on NULL.       */
void qp_destroy(qp_ctx *ctx);

/* Influence coefficients eta_0 .. eta_{n-1} from a spectral density (paper
 * Eq. inf_fun; explicit forms per its refs): with the point q_k held on the
 * box ((k-1) dt, k dt] and alpha(t) = (1/pi) int J [coth(beta w/2) cos wt -
 * i sin wt] dw,
 *   eta_0 = (1/pi) int J/w^2 [coth(beta w/2)(1 - cos w dt) - i (w dt - sin w dt)] dw
 *   eta_d = (4/pi) int J/w^2 sin^2(w dt/2) [coth(beta w/2) cos(w d dt) - i sin(w d dt)] dw.
 * Host FP64 adaptive Gauss-Legendre quadrature; no GPU needed.  re/im: [n]
 * caller-owned outputs.                                                     */
qp_status qp_eta_from_bath(const qp_bath *bath, double dt, int n, double *eta_re, double *eta_im);

/* Set eta_0 .. eta_{dkmax-1} (n >= dkmax; extra entries ignored).  Builds the
 * device tables of the history sum and of propagator x new-point influence. */
qp_status qp_set_eta(qp_ctx *ctx, const double *eta_re, const double *eta_im, int n);

/* Q(t) = int_0^t dt' int_0^t' dt'' alpha(t'') at t = j h, j = 0 .. n-1 (the
 * double integral of the bath correlation function of qp_eta_from_bath, whose
 * second differences are the coefficients of full intervals).  Host FP64
 * quadrature, no GPU needed; re/im: [n] caller-owned; 1 <= n <= 8192.      */
qp_status qp_Q_from_bath(const qp_bath *bath, double h, int n, double *re, double *im);

/* The symmetric Trotter splitting of Eq. quapi_red_rho ("applying a
 * symmetric Trotter splitting"; Eq. inf_fun sums from point 0 to point N)
 * instead of the right-box reading of qp_eta_from_bath: point k holds the
 * bath over the interval centred on k dt, point 0 over [0, dt/2] and the
 * newest point over [t - dt/2, t].  Given Q at multiples of dt/2,
 * Qh[j] = Q(j dt/2) for j = 0 .. n-1 (n >= 2 dkmax + 1, Qh[0] = 0; e.g. from
 * qp_Q_from_bath with h = dt/2), the library forms the interior coefficients
 * (which replace those of qp_set_eta), the coefficients of point 0 and of
 * the newest point with every other point, and the half-interval self terms
 * (memory cut at lags >= dkmax).  The stored amplitudes carry point 0's half
 * interval and treat the newest point as interior (as it will be once later
 * points exist); rho(t) multiplies every surviving child by the difference
 * between its newest point's end-point and interior factors.  Merge-table
 * engine, pre-merging order, single problems (QP_ERR_STATE otherwise: set
 * engine QP_ENGINE_HASH or QP_ENGINE_AUTO).  Takes effect at the next
 * qp_set_rho0; qp_set_eta returns to the right-box reading.  Host arrays
 * copied before the call returns.                                          */
qp_status qp_set_end_points(qp_ctx *ctx, const double *qh_re, const double *qh_im, int n);

/* eta of one instance of a batched context (after qp_set_eta, which sets
 * every instance).  inst in [0, n_inst).                                    */
qp_status qp_set_eta_instance(qp_ctx *ctx, int inst, const double *eta_re, const double *eta_im, int n);

/* MACGIC mask P: the window positions at time t (0 = newest) on which paths
 * must agree to merge (Sec. 2.1).  Must contain 0, and 1 when dkmax >= 2;
 * positions in [0, dkmax).  The pre-merge uses P' = {p-1 : p in P, p >= 1}
 * plus position 0 (the paper's mask[i] -> mask[i]+1 shift, Sec. 3.1).
 * positions == NULL or n == 0: the full mask (plain iQUAPI).  Takes effect
 * from the next qp_step.                                                     */
qp_status qp_set_mask(qp_ctx *ctx, const int *positions, int n);

/* Restart the propagation at t = 0 from rho(0) (M*M row-major, Hermitian):
 * one stored path per nonzero element.  im may be NULL (real rho0).  Clears
 * any device error state.  Requires qp_set_eta to have been called.         */
qp_status qp_set_rho0(qp_ctx *ctx, const double *rho0_re, const double *rho0_im);

/* Enqueue nsteps propagation steps on the context's stream (asynchronous;
 * errors raised on the device surface at the next synchronising call).     */
qp_status qp_step(qp_ctx *ctx, int nsteps);

/* Wait for the stream; report a device-side error if one was raised.       */
qp_status qp_sync(qp_ctx *ctx);

/* Current time step and number of stored paths (synchronises).              */
qp_status qp_current(qp_ctx *ctx, int64_t *t, int64_t *n_paths);

/* rho(t) for count consecutive steps t0 .. t0+count-1 (synchronises): the
 * reduced density matrix of Eq. quapi_red_rho, the surviving children of
 * each step summed by end point (Sec. 3.2).  Each step must be among the
 * last rho_history steps (QP_ERR_ARG otherwise).  re/im:
 * [count][n_inst][M*M] (n_inst = 1 for a single problem), caller-owned.
 * The device state and the rows are copied in one round trip.              */
qp_status qp_read_rho(qp_ctx *ctx, int64_t t0, int count, double *rho_re, double *rho_im);

/* The same rows without waiting: enqueues on the context's stream the sum of
 * the last step's block partials (stream engine) and the copy of rho(t) for
 * t = t0 .. t0+count-1 into dst, interleaved (re, im) FP64,
 * [count][n_inst][M*M] (the layout of a complex128 array).  dst is host
 * memory owned by the caller, at least count*n_inst*M*M*16 bytes.
 * Page-locked memory that the device can address (cudaMallocHost, a pinned
 * tensor) is written by the finalising kernel itself; other memory receives
 * a cudaMemcpyAsync (synchronous for pageable memory).
 * The values are in place once qp_sync (or any synchronising call) returns;
 * device errors are reported there.  The range is checked against the steps
 * enqueued since qp_set_rho0 (QP_ERR_ARG outside the last rho_history).    */
qp_status qp_read_rho_async(qp_ctx *ctx, int64_t t0, int count, double *dst);

/* Stored paths of each instance after step t: kept[n_inst] (synchronises). */
qp_status qp_read_instance_counts(qp_ctx *ctx, int64_t t, int64_t *kept);

/* Per-step path counts for steps t0 .. t0+count-1 (1 <= t, synchronises);
 * totals over all instances.                                               */
qp_status qp_read_stats(qp_ctx *ctx, int64_t t0, int count, qp_step_stats *out);

/* Copy the stored path set Omega(t) to host arrays: keys[cap] packed keys,
 * amps[2*cap] interleaved (re, im) as FP64 whatever the precision.  *n gets
 * the number of stored paths; QP_ERR_CAPACITY (nothing copied) if > cap.
 * The order of the entries is unspecified.                                   */
qp_status qp_export_paths(qp_ctx *ctx, uint64_t *keys, double *amps, int64_t cap, int64_t *n);

/* Run nsteps propagation steps like qp_step, but launch the kernels one by
 * one with CUDA events between them, and add each kernel's elapsed time in
 * milliseconds to kernel_ms[k] (synchronises).  Kernel order, merge-table
 * engine: k = 0 merge insert, 1 merge tie-break, 2 extension/filter/rho,
 * 3 step finalisation; stream engine: k = 0 regular map (no time where it is
 * not launched), 2 tile kernel.  Each step starts with a 50 us delay kernel,
 * so that the intervals hold device time, not host enqueue time.
 * nk = length of kernel_ms (at most 4 entries are written).               */
qp_status qp_profile_steps(qp_ctx *ctx, int nsteps, double *kernel_ms, int nk);

/* Current launch shape and table size.                                      */
qp_status qp_get_tuning(qp_ctx *ctx, qp_tuning *out);

/* Set the launch shape and table size (validated against the device: the
 * persistent grid must be co-resident, the table at most the workspace's).  */
qp_status qp_set_tuning(qp_ctx *ctx, const qp_tuning *t);

/* Autotuner: time trial_steps steps for each candidate launch shape and
 * table size (graph mode with 2/4/8 blocks per SM for the pre-merge and
 * extension kernels and, for hashed tables, smaller tables; persistent mode
 * with 1/2/4 blocks per SM) and keep the fastest.  The propagation advances
 * by (trial_steps + 1) steps per candidate.  Results are cached per problem
 * bucket (M, dkmax, n_inst, precision, mask, filter on/off, log2 of the path
 * count); with use_cache the cached choice is applied without trials
 * (*best_ms_per_step = -1 then).  best / best_ms_per_step may be NULL.    */
qp_status qp_autotune(qp_ctx *ctx, int trial_steps, int use_cache, qp_tuning *best, double *best_ms_per_step);

/* Test hook for the bounded waits of the persistent kernel: corrupts the grid
 * barrier's arrival count so that the next persistent launch cannot complete
 * its first barrier; every block gives up after about two seconds, the step
 * is not applied and the next synchronising call returns QP_ERR_TIMEOUT.
 * qp_set_rho0 restores a usable context.                                    */
qp_status qp_test_stall_barrier(qp_ctx *ctx);

/* Sharded propagation over several GPUs (the distributed pre-merge of
 * Sec. 3.2 in a GPU form).  One context per rank holds the stored paths the
 * rank owns: a path belongs to the owner of its next pre-merge group,
 *   owner = ((key & B) * 0x9E3779B97F4A7C15 mod 2^64) / 2^32  mod n_ranks,
 * B = the key bits of the pre-merge positions P' (qp_set_mask), so every
 * group of the next pre-merge lies on one rank.  A step on n ranks: each
 * rank runs qp_step(ctx, 1) on its paths (rho(t) of the context is the
 * rank's part: the sum over ranks is rho(t)), partitions its stored set by
 * owner (qp_partition_paths), exchanges the parts (an all-to-all, outside
 * the library) and replaces its set with what it received
 * (qp_import_paths).  Needs the merge-table engine (QP_ENGINE_HASH), the
 * pre-merging order and a single problem (QP_ERR_STATE otherwise).
 *
 * qp_partition_paths: copies the stored set Omega(t) into d_keys (uint64)
 * and d_amps (interleaved (re, im) in the context's precision: FP64 or FP32)
 * grouped by owner, rank 0's paths first; counts[n_ranks] gets the paths per
 * rank.  Device buffers owned by the caller, cap entries each
 * (QP_ERR_CAPACITY when the set is larger).  1 <= n_ranks <= 1024.
 * Synchronises.                                                            */
qp_status qp_partition_paths(qp_ctx *ctx, int n_ranks, uint64_t *d_keys, void *d_amps, int64_t cap, int64_t *counts);

/* Replaces the stored set of the current time step with n paths from device
 * arrays (the layout qp_partition_paths writes), copied before the call
 * returns (synchronises).  n <= max_paths (QP_ERR_CAPACITY).              */
qp_status qp_import_paths(qp_ctx *ctx, const uint64_t *d_keys, const void *d_amps, int64_t n);

/* Test hook for the bounded wait of the stream engine's look-back (the wait
 * of a tile for the survivor counts of the tiles before it, Sec. 3.1 order
 * of the stored set): the first tile of the next stream-engine step publishes
 * no count, so the step's other tiles wait for it until their bounded wait
 * gives up (about two seconds).  Tiles whose wait gave up write nothing, the
 * step is not applied and the next synchronising call returns
 * QP_ERR_TIMEOUT; qp_set_rho0 restores a usable context.  QP_ERR_STATE when
 * the running propagation is not on the stream engine.                    */
qp_status qp_test_stall_lookback(qp_ctx *ctx);

/* Test hook: out[i] = in[i] widened from FP32 to FP64 exactly as the step
 * kernels widen FP32 amplitudes and partial sums before FP64 arithmetic
 * (IEEE-754 field arithmetic in integer registers, all classes: zeros,
 * subnormals, normals, infinities, NaNs).  in, out: device pointers, n
 * entries (0 <= n <= 2^31); asynchronous on stream (NULL = default stream).
 * QP_ERR_ARG for bad arguments, QP_ERR_CUDA if the launch fails.            */
qp_status qp_test_widen(const float *in, double *out, int64_t n, void *stream);

/* Last error message of the context ("" if none).                           */
const char *qp_last_error(const qp_ctx *ctx);

/* One propagation step t -> t+1 that allocates nothing and needs no context.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory -- a plug-in running inside a host program
 * that owns all GPU memory through its own pool and offers no allocator, a
 * real-time loop that may not call cudaMalloc (it can block and synchronise
 * the device), or a process under a hard device-memory quota.
 *
 * It runs the same step kernels as qp_step (FP64 path only) on the caller's
 * buffers.  All scratch (merge table, eta tables, partial sums) lives in one
 * fixed array of 20 MiB of device memory inside the library, which every GPU
 * that loads the library holds until the process exits.  Limits set by that
 * array: n_in <= 2^20 stored paths, at most 2^16 merge groups in the step,
 * dkmax <= 16 (and 2 <= M <= 4 as everywhere).  Larger inputs return
 * QP_ERR_ARG; more than 2^16 groups or more survivors than cap_out return
 * QP_ERR_CAPACITY (*n_out = 0).  No cudaMalloc, cudaFree or other allocating
 * routine is called.
 *
 *   cfg          as for qp_create; precision must be QP_FP64; max_paths,
 *                max_groups, rho_history and engine are ignored
 *   eta_re/im    host [n_eta >= dkmax] influence coefficients eta_0..
 *   mask/n_mask  as for qp_set_mask (NULL/0 = full mask)
 *   t            time index of the input set (it holds the newest
 *                min(t+1, dkmax) points of each path)
 *   d_keys_in    device [n_in] packed keys of the input set
 *   d_amps_in    device [2*n_in] amplitudes, (re, im) interleaved
 *   d_keys_out   device [cap_out] keys of the set at t+1 (no aliasing)
 *   d_amps_out   device [2*cap_out] its amplitudes, (re, im) interleaved
 *   n_out        host: number of stored paths at t+1
 *   rho_re/im    host [M*M]: rho(t+1)
 *   cuda_stream  cudaStream_t or NULL; the call synchronises it
 *
 * The first call on a device looks up the device address of the array
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call reuses the same array and clears
 * what must start at zero; calls that overlap on one GPU (several host
 * threads or streams) race on the array and must be serialised by the
 * caller.                                                                   */
qp_status qp_step_noalloc(const qp_config *cfg, const double *eta_re, const double *eta_im, int n_eta,
                          const int *mask, int n_mask, int64_t t,
                          const uint64_t *d_keys_in, const double *d_amps_in, int64_t n_in,
                          uint64_t *d_keys_out, double *d_amps_out, int64_t cap_out,
                          int64_t *n_out, double *rho_re, double *rho_im, void *cuda_stream);

/* ===================================================================== */
/* Learned surrogate of rho(t).  The paper has no counterpart: a small MLP
 * over the last L steps of rho(t) and the bath parameters, trained on
 * trajectories of the path update above, extends propagation in time; the
 * path update checks it at checkpoints and is its fallback.
 *
 * Network: x (d_in) -> tanh(x W1 + b1) (width) -> tanh(. W2 + b2) (width)
 * -> . W3 + b3 (d_out); loss = mean squared error.  Parameters are FP32;
 * every matrix product reads BF16 copies of weights and activations and
 * accumulates in FP32 on the tensor cores.  Parameter vector layout (FP32):
 * W1 [d_in x width] row-major, b1 [width], W2 [width x width], b2 [width],
 * W3 [width x d_out], b3 [d_out].  Device workspace and stream as for
 * qp_create (caller-owned; the library allocates nothing).               */
typedef struct qp_mlp qp_mlp;

qp_status qp_mlp_workspace_size(int d_in, int width, int d_out, int max_batch, size_t *bytes);
qp_status qp_mlp_create(int d_in, int width, int d_out, int max_batch, void *d_workspace, size_t bytes,
                        void *cuda_stream, qp_mlp **out);
/* Release the host side (as qp_destroy: synchronise the stream before the
 * workspace is freed or reused).                                           */
void qp_mlp_destroy(qp_mlp *m);
qp_status qp_mlp_num_params(const qp_mlp *m, int64_t *n);
/* Host FP32 parameters in (resets the Adam moments and step count) / out. */
qp_status qp_mlp_set_params(qp_mlp *m, const float *params);
qp_status qp_mlp_get_params(qp_mlp *m, float *params);
/* y = net(x): d_x [batch x d_in], d_y [batch x d_out], FP32 device, async.  */
qp_status qp_mlp_forward(qp_mlp *m, const float *d_x, int batch, float *d_y);
/* Forward and backward without update (synchronises): gradients of the loss
 * w.r.t. all parameters into host grads [num_params] (NULL = skip), loss.   */
qp_status qp_mlp_gradients(qp_mlp *m, const float *d_x, const float *d_target, int batch, float *grads,
                           double *loss);
/* One Adam step (bias-corrected) on the batch; loss != NULL synchronises
 * and returns the loss before the update.                                 */
qp_status qp_mlp_train_step(qp_mlp *m, const float *d_x, const float *d_target, int batch, float lr, float beta1,
                            float beta2, float eps, double *loss);
const char *qp_mlp_last_error(const qp_mlp *m);

/* Training windows from device rho trajectories d_rho [T][n_inst][4]
 * (complex FP64, the layout of qp_read_rho's output for M = 2): for
 * instances inst0 .. inst0+ninst_used-1 and target times t_begin <= t <
 * t_end (t_begin >= L): features = Re, Im of rho_00, rho_01, rho_10, rho_11
 * at t-L .. t-1 (8 L values), then the instance's n_par parameters
 * d_par [n_inst x n_par]; target = (rho(t) - rho(t-1)) * out_scale (8
 * values).  d_x [rows x (8 L + n_par)], d_target [rows x 8], rows =
 * ninst_used * (t_end - t_begin), instance-major.  Async on the stream.   */
qp_status qp_surrogate_windows(const double *d_rho, int n_inst, int L, const float *d_par, int n_par, int t_begin,
                               int t_end, int inst0, int ninst_used, float out_scale, float *d_x, float *d_target,
                               void *cuda_stream);

/* Autoregressive rollout of n trajectories held in d_hist [n][T][8] (FP32,
 * same 8 reals as above; steps < t_from must be filled): for t = t_from ..
 * t_to-1, rho(t) = rho(t-1) + net(window) / out_scale with the increment
 * made traceless, projected onto Hermitian matrices and then onto positive
 * semidefinite ones of the same trace (a density matrix).  d_xbuf [n x d_in]
 * and d_ybuf [n x 8] (device floats) are kept in the signature; the rollout
 * packs its input in the model's workspace and does not write them.  The steps run
 * in one cluster launch (qp_mlp_set_rollout_mode below) or as CUDA graphs
 * of up to 32 steps captured on the model's stream at the first call with
 * these arguments and replayed (the step index lives on the device; on the
 * legacy default stream they are launched one by one).  Synchronous: the
 * rollout is complete when the call returns.                              */
qp_status qp_surrogate_rollout(qp_mlp *m, float *d_hist, int n, int T, int L, const float *d_par, int n_par,
                               int t_from, int t_to, float out_scale, float *d_xbuf, float *d_ybuf);

/* How qp_surrogate_rollout runs its steps.  QP_ROLLOUT_AUTO (the default):
 * all steps in one launch of a two-block cluster (k_rollout_fused: block 0
 * holds W1^T in shared memory and packs the features, runs layer 1 and the
 * update; block 1 holds W2^T and W3^T and runs layers 2 and 3; the
 * activations cross through distributed shared memory, two cluster
 * barriers per step, no launch per step) when n <= 32, the model has 8
 * outputs and the weights fit shared memory; otherwise the CUDA graphs of
 * step kernels described above.  QP_ROLLOUT_GRAPH forces the graphs;
 * QP_ROLLOUT_FUSED forces the cluster kernel (QP_ERR_ARG when it does not
 * fit).  Both use the same rounding points and the same order of the
 * k-steps, and give the same trajectories.                                 */
enum { QP_ROLLOUT_AUTO = 0, QP_ROLLOUT_GRAPH = 1, QP_ROLLOUT_FUSED = 2 };
qp_status qp_mlp_set_rollout_mode(qp_mlp *m, int mode);

/* ------------------------------------------------------------------------
 * Wide keys: the path update with keys of up to 128 bits (M <= 8 states,
 * dkmax <= 16 points; the production models of Sec. 4.3 need M = 8 at
 * dkmax = 12, beyond one 64-bit word).  A separate context over the same
 * qp_config (precision, theta, max_paths, max_groups, rho_history; single
 * problems, pre-merging order): the merge-table form, with the pre-merge on
 * a 64-bit key of 6 bits per position of P' (so P' may hold at most 10
 * positions, and at most 10 positions may lie outside it) and the tie rule
 * of the narrow engines (reading R4: the smallest key among the members
 * within the tie window of the largest weight).
 *
 * Key layout (exported as two words per path, lo then hi): one byte per
 * window position p = 0 .. dkmax-1 (0 = newest point), byte p of the
 * 128-bit number lo + 2^64 hi; forward state in its low nibble, backward
 * state in its high nibble.  Numerically this orders keys as the narrow
 * packing does (oldest position first, backward state before forward).
 * Semantics of eta, the mask and rho0 as the narrow calls above.          */
typedef struct qp_wide qp_wide;
qp_status qp_wide_workspace_size(const qp_config *cfg, size_t *bytes);
/* d_workspace: device memory of at least qp_wide_workspace_size bytes,
 * owned by the caller and alive until qp_wide_destroy; q and hs are copied. */
qp_status qp_wide_create(const qp_config *cfg, void *d_workspace, size_t bytes, void *cuda_stream, qp_wide **out);
/* Release the host side (as qp_destroy: synchronise the stream before the
 * workspace is freed or reused).                                           */
void qp_wide_destroy(qp_wide *w);
qp_status qp_wide_set_eta(qp_wide *w, const double *eta_re, const double *eta_im, int n);
/* Default: the full mask, refused at qp_wide_set_rho0 when its P' holds more
 * than 10 positions (set a mask first).                                    */
qp_status qp_wide_set_mask(qp_wide *w, const int *positions, int n);
qp_status qp_wide_set_rho0(qp_wide *w, const double *rho0_re, const double *rho0_im);
/* nsteps steps on the context's stream; reads the step index first
 * (synchronises once per call).  Capacity overflows surface as
 * QP_ERR_CAPACITY at the next synchronising call.                          */
qp_status qp_wide_step(qp_wide *w, int nsteps);
qp_status qp_wide_current(qp_wide *w, int64_t *t, int64_t *n);
qp_status qp_wide_read_rho(qp_wide *w, int64_t t0, int count, double *re, double *im);
qp_status qp_wide_read_stats(qp_wide *w, int64_t t0, int count, qp_step_stats *out);
/* keys[2 cap] (lo, hi per path), amps[2 cap] (re, im, FP64).               */
qp_status qp_wide_export_paths(qp_wide *w, uint64_t *keys, double *amps, int64_t cap, int64_t *n);
const char *qp_wide_last_error(const qp_wide *w);

#ifdef __cplusplus
}
#endif
#endif /* QP_H */
