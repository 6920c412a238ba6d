/*
 * ess.h -- C ABI of the GB300 linear elliptical slice sampler.
 *
 * Samples x ~ N(0, I_d) restricted to the polytope D = {x : A x <= b},
 * A of shape m x d (Wu & Gardner, arXiv 2407.10449, Sec. 1), by running many
 * independent elliptical-slice chains (Alg. 1).  Each chain step:
 *   1. draws nu ~ N(0, I_d)                                  (Alg. 1)        
 *   2. forms q = A nu for all chains (one GEMM) and carries p = A x as
 *      p cos(theta) + q sin(theta), refreshed every refresh_k steps
 *   3. solves a_i.x cos(theta) + a_i.nu sin(theta) = b_i in closed form
 *      (Eq. trigonometry-equation, App. B) with the Sec. 3.2 edge cases
 *   4. builds the active intervals I_act by sorting the left endpoints and a
 *      cumulative max of the right endpoints (Alg. 3, Prop. 1)
 *   5. draws theta uniformly on I_act                        (Alg. 1)        
 *   6. moves x <- x cos(theta) + nu sin(theta)                (Alg. 1)        
 *      and rejects an infeasible move (Sec. 3.3).
 *
 * Conventions for every entry point:
 *   - Matrices are dense and row-major.  "device" pointers are CUDA global
 *     memory of the current device; "host" pointers are ordinary CPU memory.
 *   - The library never takes ownership of caller memory; ess_create copies
 *     A and b.  Work buffers belong to the ess_state and are freed by
 *     ess_destroy.
 *   - Every function returns an ess_status.  On failure ess_last_error()
 *     returns a human-readable message for the calling thread.  No function
 *     aborts the process or traps the GPU.
 *   - cuda_stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is enqueued on that stream; the call returns
 *     after the work is complete only where stated.
 */
#ifndef ESS_GB300_H
#define ESS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ess_state ess_state;

typedef enum {
    ESS_OK = 0,
    ESS_ERR_ARG = 1,            /* bad size, NULL pointer, NaN/Inf input */
    ESS_ERR_INFEASIBLE_X0 = 2,  /* a start point violates A x <= b (Alg. 1 needs x0 in D) */
    ESS_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    ESS_ERR_NUMERIC = 4,        /* NaN/Inf appeared in theta or x on the device */
    ESS_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up */
    ESS_ERR_OOM = 6,            /* device allocation failed */
    ESS_ERR_UNSUPPORTED = 7     /* size or mode outside what the kernels support */
} ess_status;

typedef enum {
    ESS_PREC_FP64 = 0,          /* every step in double precision */
    ESS_PREC_MIXED = 1          /* q = A nu by FP16x3 tensor cores, FP32 step,
                                   FP64 near-tangent arccos, A x refresh and
                                   feasibility residual */
} ess_precision;

typedef enum {
    ESS_REFRESH_FP64 = 0,       /* p = A x with FP64 fused multiply-adds */
    ESS_REFRESH_SPLIT = 1       /* p = A x exactly on BF16 tensor cores with an
                                   error-free fixed-point split, rounded once */
} ess_refresh_mode;

typedef enum {
    ESS_PRODUCTS_DFMA = 0,      /* FP64 form: q = A nu and p = A x with FP64
                                   fused multiply-adds (plain FP64) */
    ESS_PRODUCTS_SPLIT = 1      /* FP64 form: both products on BF16 tensor
                                   cores from 56-bit fixed-point splits of both
                                   operands (integer slices of w <= 8 bits,
                                   every slice product exact in the FP32
                                   accumulator, the pairs combined error-free,
                                   rounded once to double): error below
                                   d (3 + K(K-1)/2) 2^-(wK) max|a_i| max|x|
                                   (e.g. 4e-13 relative to that at d = 1000)
                                   plus N^2 2^-48 sum_j |a_ij x_j| for the
                                   N = K(K+1)/2 slice products */
} ess_products_mode;

typedef struct {
    int precision;              /* ess_precision; default ESS_PREC_FP64 */
    int refresh_k;              /* p = A x recomputed when t % refresh_k == 0;
                                   default 32; 1 = every step */
    int refresh_mode;           /* ess_refresh_mode; default ESS_REFRESH_SPLIT
                                   for the mixed form (the FP64 form always
                                   uses ESS_REFRESH_FP64) */
    double tangent_thresh;      /* mixed form: arccos argument b/r evaluated in
                                   FP64 when |b/r| > 1 - tangent_thresh;
                                   default 1e-4 */
    double trim_eps;            /* Sec. 3.3 trimming of constraint endpoints
                                   (radians); default 0 */
    double residual_margin;     /* rows with p_i > b_i - residual_margin*||a_i||
                                   get their residual a_i.x - b_i recomputed in
                                   FP64; default 1e-8 (FP64 form), 2e-4 (mixed) */
    int sort_threads;           /* 0 (default): one warp per chain, with a
                                   CTA per chain for chains that keep more than
                                   128 arcs after the domination prune;
                                   > 0: a CTA per chain for every chain, of
                                   sort_threads threads rounded up to a power
                                   of two (at least the width that holds m
                                   arcs, at most 1024).  For m > 8192 the CTA
                                   per chain is the wide-row kernel (512
                                   threads, rows streamed), whatever the value */
    int autotune;               /* 0 (default): tile widths and the sort path
                                   from a cost model; 1: ess_chains_init times
                                   the candidates on the loaded chains and keeps
                                   the fastest (see ess_get_tuning) */
    int q_tile;                 /* mixed form, tile of the q = A nu GEMM:
                                   0 (default): cost model (or the autotuner);
                                   BN in {64, 128, 160, 192, 224, 256}: one SM
                                   per tile of 128 chains x BN rows of A;
                                   2000 + BN, BN in {128, ..., 256}: a pair of
                                   SMs (tcgen05 cta_group::2) per tile of 256
                                   chains x BN rows, one launch per tile;
                                   3000 + BN: the same tiles in a persistent
                                   kernel, one cluster per SM pair (when m is
                                   not a multiple of 4, 2000 + BN runs).  Any
                                   other value is ESS_ERR_ARG. */
    int fp64_products;          /* FP64 form: ess_products_mode; default
                                   ESS_PRODUCTS_DFMA (ignored by the mixed
                                   form) */
    int wait_limit_us;          /* bounded device waits of the persistent
                                   kernels (ess_run_few's grid barriers; the
                                   batched persistent launch's q dependency
                                   counters and grid barriers): a wait gives
                                   up after this many microseconds and the
                                   call returns ESS_ERR_TIMEOUT; 0 (default):
                                   2 s */
    int reserved[4];
} ess_config;

typedef struct {
    long long steps;            /* chain-steps executed */
    long long rejections;       /* Sec. 3.3 safeguard rejections */
    long long residual_rechecks;/* rows whose FP64 residual was recomputed */
    long long tangent_fp64;     /* near-tangent roots evaluated in FP64 */
    double max_refresh_drift;   /* max |p_carried - p_refresh| / ||a_i|| seen */
    double max_residual;        /* max a_i.x' - b_i over the candidate moves whose row was
                                   rechecked in FP64, including moves the check then
                                   rejected (a positive value means a rejection, not
                                   an infeasible emitted iterate) */
    long long numeric_errors;   /* chains that produced NaN/Inf */
    long long sort_keys;        /* arcs left to sort after dropping dominated ones */
} ess_stats;

/* Fills cfg with the defaults above for the given precision. */
ess_status ess_default_config(int precision, ess_config *cfg);

/*
 * Creates a sampler for D = {x in R^d : A x <= b} (Sec. 1).
 *   A    host, m x d row-major doubles; copied.
 *   b    host, m doubles; copied.
 *   cfg  NULL for ess_default_config(ESS_PREC_FP64).
 *   out  receives the new state.
 * Errors: ESS_ERR_ARG for d < 1, m < 1, NULL pointers or non-finite entries;
 * ESS_ERR_UNSUPPORTED for m or d beyond the kernels' limits (see
 * ess_limits); ESS_ERR_OOM / ESS_ERR_CUDA for device failures.
 */
ess_status ess_create(const double *A, const double *b, int d, int m,
                      const ess_config *cfg, ess_state **out);

/* Releases the state and all its device memory.  NULL is ignored. */
void ess_destroy(ess_state *state);

/*
 * Normal probability Z = P(A x <= b) of the state's polytope for x ~ N(0, I_d)
 * (the normaliser of the truncated normal of Sec. 2), by the
 * Holmes-Diaconis-Ross splitting estimator driven by the chain steps (the use
 * of the sampler the paper cites; the paper gives no algorithm, the steps
 * follow the published method).  Nested domains D_t = {x : A x <= b +
 * gamma_t}, gamma_1 > ... > gamma_T = 0, and Z = prod_t P(D_t | D_(t-1)),
 * each factor estimated by the fraction of n_samples samples of the
 * truncated normal on D_(t-1) lying in D_t; level t's samples come from
 * n_between chain steps on D_(t-1) started from level t - 1's samples inside
 * it (sample j restarts from the (j mod count)-th of them).
 *   Stage 1 (subset simulation) sets the shifts: gamma_t is the midpoint of
 *   the k-th and (k + 1)-th smallest level value g(x) = max_i (a_i.x - b_i)
 *   (k = ceil(rho n_samples)), or 0 once the k-th is <= 0 (the last level).
 *   Stage 2 (HDR) repeats the levels at those shifts with fresh draws.
 * Random numbers: a stage's start samples are the normals of (seed_s, chain
 * j, t = 0, problem 1) of ess_draw_normals' generator; the chains of the step
 * from level t (0-based) take the steps t n_between .. (t + 1) n_between - 1
 * of ess_run's map; seed_s = seed (stage 1), seed + 1 (stage 2).  g is taken
 * in FP64 from FP64 products A x (the exact split of the refresh in the mixed
 * form).
 *   n_samples   samples per level, >= 2, with 1 <= ceil(rho n_samples) <= n_samples - 1
 *   rho         target fraction of samples inside each next domain, 0 < rho < 1
 *   n_between   chain steps between levels, >= 1
 *   max_levels  capacity of shifts / counts / counts_ss
 *   shifts      host, out: gamma_1 .. gamma_T
 *   counts      host, out (or NULL): stage 2's samples inside each level
 *   counts_ss   host, out (or NULL): stage 1's counts
 *   n_levels    host, out: T
 *   log_z       host, out: log of the HDR estimate, sum_t log(counts_t / n_samples)
 *               (-inf if a level held no sample)
 *   log_z_ss    host, out (or NULL): log of stage 1's estimate
 * The state's loaded chains are dropped (load new ones with ess_chains_init);
 * b is restored on return.  Errors: ESS_ERR_ARG; ESS_ERR_UNSUPPORTED when no
 * level reaches the domain within max_levels (the domain may be empty);
 * ESS_ERR_NUMERIC from the chain steps; ESS_ERR_OOM / ESS_ERR_CUDA.
 */
ess_status ess_hdr(ess_state *state, int n_samples, double rho, int n_between, uint64_t seed,
                   int max_levels, double *shifts, int *counts, int *counts_ss, int *n_levels,
                   double *log_z, double *log_z_ss, void *cuda_stream);

/*
 * Largest supported m and d for the state's precision and row count: m up to
 * 2^22 rows; d bounded by the shared memory of the chain-step kernel that
 * takes the state's m (m <= 8192: the CTA-per-chain kernel; larger m: the
 * wide-row kernel, which streams the rows).
 */
ess_status ess_limits(const ess_state *state, int *max_m, int *max_d);

/*
 * Runs n_chains independent chains for n_iter steps (Alg. 1 loop).
 *   X          device, n_chains x d doubles, in/out: start points on entry
 *              (each must satisfy A x <= b), states after the last step on
 *              return.
 *   t0         global index of the first step (chains are reproducible:
 *              the draws of chain c at step t depend only on (seed, c, t));
 *              a run split at a multiple of refresh_k reproduces the unsplit
 *              run bit for bit.
 *   seed       Philox4x32-10 key.
 *   samples    device or NULL; if record_every > 0, receives the state after
 *              every record_every-th step: n_chains x (n_iter / record_every)
 *              x d elements, double for ESS_PREC_FP64, float for
 *              ESS_PREC_MIXED.
 *   cuda_stream  stream for all device work.
 * Synchronous: returns after the work completes (status words are read
 * back).  Errors: ESS_ERR_INFEASIBLE_X0 if a start point is infeasible in
 * FP64; ESS_ERR_NUMERIC if a chain produced NaN/Inf; ESS_ERR_ARG for bad
 * sizes.
 */
ess_status ess_run(ess_state *state, double *X, int n_chains, int t0, int n_iter,
                   uint64_t seed, void *samples, int record_every, void *cuda_stream);

/*
 * The three stages of ess_run, for callers that keep the chains on the device
 * across calls (e.g. to time or graph-capture the steps):
 *   ess_chains_init  copies n_chains start points X (device doubles) into the
 *                    state, checks them in FP64 (ESS_ERR_INFEASIBLE_X0) and
 *                    computes p = A x; the next step has global index t0.
 *                    Synchronous.
 *   ess_chains_step  enqueues n_iter steps of the loaded chains on the stream
 *                    and returns without waiting (samples as in ess_run).
 *                    Device-side errors surface in the next ess_chains_get.
 *                    Unless per-phase timing is on, the steps run on two
 *                    internal streams of the state (the draw of step t + 1
 *                    beside step t), forked from the stream at the call and
 *                    joined back into it before the call returns: work the
 *                    caller enqueues on the stream afterwards runs after
 *                    them, as with plain launches.
 *   ess_chains_get   copies the current states to X (device doubles, may be
 *                    NULL) and reports device-side errors.  Synchronous.
 * ess_step_with_draws and ess_products reuse the work buffers and unload the
 * chains.
 */
ess_status ess_chains_init(ess_state *state, const double *X, int n_chains, int t0,
                           void *cuda_stream);
ess_status ess_chains_step(ess_state *state, int n_iter, uint64_t seed, void *samples,
                           int record_every, void *cuda_stream);
ess_status ess_chains_get(ess_state *state, double *X, void *cuda_stream);

/* Same as ess_run with X and samples in HOST memory: copies X to the device,
 * runs, and copies the final states (and samples) back.  Each record is copied
 * to the host (from one of two device slots, on a stream of its own) while the
 * next record_every steps run; with pinned host buffers the copies overlap the
 * steps.  The device buffers are kept in the state for the next call.  Returns
 * after every copy has finished. */
ess_status ess_run_host(ess_state *state, double *X_host, int n_chains, int t0, int n_iter,
                        uint64_t seed, void *samples_host, int record_every,
                        void *cuda_stream);

/*
 * One chain step with caller-supplied draws (for testing the step map in
 * isolation from the random number generator).
 *   X          device, n_chains x d doubles: current states (must be feasible).
 *   nu         device, n_chains x d doubles: the Gaussian directions.
 *   u          device, n_chains doubles in [0, 1): the theta draw.
 *   X_next     device, n_chains x d doubles: next states.
 *   theta      device or NULL, n_chains doubles.
 *   pieces     device or NULL, n_chains x max_pieces x 2 doubles: the
 *              positive-length pieces [lo, hi] of I_act (after trimming) in
 *              ascending order.
 *   n_pieces   device or NULL, n_chains ints: number of pieces (may exceed
 *              max_pieces; only the first max_pieces are written).
 *   rejected   device or NULL, n_chains ints: 1 if the Sec. 3.3 safeguard
 *              rejected the move.
 * In the mixed form X and nu are rounded to float first, exactly as a run
 * stores them.  p = A x is computed by the refresh path.  Synchronous.
 */
ess_status ess_step_with_draws(ess_state *state, const double *X, const double *nu,
                               const double *u, int n_chains, double *X_next,
                               double *theta, double *pieces, int max_pieces,
                               int *n_pieces, int *rejected, void *cuda_stream);

/*
 * The products the step uses, as the state computes them (for verification):
 * p = A x by the refresh path and q = A nu by the step's GEMM (FP64 FMAs in
 * the FP64 form, the FP16x3 tensor-core GEMM in the mixed form).
 *   X, nu   device, n_chains x d doubles (rounded to float first in the mixed
 *           form, as a run stores them).
 *   P, Q    device, n_chains x m doubles; either may be NULL.
 * Synchronous.  Reference: Sec. 2.2 (the cached A x and A nu).
 */
ess_status ess_products(ess_state *state, const double *X, const double *nu, int n_chains,
                        double *P, double *Q, void *cuda_stream);

/*
 * Philox4x32-10 (Salmon et al., SC'11) as used for all draws, exposed for
 * verification: out[4*i .. 4*i+3] is the block for counter
 * (n_i, chain, t, (problem << 8) | stream) with n_i = i, i < n_blocks.
 * out is device memory (n_blocks x 4 uint32).
 */
ess_status ess_philox_blocks(uint64_t seed, uint32_t chain, uint32_t t, uint32_t problem,
                             uint32_t stream, int n_blocks, uint32_t *out, void *cuda_stream);

/* The normals nu of chains [0, n_chains) at step t, as a run draws them:
 * device n_chains x d, double (FP64 form) or float (mixed form). */
ess_status ess_draw_normals(const ess_state *state, int n_chains, int t, uint64_t seed,
                            void *out, void *cuda_stream);

/*
 * Per-phase device time of ess_chains_step (and ess_run), measured with CUDA
 * events on the run's stream when enabled.  Phases: ESS_PHASE_DRAW (nu),
 * ESS_PHASE_GEMM (q = A nu), ESS_PHASE_CHAIN (roots, sort, sweep, theta,
 * move), ESS_PHASE_REFRESH (p = A x).  ess_get_timing fills up to n_phases
 * entries of ms (total milliseconds) and launches (kernel launches) and
 * synchronizes the device.  Timing is off by default.
 */
#define ESS_PHASE_DRAW 0
#define ESS_PHASE_GEMM 1
#define ESS_PHASE_CHAIN 2
#define ESS_PHASE_REFRESH 3
#define ESS_N_PHASES 4
ess_status ess_set_timing(ess_state *state, int enable);
ess_status ess_get_timing(ess_state *state, double *ms, long long *launches, int n_phases);
ess_status ess_reset_timing(ess_state *state);

/* Accumulated statistics since create or the last ess_reset_stats. */
ess_status ess_get_stats(const ess_state *state, ess_stats *out);
ess_status ess_reset_stats(ess_state *state);

/*
 * App. A change of variables for N(mu, Sigma) with Sigma = L L^T, host side:
 *   A_out = A L (m x d), b_out = b - A mu (m).  mu may be NULL (zero).
 * Sampling u under A_out u <= b_out and mapping x = L u + mu samples the
 * truncation of N(mu, Sigma) by A x <= b.
 */
ess_status ess_whiten(const double *A, const double *b, const double *mu, const double *L,
                      int d, int m, double *A_out, double *b_out);

/* x = L u + mu for each of the n rows of U (host, n x d); mu may be NULL. */
ess_status ess_unwhiten(const double *L, const double *mu, int d, int n, const double *U,
                        double *X);

/*
 * App. A map x = L u + mu on the GPU for many samples (e.g. the recorded
 * samples of a run in whitened coordinates).  ess_whitener_create copies L
 * (host, d x d row-major, any square matrix) and mu (host, d, or NULL) to the
 * current device; ess_whitener_apply computes X = U L^T + mu row by row for
 * n rows of U (device, n x d, row-major):
 *   u_double = 0: U and X float; the product runs on the tensor cores as the
 *                 scaled FP16x3 GEMM of q = A nu (|error| <= (16 + d / 16)
 *                 2^-24 sum_j |L_ij| |u_j| before the FP32 rounding of + mu);
 *   u_double = 1: U and X double; FP64 fused multiply-adds.
 * X must not overlap U.  Synchronous.  Errors: ESS_ERR_ARG for bad sizes or
 * non-finite L or mu, ESS_ERR_TIMEOUT if a bounded device wait gave up.
 */
typedef struct ess_whitener ess_whitener;
ess_status ess_whitener_create(const double *L, const double *mu, int d, ess_whitener **out);
void ess_whitener_destroy(ess_whitener *whitener);
ess_status ess_whitener_apply(ess_whitener *whitener, const void *U, int u_double, int n,
                              void *X, void *cuda_stream);

/*
 * One FP64 chain step that allocates no device memory (the paper has no
 * counterpart; this is a service for callers that may not call cudaMalloc,
 * e.g. plugins whose host framework owns the device-memory budget, or request
 * paths that must stay off the allocator and its implicit synchronization).
 * Same map and results as ess_step_with_draws in the FP64 form, without an
 * ess_state:
 *   A, b        device, m x d row-major and m doubles (the polytope A x <= b).
 *   X, nu, u    device inputs as in ess_step_with_draws (n_chains x d, n_chains x d,
 *               n_chains doubles, row-major, contiguous).
 *   X_next      device output, n_chains x d doubles (must not overlap X).
 *   theta, rejected   device outputs (n_chains doubles / ints) or NULL.
 * All scratch lives in one library-owned device array of
 * ESS_NOALLOC_SCRATCH_BYTES per GPU (allocated when the library is loaded,
 * kept until exit), every region rounded up to 256 bytes: with r(v) = v
 * rounded up to a multiple of 256, 512 + r(8 m) + 2 r(8 n_chains m) bytes
 * must fit (e.g. 512 chains at m = 2000), else ESS_ERR_ARG.  m > 8192, or a d
 * whose x' does not fit the chain-step kernel's shared memory beside the
 * arcs, gives ESS_ERR_UNSUPPORTED (as in ess_create).  Calls share that
 * array: calls that overlap on the GPU race, so serialize them.  The start
 * points are checked in FP64 first: an infeasible X gives
 * ESS_ERR_INFEASIBLE_X0 with X_next, theta and rejected untouched.
 * Synchronous (reads a status word back and waits for cuda_stream).
 */
#define ESS_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
ess_status ess_step_noalloc(const double *A, const double *b, int d, int m, const double *X,
                            const double *nu, const double *u, int n_chains, double *X_next,
                            double *theta, int *rejected, void *cuda_stream);

/*
 * A few FP64 chains (1 to 16) of the state's polytope for n_iter steps of
 * Alg. 1, every step in one persistent cooperative kernel (the paper's
 * single-chain and ten-chain experiments of Sec. 4.2).  The map and the draws
 * are those of ess_run in the FP64 form (Philox counters (chain, step), the
 * App. B roots, Alg. 3, the Sec. 3.3 rejection), laid out for few chains:
 * all SMs stream the rows of A once per step for q = A nu of every chain
 * and take the exact roots of every row, arcs are merged per angle bucket,
 * one CTA per chain sweeps the merged arcs (Alg. 3) and draws theta (with
 * one chain every CTA does, so the move follows without a grid barrier),
 * grid barriers separate the other phases.  p = A x is recomputed at step
 * t0 and whenever t % refresh_k == 0.
 *   X          device, n_chains x d doubles: start points in, final states
 *              out.
 *   samples    device or NULL; with record_every > 0, n_chains x
 *              (n_iter / record_every) x d doubles: the state after every
 *              record_every-th step.
 * Synchronous.  Errors: ESS_ERR_UNSUPPORTED for the mixed form or m > 6144,
 * ESS_ERR_ARG for n_chains outside 1..16, ESS_ERR_INFEASIBLE_X0 for a start
 * point outside the polytope (checked in FP64 at step t0; X unchanged),
 * ESS_ERR_NUMERIC if NaN/Inf appeared (that chain stays), ESS_ERR_TIMEOUT if
 * a grid barrier waited longer than cfg.wait_limit_us (default 2 s).
 */
ess_status ess_run_few(ess_state *state, double *X, int n_chains, int t0, int n_iter,
                       uint64_t seed, double *samples, int record_every, void *cuda_stream);

/*
 * App. A's factor on the GPU: the lower Cholesky factor L of a symmetric
 * positive definite Sigma = L L^T (the change of variables x = L u + mu).
 *   A     device, n x n row-major doubles with leading dimension lda >= n;
 *         only the lower triangle is read, and it is overwritten with L (the
 *         strict upper triangle is left as it is).
 *   info  host int or NULL: 0, or the 1-based row whose pivot is not positive.
 * Blocked FP64 factorisation (64 x 64 blocks: diagonal block, panel solve,
 * trailing update).  Synchronous.  Errors: ESS_ERR_ARG for bad sizes or a
 * matrix that is not positive definite (A then holds a partial factor).
 */
ess_status ess_cholesky(double *A, int n, int lda, int *info, void *cuda_stream);

/*
 * Self-test of the bounded waits (the paper has no counterpart): runs the
 * persistent few-chain kernel of ess_run_few on the state with one chain of
 * zeros and one CTA withholding its arrival at the first grid barrier (a
 * dependency nothing releases).  Every CTA's wait runs out after
 * cfg.wait_limit_us, the kernel returns, and so must this call, with
 * ESS_ERR_TIMEOUT; the device stays usable.  FP64 states only
 * (ESS_ERR_UNSUPPORTED otherwise).
 */
ess_status ess_selftest_wait(ess_state *state);

/*
 * CUDA-graph replay of whole refresh periods in ess_chains_step / ess_run
 * (on by default).  A period -- the A x refresh and refresh_k steps -- is
 * captured once per (chain count, seed, p buffer) and replayed, the step index
 * coming from a device counter that the graph advances; it applies when
 * refresh_k is even, no samples are recorded and phase timing is off.  The
 * chains are bit-identical with and without graphs.  ess_graph_launches
 * reports the replays since the state was created.
 */
ess_status ess_set_graphs(ess_state *state, int enable);

/*
 * The chain-step kernel of ess_chains_step / ess_run / ess_step_with_draws
 * when ess_config.sort_threads = 0 (the paper has no counterpart: this is the
 * GPU layout of the per-chain work of Alg. 1, roots of App. B and Alg. 3).
 *   ESS_CHAIN_AUTO (default): one warp per chain, rows read from global
 *       memory (the fastest form measured at d = 1000, m = 2000, 8192 chains;
 *       the autotuner of ess_config.autotune times both forms).
 *       With fewer chains than SMs and m > 256 it runs one CTA per chain
 *       instead (the step is then the latency of one chain: at m = 2000, one
 *       chain, 33 us per step against 81 with one warp).
 *   ESS_CHAIN_WARP: the warp kernel, chosen explicitly (for any chain count).
 *   ESS_CHAIN_STREAM: in the mixed form, when m and d are multiples of 4 and
 *       m is at most 4096, one warp per chain with the chain's p and q rows
 *       streamed through shared memory in chunks by 1-D bulk copies (for the
 *       classification and again, with x and nu, for the move); other shapes
 *       and the FP64 form use the warp kernel.
 * In both, chains with more than 128 arcs left after the domination prune go
 * to the CTA-per-chain kernel.  For m > 8192 the CTA per chain is the
 * wide-row kernel (rows streamed); there ESS_CHAIN_AUTO and ESS_CHAIN_STREAM
 * run it for every chain (measured faster at m = 12000 and 16384, where most
 * chains keep more than 128 arcs), ESS_CHAIN_WARP runs the warp kernel first,
 * and so does ESS_CHAIN_AUTO when some b_i <= 0 (those rows' arcs, half a
 * circle or more, form one arc that the warp kernel keeps as its two extreme
 * rows, so such chains rarely keep more than 128 arcs).
 * The kernels compute the same map; their results can differ in the last bits
 * (the order of FP32 roundings).  ess_get_chain_kernel reports the kernel in
 * use for the loaded chains: ESS_CHAIN_STREAM, ESS_CHAIN_WARP, or
 * ESS_CHAIN_CTA (sort_threads > 0, fewer chains than SMs under
 * ESS_CHAIN_AUTO, or m > 8192 with the wide-row kernel for every chain).
 * Changing the kernel drops the captured CUDA graphs.  Errors: ESS_ERR_ARG.
 */
enum { ESS_CHAIN_AUTO = 0, ESS_CHAIN_WARP = 1, ESS_CHAIN_STREAM = 2, ESS_CHAIN_CTA = 3 };
ess_status ess_set_chain_kernel(ess_state *state, int kind);
ess_status ess_get_chain_kernel(const ess_state *state, int *kind);

/*
 * Autotuner (cfg.autotune = 1): when chains are loaded, ess_chains_init
 * (and so ess_run) times, on the loaded chains and their first draw,
 *   - every tile width of the q = A nu tensor-core GEMM (mixed form), and
 *   - the chain-step kernels: one warp per chain with the CTA-per-chain
 *     fallback, or a CTA per chain for every chain at the minimum and at twice
 *     the minimum width,
 * without advancing any chain, and keeps the fastest for that chain count.
 * Different choices can change results in the last bits (different sums), so
 * the tuning is opt-in.  ess_get_tuning reports the choice in use: the q GEMM
 * tile code as in ess_config.q_tile (0 in the FP64 form) and sort_threads
 * (0: warp per chain).
 */
ess_status ess_get_tuning(const ess_state *state, int *q_width, int *sort_threads);
ess_status ess_graph_launches(const ess_state *state, long long *launches);

/* ---- Batched problems -------------------------------------------------------
 * Many independent polytopes {x : A_p x <= b_p} of uneven sizes d_p x m_p,
 * each with its own chains, advanced together: per step one grouped GEMM for
 * q = A_p nu over all problems (mixed form: tcgen05 items of 128 rows of A_p
 * x up to 64 of its chains walked by one persistent CTA per SM; FP64 form:
 * items of up to 4096 row-chain pairs taken from a device work queue by a
 * persistent grid), one chain-step launch for all chains, and whole refresh
 * periods replayed from a CUDA graph (or, with ess_batch_set_persistent, run
 * as one cooperative launch per period).  The sampler
 * of every chain is the one of ess_run (Alg. 1 with the roots of App. B and
 * the intersection of Alg. 3); the batch only changes how the work is laid
 * out.  The paper runs one polytope at a time and has no counterpart.
 *
 * Packing.  A holds the problems' m_p x d_p row-major matrices one after
 * another, b their right-hand sides one after another.  Chain states are
 * packed problem by problem, chain-major: problem p's n_p chains occupy
 * n_p x d_p consecutive doubles; products P, Q likewise with n_p x m_p.
 * Chain k of problem p draws from Philox with chain counter k and problem
 * index p, so its trajectory is the one-problem trajectory with that
 * problem index.
 *
 * Precision.  cfg->precision as for ess_create.  Mixed form: q = A nu on the
 * tensor cores, the scaled FP16x3 products of ess_create (tcgen05, FP32
 * accumulation in tensor memory; within (16 + d_p / 16) 2^-24 sum |a||nu|),
 * FP32 step, near-tangent roots, the refresh of p = A x (every refresh_k
 * steps, in double-float arithmetic on the FP32 pipe, FP64-class accuracy)
 * and the feasibility residual as in ess_create.  FP64 form: everything in
 * double (q by FP64 fused multiply-adds).  cfg->sort_threads and
 * cfg->refresh_mode are ignored.
 */
typedef struct ess_batch ess_batch;

/* Copies the n_problems polytopes (host arrays) to the current device.
 * Errors: ESS_ERR_ARG (n_problems < 1, some d_p or m_p < 1, non-finite A or
 * b, NULL pointers); ESS_ERR_UNSUPPORTED when the largest problem exceeds the
 * chain-step kernels (m_p up to 8192, d_p up to the shared-memory limit). */
ess_status ess_batch_create(int n_problems, const int *d, const int *m, const double *A,
                            const double *b, const ess_config *cfg, ess_batch **out);
void ess_batch_destroy(ess_batch *batch);

/* n_iter steps of every chain.
 *   n_chains  host, n_problems counts (0 allowed).
 *   X         device, packed chain states (doubles); every state must satisfy
 *             A_p x <= b_p (FP64 check; ESS_ERR_INFEASIBLE_X0 otherwise);
 *             overwritten with the final states.
 *   samples   NULL or device buffer of (n_iter / record_every) records, each
 *             the packed states after every record_every-th step, in the
 *             run's precision (float in the mixed form, double in FP64).
 * Steps t0 .. t0 + n_iter - 1; p = A x is recomputed when t % refresh_k == 0.
 * Without sample recording and with refresh_k even, full refresh periods run
 * as CUDA-graph replays.  Unless per-phase timing is on, the steps run on two
 * internal streams (the draw of step t + 1 beside step t), forked from
 * cuda_stream and joined back into it.  Synchronous on return.
 * Reference: Alg. 1. */
ess_status ess_batch_run(ess_batch *batch, const int *n_chains, double *X, int t0, int n_iter,
                         uint64_t seed, void *samples, int record_every, void *cuda_stream);

/* One step with caller-supplied draws (packed device arrays): nu like X,
 * u one uniform per chain; X_next, theta (per chain, may be NULL) and
 * rejected (per chain, may be NULL) are written.  Synchronous. */
ess_status ess_batch_step_with_draws(ess_batch *batch, const int *n_chains, const double *X,
                                     const double *nu, const double *u, double *X_next,
                                     double *theta, int *rejected, void *cuda_stream);

/* The products the batched step uses (verification): P = A x by the refresh
 * path (double result) and Q = A nu by the step's grouped GEMM, packed per
 * problem (n_p x m_p doubles each); either may be NULL.  Synchronous. */
ess_status ess_batch_products(ess_batch *batch, const int *n_chains, const double *X,
                              const double *nu, double *P, double *Q, void *cuda_stream);

/* Statistics and per-phase timing as for a single state (timing disables
 * graph replays, so every phase is timed by events); graphs can be switched
 * off to compare with plain launches. */
ess_status ess_batch_get_stats(const ess_batch *batch, ess_stats *out);
ess_status ess_batch_reset_stats(ess_batch *batch);
ess_status ess_batch_set_graphs(ess_batch *batch, int enable);
ess_status ess_batch_set_timing(ess_batch *batch, int enable);
ess_status ess_batch_get_timing(ess_batch *batch, double *ms, long long *launches, int n_phases);
ess_status ess_batch_reset_timing(ess_batch *batch);
/* Persistent launch of whole refresh periods (mixed form; enable = 1):
 * instead of the graph of per-step launches (draw, grouped GEMM, warp step,
 * CTA step for each step), a refresh period replays as the refresh of p and
 * the draw of step 0, then ONE cooperative kernel with one 1024-thread CTA
 * per SM for all refresh_k steps.  Per step its warps 0..5 run the grouped
 * q GEMM on the tensor cores, warps 6..21 draw nu of the next step, and
 * warps 22..31 -- then warps 0..21 too, once the CTA's own q items are done
 * -- take chains from a device work queue (problems in the order their q
 * items finish) for the warp-per-chain step, each chain after its problem's
 * q is complete (a per-problem counter of finished q items); whole CTAs
 * then take the chains left with too many arcs.  Steps are joined by grid
 * barriers; every dependency and barrier wait is bounded by
 * cfg->wait_limit_us (ESS_ERR_TIMEOUT on expiry).  The
 * chains are the ones of the graph of per-step launches (the same products,
 * roots, prune, sort and draws); the chains left with too many arcs take the
 * same CTA step at 1024 threads (more merge buckets, another summation order
 * of the piece lengths, FP32 subnormals flushed), which can change their
 * theta in the last bits.  It applies to runs that
 * replay graphs (no sample recording, no per-phase timing, refresh_k even).
 * Errors: ESS_ERR_UNSUPPORTED for the FP64 form, or when the device cannot
 * hold the launch (cooperative launch, one CTA of 1024 threads and ~217 KB of
 * shared memory per SM; largest m_p up to 8192).  Default: on for the mixed
 * form where the device holds the launch (512 problems, 18,687 chains:
 * 0.176 ms per step against 0.178 for the per-step graph);
 * enable = 0 returns to the per-step graph.
 * Reference: Alg. 1 (the batch itself has no counterpart in the paper). */
ess_status ess_batch_set_persistent(ess_batch *batch, int enable);

/* Self-test of the persistent launch's bounded dependency waits (the paper
 * has no counterpart): lays out n_chains and runs 2 refresh_k steps of X
 * (device, packed as in ess_batch_run) with every problem's q dependency
 * raised by one count that nothing releases.  The first refresh_k steps run
 * as plain launches; in the persistent launch of the second period every
 * chain step's wait runs out after cfg->wait_limit_us, the kernel returns,
 * and so must this call, with ESS_ERR_TIMEOUT; the batch stays usable (X is
 * left unspecified).  ESS_ERR_UNSUPPORTED unless the persistent launch is on
 * (mixed form) and refresh_k is even.  Synchronous. */
ess_status ess_batch_selftest_wait(ess_batch *batch, const int *n_chains, double *X);

/* Sizes of the current chain layout: packed state and product lengths, GEMM
 * work items, and the graph replays since the last timing reset. */
ess_status ess_batch_info(const ess_batch *batch, long long *total_x, long long *total_p,
                          int *n_items, long long *graph_launches);

/* Message describing the last failure of the calling thread ("" if none). */
const char *ess_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ESS_GB300_H */
