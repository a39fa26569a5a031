/*
 * sadi.h -- C ABI of the S-ADI library (splitting ADI scheme for the 2D
 * fractional Laplacian wave equation, arXiv 2312.06206), GB300 / sm_103a.
 *
 * Problem (Sec. 1, eq. "wave equation"): on Omega = (a, b)^2,
 *     u_tt = -kappa (-Delta)^{alpha/2} u + g(u),  u = 0 outside Omega,
 *     u(x, y, 0) = phi1,  u_t(x, y, 0) = phi2,
 * discretised on N x N interior points with h = (b - a)/(N + 1) (Sec. 2) and
 * advanced by the S-ADI scheme in its factored increment form (Sec. 3, eq.
 * "ADI scheme equivalent"):
 *     (1 + tau^2 kappa/2 delta_x)(1 + tau^2 kappa/2 delta_y) uhat^n = B^n,
 * with both ADI factors solved by the Gohberg-Semencul formula (Proposition 1,
 * Algorithm 1) and L_h u^n applied by a zero-padded 2D FFT convolution (Sec. 3).
 *
 * Conventions shared by every entry point:
 *  - Grid functions are N x N row-major arrays of double, element [j*N + i] is
 *    the value at (x_{i+1}, y_{j+1}): i is the x index (contiguous), j the y
 *    index.  Host arrays are read or written synchronously and are owned by
 *    the caller; the library never keeps a host pointer.
 *  - The context owns all of its device memory and frees it in sadi_destroy.
 *  - Every call returns a status and never aborts or exits; on failure the
 *    context keeps a message readable with sadi_last_error.  After a CUDA
 *    error (SADI_ECUDA) the context refuses further steps with SADI_ESTATE.
 *  - All device work of a context is issued on its stream (sadi_set_stream);
 *    calls on one context must not run concurrently from several host threads.
 *    Different contexts may be driven at the same time, from several host
 *    threads or on several streams: a context's results do not depend on
 *    what runs beside it (sadi_step_noalloc excepted, see there).
 */
#ifndef SADI_H
#define SADI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sadi_ctx sadi_ctx;

typedef enum {
  SADI_OK = 0,
  SADI_EINVAL = 1,        /* invalid argument (message names it)                */
  SADI_ENOMEM = 2,        /* device or host allocation failed                   */
  SADI_ECUDA = 3,         /* a CUDA call failed; the context is now unusable    */
  SADI_ENOTSPD = 4,       /* generator solve broke down (H not SPD numerically) */
  SADI_ESTATE = 5,        /* call out of order (e.g. step before set_initial)   */
  SADI_ETIMEOUT = 6,      /* a bounded device wait ran out                      */
  SADI_ENONFINITE = 7,    /* non-finite value detected in the state             */
  SADI_EUNSUPPORTED = 8   /* valid request this library version does not implement */
} sadi_status;

/* Nonlinearity g(u) of Sec. 1 (Sec. 6 uses -sin u and -u^3).
 * SADI_G_GENERAL: g(u) = c1 u + c3 u^3 + cs sin u with the coefficients of
 * sadi_set_nonlinearity (all 0 until set), e.g. the linear Klein-Gordon term
 * -u, the phi^4 term -u - u^3, or a scaled sine-Gordon term. */
typedef enum { SADI_G_ZERO = 0, SADI_G_NEG_CUBE = 1, SADI_G_NEG_SIN = 2, SADI_G_GENERAL = 3 } sadi_g;

/* Arithmetic of the per-step path.  Setup (weights, generator, spectra, the
 * dense inverse) is always FP64.
 * SADI_PREC_FP64: FFTs, sweeps and state in double.
 * SADI_PREC_FP32: FFTs and Gohberg-Semencul sweeps in float; the state kept
 *   as a double-float pair with a compensated leapfrog (float storage), and
 *   the remainder -kappa tau^2 L_h u^n carried as a double-float pair that
 *   each step advances by the FFT convolution of the increment u^n - u^{n-1}
 *   (started from an FP64 evaluation of L_h phi1 when N' <= 4096; FP32 above).
 *   FFT rounding then scales with the increment instead of u^n.
 * SADI_PREC_FP32_DENSE: as FP32, but both sweeps apply the precomputed dense
 *   inverse H^-1 = I + E to all rows / columns at once: W = B + B E and
 *   uhat = W + E W, each product a split-BF16 GEMM on the tensor cores
 *   (E and the right-hand side split into BF16 hi + lo pairs, three products,
 *   FP32 accumulation).  E comes from the FP64 generator of the N x N matrix.
 *   Any N up to 8192 (E and the operands take 12 N_p^2 bytes, N_p = N rounded
 *   up to 256).  Its error is relative to E, whose size grows with
 *   s = kappa tau^2 / (2 h^alpha): near-FP32 while s a_0 is small (a_0 the
 *   first 1D weight), visibly coarser once E is O(1) (s a_0 of order 1 or
 *   more); prefer SADI_PREC_FP32 there. */
typedef enum {
  SADI_PREC_AUTO = -1,    /* sadi_batch_create only: the autotuner's choice per N */
  SADI_PREC_FP64 = 0, SADI_PREC_FP32 = 1, SADI_PREC_FP32_DENSE = 2
} sadi_prec;

/* Create a context for N interior points per direction, fractional order
 * alpha in (1, 2] (2 = the classical wave equation limit; the paper states
 * (1, 2)), kappa > 0, time step tau > 0 and Omega = (domain[0], domain[1])^2.
 * Runs the FP64 setup on the current CUDA device: the 1D Riesz weights a_i
 * (Sec. 2, eq. "single coefficient discrete Riesz"), the 2D weights a_ij
 * (Sec. 2, eq. "center discretization"; trapezoid rule + Richardson), the
 * symbol of the block-circulant embedding of L_h (Sec. 3), and the
 * Gohberg-Semencul generator c = H^-1 e_1 with its spectra (Proposition 1,
 * eq. "eigenvalue of CS").  Defaults: g = SADI_G_ZERO, precision FP64, a
 * stream owned by the context.  N must be in [1, 4096] (FP64 path) or
 * [1, 8192] (FP32 path).  On success *out receives the context; on failure
 * *out is NULL and the status says why (no context is left behind). */
sadi_status sadi_create(int N, double alpha, double kappa, double tau,
                        const double domain[2], sadi_ctx **out);

/* A context for the fractional Laplacian diffusion equation
 *     u_t = -kappa (-Delta)^{alpha/2} u + g(u) + f on Omega, u = 0 outside,
 *     u(., 0) = phi1,
 * the further application of the S-ADI idea that the paper names in its
 * conclusion (Sec. 7) without giving a scheme.  This library takes the
 * splitting of Secs. 2-3 with the Riesz parts delta_x + delta_y by
 * Crank-Nicolson, the remainder L_h - delta_x - delta_y and g explicit at
 * t_{n+1/2} by the extrapolation u~ = u^n + (u^n - u^{n-1})/2, and the
 * factorisation term (kappa^2 tau/4) delta_x delta_y on the second
 * difference, so that each step is
 *     (I + kappa tau/2 delta_x)(I + kappa tau/2 delta_y) Delta
 *         = tau (-kappa L_h u~ + g(u~) + f^{n+1/2}) - (u^n - u^{n-1}),
 *     u^{n+1} = 2u^n - u^{n-1} + Delta      (n = 0: u~ = u^0, u^1 = u^0 + Delta),
 * second order in tau, with the same operators, Gohberg-Semencul sweeps and
 * step forms as the wave equation (tau in place of tau^2 in the ADI factor
 * and the symbol).  Arguments, set-up and every other call as sadi_create;
 * sadi_set_initial takes phi2 = NULL (SADI_EINVAL otherwise); sources are
 * sampled at the step midpoints t_{n+1/2} (sadi_set_source) or given for
 * them (sadi_step_source).  The dense-inverse form's accuracy limit applies
 * with s = kappa tau / (2 h^alpha), usually far larger than the wave's. */
sadi_status sadi_create_diffusion(int N, double alpha, double kappa, double tau,
                                  const double domain[2], sadi_ctx **out);

/* *eq = 0 for a context of sadi_create (wave), 1 for sadi_create_diffusion. */
sadi_status sadi_get_equation(const sadi_ctx *ctx, int *eq);

/* Choose g and the step precision.  Must be called before sadi_set_initial
 * (SADI_ESTATE otherwise). */
sadi_status sadi_set_options(sadi_ctx *ctx, int g, int prec);

/* g(u) = c1 u + c3 u^3 + cs sin u (finite coefficients, else SADI_EINVAL):
 * selects SADI_G_GENERAL with these coefficients; the nonlinear term enters
 * B^n as the paper's g does (Sec. 3), evaluated in the step's precision (the
 * FP32 register path uses the hardware sine, whose error is scaled by
 * tau^2).  Must precede sadi_set_initial (SADI_ESTATE otherwise). */
sadi_status sadi_set_nonlinearity(sadi_ctx *ctx, double c1, double c3, double cs);

/* Current g and precision of ctx (either pointer may be NULL). */
sadi_status sadi_get_options(const sadi_ctx *ctx, int *g, int *prec);

/* Optional source term (an extension beyond the paper's problem statement,
 * used for manufactured-solution checks): the equation becomes
 * u_tt = -kappa (-Delta)^{alpha/2} u + g(u) + f with
 *     f(x, y, t_n) = cos(omega t_n + phase) * F(x, y),  t_n = n tau,
 * and f^n enters B^n exactly as g(u^n) does (tau^2 f^n for n >= 1,
 * tau^2/2 f^0 at n = 0).  F: host N*N doubles (copied; layout above), or NULL
 * to remove the source.  Call after sadi_set_options; changing the precision
 * afterwards returns SADI_ESTATE. */
sadi_status sadi_set_source(sadi_ctx *ctx, const double *F, double omega, double phase);

/* One time step (as sadi_step(ctx, 1)) with a source term given as a grid
 * function for this step: the equation u_tt = -kappa (-Delta)^{alpha/2} u +
 * g(u) + f (an extension beyond the paper's problem statement, e.g. for
 * manufactured solutions or driven problems), f^n = f at t_n = n tau
 * entering B^n as g(u^n) does: tau^2 f^n for n >= 1, tau^2/2 f^0 at n = 0,
 * fused into the B^n epilogue.  f: device memory on the context's device,
 * N*N elements (layout above) of dtype 0 = double or 1 = float, owned by the
 * caller and read by the step on the context's stream (keep it unchanged
 * until the step has run).  A dtype other than the step's precision is
 * converted into a buffer of the context (allocated on first use) first.
 * SADI_EINVAL if f is not such a buffer; SADI_ESTATE while a separable source
 * (sadi_set_source) is set or before sadi_set_initial. */
sadi_status sadi_step_source(sadi_ctx *ctx, const void *f, int dtype);

/* Issue all further device work on cuda_stream (a cudaStream_t, e.g. a torch
 * stream's handle); NULL selects the context's own stream.  The caller keeps
 * ownership of the stream and must keep it alive while the context uses it. */
sadi_status sadi_set_stream(sadi_ctx *ctx, void *cuda_stream);

/* Copy the initial data phi1 = u(., 0) and phi2 = u_t(., 0) (host, N*N doubles
 * each, layout above) to the device and reset the step counter n to 0.  phi2
 * may be NULL (meaning 0).  Synchronous with respect to the host buffers. */
sadi_status sadi_set_initial(sadi_ctx *ctx, const double *phi1, const double *phi2);

/* Advance nsteps >= 0 time steps (asynchronous on the context's stream).  The
 * first step after sadi_set_initial uses the n = 0 formula of Sec. 3
 * (u^1 - u^0 with B^0 = tau phi2 - tau^2/2 kappa L_h u^0 + tau^2/2 g(u^0)),
 * every later step the n >= 1 formula (u^{n+1} - 2u^n + u^{n-1} with
 * B^n = -tau^2 kappa L_h u^n + tau^2 g(u^n)). */
sadi_status sadi_step(sadi_ctx *ctx, int nsteps);

/* Advance each of count contexts by nsteps time steps (asynchronous), as
 * sadi_step would, but batched: FP32 contexts with FFT length N' <= 1024 and
 * FP32_DENSE contexts with N' <= 2048 (unless explicit tiles keep them on
 * the shared-memory engine, see sadi_set_tiles) are grouped by precision
 * and N' (at most 32 per group) and each
 * group runs one launch per kernel for all its members (independent problems
 * of possibly different N, alpha, kappa, tau and g; both dense sweeps of up
 * to 8 members in one GEMM launch); the other contexts step one after
 * another.
 * All contexts must be initialised and distinct (SADI_EINVAL / SADI_ESTATE
 * otherwise).  The work
 * is issued on the first context's stream, ordered after the work already
 * queued on the other contexts' streams and before their later work (event
 * waits).  Results are identical to stepping each context alone. */
sadi_status sadi_batch_step(sadi_ctx **ctxs, int count, int nsteps);

/* A batch of independent instances behind one handle (the batched pattern:
 * many problems of uneven N, alpha, kappa, tau advanced together; the paper
 * solves one problem at a time, Sec. 6).  Member k is the problem
 * sadi_create(N[k], alpha[k], kappa[k], tau[k], domains + 2k) would set up
 * (domains NULL: every member on (-1, 1)^2), all with nonlinearity g, and
 * the step form prec, or with prec = SADI_PREC_AUTO the form and tiles that
 * sadi_autotune picks per N (FP32 or FP32_DENSE).  All members share one
 * stream owned by the batch (sadi_batch_set_stream replaces it; NULL
 * restores it).  On failure *out is NULL, nothing is left allocated, and
 * sadi_batch_last_error(NULL) says which member failed and why. */
typedef struct sadi_batch sadi_batch;
sadi_status sadi_batch_create(int count, const int *N, const double *alpha, const double *kappa,
                              const double *tau, const double *domains, int g, int prec,
                              sadi_batch **out);

/* Initial data of member k (0 <= k < count), as sadi_set_initial.  Members
 * may be (re)initialised at any time between runs; a member at n = 0 takes
 * the n = 0 step in the next sadi_batch_run. */
sadi_status sadi_batch_set_initial(sadi_batch *batch, int k, const double *phi1, const double *phi2);

/* Advance every member by nsteps >= 0 steps (asynchronous on the batch's
 * stream): batched launches as sadi_batch_step makes them (one launch per
 * kernel for each group of equal FFT length on the register path), and once every member
 * is past its n = 0 step, replays of a CUDA graph of one batched step
 * (captured on first use; FP32 forms without source terms or profiling --
 * otherwise the steps are launched directly).  Results are identical to
 * stepping each member alone.  SADI_ESTATE if a member has no initial data. */
sadi_status sadi_batch_run(sadi_batch *batch, int nsteps);

/* u^n of member k to the host (N_k * N_k doubles) and its step count, as
 * sadi_get (synchronous; the member's watchdog and wait errors surface
 * here). */
sadi_status sadi_batch_get(sadi_batch *batch, int k, double *u_out, long long *n_out);

/* The context of member k (owned by the batch: do not destroy it), for the
 * per-context calls (sadi_get_async, sadi_set_source, sadi_profile, ...).
 * The batch captures its step graph anew after this call. */
sadi_status sadi_batch_member(sadi_batch *batch, int k, sadi_ctx **ctx);
sadi_status sadi_batch_count(const sadi_batch *batch, int *count);
sadi_status sadi_batch_set_stream(sadi_batch *batch, void *cuda_stream);
/* Last error of the batch ("" if none); NULL: the last failed
 * sadi_batch_create on this thread. */
const char *sadi_batch_last_error(const sadi_batch *batch);
/* Waits for the batch's stream, then frees every member and the batch. */
void sadi_batch_destroy(sadi_batch *batch);

/* Checkpoint and resume (no paper counterpart).  sadi_save_state writes the
 * step state of an initialised context into buf (host memory of *bytes
 * bytes, owned by the caller): a header (N, precision, g, alpha, kappa, tau,
 * domain, step counter n) followed by the device arrays the next step reads
 * (FP64: u^n, u^{n-1}, phi2; FP32 forms: u_hi, u_lo, the increment, the
 * remainder pair, phi2).  With buf NULL it only stores the size needed in
 * *bytes; a buffer that is too small returns SADI_EINVAL with the size in
 * *bytes.  sadi_load_state restores such a blob into a context created with
 * the same N, alpha, kappa, tau and domain and set to the same g and
 * precision (SADI_EINVAL otherwise); the context continues exactly as the
 * saved one would (bitwise).  Both are synchronous on the context's stream.
 * The blob is tied to this library version's layout; it is not an interchange format. */
sadi_status sadi_save_state(sadi_ctx *ctx, void *buf, size_t *bytes);
sadi_status sadi_load_state(sadi_ctx *ctx, const void *buf, size_t bytes);

/* CUDA-graph replay of batched steps (no paper counterpart; it removes the
 * per-step host launch cost when many small instances advance together).
 * sadi_graph_create captures nsteps >= 1 steps of the count contexts, issued
 * exactly as sadi_batch_step(ctxs, count, nsteps) would issue them, into a
 * CUDA graph on the first context's stream; nothing runs at capture time and
 * the contexts' step counters are unchanged.  Requirements (SADI_ESTATE /
 * SADI_EINVAL / SADI_EUNSUPPORTED otherwise): every context initialised and
 * past its n = 0 step (n >= 1), no source term, profiling off, all contexts
 * on one stream, distinct.  FP32 and FP32_DENSE contexts update their state
 * in place, so one captured step fits every later step; FP64 contexts keep
 * u^n and u^{n-1} in two buffers that swap every step, so they need an even
 * nsteps, and a launch after an odd number of other steps since the capture
 * returns SADI_ESTATE.
 * sadi_graph_launch replays the graph reps >= 0 times (asynchronous) and
 * advances every context's n by nsteps * reps; it re-checks the requirements
 * first.  The graph holds the contexts' device pointers: destroy it before
 * any of its contexts, and re-create it after sadi_set_options on any of
 * them.  sadi_graph_destroy waits for the stream and frees the graph (NULL
 * is a no-op). */
typedef struct sadi_graph sadi_graph;
sadi_status sadi_graph_create(sadi_ctx **ctxs, int count, int nsteps, sadi_graph **out);
sadi_status sadi_graph_launch(sadi_graph *graph, int reps);
/* Number of kernel launches one replay of graph performs (*kernels). */
sadi_status sadi_graph_kernels(const sadi_graph *graph, int *kernels);
void sadi_graph_destroy(sadi_graph *graph);

/* Autotuner (no paper counterpart): for the count contexts, grouped by N,
 * time the candidate step forms on zero data with the group stepped as
 * sadi_batch_step steps it (up to 32 contexts per group) -- SADI_PREC_FP32
 * (Gohberg-Semencul FFT sweeps) and, unless flags bit 0 is set or
 * s a_0 > 0.2 (the dense form's accuracy limit above),
 * SADI_PREC_FP32_DENSE (tensor-core dense-inverse sweeps) -- and, for a
 * form on the shared-memory FFT engine (FP32 at N' > 1024, FP32_DENSE at
 * N' > 2048), the work decomposition of sadi_set_tiles by coordinate
 * descent.  flags bit 1 keeps the precision the
 * contexts already have (FP32 or FP32_DENSE, equal within each N) and tunes
 * only the tiles.  Each context is left with g, the fastest precision and
 * tiles of its group, uninitialised (call sadi_set_initial next).  Must precede sadi_set_initial and
 * sadi_set_source.  The choice and the timings are readable with
 * sadi_tuning_log.  Synchronous. */
sadi_status sadi_autotune(sadi_ctx **ctxs, int count, int g, int flags);

/* Text record of the last sadi_autotune choice for ctx ("" if none). */
const char *sadi_tuning_log(const sadi_ctx *ctx);

/* Copy u^n to the host (N*N doubles) after the stream's pending work; *n_out
 * (may be NULL) receives n.  Synchronous.  Returns SADI_ETIMEOUT (and the
 * context becomes unusable) if a bounded wait inside a tensor-core sweep of
 * the dense-inverse form ran out since the context was created. */
sadi_status sadi_get(sadi_ctx *ctx, double *u_out, long long *n_out);

/* Asynchronous read of the state u^n = phi^n (the scheme's solution after n
 * steps, Sec. 3): queue the copy of u^n (N*N doubles, row-major, x fastest)
 * into host memory u_out and return at once.  u_out should be page-locked
 * (pinned) host memory; it is written when sadi_wait returns and must not be
 * read or freed before.  The state is first joined into the context's
 * staging buffer on its stream, then copied to the host on a stream of the
 * context's own, so steps queued after this call run while the copy is in
 * flight; a later sadi_get_async, sadi_get, sadi_set_initial or
 * sadi_set_source waits for the copy before reusing the buffer.  Not to be
 * called while the context's stream is being captured into a CUDA graph.
 * SADI_EINVAL for u_out NULL, SADI_ESTATE before sadi_set_initial. */
sadi_status sadi_get_async(sadi_ctx *ctx, double *u_out);

/* Wait for all work queued on the context's stream and for its
 * sadi_get_async copies.  Returns SADI_ETIMEOUT (the context then becomes
 * unusable) under the same condition as sadi_get. */
sadi_status sadi_wait(sadi_ctx *ctx);

/* Copy u^n device-to-device into dst (N*N contiguous elements of dtype 0 =
 * double or 1 = float, device memory owned by the caller), on the context's
 * stream (asynchronous). */
sadi_status sadi_get_device(sadi_ctx *ctx, void *dst, int dtype);

/* Setup tables for parity tests, FP64, copied to the host (synchronous):
 *   which = 0: a_i, 0 <= i < N                         (count N)
 *   which = 1: a_ij, 0 <= i, j < N, row-major          (count N*N)
 *   which = 2: generator c' = H'^-1 e_1 of the bordered Toeplitz matrix
 *              H' = I + s T(a_0 .. a_{N'-1}), N' = the FFT length (count N')
 *   which = 3: symbol Lambda(k1, k2) of the block-circulant embedding of
 *              size 2N' x 2N' (unscaled), 0 <= k1, k2 <= N'  (count (N'+1)^2)
 *   which = 4: E = H^-1 - I of the N x N matrix H = I + s T(a_0 .. a_{N-1})
 *              as the dense-inverse form stores it (E_hi + E_lo, the BF16
 *              pair, summed in double), row-major (count N*N); only after
 *              SADI_PREC_FP32_DENSE was selected (SADI_ESTATE otherwise)
 * count must equal the stated size.  N' is returned by sadi_get_info. */
sadi_status sadi_get_setup(sadi_ctx *ctx, int which, double *out, size_t count);

/* Sizes chosen at create: fft_len = N' (power of two >= N, >= 8) and the
 * border rank r = N' - N of the Gohberg-Semencul solve.  Either pointer may
 * be NULL. */
sadi_status sadi_get_info(const sadi_ctx *ctx, int *fft_len, int *border_rank);

/* Work decomposition of the four step kernels for the precision currently
 * selected: grid rows per block of the row kernels, spectrum slots per block
 * of the column convolution (a divisor of N'), grid columns per block of the
 * y sweep.  conv_cols = -1 selects the three-pass column convolution (a
 * four-step FFT through HBM; FP32 forms, N' = 2048 .. 8192; the default at
 * N' = 8192; its buffers, about 24 N'^2 bytes, are allocated on first use).
 * All zero restores the defaults.  Invalid combinations (shared memory above
 * 227 KB per block, more rows than the row kernel stages, -1 elsewhere)
 * return SADI_EINVAL and leave the setting unchanged.  The tiles change the
 * order of some rounding steps (the column convolution multiplies the symbol
 * fused into its transforms or in a separate pass), so results of different
 * tiles agree to rounding, not bitwise.  The tiles are those of the
 * shared-memory FFT engine; the register path (FP32 at N' <= 1024,
 * FP32_DENSE at N' <= 2048) has none.  At N' = 2048 the dense form's FFT
 * part runs on the register path by default, and explicit (non-zero) tiles
 * move it to the shared-memory engine (all zero moves it back); such a
 * change re-lays the state and must precede sadi_set_initial and
 * sadi_set_source (SADI_ESTATE otherwise).  Call after sadi_set_options. */
sadi_status sadi_set_tiles(sadi_ctx *ctx, int rows, int conv_cols, int solve_cols);

/* Current tiles of the selected precision: tiles[0..2] = rows, conv_cols,
 * solve_cols. */
sadi_status sadi_get_tiles(const sadi_ctx *ctx, int tiles[3]);

/* Per-kernel timing (a tracing aid).  enable != 0: every later step records
 * CUDA events on the context's stream around each of its four phases
 * (0 row FFT, 1 column convolution, 2 row inverse FFT + RHS + x sweep,
 * 3 y sweep + leapfrog; in the dense-inverse form 2 is the row inverse FFT +
 * RHS alone and 3 both sweep GEMMs, which run as one launch); enable = 0
 * stops recording.  Recording adds event records between the kernels, so
 * time throughput with it disabled. */
sadi_status sadi_profile(sadi_ctx *ctx, int enable);

/* Wait for the context's stream, then return in ms[4] the milliseconds
 * accumulated per kernel since the last call (or since sadi_profile), and
 * in *nsteps (may be NULL) the number of steps they cover; resets the
 * accumulators. */
sadi_status sadi_get_phase_times(sadi_ctx *ctx, double ms[4], long long *nsteps);

/* State watchdog (failure detection; no paper counterpart).  After every
 * stepping call (sadi_step, sadi_batch_step, sadi_graph_launch,
 * sadi_batch_run) in which the step counter n reaches or passes a multiple
 * of `every`, one small kernel on the context's stream sums u_ij^2 of the
 * state u^n over the grid in double (FP32 forms: the float hi part of u^n)
 * and latches a flag if the sum is not finite (a NaN or an infinity in u^n,
 * or a blow-up past ~1e154).  The next synchronising call (sadi_get,
 * sadi_wait) then returns SADI_ENONFINITE, naming the step of the first
 * check that saw it, and the context needs new data (sadi_set_initial or
 * sadi_load_state, which clear the flag) before it steps again.
 * every >= 0; 0 switches the checks off; a new context checks every 100
 * steps.  The checks only read the state: results are unchanged. */
sadi_status sadi_set_watchdog(sadi_ctx *ctx, int every);

/* Result of the last watchdog check of ctx (waits for its stream): the
 * discrete L2 norm h (sum_ij u_ij^2)^(1/2) of u^n (Sec. 4 norm) in *l2norm
 * and its step n in *step (0 and 0 before the first check); either pointer
 * may be NULL. */
sadi_status sadi_get_watchdog(sadi_ctx *ctx, double *l2norm, long long *step);

/* Test hook for the bounded device waits of the dense-inverse form (no paper
 * counterpart).  The next step of ctx (SADI_PREC_FP32_DENSE only, else
 * SADI_EUNSUPPORTED) launches its sweep GEMM with every bounded wait limited
 * to wait_limit_ns (1e5 .. 1e9, else SADI_EINVAL) instead of 1 s, and with
 * its y-sweep tiles waiting for an x-sweep panel count that no tile reaches.
 * Those waits run out: the kernel's CTAs stop, wait (bounded) for their own
 * copies and tensor-core work in flight, free their tensor memory and
 * return, and the next sadi_get or sadi_wait returns SADI_ETIMEOUT; the
 * context is then unusable (SADI_ESTATE), other contexts and the CUDA
 * context are not affected.  One-shot: the hook applies to one step. */
sadi_status sadi_debug_expire_waits(sadi_ctx *ctx, long long wait_limit_ns);

/* Last error message of ctx ("" if none).  ctx may be NULL: then the message
 * of the last failed sadi_create on this thread is returned. */
const char *sadi_last_error(const sadi_ctx *ctx);

/* Free the context and all its device memory (waits for its stream). NULL is
 * a no-op. */
void sadi_destroy(sadi_ctx *ctx);

/* Split-BF16 tensor-core product (no paper counterpart: the contraction of the
 * dense-inverse sweeps, exposed so that it can be tested on its own).
 * A: M x K, B: N x K, C: M x N, all FP32, row-major, contiguous, device
 * memory on the current device, owned by the caller.  Each operand is split
 * into BF16 pairs X = X_hi + X_lo (X_hi = X rounded to nearest BF16, X_lo = the
 * remainder rounded to BF16) and
 *     C = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T
 * is accumulated in FP32 by tcgen05 MMAs (the A_lo B_lo^T term is dropped).
 * 1 <= M, N, K <= 65536.  Allocates and frees temporary device buffers (zero-
 * padded operand copies); runs on `stream` (a cudaStream_t, NULL = the legacy
 * default stream) and returns after it has finished.  SADI_ETIMEOUT if a
 * bounded device wait ran out (C is then unspecified). */
sadi_status sadi_gemm_split_bf16(const float *A, const float *B, float *C,
                                 int M, int N, int K, void *stream);

/* One time step on caller-owned device state that allocates and frees no
 * device memory.  The paper has no counterpart: this is a service entry point
 * of the library.
 *
 * Who needs it: a caller that cannot allocate device memory while it steps,
 * for example one whose free HBM is already reserved by another allocator (a
 * framework's caching pool), or a latency-critical loop in which a cudaMalloc
 * or cudaFree would synchronise the device and stall its other streams.  It
 * also lets the caller keep the state in its own buffers instead of the
 * context's.
 *
 * Computes u_next = u^{n+1} = 2 u^n - u^{n-1} + uhat^n by the n >= 1 formula
 * of Sec. 3 (B^n = -tau^2 kappa L_h u^n + tau^2 g(u^n), plus tau^2 f^n with a
 * source) from u_prev = u^{n-1} and u_cur = u^n, with the context's setup
 * (N, alpha, kappa, tau, g, source, tiles) and its FP64 step kernels: the
 * same arithmetic as sadi_step.  n >= 1 is the time level of u_cur; it only
 * sets the source time t_n = n tau.  The context's own state (sadi_set_initial,
 * sadi_step, sadi_get) is neither read nor changed; sadi_set_initial need not
 * have been called.
 *
 * u_prev, u_cur, u_next: device memory on the context's device, N*N doubles
 * each (layout above), owned by the caller.  u_next may equal u_prev (in
 * place) but must not overlap u_cur; other overlaps are rejected
 * (SADI_EINVAL).  The step is queued on the context's stream (asynchronous).
 * The context's device must be current.  FP64 contexts only
 * (SADI_EUNSUPPORTED otherwise).
 *
 * Scratch: a fixed 32 MiB array compiled into the library, which every GPU
 * that loads the library's device code holds until the process exits.  A step
 * needs 16 N N' + 8 N^2 bytes (+ alignment), N' the FFT length, so N <= 1024
 * fits (25 MB at N = 1023); a larger N returns SADI_EINVAL naming both sizes.
 * The array keeps what the previous call left in it; nothing in it has to
 * start at zero, as each call writes every scratch element before reading it.
 * All calls share the one array: calls that overlap in time (on several
 * streams or host threads, whatever the contexts) race on it and produce
 * wrong results, so order them (one stream, or events).
 *
 * The first call on a device does a per-device set-up (it looks up the
 * array's device address, which can load the library's device code on that
 * device); make that first call before any stream capture begins. */
sadi_status sadi_step_noalloc(sadi_ctx *ctx, const double *u_prev,
                              const double *u_cur, double *u_next,
                              long long n);

#ifdef __cplusplus
}
#endif

#endif /* SADI_H */
