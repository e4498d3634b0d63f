/*
 * gwl.h -- C ABI of the GB300 batched gravitational-wave likelihood library.
 *
 * The library evaluates, for many parameter vectors at once, the
 * frequency-domain Gaussian-noise log-likelihood of Smith, Ashton, Vajpeyi &
 * Talbot (2020), Eq. 2, read as the log-likelihood ratio
 *
 *     lnL(theta) = sum_det [ <d|h(theta)> - 1/2 <h(theta)|h(theta)> ],
 *     <a|b> = 4 df Re sum_j conj(a_j) b_j / S_j,
 *
 * with an aligned-spin TaylorF2 inspiral template (Newtonian amplitude,
 * 3.5PN phase, h = 0 above the ISCO frequency), and the constrained
 * random-walk replacement step of static parallel nested sampling
 * (Section 3, Algorithm 1: candidates are accepted iff lnL >= L*).
 *
 * Conventions
 *   - Every function returns an int status: GWL_OK (0) or a negative
 *     GWL_ERR_* code; gwl_last_error() returns a text for the calling thread's
 *     last failure.  Argument errors are reported synchronously.  Errors that
 *     kernels detect (a bounded wait that ran out) are latched in the context
 *     and reported by the next gwl_sync().
 *   - "dev" pointers are device pointers owned by the caller (e.g. torch
 *     tensors); "host" pointers are ordinary host memory.  Compute calls
 *     enqueue on the caller's CUDA stream (a cudaStream_t passed as void*;
 *     NULL = legacy default stream) and return without synchronising, except
 *     the *_host variants, which copy, compute and synchronise.
 *   - Parameter order of the full 11-D vector (GWL_P_*):
 *       Mc [detector-frame Msun], q = m2/m1 in (0,1], chi1z, chi2z,
 *       dL [Mpc], iota, psi, ra, dec [rad], tc [s, relative to t_ref],
 *       phic [rad].
 *     A context samples n_dim of them (param_map); the others keep
 *     fixed_theta.  theta arrays passed to the library hold the n_dim sampled
 *     coordinates per row, row-major [B][n_dim], FP64.
 *   - An unphysical row (q outside (0,1], Mc <= 0 or dL <= 0, or a non-finite
 *     value) yields lnL = -inf and a zero gradient; it is not an error.
 *   - A context is not thread-safe; calls on one context must not overlap
 *     (they share its scratch buffers).
 */
#ifndef GWL_H
#define GWL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GWL_OK 0
#define GWL_ERR_ARG (-1)       /* invalid argument (null pointer, size, option) */
#define GWL_ERR_CUDA (-2)      /* a CUDA runtime call failed */
#define GWL_ERR_TIMEOUT (-3)   /* a kernel's bounded wait ran out (latched) */
#define GWL_ERR_NONFINITE (-4) /* reserved */
#define GWL_ERR_NOMEM (-5)     /* device allocation failed */

#define GWL_FP64 0  /* plain FP64: phase, sincos and sums in double precision */
#define GWL_MIXED 1 /* float-float phase, exact mod-1 reduction, FP32 sincos and
                       sums, FP64 combination */
#define GWL_MIXED_F64PHASE 2 /* the phase in FP64 per bin and detector, reduced
                       exactly modulo one cycle in FP64, then FP32 sincos and FP32
                       sums, FP64 combination: the split without the float-float
                       anchors of GWL_MIXED, for comparison.  Likelihood only
                       (gwl_loglike, gwl_loglike_host, gwl_loglike_static, and the
                       random walks of ns_replace / ns_run); gwl_grad, the Galilean
                       walk, the calibration model and multi-event batches refuse it
                       with GWL_ERR_ARG. */

#define GWL_FCUT_ISCO 0 /* h = 0 above f_ISCO = 1/(6^{3/2} pi M) */
#define GWL_FCUT_BAND 1 /* template continued to the top of the band */

#define GWL_N_PARAM 11
#define GWL_MAX_DET 4

enum {
  GWL_P_MC = 0, GWL_P_Q, GWL_P_CHI1, GWL_P_CHI2, GWL_P_DL, GWL_P_IOTA,
  GWL_P_PSI, GWL_P_RA, GWL_P_DEC, GWL_P_TC, GWL_P_PHIC
};

/* Unit-cube prior maps used by ns_replace (u in [0,1] -> parameter). */
#define GWL_PRIOR_UNIFORM 0 /* lo + u (hi - lo) */
#define GWL_PRIOR_VOLUME 1  /* [lo^3 + u (hi^3 - lo^3)]^{1/3} (uniform in volume) */
#define GWL_PRIOR_SINE 2    /* arccos(1 - 2u), on [0, pi] */
#define GWL_PRIOR_COSINE 3  /* arcsin(2u - 1), on [-pi/2, pi/2] */

/* One L-shaped detector in Earth-fixed Cartesian axes: vertex position [m]
 * and unit vectors along the two (perpendicular) arms.  The detector tensor
 * is D = (x x - y y)/2, F+ = D:e+, Fx = D:ex, and the arrival delay relative
 * to the Earth's centre is dt = -(vertex . n)/c for a source in direction n. */
typedef struct {
  double vertex[3];
  double xarm[3];
  double yarm[3];
} gwl_detector;

typedef struct {
  int precision;     /* GWL_FP64, GWL_MIXED or GWL_MIXED_F64PHASE */
  int fcut_mode;     /* GWL_FCUT_ISCO or GWL_FCUT_BAND */
  double gmst;       /* Greenwich sidereal angle [rad]; Earth rotation over the
                        segment is ignored; ra enters as ra - gmst */
  double t_ref;      /* reference time [s] from the segment start; the template's
                        coalescence time is t_ref + tc */
  int n_dim;         /* number of sampled parameters, 1..11 */
  int param_map[GWL_N_PARAM];      /* [n_dim] index into the 11-D vector */
  double fixed_theta[GWL_N_PARAM]; /* values of the parameters not sampled */
  /* unit-cube prior of each sampled coordinate (used by ns_replace) */
  int prior_kind[GWL_N_PARAM];
  double prior_lo[GWL_N_PARAM];
  double prior_hi[GWL_N_PARAM];
  int periodic[GWL_N_PARAM]; /* 1: the coordinate wraps in the unit cube */
} gwl_options;

typedef struct gwl_ctx gwl_ctx;

/* Create a context for one data segment (Eq. 2's d, S and detectors).
 *   freqs  host [n_bins]          uniformly spaced ascending frequencies [Hz]
 *                                 f_j = f_0 + j df, f_0 > 0 (checked to 1e-9 df)
 *   strain host [n_det][n_bins][2] complex frequency-domain data d_j (re, im)
 *   psd    host [n_det][n_bins]   one-sided noise PSD S_j > 0
 *   dets   host [n_det]           detector geometry, 1 <= n_det <= GWL_MAX_DET
 *   opt    host                   options (copied)
 * The library copies the inputs to the device, builds its tables there
 * (basis functions of the PN phase, data weights, <h|h> prefix sums) and owns
 * them until gwl_destroy.  Uses the current CUDA device.  *out receives the
 * context, or NULL on failure. */
int gwl_create(const double* freqs, int64_t n_bins, const double* strain, const double* psd,
               const gwl_detector* dets, int n_det, const gwl_options* opt, gwl_ctx** out);

/* Batched log-likelihood (Eq. 2 as the log-likelihood ratio).
 *   theta_dev dev [B][n_dim] FP64 sampled coordinates (with the calibration
 *             model: [B][n_dim + 2 n_nodes n_det], see gwl_set_calibration)
 *   lnl_dev   dev [B]        FP64 output
 * B >= 0 (B = 0 is a no-op). */
int gwl_loglike(gwl_ctx* ctx, const double* theta_dev, int64_t B, double* lnl_dev, void* stream);

/* As gwl_loglike with host buffers, synchronising the stream before
 * returning.  Page-locked (pinned) buffers are read and written in place by
 * the kernels (device-accessible under unified addressing; on GB300 over the
 * CPU-GPU link), so no staging copies are made; pageable buffers are copied
 * through device memory. */
int gwl_loglike_host(gwl_ctx* ctx, const double* theta_host, int64_t B, double* lnl_host,
                     void* stream);

/* Calibration model (Section 2.2 of the paper: the calibration uncertainty
 * of each interferometer's data is modelled by amplitude and phase
 * corrections at frequency nodes, ten nodes and twenty parameters per
 * detector in the paper's analyses).  With n_nodes > 0 the template of
 * detector d is multiplied bin by bin by
 *   C_d(f) = (1 + dA_d(f)) exp(i dphi_d(f)),
 * dA_d and dphi_d [rad] natural cubic splines in ln f through the node values
 * (the end cubics continued outside the nodes), and each row of theta for
 * gwl_loglike, gwl_loglike_host and gwl_loglike_static holds
 * n_dim + 2 n_nodes n_det doubles: the n_dim sampled coordinates, then for
 * each detector d (gwl_create's order) dA at the nodes followed by dphi at
 * the nodes.
 *   n_nodes     0 (off, the default) or 2 .. GWL_MAX_CAL_NODES
 *   node_freqs  host [n_nodes] positive, strictly increasing [Hz]; copied
 *   sigma_amp, sigma_phase  > 0: widths of the zero-mean Gaussian priors of
 *               the amplitude and phase [rad] corrections, used where
 *               ns_replace / ns_run map unit-cube coordinates to parameters
 *               (theta = sigma Phi^{-1}(u); never periodic)
 * A set-up call like gwl_create: it synchronises the device and builds
 * per-bin tables there (about 70 bytes per bin).  gwl_grad then also returns
 * the derivatives with respect to the calibration parameters, and ns_replace
 * and ns_run walk in the n_dim + 2 n_nodes n_det coordinates (random or
 * Galilean walk).  Multi-event batches take calibrated contexts when all of
 * them have the same number of nodes (see gwl_multi_create); gwl_waveform
 * returns the template without the calibration factor.  A non-finite calibration
 * parameter gives a non-finite lnL.  The likelihood and gradient windows
 * (gwl_tuning.window, .grad_window) shrink, if needed, so that the
 * calibration rows fit in shared memory.  An argument error leaves the
 * context unchanged. */
#define GWL_MAX_CAL_NODES 16
int gwl_set_calibration(gwl_ctx* ctx, int n_nodes, const double* node_freqs, double sigma_amp,
                        double sigma_phase);

/* The context's calibration nodes (0: off) and doubles per row of theta
 * (either pointer may be null). */
int gwl_get_calibration(const gwl_ctx* ctx, int* n_nodes, int64_t* theta_stride);

/* Log-likelihood and its gradient with respect to the n_dim sampled
 * coordinates (adjoint accumulation over bins; the ISCO cut index is held
 * fixed, i.e. the gradient of the piecewise-smooth lnL).  With the calibration
 * model the rows of theta and of the gradient hold n_dim + 2 n_nodes n_det
 * doubles (gwl_set_calibration's layout): the calibration derivatives are
 * accumulated as moments of the spline weights over each spline interval,
 * then mapped to the node values through the spline's linear dependence on
 * them.
 *   theta_dev dev [B][theta_stride] FP64 (see gwl_get_calibration)
 *   lnl_dev   dev [B] FP64 output
 *   grad_dev  dev [B][theta_stride] FP64 output
 * GWL_MIXED_F64PHASE contexts are refused with GWL_ERR_ARG. */
int gwl_grad(gwl_ctx* ctx, const double* theta_dev, int64_t B, double* lnl_dev, double* grad_dev,
             void* stream);

/* Detector-projected template h_d(f_j) of each row, as evaluated by the
 * device path (zero above the cut).
 *   h_dev dev [B][n_det][n_bins][2] FP64 output */
int gwl_waveform(gwl_ctx* ctx, const double* theta_dev, int64_t B, double* h_dev, void* stream);

/* Constrained random-walk replacement (Algorithm 1's parallel sampling step
 * with a fixed-length random walk).  Each of n_chains chains starts at a live
 * point chosen uniformly among the K - 1 points other than `worst`, then makes
 * walk_len steps u' = u + scale * chol z in the unit cube (z standard normal);
 * periodic coordinates wrap, any other coordinate outside [0,1] rejects the
 * step; a step is accepted iff lnL(theta(u')) >= lnl_star.  D below is the
 * walk dimension: n_dim, plus 2 n_nodes n_det with the calibration model.
 *   live_u   dev [K][D]          unit-cube coordinates of the live points
 *   live_lnl dev [K]             their lnL
 *   chol     dev [D][D]          lower-triangular step matrix (row-major)
 *   out_u    dev [n_chains][D], out_lnl dev [n_chains],
 *   out_nacc dev [n_chains] int32 accepted steps (0 = the chain returns its
 *            start point), out_start dev [n_chains] int32 (may be NULL).
 * Random numbers: Philox4x32-10 (Salmon et al. 2011) with key = (seed low,
 * seed high 32 bits) and counter = (block, step, chain, counter low 32 bits);
 * step 0 block 0 word 0 picks the start (index = floor(w (K-1) / 2^32),
 * skipping `worst`); step s >= 1, block b gives normals 4b..4b+3 by
 * Box-Muller on word pairs: u1 = (w0 + 1) 2^-32, u2 = w1 2^-32,
 * z = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2). */
int ns_replace(gwl_ctx* ctx, const double* live_u, const double* live_lnl, int64_t K, int64_t worst,
               double lnl_star, uint64_t seed, uint64_t counter, int64_t n_chains, int walk_len,
               double scale, const double* chol, double* out_u, double* out_lnl, int32_t* out_nacc,
               int32_t* out_start, void* stream);

/* Result of ns_run. */
typedef struct {
  double lnZ;                 /* log evidence (natural log, likelihood-ratio units) */
  double lnZ_err;             /* sqrt(H / K) */
  double H;                   /* information, sum_i p_i ln L_i - ln Z */
  int64_t n_dead;             /* dead points including the final live set */
  int64_t n_proposals;        /* K + rounds * n_chains * walk_len */
  int64_t rounds;             /* parallel sampling rounds that changed the state */
  double scale;               /* walk scale at the end */
  double acceptance;          /* mean fraction of accepted walk steps per round */
  double consumed_per_round;  /* mean candidates used per round (Eq. 5 predicts K ln(1 + n_chains/K)) */
  double dlogz;               /* ln(Z + Lmax X) - ln Z at the last round */
  int64_t n_dead_returned;    /* dead points copied to the optional output arrays */
} gwl_ns_result;

/* Static parallel nested sampling (Section 3, Algorithm 1) on the context's
 * likelihood and prior, all state on the device.  K live points are drawn
 * from the prior (Philox words with step word 0xFFFFFFFF, point index k and
 * call word 0xFFFFFFFF; u = (w + 1/2) 2^-32).  Each round r: L* = worst live
 * lnL; the walk step matrix is scale times the Cholesky factor of the
 * live-set covariance in the unit cube; ns_replace's walks run with call
 * counter r; the candidates then replace successive worst points in chain
 * order, a candidate not above the current worst being discarded, until they
 * run out.  Dead point i has weight dX_i = X_{i-1} - X_i, X_i = e^{-i/K}; the
 * final live points enter with X_N/(K+1) each.  The walk scale adapts as
 * scale <- scale exp(acceptance - 1/2), clamped to [1e-3, 1].  The run stops
 * when ln(Z + Lmax X) - ln Z < dlogz or after max_rounds rounds.
 *   dead_lnl, dead_logwt host [max_dead], dead_u host [max_dead][D] (D as for ns_replace)
 *   (may be NULL; the first min(n_dead, max_dead) dead points in death order,
 *   the final live points last with their equal weights).
 * Synchronises the stream before returning. */
int ns_run(gwl_ctx* ctx, int64_t K, int64_t n_chains, int walk_len, uint64_t seed, double dlogz,
           int64_t max_rounds, double scale0, int64_t max_dead, double* dead_lnl, double* dead_logwt,
           double* dead_u, gwl_ns_result* out, void* stream);

/* Checkpoint and resume of ns_run (an interface addition without a
 * counterpart in the paper).  The state of a run between rounds is its live
 * set (u and lnL), the walk's L*, scale, worst index and round counter, the
 * evidence and information accumulators, and the dead points so far.  The
 * walk's normals come from a counter-based generator keyed by the round
 * counter, so a run split into calls continues bit for bit: calls with
 * max_rounds R1, R2, ..., each resuming from the previous call's checkpoint
 * and all other arguments equal, give the same results, dead points and
 * checkpoints as one call with R1 + R2 + ....
 *   resume      host [ns_state_doubles(K, D, m)] or NULL: a checkpoint written
 *               by an earlier call with the same K and walk dimension D (m
 *               that call's max_dead); the run continues from it, so scale0
 *               and the seed's initial draw are unused
 *   checkpoint  host [ns_state_doubles(K, D, max_dead)] or NULL: receives the
 *               state after this call's last round, before the final live
 *               points join the dead list
 * out and the dead-point arrays are filled as by ns_run, as if the run
 * stopped after this call.  Dead points beyond the max_dead of the call that
 * wrote a checkpoint are not carried in it.  A resume buffer of another
 * format, K or D gives GWL_ERR_ARG.  Synchronises the stream. */
int ns_run_resumable(gwl_ctx* ctx, int64_t K, int64_t n_chains, int walk_len, uint64_t seed, double dlogz,
                     int64_t max_rounds, double scale0, int64_t max_dead, double* dead_lnl, double* dead_logwt,
                     double* dead_u, gwl_ns_result* out, const double* resume, double* checkpoint, void* stream);

/* Doubles in a checkpoint of a run with K live points in D walk dimensions
 * keeping up to max_dead dead points; -1 for K < 2, D < 1 or max_dead < 0. */
int64_t ns_state_doubles(int64_t K, int64_t D, int64_t max_dead);

/* Diagnostic: the float-float elementary functions of the mixed prologue
 * (about 48 significant bits on the FP32 pipe) on n arguments, for checking
 * their accuracy against FP64 references, and the FP32 sin(pi x), cos(pi x)
 * of the mixed gradient's bin loop.  (An interface addition without a
 * counterpart in the paper.)
 *   x_dev   dev [n] FP64 arguments (split into float pairs first; rounded to
 *           FP32 for GWL_F32_SINPI and GWL_F32_COSPI); the domains of the
 *           functions: exp |x| < 87 (a normal float result), ln 2^-126 < x <
 *           2^127, sin and cos |x| < 2^11 (the reduction by pi/2 is exact
 *           there), sinpi and cospi |x| <= 1.5; outside them the results are
 *           unspecified
 *   fn      GWL_FF_EXP, GWL_FF_LOG, GWL_FF_SIN, GWL_FF_COS, GWL_F32_SINPI or
 *           GWL_F32_COSPI
 *   out_dev dev [n] FP64 results (the float pair summed in FP64, or the
 *           FP32 result widened)
 * Enqueues one kernel on the stream and returns. */
#define GWL_FF_EXP 0
#define GWL_FF_LOG 1
#define GWL_FF_SIN 2
#define GWL_FF_COS 3
#define GWL_F32_SINPI 4
#define GWL_F32_COSPI 5
int gwl_ff_eval(const double* x_dev, int64_t n, int fn, double* out_dev, void* stream);

/* Diagnostic: the Philox4x32-10 generator of ns_replace and ns_run (Salmon,
 * Moraes, Dror & Shaw 2011) on given counters and keys, so that the device
 * generator can be checked against the generator's published known-answer
 * vectors.  (An interface addition without a counterpart in the paper.)
 *   in_dev  dev [n][6] uint32: counter words c0..c3, then key words k0, k1
 *   out_dev dev [n][4] uint32: the output block x0..x3
 * GWL_ERR_ARG for n < 0 or a null pointer with n > 0.  Enqueues one kernel
 * on the stream and returns. */
int gwl_test_philox(const uint32_t* in_dev, int64_t n, uint32_t* out_dev, void* stream);

/* ---- many events in one batch ----
 * A multi-event context groups n_events contexts (same device, detector
 * count, precision, sampled dimension and number of calibration nodes;
 * different segment lengths, priors, calibration node frequencies and
 * calibration prior widths allowed).  GWL_MIXED_F64PHASE contexts are
 * refused with GWL_ERR_ARG.  It borrows the contexts: they must outlive it.
 * A context's calibration may be changed afterwards (the batch rebuilds its
 * device descriptors on its next call), but gwl_multi_loglike and
 * gwl_multi_ns_run return GWL_ERR_ARG while the contexts' node counts
 * differ. */
typedef struct gwl_multi gwl_multi;

int gwl_multi_create(gwl_ctx* const* ctxs, int n_events, gwl_multi** out);

/* Batched lnL of n_per proposals of every event in one launch sequence
 * (prologue, a persistent bin loop over (event, window) tasks, combination).
 *   theta_dev dev [n_events][n_per][theta_stride] (n_dim sampled coordinates,
 *             then with the calibration model each event's calibration
 *             parameters in gwl_set_calibration's layout)
 *   lnl_dev   dev [n_events][n_per] */
int gwl_multi_loglike(gwl_multi* m, const double* theta_dev, int64_t n_per, double* lnl_dev, void* stream);

/* ns_run for all events at once: every round is one sequence of launches
 * (CUDA graph) covering all events; each event has its own live set, walk
 * scale and Philox key seed + e * 0x9E3779B97F4A7C15, and walks in its
 * theta_stride unit-cube coordinates (random walk).  Stops when every
 * event's stopping rule holds or after max_rounds.  out: [n_events] results
 * (no dead-point arrays).  Synchronises the stream. */
int gwl_multi_ns_run(gwl_multi* m, int64_t K, int64_t n_chains, int walk_len, uint64_t seed, double dlogz,
                     int64_t max_rounds, double scale0, gwl_ns_result* out, void* stream);

/* gwl_multi_ns_run continued from a checkpoint and/or writing one (the
 * counterpart of ns_run_resumable for a batch of events; no dead points).
 *   resume      host [gwl_multi_ns_state_doubles(m, K)] or NULL: a state
 *               written by an earlier call on the same batch with the same K;
 *               the run continues from it bit for bit (the walks' random
 *               numbers are keyed by each event's round counter, which the
 *               state carries)
 *   checkpoint  host [gwl_multi_ns_state_doubles(m, K)] or NULL: receives
 *               every event's state after this call's rounds, before the
 *               final live points are added to the evidence
 * A resume buffer of another format, event count, K or walk dimension gives
 * GWL_ERR_ARG.  Synchronises the stream. */
int gwl_multi_ns_run_resumable(gwl_multi* m, int64_t K, int64_t n_chains, int walk_len, uint64_t seed, double dlogz,
                               int64_t max_rounds, double scale0, gwl_ns_result* out, const double* resume,
                               double* checkpoint, void* stream);

/* Doubles in a checkpoint of gwl_multi_ns_run_resumable for this batch and
 * K (5 + n_events (10 + NS statistics + K (D + 1)) with D the batch's walk
 * dimensions); -1 for a null batch or K < 2. */
int64_t gwl_multi_ns_state_doubles(const gwl_multi* m, int64_t K);

/* Kernel launches issued by the multi-event context. */
int64_t gwl_multi_launch_count(const gwl_multi* m);

void gwl_multi_destroy(gwl_multi* m);

/* Size of the fixed device array used by gwl_loglike_static (16 MiB). */
#define GWL_STATIC_SCRATCH_BYTES (16u << 20)

/* gwl_loglike for callers that cannot allocate device memory at call time.
 * (The paper has no counterpart; this is an interface addition.)  Some hosts
 * hand all free device memory to their own caching allocator, so a raw
 * cudaMalloc can fail; others run in loops that must not block, and
 * cudaMalloc/cudaFree may synchronise the device.  This entry point computes
 * exactly what gwl_loglike computes, with the same kernels, but takes its
 * per-call scratch (per-proposal coefficients and per-window partial sums)
 * from a fixed file-scope device array of GWL_STATIC_SCRATCH_BYTES, which the
 * library's CUDA module reserves on every device that loads it and keeps until
 * the process exits.  It calls no cudaMalloc, cudaFree or allocating routine;
 * per-kernel profiling (gwl_profile) is suspended for the call.
 *   - gwl_create looks up the array's device address (cudaGetSymbolAddress)
 *     on its device, afresh each time, so a context created after a
 *     cudaDeviceReset uses the new array (a reset frees every context's
 *     tables too: contexts from before it must not be used).  Only if that
 *     look-up failed does the first call on the device repeat it; such a
 *     first call must come before any stream capture.
 *   - A batch needs about (276 + 16 n_det ceil(n_bins / window)) bytes per
 *     proposal (24 n_det with the calibration model), window being the
 *     context's bin window (gwl_tuning.window); a
 *     batch that does not fit returns GWL_ERR_ARG with the sizes in the error
 *     text and launches nothing.
 *   - All calls on a device share the array and it keeps the previous call's
 *     contents (each call rewrites what it reads; the batch's work counters
 *     are cleared on the stream first).  Calls whose kernels overlap on the
 *     GPU -- from different streams, threads or contexts -- race on the array
 *     and must be serialised by the caller. */
int gwl_loglike_static(gwl_ctx* ctx, const double* theta_dev, int64_t B, double* lnl_dev, void* stream);

/* Walk used by ns_replace and ns_run. */
#define GWL_WALK_RANDOM 0   /* Gaussian random walk (default) */
#define GWL_WALK_GALILEAN 1 /* gradient-informed Galilean walk (Skilling 2012): chains
                               carry a velocity v, initially scale * chol z (normals of
                               step word 0x40000000) and from the second step on partly
                               refreshed, v <- rho v + sqrt(1 - rho^2) scale chol z
                               (normals of the step's word; rho: gwl_set_galilean).  A
                               step tries x1 = u + v and moves there if x1 is in the cube
                               with lnL >= L*.  Otherwise v is reflected off the surface
                               at x1 -- the contour (g = d lnL / du at x1) inside the cube,
                               the crossed walls (g = their outward normals summed)
                               outside it -- in the metric of Sigma = chol chol^T,
                               v' = v - 2 (v.g) / (g.Sigma g) Sigma g, and x2 = x1 + v' is
                               tried: the chain moves to x2 with v' if x2 is in the cube
                               with lnL >= L*, else stays with v <- -v.  The map keeps the
                               uniform distribution inside the contour and the velocity
                               distribution invariant.  out_nacc counts moves. */
int gwl_set_walk(gwl_ctx* ctx, int walk_kind);

/* Velocity persistence rho of the Galilean walk, in [0, 1] (1: never
 * refreshed; 0: a fresh velocity every step).  Default
 * GWL_GALILEAN_PERSISTENCE.  GWL_ERR_ARG outside [0, 1]. */
#define GWL_GALILEAN_PERSISTENCE 0.5
int gwl_set_galilean(gwl_ctx* ctx, double persistence);

/* Synchronise the context's last stream and return the latched device
 * status (GWL_OK or GWL_ERR_TIMEOUT); clears the latch. */
int gwl_sync(gwl_ctx* ctx);

/* Diagnostic (an interface addition without a counterpart in the paper):
 * exercises the timeout path of the kernels' bounded waits.  One thread
 * waits on a shared-memory barrier phase that nothing completes, for about
 * `seconds` of SM clock (0 < seconds <= 2), then latches the timeout status
 * and leaves, as a kernel whose bulk copy never landed would; the next
 * gwl_sync returns GWL_ERR_TIMEOUT and clears it, and the context stays
 * usable.  Enqueues one kernel on the stream and returns; GWL_ERR_ARG for a
 * null context or seconds outside (0, 2]. */
int gwl_test_wait_timeout(gwl_ctx* ctx, double seconds, void* stream);

/* Diagnostic (an interface addition without a counterpart in the paper):
 * counts the 32-bin blocks of the mixed likelihood bin loop whose phase
 * deltas take the float-float form (blocks whose phase excursion bound is 16
 * cycles or more: long signals in short segments, the low-frequency blocks
 * of BNS signals), one count per block and proposal, so that tests can check
 * that this path ran.  Counted on gwl_loglike and gwl_loglike_host calls.
 *   enable  1: clear the counter and count from now on (synchronises the
 *           device; allocates 8 bytes once); 0: stop counting; -1: unchanged
 *   count   (may be NULL) receives the blocks counted since enabling; reading
 *           it synchronises the device first (done before `enable` applies)
 * GWL_ERR_ARG for a null context or another enable value. */
int gwl_test_ffdelta_blocks(gwl_ctx* ctx, int enable, int64_t* count);

/* Launch shape of the bin loops (the tile the hardware sees: a window of
 * `window` frequency bins staged in shared memory, drained by warps of 32
 * lanes, one proposal per warp; the grid is sized in CTAs per SM).  The
 * result of gwl_loglike/gwl_grad depends on the shape only through the FP32
 * (mixed) or FP64 summation order, within the parity tolerances. */
typedef struct gwl_tuning {
  int window;        /* likelihood bin loop: bins per window; 0 keeps (set) */
  int ctas_per_sm;   /* likelihood bin loop: grid = ctas_per_sm x SMs; 0 keeps */
  int grad_window;   /* gradient bin loop: bins per window; 0 keeps */
  double ms_loglike; /* gwl_autotune output: best time of one gwl_loglike call
                        (ms) at the tuned batch; gwl_get_tuning: last tuned value or 0 */
  double ms_grad;    /* same for gwl_grad */
  int n_tried;       /* gwl_autotune output: launch shapes timed */
  int bin_kernel;    /* likelihood bin loop layout, GWL_BINS_*; 0 keeps (set) */
  int lane_chunk;    /* GWL_BINS_LANE: bins per chunk (a multiple of 32 dividing the
                        window; chunks of one window on segments whose per-chunk sums
                        would exceed 64 MB); 0 keeps (set) */
} gwl_tuning;

/* Layouts of the likelihood bin loop (gwl_tuning.bin_kernel).  Both compute
 * the same sums (the anchored phase of the mixed path); they differ in the
 * order in which the FP32 terms are added, within the parity tolerances.
 *   WARP: one proposal per warp, its lanes striding over the bins of a
 *         window (every precision, the calibration model, any batch).
 *   LANE: one proposal per lane, the 32 lanes of a warp walking the same bins
 *         together; proposals are grouped by their cut (the prologue files
 *         them in buckets of their last chunk of 64 bins, or of one window on
 *         long segments) and chunks of several proposals' sums are added in
 *         FP64 in chunk order.  Mixed precision without the calibration
 *         model; segments of at most 2048 chunks.  Elsewhere WARP runs.
 *   AUTO: LANE for mixed batches of 2048 proposals or more where it is
 *         available, WARP otherwise (the default). */
#define GWL_BINS_AUTO 1
#define GWL_BINS_WARP 2
#define GWL_BINS_LANE 3

/* Set the launch shape (fields as above; the ms/n_tried fields are ignored).
 * Windows and lane chunks are multiples of 32 bins.  A window or chunk that
 * is not, a window whose rows exceed 200 KB of shared memory, a negative
 * value, a ctas_per_sm above 16 or a bin_kernel outside 0..3 returns
 * GWL_ERR_ARG and changes nothing.  A chunk that does not divide the window
 * falls back to chunks of one window. */
int gwl_set_tuning(gwl_ctx* ctx, const gwl_tuning* t);

/* Read the context's current launch shape into *out. */
int gwl_get_tuning(const gwl_ctx* ctx, gwl_tuning* out);

#define GWL_TUNE_LOGLIKE 1
#define GWL_TUNE_GRAD 2

/* Autotuner: times gwl_loglike (what & GWL_TUNE_LOGLIKE) over every window in
 * {128, 192, ..., 1536} bins that fits in shared memory (at most the segment),
 * every ctas_per_sm in {1, 2, 3, 4} and both bin-loop layouts (GWL_BINS_WARP,
 * and GWL_BINS_LANE with chunks of 32 and 64 bins where it is available),
 * and gwl_grad
 * (what & GWL_TUNE_GRAD) over the same windows (those whose calibration
 * scratch fits, with the calibration model), on the caller's batch
 * theta_dev (B x theta_stride, device, row-major, read only) on `stream`, and keeps
 * the fastest shape of each in the context.  Each shape is timed with CUDA
 * events as the best of two runs of three back-to-back calls after one
 * warm-up call.  Outputs go to a device buffer the call allocates and frees;
 * scratch grows to the largest need of the shapes tried and is kept.  The
 * results are not used; windows whose per-window partial sums would exceed
 * 2 GB at this batch are skipped.  The call synchronises
 * the stream.  *out (may be NULL) receives the chosen shape and its times.  On
 * any error the previous shape is restored. */
int gwl_autotune(gwl_ctx* ctx, const double* theta_dev, int64_t B, int what, gwl_tuning* out, void* stream);

/* Kernel classes for gwl_profile_read. */
#define GWL_KERNEL_PROLOGUE 0 /* per-proposal coefficients */
#define GWL_KERNEL_BINS 1     /* windowed bin loop of gwl_loglike */
#define GWL_KERNEL_COMBINE 2  /* per-proposal combination */
#define GWL_KERNEL_GRAD 3     /* windowed bin loop of gwl_grad */
#define GWL_KERNEL_WALK 4     /* random-walk proposal/accept steps of ns_replace */
#define GWL_KERNEL_CALGRAD 5  /* calibration-moment pass of gwl_grad (calibration model) */
#define GWL_KERNEL_KINDS 6

/* Enable (1) or disable (0) per-kernel timing: while enabled, the library
 * records a CUDA event pair around every launch of its kernels on the launch
 * stream.  Enabling resets the accumulated totals. */
int gwl_profile(gwl_ctx* ctx, int enable);

/* Wait for the recorded events and return the accumulated device time [ms]
 * and launch count of one kernel class since profiling was enabled. */
int gwl_profile_read(gwl_ctx* ctx, int kind, double* total_ms, int64_t* count);

/* Device bytes held by the context (tables + scratch). */
int64_t gwl_device_bytes(const gwl_ctx* ctx);

/* Number of kernel launches the context has issued since creation. */
int64_t gwl_launch_count(const gwl_ctx* ctx);

/* Free the context's device memory.  NULL is ignored. */
void gwl_destroy(gwl_ctx* ctx);

/* Text of the calling thread's last error ("" if none). */
const char* gwl_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GWL_H */
