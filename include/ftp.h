/*
 * ftp.h - C ABI of the GB300 (sm_103a) Fast Template Periodogram library.
 *
 * The Fast Template Periodogram (Hoffman, VanderPlas, Hartman & Bakos,
 * arXiv 2101.12348) fits a fixed-shape periodic template
 *     M(x) = sum_{n=1..H} c_n cos(n x) + s_n sin(n x)            (Section 2)
 * to an irregularly sampled series S = {(t_i, y_i, sigma_i)} with the model
 *     y ~ theta1 * M(omega t - theta2) + theta3,                  (Section 2)
 * and reports at each trial frequency the power
 *     P(omega) = 1 - chi^2_min / chi^2_0  in [0, 1]               (Eq. lsp)
 * together with the best (theta1, theta2, theta3).  For every frequency the
 * library runs three steps, all as CUDA kernels on one GPU:
 *   (a) the weighted trigonometric sums at the harmonics h*omega, h <= 2H
 *       (Eqs. CCdef-YSdef), by an adjoint NFFT: Kaiser-Bessel spreading onto an
 *       oversampled grid, an equispaced FFT (cuFFT), deconvolution + gather;
 *   (b) assembly of MM' = psi^{2H} MM and YM' = psi^H YM and of the final
 *       polynomial 2 MM' d(YM') - YM' d(MM') in psi = exp(i theta2)
 *       (Section 2, Eq. finalpoly), of degree 6H-2;
 *   (c) all zeros of that polynomial by Aberth-Ehrlich iteration, scaled onto
 *       the unit circle (Section 2, end), P evaluated at every candidate,
 *       the best one polished by a Newton step (FP64 on the FP64 path,
 *       float-float on the mixed one).
 *
 * Conventions shared by every entry point
 *   - Frequencies are in cycles per unit time, omega = 2 pi f.  The grid is
 *     f_k = (k0 + k) * df, k = 0..nf-1, with k0 >= 1 (the NFFT needs the
 *     harmonics h * f_k on the same integer lattice j * df; f = 0 excluded).
 *   - theta2 is in radians in [0, 2 pi), relative to t = 0.
 *   - Weights are w_i = sigma_i^-2 / sum sigma^-2.  All sigma_i = 0 means
 *     unit weights (Section 2); a mix of zero and non-zero sigma returns
 *     FTP_ERR_MIXED_ZERO_SIGMA; all-equal y (Var(y) = 0, P undefined) returns
 *     FTP_ERR_ZERO_VARIANCE (Section 2); negative or non-finite inputs return
 *     FTP_ERR_NONFINITE; fewer than 2 observations FTP_ERR_INVALID_ARG.
 *   - Pointers to observation and output arrays may be host or device memory
 *     of the plan's device; the library asks the CUDA runtime which.  Host
 *     arrays are staged through the plan's workspace.  Every call returns
 *     only after its results are in the caller's arrays (it synchronises the
 *     plan's stream), so a returned status covers the whole computation.
 *   - Ownership: the caller owns every array it passes; the plan owns its
 *     device workspace, its cuFFT plan and its stream (unless the caller
 *     supplied one).  Nothing is retained after a call returns.
 *   - Errors: a non-FTP_OK status means the outputs were not written.  No
 *     C++ exception crosses the ABI.  Per-frequency conditions are not errors:
 *     they set bits in the optional flags array (FTP_FLAG_*).
 *   - A plan is not thread-safe: use one plan per host thread / stream.
 */
#ifndef FTP_GB300_H
#define FTP_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ftp_plan_s* ftp_plan_t;

typedef enum {
  FTP_OK = 0,
  FTP_ERR_INVALID_ARG = 1,      /* bad size, null pointer, H out of range, k0 < 1 ... */
  FTP_ERR_ZERO_VARIANCE = 2,    /* all y equal: P undefined (Section 2) */
  FTP_ERR_MIXED_ZERO_SIGMA = 3, /* some sigma = 0 and some > 0 (Section 2) */
  FTP_ERR_NONFINITE = 4,        /* NaN/Inf in t, y or sigma, or sigma < 0 */
  FTP_ERR_OOM = 5,              /* device allocation failed */
  FTP_ERR_CUDA = 6,             /* CUDA runtime or cuFFT failure */
  FTP_ERR_TIMEOUT = 7,          /* a bounded device-side wait gave up */
  FTP_ERR_UNSUPPORTED = 8       /* request exceeds what the plan was built for */
} ftp_status;

typedef enum {
  FTP_FP64 = 0,  /* FP64 everywhere: sums, assembly, roots, candidates */
  FTP_MIXED = 1  /* FP32 NFFT sums (FP64 phase reduction); assembly of MM'
                    and YM' in float-float (FMA-based two-word FP32, about
                    44 significant bits); FP32 final polynomial, Aberth and
                    candidate screening; Newton polish and evaluation of the
                    chosen phase in float-float; ill-conditioned frequencies
                    re-solved from FP64 sums */
} ftp_precision;

/* Per-frequency flag bits (uint8). */
#define FTP_FLAG_NONCONVERGED 1u  /* the root solver hit its iteration cap with a root
                                     that is not a zero of the final polynomial to the
                                     working precision, and no re-solve cleared it */
#define FTP_FLAG_DEGENERATE_MM 2u /* MM ~ 0 at the chosen phase: P set to 0 */
#define FTP_FLAG_CONSTANT_P 4u    /* final polynomial ~ 0: P independent of theta2 */
#define FTP_FLAG_NEGATIVE_AMP 8u  /* best theta1 < 0 (Section 2.1: allowed, reported) */
#define FTP_FLAG_UNRESOLVED 16u   /* ill-conditioned (or at the iteration cap) but not
                                     re-solved: the batch's re-solve list was full, or
                                     the call cannot re-solve
                                     (ftp_periodogram_sums_noalloc) */
#define FTP_FLAG_SCREENED_OUT 32u /* not evaluated: screened out by the surrogate
                                     (ftp_batch_screened); P and theta are NaN */
#define FTP_FLAG_NO_POSITIVE 64u  /* positive-amplitude mode: no candidate with
                                     theta1 > 0, so P = 0 (ftp_set_positive_amplitude) */
#define FTP_FLAG_RESOLVED 128u    /* result of a re-solve from direct FP64 sums: the
                                     frequency was ill-conditioned, or an item of it hit
                                     the Aberth cap */

#define FTP_MAX_H 16

/* Trial-frequency grid f_k = (k0 + k) * df, k = 0..nf-1, k0 >= 1.  The last
 * bin k0 + nf - 1 may be at most FTP_MAX_BIN: a grid beyond it would need an
 * FFT of more than 2^31 cells, and ftp_plan and ftp_batch return
 * FTP_ERR_UNSUPPORTED for it (df <= 0, k0 < 1 or nf < 1 are
 * FTP_ERR_INVALID_ARG). */
#define FTP_MAX_BIN ((int64_t)1 << 30)
typedef struct {
  double df;
  int64_t k0;
  int64_t nf;
} ftp_grid;

/* Template: c[n-1], s[n-1] are the cos / sin coefficients of harmonic n,
 * n = 1..H, host memory, 1 <= H <= FTP_MAX_H.  No constant term: a constant
 * is absorbed by theta3 (Section 2). */
typedef struct {
  int H;
  const double* c;
  const double* s;
} ftp_template;

/*
 * ftp_plan - create a plan for lightcurves of at most max_nobs observations,
 * templates of at most max_H harmonics, a fixed frequency grid and at most
 * max_templates templates per call.  Allocates all device workspace (the
 * NFFT grid, the sum tiles, staging for host arrays) and the cuFFT plan on
 * `device`.  cuda_stream is a cudaStream_t of that device, or NULL to let
 * the plan create its own.  On success *out receives the plan.
 */
ftp_status ftp_plan(ftp_plan_t* out, int64_t max_nobs, int max_H, ftp_grid grid,
                    int max_templates, ftp_precision prec, int device, void* cuda_stream);

/*
 * ftp_sums - step (a) only: the trig sums of Eqs. CCdef-YSdef in complex form,
 *   Z_h(f_k) = sum_i w_i exp(i h omega_k t_i),            h = 1..2*H_sums
 *   Y_h(f_k) = sum_i w_i (y_i - ybar) exp(i h omega_k t_i), h = 1..H_sums
 * (so C_h = Re Z_h, S_h = Im Z_h, YC_h = Re Y_h, YS_h = Im Y_h; CC, CS, SS
 * follow by product-to-sum identities).  sums_out (host or device) receives
 * complex values of the plan's sum type - float2 (8 bytes) for FTP_MIXED,
 * double2 (16 bytes) for FTP_FP64 - laid out row-major as [3*H_sums][nf]:
 * rows 0..2H_sums-1 hold Z_1..Z_2H_sums, rows 2H_sums..3H_sums-1 hold
 * Y_1..Y_H_sums.  moments_out (host or device, nullable) receives
 * {ybar, YY} as two doubles.  1 <= H_sums <= max_H.
 */
ftp_status ftp_sums(ftp_plan_t plan, const double* t, const double* y, const double* dy,
                    int64_t nobs, int H_sums, void* sums_out, double* moments_out);

/*
 * ftp_periodogram - the full path (a)-(c) for one lightcurve and ntemplates
 * templates sharing its sums.  Outputs are [ntemplates][nf] arrays of double
 * (host or device): power P, theta1 (amplitude), theta2 (phase, radians,
 * [0, 2 pi)), theta3 (offset); flags (uint8, same shape) is nullable.
 */
ftp_status ftp_periodogram(ftp_plan_t plan, const double* t, const double* y, const double* dy,
                           int64_t nobs, const ftp_template* tpl, int ntemplates,
                           double* power, double* theta1, double* theta2, double* theta3,
                           uint8_t* flags);

/*
 * ftp_batch - many lightcurves in one call.  Curve c owns observations
 * [obs_off[c], obs_off[c+1]) of t, y, dy and the frequency grid grids[c]
 * (each with nf <= the plan's grid.nf and a grid-size no larger than the
 * plan's); its results start at element out_off[c] of power/theta1/theta2/
 * theta3/flags and hold, per template it is run with, grids[c].nf values
 * (template-major).  tpl_of_curve[c] selects one template of `bank` for curve
 * c; NULL runs every template of the bank on every curve.  obs_off, grids,
 * out_off, tpl_of_curve and bank are host arrays; t, y, dy and the outputs
 * may be host or device.
 *
 * Execution: the curves are cut into chunks whose sum tiles fit the plan's
 * chunk budget (ftp_set_batch_options; 8 GiB by default).  Per chunk, one
 * launch prepares every curve of step (a) (weights, moments, grid cells and
 * tile order, one CTA per curve); spreading, FFT and gather then run curve by
 * curve, several curves at once on concurrent streams (ftp_set_batch_tuning),
 * into the chunk's sum tiles, then steps (b)-(c) run
 * as one persistent kernel launch per harmonic count H over every
 * (frequency, template) item of every curve of the chunk, and the chunk's
 * ill-conditioned frequencies are re-solved from direct FP64 sums in one more
 * launch per H (at most 2^18 per chunk; beyond that they keep their result
 * and get FTP_FLAG_UNRESOLVED).  When every array is device memory and a call
 * repeats the previous one exactly (same pointers, offsets, grids and
 * templates), the second call captures the device work into a CUDA graph and
 * later calls replay it.  The plan's batch workspace (sum tiles of one chunk,
 * staging for host arrays) is allocated on first use and kept.  A
 * device-side error (e.g. zero variance of one curve) stops the batch and is
 * returned.
 */
ftp_status ftp_batch(ftp_plan_t plan, int64_t ncurves, const int64_t* obs_off, const double* t,
                     const double* y, const double* dy, const ftp_grid* grids,
                     const int64_t* out_off, const ftp_template* bank, int nbank,
                     const int32_t* tpl_of_curve, double* power, double* theta1,
                     double* theta2, double* theta3, uint8_t* flags);

/*
 * ftp_set_batch_options - chunk budget of ftp_batch in bytes of sum tiles
 * (0 keeps the current value) and whether repeated all-device calls may be
 * captured into and replayed from a CUDA graph (default 1).
 * ftp_batch_info - of the last ftp_batch call: the number of chunks and how
 * its device work ran (0 eagerly, 1 captured into a graph and launched,
 * 2 replayed from the graph).  Each pointer is nullable.
 */
ftp_status ftp_set_batch_options(ftp_plan_t plan, int64_t chunk_bytes, int use_graph);
ftp_status ftp_batch_info(ftp_plan_t plan, int64_t* chunks, int* graph);

/*
 * ftp_multiband_periodogram - the multi-phase multi-band periodogram (Section
 * 2.2, Eq. multibandmultiphase): band b owns observations [obs_off[b],
 * obs_off[b+1]) of t, y, dy and its own amplitude, phase and offset at a
 * shared trial frequency (the plan's grid), fitted with template
 * bank[tpl_of_band[b]] (NULL: template 0 for every band).  The combined
 * power is P = sum_b chi2_0,b P_b / sum_b chi2_0,b with chi2_0,b the weighted
 * sum of squared deviations of band b from its weighted mean (raw weights
 * sigma^-2, unit weights when a band's sigma are all zero).  power [nf] and
 * the nullable per-band outputs [nbands][nf] may be host or device memory;
 * obs_off, bank and tpl_of_band are host arrays.  The bands run as one
 * ftp_batch over the plan's grid (same validation and errors).
 */
ftp_status ftp_multiband_periodogram(ftp_plan_t plan, int nbands, const int64_t* obs_off,
                                     const double* t, const double* y, const double* dy,
                                     const ftp_template* bank, int nbank,
                                     const int32_t* tpl_of_band, double* power,
                                     double* band_power, double* band_theta1,
                                     double* band_theta2, double* band_theta3,
                                     uint8_t* band_flags);

/*
 * ftp_shared_multiband - the shared-phase multi-band template periodogram
 * (Appendix A, the model of Sesar et al. 2016): band b owns observations
 * [obs_off[b], obs_off[b+1]) of t, y, dy and a template
 * bank[tpl_of_band[b]] (NULL: template 0 for every band); one amplitude
 * theta1, phase theta2 and offset theta3 are shared by all bands,
 *     y^(b) ~ theta1 M^(b)(omega t - theta2) + theta3 + offsets[b],
 * with the fixed band offsets (host array, nullable = 0) subtracted first.
 * Weights are normalised over all observations, so the polynomials MM', YM'
 * are band-weighted sums of the single-band ones (y centred on the pooled
 * mean) and the root stage is the single-band one.  Step (a) runs per band on
 * the plan's grid; the pooled polynomial coefficients are formed in FP64 and
 * the roots found with FP64 polish on both precision paths.  Outputs are [nf]
 * arrays (host or device, flags nullable) of the combined fit.  Every band
 * must fit the plan (N_obs <= max_nobs, H <= max_H); mixing bands with and
 * without uncertainties returns FTP_ERR_MIXED_ZERO_SIGMA.
 */
ftp_status ftp_shared_multiband(ftp_plan_t plan, int nbands, const int64_t* obs_off,
                                const double* t, const double* y, const double* dy,
                                const double* offsets, const ftp_template* bank, int nbank,
                                const int32_t* tpl_of_band, double* power, double* theta1,
                                double* theta2, double* theta3, uint8_t* flags);

/*
 * ftp_set_positive_amplitude - constrain the template amplitude to
 * theta1 >= 0 in every later call of the plan (Section 2.1 allows negative
 * amplitudes and leaves the choice to the user; default off).  At a fixed
 * phase the best theta1 >= 0 is YM/MM when YM > 0 and 0 otherwise, so the
 * constrained power is P(theta2) [YM(theta2) > 0]; since P vanishes where YM
 * does, its maximum on each arc with YM > 0 is a stationary point, i.e. one of
 * the polynomial's candidates, and the best candidate with theta1 > 0 is the
 * exact constrained optimum.  Frequencies without one get P = 0, theta1 = 0,
 * theta2 = 0, theta3 = ybar and FTP_FLAG_NO_POSITIVE.  Costs nothing extra.
 */
ftp_status ftp_set_positive_amplitude(ftp_plan_t plan, int enable);

/*
 * Batch tuning.  Two choices of ftp_batch depend on the GPU and the shape of
 * the batch: how many curves run step (a) at once (sum_lanes, 1..8: each lane
 * has its own stream, workspace and FFT plans; default 4) and how many CTAs
 * per SM the persistent root-finding launches use (roots_ctas_per_sm; 0 = as
 * many as fit, the default).  ftp_set_batch_tuning / ftp_get_batch_tuning
 * set and read them.
 *
 * ftp_batch_autotune - picks both by timing them on the given batch
 * (arguments as ftp_batch; the outputs are used as scratch and overwritten):
 * each lane count in {1, 2, 4, 8} by the device time of step (a), then each
 * CTA count in {all that fit, 4, 3, 2} by the time of the root stage; the
 * fastest (a later candidate must win by 3 % / 2 %) is kept for the plan.
 * cache_path (nullable) names a JSON file of earlier results keyed by the
 * device, precision, largest H, template mode and log2 classes of the curve
 * count, median N_obs and median N_f: a cached class is applied without
 * timing (*from_cache = 1), a new one is timed and added.  Costs about ten
 * ftp_batch calls when it times.
 */
ftp_status ftp_set_batch_tuning(ftp_plan_t plan, int sum_lanes, int roots_ctas_per_sm);
ftp_status ftp_get_batch_tuning(ftp_plan_t plan, int* sum_lanes, int* roots_ctas_per_sm);
ftp_status ftp_batch_autotune(ftp_plan_t plan, int64_t ncurves, const int64_t* obs_off,
                              const double* t, const double* y, const double* dy,
                              const ftp_grid* grids, const int64_t* out_off,
                              const ftp_template* bank, int nbank, const int32_t* tpl_of_curve,
                              double* power, double* theta1, double* theta2, double* theta3,
                              const char* cache_path, int* from_cache);

/* Release the plan's device memory, cuFFT plan and owned stream.  NULL is a no-op. */
void ftp_destroy(ftp_plan_t plan);

/* Static, human-readable name of a status code. */
const char* ftp_status_string(ftp_status status);

/*
 * ftp_plan_info - introspection for tests and benchmarks: fills (each
 * pointer nullable) the NFFT grid length n, the Kaiser-Bessel half-width m,
 * the number of spreading tiles, and the number of kernel launches the last
 * ftp_periodogram / ftp_sums call issued (cuFFT's own kernels excluded).
 */
ftp_status ftp_plan_info(ftp_plan_t plan, int64_t* grid_len, int* half_width, int64_t* ntiles,
                         int* last_launches);

/*
 * ftp_solver_stats - root-solver statistics of the last call:
 *   items          (frequency, template) items solved by the main pass;
 *   mean_iterations mean Aberth iterations per item (iterations of the warp
 *                  that solved it);
 *   nonconverged   items whose main-pass iteration hit the cap with a root
 *                  that is not a zero of the final polynomial to the working
 *                  precision (|F(z)| above 8 D eps sum_k |F_k| |z|^k);
 *   resolved       frequencies re-solved from direct FP64 sums: those where
 *                  the a-posteriori estimate of the error of P caused by the
 *                  NFFT sums exceeded 2.5e-5 (FTP_MIXED) or 1e-10 (FTP_FP64) -
 *                  clustered phases make MM = Var(M) a small difference of
 *                  O(1) sums - and those with a non-converged item;
 *   resolved_nonconverged  the latter kind among them;
 *   still_nonconverged  items left at the cap after their re-solve, or not
 *                  re-solved at all (these keep FTP_FLAG_NONCONVERGED).
 * Section 2 takes every stationary point as a candidate, so an item whose
 * roots did not all converge is re-solved rather than only reported: from
 * direct FP64 sums with the re-solve cap of ftp_set_solver_limits, accepting
 * a root whose correction has stalled once F's value there is at the rounding
 * level of its evaluation (clustered and multiple roots); on FTP_MIXED the
 * re-solve iterates in FP32 and items still at the cap after it get one more
 * re-solve with FP64 iterations.  Each pointer is nullable.
 */
ftp_status ftp_solver_stats(ftp_plan_t plan, int64_t* items, double* mean_iterations,
                            int64_t* nonconverged, int64_t* resolved,
                            int64_t* resolved_nonconverged, int64_t* still_nonconverged);

/*
 * ftp_set_solver_limits - iteration caps and wait bounds of the root stage
 * for later calls of the plan (0 restores a default):
 *   maxit        Aberth iteration cap of the main pass (default 60 on
 *                FTP_MIXED, 80 on FTP_FP64; 1..100000);
 *   redo_maxit   cap of the re-solve passes (default 200; 1..100000);
 *   wait_polls   polls of each bounded wait of the roots kernels for their
 *                staged sum tiles before they give up and the call returns
 *                FTP_ERR_TIMEOUT (default 2^20; >= 1).
 * Errors: FTP_ERR_INVALID_ARG for a null plan or a value out of range.
 */
ftp_status ftp_set_solver_limits(ftp_plan_t plan, int maxit, int redo_maxit, int wait_polls);

/*
 * ftp_set_fault_injection - for tests of the failure path, without any GPU
 * fault.  mode 1: the roots kernels arm their waits for the staged sum tiles
 * but never issue the copies, so every wait runs out after the plan's
 * wait_polls polls, the kernels return early and the call returns
 * FTP_ERR_TIMEOUT; no copy is in flight when a kernel gives up.  mode 0
 * (default) turns it off, and the next call runs normally.  Errors:
 * FTP_ERR_INVALID_ARG for a null plan or another mode.
 */
ftp_status ftp_set_fault_injection(ftp_plan_t plan, int mode);

/*
 * ftp_stage_times - per-stage device times (milliseconds) of the last
 * ftp_periodogram call when timing was enabled with ftp_set_timing(plan, 1),
 * measured with CUDA events on the plan's stream: [0] moments, phase
 * reduction and binning, [1] spreading, [2] FFT, [3] deconvolution + gather,
 * [4] assembly + roots + candidates + polish (all template groups),
 * [5] re-solve of ill-conditioned frequencies from direct FP64 sums.
 * After ftp_batch (timed calls run eagerly, without a graph): [0] all of
 * step (a) for every curve, [1] features, surrogate scores and selection
 * (screened and features-only batches; zero otherwise), [2]-[3] zero, [4]
 * and [5] as above, summed over the chunks.
 */
ftp_status ftp_set_timing(ftp_plan_t plan, int enable);
ftp_status ftp_stage_times(ftp_plan_t plan, float* ms6);

/*
 * ftp_roots_first_phase_ms - device time (milliseconds, CUDA events on the
 * plan's stream) of the first of the two root-stage kernels in the last
 * timed ftp_periodogram call, summed over its template groups: assembly of
 * the polynomial of Section 2, the Aberth-Ehrlich iterations and the choice of
 * the best candidate root (Section 2, final polynomial and its roots).  The
 * second kernel (FP64-class polish and evaluation at that root, outputs)
 * takes the rest of stage [4] of ftp_stage_times.  The re-solve pass is not
 * included.  Zero unless timing was enabled with ftp_set_timing(plan, 1);
 * not recorded by ftp_batch.  Errors: FTP_ERR_INVALID_ARG for a null plan or
 * pointer.
 */
ftp_status ftp_roots_first_phase_ms(ftp_plan_t plan, float* ms);

/*
 * ftp_periodogram_sums_noalloc - steps (b)-(c) on sums the caller already
 * holds, allocating nothing.  The paper has no counterpart: this is an entry
 * point for callers that cannot call cudaMalloc - a process whose device
 * memory belongs to another runtime's pool allocator, a latency-bound loop
 * where cudaMalloc/cudaFree (which may synchronise the device) are not
 * acceptable, or a service under a hard device-memory cap.  It needs no plan.
 *
 *   sums        device pointer, 16-byte aligned: the layout ftp_sums writes
 *               (rows 0..2H_sums-1 = Z_1..Z_2H_sums, then H_sums rows
 *               Y_1..Y_H_sums) with consecutive rows row_stride elements
 *               apart; elements are float2 for FTP_MIXED, double2 for FTP_FP64
 *   row_stride  >= nf rounded up to a multiple of 64, and row_stride times
 *               the element size a multiple of 16 bytes (whole work units are
 *               read; the padding may hold anything)
 *   ybar, YY    the weighted mean and variance (ftp_sums' moments_out)
 *   tpl         1..FTP_NOALLOC_MAX_TEMPLATES templates with H <= H_sums
 *   outputs     device arrays [ntemplates][nf], as ftp_periodogram (flags
 *               nullable)
 *   device, cuda_stream   the device the pointers belong to and a stream of
 *               it (NULL = default stream); the call returns after the stream
 *               has finished its work
 *
 * Scratch: a fixed FTP_NOALLOC_SCRATCH_BYTES-byte array in the library's own
 * device memory, held by every GPU that loads the library until the process
 * exits.  The first call on a device looks up its address (make that first
 * call before any stream capture).  Calls share the array: every value the
 * kernel reads is written at the start of each call, and calls that overlap
 * on the GPU race on it.  Requests beyond the array (more than
 * FTP_NOALLOC_MAX_TEMPLATES templates) return FTP_ERR_UNSUPPORTED before any
 * device work; bad sizes, strides, alignment or host pointers return
 * FTP_ERR_INVALID_ARG, and so do pointers to another GPU's memory.
 * Unlike ftp_periodogram it cannot re-solve anything from the observations,
 * which it does not see: items whose estimated error of P from the sums
 * exceeds 2.5e-5 (FTP_MIXED) or 1e-10 (FTP_FP64) get FTP_FLAG_UNRESOLVED, and
 * items that hit the Aberth iteration cap keep FTP_FLAG_NONCONVERGED.  The
 * flags array is the only per-item report of either.  Each call copies its
 * small parameter tables from host memory into the scratch array and waits
 * for the stream before it returns.
 */
#define FTP_NOALLOC_MAX_TEMPLATES 64
#define FTP_NOALLOC_SCRATCH_BYTES (512 + FTP_NOALLOC_MAX_TEMPLATES * FTP_MAX_H * 16)
ftp_status ftp_periodogram_sums_noalloc(const void* sums, int64_t row_stride,
                                        ftp_precision prec, int64_t nf, int H_sums, double ybar,
                                        double YY, const ftp_template* tpl, int ntemplates,
                                        double* power, double* theta1, double* theta2,
                                        double* theta3, uint8_t* flags, int device,
                                        void* cuda_stream);

/*
 * ftp_alu_peak - a measurement utility, not part of the paper's method: the
 * peak rate of the plain ALUs on `device`, the denominator of the root
 * stage's roofline.  One launch of independent fused multiply-add chains
 * (every SM, 32 warps each) runs `iters` outer iterations (1..2^26) after a
 * short warm-up launch; *flops receives the floating-point operations it
 * performed (2 per FMA) and *ms its device time (CUDA events).  kind 0: FP32
 * fma.rn.f32; 1: packed FP32 pairs fma.rn.f32x2; 2: FP64 fma.rn.f64.  It
 * allocates a few bytes of device memory for the kernel's guarded store.
 * Errors: FTP_ERR_INVALID_ARG for a bad kind, count, pointer or device;
 * FTP_ERR_CUDA if the launch fails.
 */
ftp_status ftp_alu_peak(int device, int kind, int iters, double* flops, float* ms);

/* ------------------------------------------------------------------------
 * Learned screening.  The paper has no surrogate: these entry points rank the
 * trial frequencies of a lightcurve with a small network so that the exact
 * solve of steps (b)-(c) runs only on the most promising ones and their
 * neighbours.  The network reads 2 H_f + 2 features per frequency taken from
 * the step (a) sums (so they cost no extra pass over the observations):
 *   x[h-1]      the floating-mean Lomb-Scargle power at h*omega (the H = 1
 *               template periodogram, Section 2.1), h = 1..H_f
 *   x[H_f+h-1]  |Y_h|^2 / YY, h = 1..H_f
 *   x[2 H_f]    the multi-harmonic least-squares power with H_f harmonics
 *               (Section 2.1), an upper bound of the template power
 *   x[2 H_f+1]  log10(N_obs)
 * and predicts the template power P.  It is 2H_f+2 -> 128 -> 128 -> 1 with
 * ReLU, BF16 weights and activations and FP32 accumulation on the tensor
 * cores.  Parameters are a flat FP32 array:
 *   W1 [128][nfeat] | b1 [128] | W2 [128][128] | b2 [128] | w3 [128] | b3
 * (row-major, W2[j][i] maps input i to output j).
 * ------------------------------------------------------------------------ */
typedef struct ftp_mlp_s* ftp_mlp_t;

/* Number of parameters for nfeat inputs (1 <= nfeat <= 18), or -1. */
int64_t ftp_mlp_param_count(int nfeat);

/*
 * ftp_mlp_create - a network of nfeat inputs on `device`, with its FP32
 * master parameters, Adam moments and gradient workspace.  params (host or
 * device, nullable) gives the initial parameters; NULL draws each layer's
 * weights and biases uniformly in +-1/sqrt(fan_in) from `seed`.
 * cuda_stream: a stream of that device, or NULL for one of its own.
 */
ftp_status ftp_mlp_create(ftp_mlp_t* out, int nfeat, const float* params, uint64_t seed,
                          int device, void* cuda_stream);
void ftp_mlp_destroy(ftp_mlp_t mlp);
/* Copy the parameters out / in (host or device arrays of
 * ftp_mlp_param_count floats); set also resets the Adam state. */
ftp_status ftp_mlp_get_params(ftp_mlp_t mlp, float* params);
ftp_status ftp_mlp_set_params(ftp_mlp_t mlp, const float* params);
/*
 * ftp_mlp_get_state / ftp_mlp_set_state - the whole training state, for a
 * checkpoint: the parameters and Adam's first and second moments (host or
 * device arrays of ftp_mlp_param_count floats each, none nullable) and the
 * number of Adam steps taken, which keys the minibatch draws of
 * ftp_mlp_train and Adam's bias correction.  A handle given the state that
 * another handle of the same nfeat returned continues training bit for bit
 * as that handle would have (the gradient reductions have a fixed order).
 * set_state: steps must lie in [0, 2^31 - 2^20]; FTP_ERR_INVALID_ARG
 * otherwise or for a null pointer.  Both calls synchronise the handle's
 * stream.
 */
ftp_status ftp_mlp_get_state(ftp_mlp_t mlp, float* params, float* adam_m, float* adam_v,
                             int64_t* steps);
ftp_status ftp_mlp_set_state(ftp_mlp_t mlp, const float* params, const float* adam_m,
                             const float* adam_v, int64_t steps);

/* Scores of n rows of X [n][nfeat] (FP32, host or device) into scores [n]. */
ftp_status ftp_mlp_forward(ftp_mlp_t mlp, const float* X, int64_t n, float* scores);

/*
 * ftp_mlp_gradient - gradient (nullable, ftp_mlp_param_count floats, host or
 * device) and value (loss, nullable, host or device) of the mean squared
 * error mean_i (s(X[r_i]) - target[r_i])^2 over the n rows r_i = idx[i]
 * (idx nullable: r_i = i) of X [rows][nfeat] / target [rows].  The error
 * signals of the backward pass are rounded to BF16 where they enter the
 * weight-gradient products, as the tensor cores consume them.
 */
ftp_status ftp_mlp_gradient(ftp_mlp_t mlp, const float* X, const float* target, int64_t rows,
                            const int64_t* idx, int64_t n, float* grad, float* loss);

/*
 * ftp_mlp_train - `steps` Adam steps (beta = 0.9 / 0.999, eps = 1e-8, rate
 * lr) on minibatches of `batch` rows of X / target (device arrays), drawn
 * with replacement by a counter-based generator keyed by `seed` and the
 * step count.  losses (host or device, nullable) receives each step's
 * minibatch loss.
 */
ftp_status ftp_mlp_train(ftp_mlp_t mlp, const float* X, const float* target, int64_t rows,
                         int64_t steps, int64_t batch, float lr, uint64_t seed, float* losses);

/*
 * ftp_batch_features - step (a) and the screening features for many curves
 * (arguments as ftp_batch); curve c's 2 H_feat + 2 features of frequency k
 * go to row row_off[c] + k of `features` (device, FP32 [rows][2 H_feat + 2]).
 * row_off is a host array.  1 <= H_feat <= min(8, the plan's max_H).
 */
ftp_status ftp_batch_features(ftp_plan_t plan, int64_t ncurves, const int64_t* obs_off,
                              const double* t, const double* y, const double* dy,
                              const ftp_grid* grids, const int64_t* row_off, int H_feat,
                              float* features);

/*
 * ftp_batch_screened - ftp_batch with screening: per curve, the features of
 * every frequency are scored by `mlp` (H_feat = (nfeat - 2) / 2), the
 * ceil(top_frac * nf) best scores and their +-neighbours frequencies are
 * selected, and steps (b)-(c) run on the work units that hold a selected
 * frequency (a unit is a few consecutive frequencies, so a little more than
 * the selection is evaluated).  Evaluated frequencies get exact results;
 * the others NaN with FTP_FLAG_SCREENED_OUT.  0 < top_frac <= 1.
 */
ftp_status ftp_batch_screened(ftp_plan_t plan, int64_t ncurves, const int64_t* obs_off,
                              const double* t, const double* y, const double* dy,
                              const ftp_grid* grids, const int64_t* out_off,
                              const ftp_template* bank, int nbank, const int32_t* tpl_of_curve,
                              ftp_mlp_t mlp, double top_frac, int neighbours, double* power,
                              double* theta1, double* theta2, double* theta3, uint8_t* flags);

/*
 * ftp_training_rows - training rows for the surrogate from exact results:
 * per curve (rows row_off[c] .. row_off[c+1]-1 of power [rows] and
 * features [rows][nfeat], device arrays; row_off on the host), the rows
 * among the ceil(top_frac * nf) largest powers and their +-neighbours, and
 * every row whose counter-based hash (keyed by seed) falls below rand_frac,
 * are appended in order to X_out [cap][nfeat] / y_out [cap] (device) from
 * row *count on; *count (host) is advanced by the rows selected (rows past
 * cap are counted, not written).
 */
ftp_status ftp_training_rows(const double* power, const float* features, int nfeat,
                             int64_t ncurves, const int64_t* row_off, double top_frac,
                             int neighbours, double rand_frac, uint64_t seed, float* X_out,
                             float* y_out, int64_t cap, int64_t* count, int device,
                             void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* FTP_GB300_H */
