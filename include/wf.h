/*
 * wf.h -- C ABI of the GB300 (sm_103a) Wiener-reconstruction library (libwf.so).
 *
 * The library computes the hot path of the ARGO Wiener reconstruction of Kitaura et al.
 * 2009 ("Cosmic cartography of the large-scale structure with SDSS DR6",
 * arXiv:0906.3978):
 *   galaxies --(Sec. 3.1.2 supersampling: CIC/TSC on a finer grid, ideal low-pass)--> n_obs
 *   n_obs, w --(Sec. 3.2 data/noise model: eq:datamodel, eq:nmean, eq:noiseav)--> d, b
 *   b, w, P(k) --(Sec. 3.3.1, Eq. eq:WF, Krylov inversion)--> s = <delta_g>_WF
 *
 * General conventions
 *   - Grids are cubic and periodic: N cells per axis, row-major [x][y][z] (z fastest), node
 *     i at position i*H, H = box/N.  N must be even, of the form 2^a 3^b, and one of the
 *     sizes wf_supported_size() accepts (16..512).
 *   - "dev" pointers are CUDA device pointers on the context's device; "host" pointers
 *     are ordinary host memory.  The caller owns every pointer it passes; the library never
 *     frees or retains them beyond the call (wf_submit copies its inputs).
 *   - stream: a cudaStream_t passed as void* (NULL = legacy default stream).  Device work
 *     is stream-ordered on it; a call returns after its device work is enqueued unless the
 *     description says it waits (calls that return host scalars wait for them).
 *   - Every call returns a wf_status.  No call aborts, exits, prints or traps; CUDA errors
 *     are returned as WF_ERR_CUDA (wf_last_error() describes the last one).
 *   - Floating point: FP64 storage for every field crossing the ABI.
 */
#ifndef WF_H_
#define WF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  WF_OK = 0,
  WF_PENDING = 1,            /* wf_poll: request not finished yet */
  WF_ERR_ARG = -1,           /* invalid argument (sizes, pointers, non-finite input) */
  WF_ERR_OOM = -2,           /* device allocation failed or HBM budget exceeded */
  WF_ERR_CUDA = -3,          /* a CUDA runtime call failed */
  WF_ERR_NOT_CONVERGED = -4, /* iteration cap reached; info is filled */
  WF_ERR_BREAKDOWN = -5,     /* CG breakdown: p.Ap <= 0 or a non-finite scalar */
  WF_ERR_TIMEOUT = -6,       /* a bounded wait gave up */
  WF_ERR_OVERFLOW = -7,      /* a fine-grid cell would exceed 2^64-1 (>= 65536 galaxies) */
  WF_ERR_BUSY = -8,          /* serving queue full */
  WF_ERR_UNSUPPORTED = -9    /* grid size not compiled into this library */
} wf_status;

typedef struct wf_ctx wf_ctx;

/* Cubic periodic grid: n cells per axis, box side (length units of the positions),
 * supersample = 1 (plain gridding) or 2 (fine grid 2n, Sec. 3.1.2). */
typedef struct {
  int n;
  double box;
  int supersample;
} wf_grid;

typedef enum { WF_CIC = 1, WF_TSC = 2 } wf_scheme;

/* Analytic survey window (the 3D mask of Sec. 3.1.3, w <= 1), evaluated at the nodes:
 *   w(x) = [angle(x-o, axis) <= half_angle] * prod_h [angle(x-o, h) >= rho_h] * f(r),
 *   r = |x - o|, w = 0 at r = 0; membership decided by dot products against cos(angle)*r.
 * axis and hole directions are unit vectors; holes points to n_holes rows of
 * (hx, hy, hz, rho_h) in host memory.
 * radial_kind 0: f = 1; 1: f = exp(-(r/p0)^2); 2: f = (r/p0)^p1 exp(p1 (1 - r/p0)). */
typedef struct {
  double observer[3];
  double axis[3];
  double half_angle;
  int n_holes;
  const double* holes;
  int radial_kind;
  double radial_params[4];
} wf_selection;

/* Prior power spectrum P(k) as a host table (k strictly increasing, all > 0), interpolated
 * log-log linearly (end segments extrapolated).  S^-1(k) = dV / P(k) on the grid, the
 * discrete form of S-hat = (2 pi)^3 P(k) delta_D of Sec. 3.3.1; S^-1(0) = 0. */
typedef struct {
  const double* k;
  const double* p;
  int n;
} wf_power;

typedef enum {
  WF_FP64 = 0,  /* every vector and transform in FP64 storage */
  WF_MIXED = 1  /* inner CG on FP32 vectors and FP32 FFTs (FP64-accumulated dots, FP64
                   alpha/beta), outer FP64 residual b - A x and iterative refinement */
} wf_precision;

typedef struct {
  double tol;         /* stop when ||b - A s||_2 / ||b||_2 <= tol (recomputed from s) */
  int max_iter;       /* cap on CG iterations (inner iterations summed for WF_MIXED) */
  wf_precision prec;
  double inner_tol;   /* WF_MIXED: largest relative reduction asked of one inner solve (<= 0:
                         1e-4; each step asks for half the remaining reduction, at most this) */
  int precond;        /* 1: CG in Fourier variables split-preconditioned by S^(1/2)
                         (same canonical system and residual); 0: plain CG on A */
  int deflate;        /* WF_MIXED only: 0 off; K in [1, 12] with 4 K < n: each inner CG is
                         preconditioned on the coarse space of the Fourier modes |k|^2 <= K^2
                         (grid units), whose Galerkin block E = Z^T (C A C) Z is formed and inverted
                         on the device once per solve (two-level "A-DEF2" form, Tang et al. 2009).
                         Same system, residual and stop rule; fewer iterations where the mask
                         couples the long-wavelength modes.  A system whose block has
                         ||E||_inf ||E^-1||_inf above 1e8 (beyond what the FP32 block holds) runs
                         its inner CG without it, and so do the later inner solves of a system
                         whose deflated inner solve broke down or reached 1200 iterations; its
                         batch-mates keep theirs.  -1: K by grid size (0 below 64, 3 at 64, 4 up to
                         128, 6 up to 192, 8 up to 256, 10 up to 384, 12 above; 0 for WF_FP64).
                         Errors: WF_ERR_ARG for any other value. */
} wf_solve_opts;

typedef struct {
  int iters;           /* CG iterations (all inner iterations for WF_MIXED) */
  int outer_iters;     /* WF_MIXED: refinement steps; WF_FP64: residual recomputations */
  double rel_residual; /* ||b - A s|| / ||b|| recomputed from the returned s in FP64 */
  double nbar;         /* nbar the solve used */
  wf_status status;
  double latency_s;    /* wf_poll results: seconds from wf_submit to completion (else 0) */
} wf_solve_info;

/* ---- context ------------------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the device memory the
 * context may hold for workspaces (0 = no cap).  *ctx receives the handle (NULL on failure); the
 * caller owns it and frees it with wf_destroy.
 * Errors: WF_ERR_ARG (ctx NULL, no such device), WF_ERR_CUDA (no CUDA device, or the pinned
 * host buffer could not be allocated). */
wf_status wf_create(wf_ctx** ctx, int device, size_t hbm_budget_bytes);

/* Free every workspace, plan and the serving thread of ctx.  Waits for its device work; serving
 * requests not yet finished are dropped with the scheduler.  Errors: WF_ERR_ARG (ctx NULL). */
wf_status wf_destroy(wf_ctx* ctx);

/* 1 if grid size n is compiled into this library, else 0.  Host only, never fails. */
int wf_supported_size(int n);

/* The coarse radius wf_solve_opts.deflate = -1 resolves to for a wf_solve / wf_solve_batch /
 * wf_submit solve of grid size n and precision prec (0: no coarse space).  Host only, never fails. */
int wf_deflate_radius(int n, wf_precision prec);

/* A static description of status s ("unknown status" for values outside wf_status). */
const char* wf_status_string(wf_status s);

/* Text of the last CUDA error seen by this thread (empty string if none). */
const char* wf_last_error(void);

/* Choose how the FP32 transforms of a CG iteration (the mixed-precision inner solves) run
 * between the two x passes (Sec. 3.3.1: the data term applied between the inverse and forward
 * transforms of the signal).  on = 0 (the default): three passes (inverse y, the real z
 * transforms with the multiplication by nbar w in between, forward y).  on = 1: where the grid
 * size allows (n = 128, 192, 256, 384, 512), one kernel per x-plane on a thread-block cluster
 * does all three, holding the plane in the cluster's distributed shared memory (fewer HBM
 * bytes, but on GB300 it measures slower than the three passes).  Both compute the same
 * operator with the same arithmetic; the choice affects speed and, where the radix plans
 * differ, the FP32 rounding.  Applies to solves started after the call.  Errors: WF_ERR_ARG. */
wf_status wf_set_fused_planes(wf_ctx* ctx, int on);

/* ---- launch autotuning (no counterpart in the paper: how the transforms of Sec. 3.3.1 map to
 * this GPU) ---------------------------------------------------------------------------------
 * The spectral passes come in launch variants (lines per tile, tiles in flight per CTA, largest
 * radix of the transform stages).  wf_autotune times every variant of every pass for grid size n
 * and precision prec (WF_MIXED tunes the FP32 inner passes, WF_FP64 the FP64 ones) on this
 * context's device, on a working set of at least 256 MB, and keeps the fastest per pass in the
 * context's tuning table; later solves of that size and precision launch it.  Results do not
 * depend on the variant beyond rounding (the transforms' stage order changes).
 *   report  host char [report_len] out: JSON array, one object per pass with each variant's
 *           milliseconds per launch and the one chosen; may be NULL
 * Allocates and frees a scratch buffer; waits for completion.
 * Errors: WF_ERR_ARG (bad precision, report too small), WF_ERR_UNSUPPORTED (size), WF_ERR_OOM,
 * WF_ERR_CUDA, WF_ERR_TIMEOUT (a kernel's bounded wait for a bulk copy ran out). */
wf_status wf_autotune(wf_ctx* ctx, int n, wf_precision prec, char* report, int report_len);
/* The context's tuning table as JSON text {"ypass/f32/512": 1, ...} (NUL-terminated) in json
 * [len]; WF_ERR_ARG if it does not fit. */
wf_status wf_tune_get(wf_ctx* ctx, char* json, int len);
/* Merge a table written by wf_tune_get into the context's (a saved tuning, reused without timing).
 * A variant index beyond a pass's variants launches variant 0.  WF_ERR_ARG on malformed text. */
wf_status wf_tune_set(wf_ctx* ctx, const char* json);

/* ---- the 3D mask from a sky completeness map (Sec. 3.1.3) ------------------------------------ */

/* Projects a sky completeness map and a radial completeness table onto the grid along rays from
 * the observer (Sec. 3.1.3 with Eq. eq:transf).  Sky pixel (i, j) of an equidistant alpha x delta
 * map has its centre at alpha_i = alpha0 + (i + 1/2) dalpha, delta_j = delta0 + (j + 1/2) ddelta
 * (radians); its ray is sampled at r_k = (k + 1/2) dr, k < n_r, at the point
 * o + r_k (cos delta cos alpha, cos delta sin alpha, sin delta).  Each sample inside the box
 * [0, box)^3 goes to its nearest-grid-point cell floor(x / H), decided in FP32 in cell units:
 * X = fl32(O + fl32((k + 1/2) g)) with O = fl32(o / H) and g = fl32(u dr / H).  Per cell, the sky
 * values and the radial values wr[k] of its samples are averaged; the mask is the product of the
 * two averages (w <= 1), and 0 in cells no sample reached.  The sums are Q32 fixed point with
 * integer atomics, so the result is exact and independent of the order of the samples; each
 * average is the sum times 2^-32 times fl(1 / count).
 *   sky       dev double [n_delta][n_alpha], values in [0, 1]
 *   observer  host double[3] (box units); wr host double [n_r], values in [0, 1]
 *   w         dev double [n^3];  counts dev int64 [n^3] (samples per cell) or NULL
 * Errors: WF_ERR_ARG (bad geometry, a value outside [0, 1]), WF_ERR_UNSUPPORTED, WF_ERR_OOM,
 * WF_ERR_CUDA.  Waits for completion. */
wf_status wf_project_mask(wf_ctx* ctx, const wf_grid* grid, const double* sky, int n_alpha, int n_delta,
                          double alpha0, double dalpha, double delta0, double ddelta, const double* observer,
                          double dr, int n_r, const double* wr, double* w, int64_t* counts, void* stream);

/* ---- signal-dependent noise (Eq. eq:noisecov; flat-prior and Jackknife-like estimators) ---- */

/* The data terms of the signal-dependent-noise Wiener filter.  With N^SD = w lambda / nbar^2 per
 * cell (Eq. eq:noisecov, lambda the expected counts of the complete sample):
 *   D = R^T N^-1 R = nbar^2 w / lambda,   b = R^T N^-1 d = nbar^2 d / lambda,   d = n_obs / nbar - w,
 * and 0, 0 where w = 0 or lambda <= 0 (no data term, as for unobserved cells).  Solve with
 * wf_solve(w = D, nbar = 1, b); the LSQ filter is the case lambda = nbar.
 *   n_obs, w   dev double [n_cells];  lambda dev double [n_cells] or NULL: the flat-prior mean
 *              estimator (n_obs + 1) / w (Sec. "flat prior"); nbar > 0 as from wf_build_noise
 *   D, b       dev double [n_cells]
 * Errors: WF_ERR_ARG, WF_ERR_CUDA.  Stream-ordered. */
wf_status wf_sd_noise(wf_ctx* ctx, int64_t n_cells, const double* n_obs, const double* w, const double* lambda,
                      double nbar, double* D, double* b, void* stream);

/* The Jackknife-like subsample of Eq. eq:selfunc as galaxy masses: galaxy g is kept when
 * u[g] < alpha / w_gal[g] and then carries mass 1 / alpha (else 0, and 0 where w_gal = 0).
 * Gridding these masses with wf_grid_assign_weighted gives N'' = N' / alpha, an unbiased estimate
 * of the complete counts lambda.  The uniform numbers u in [0, 1) are the caller's (one fresh
 * set per subsample); w_gal is the completeness at each galaxy (wf_selection_eval).
 *   w_gal, u, out  dev double [n_gal];  0 < alpha <= 1 (the paper uses alpha = 1e-3 < min w)
 * Errors: WF_ERR_ARG, WF_ERR_CUDA.  Stream-ordered. */
wf_status wf_jackknife_masses(wf_ctx* ctx, int64_t n_gal, const double* w_gal, const double* u, double alpha,
                              double* out, void* stream);

/* The Jackknife-like signal-dependent-noise filter (Sec. "Statistically unbiased Jackknife-like
 * scheme" and the mock tests of Sec. 4.2, which show the mean of 200 reconstructions).  For each
 * subsample j < n_sub: galaxy masses from u[j] (wf_jackknife_masses), their supersampled gridding
 * and low-pass N''_j (wf_grid_assign_weighted), the noise of Eq. eq:noisecov with lambda = N''_j
 * (wf_sd_noise: D_j = nbar^2 w / N''_j, b_j = nbar^2 d / N''_j, no data term where N''_j <= 0),
 * and the solve (S^-1 + diag(D_j)) s_j = b_j; s_mean = sum_j s_j / n_sub, added in subsample order
 * (deterministic).  Up to 8 subsamples are solved together.
 *   grid       the grid and supersampling of the gridding (the solve runs on the same n, box)
 *   pos        dev double [n_gal][3]; w_gal dev double [n_gal] (the completeness at each galaxy)
 *   u          dev double [n_sub][n_gal], uniform in [0, 1) (the caller's random numbers)
 *   n_obs, w   dev double [n^3] (the observed low-passed counts and the window); nbar > 0
 *   s_mean     dev double [n^3]; infos host [n_sub] or NULL (each subsample's solve)
 * Returns WF_OK if every solve converged, else the first failing status (s_mean still holds the
 * mean of what the solves returned).  Errors: WF_ERR_ARG, WF_ERR_UNSUPPORTED, WF_ERR_OOM,
 * WF_ERR_CUDA, WF_ERR_NOT_CONVERGED, WF_ERR_BREAKDOWN.  Waits for completion. */
wf_status wf_jackknife_solve(wf_ctx* ctx, const wf_grid* grid, wf_scheme scheme, const wf_power* power,
                             const double* pos, int64_t n_gal, const double* w_gal, const double* u, int n_sub,
                             double alpha, const double* n_obs, const double* w, double nbar,
                             const wf_solve_opts* opts, double* s_mean, wf_solve_info* infos, void* stream);

/* ---- inverse-weighting estimator (Sec. 4, Eq. def:ngrid with galaxy mass 1/w) ------------- */

/* The selection w (Sec. 3.1.3: cone x holes x radial law, the same formula and operation order as
 * the window of wf_build_noise) at arbitrary positions, e.g. the completeness at each galaxy.
 * reciprocal = 1 returns 1 / w instead (0 where w = 0): the galaxy masses of the
 * inverse-weighting estimator.
 *   pos  dev double [n_pts][3], out dev double [n_pts]
 * Errors: WF_ERR_ARG, WF_ERR_OOM, WF_ERR_CUDA.  Waits for completion. */
wf_status wf_selection_eval(wf_ctx* ctx, const wf_selection* sel, const double* pos, int64_t n_pts,
                            int reciprocal, double* out, void* stream);

/* Supersampled assignment with per-galaxy masses (the inverse-weighting estimator of Sec. 4
 * takes mass 1 / w(x_g)), then the same ideal low-pass as wf_grid_assign.  Each node's
 * contribution is its Q48 fixed-point weight times wgt[g], rounded once to the nearest Q32 unit,
 * so the fine grid is exact and independent of the order of the atomics.
 *   pos      dev double [n_gal][3];  wgt dev double [n_gal], each in [0, 2^32)
 *   fine_out dev uint64 [(s n)^3] or NULL: the fine grid in units of 2^-32 weighted galaxies
 *   n_obs    dev double [n^3]: the low-passed weighted counts
 * Errors: WF_ERR_ARG (bad position or weight), WF_ERR_OVERFLOW (a cell beyond 2^64 units),
 * WF_ERR_UNSUPPORTED, WF_ERR_OOM, WF_ERR_CUDA.  Waits for completion. */
wf_status wf_grid_assign_weighted(wf_ctx* ctx, const wf_grid* grid, wf_scheme scheme, const double* pos,
                                  const double* wgt, int64_t n_gal, uint64_t* fine_out, double* n_obs,
                                  void* stream);

/* ---- redshift distortions and the deconvolution (Sec. 3.3.2-3.3.3, Eq. eq:DEC) --------------------- */

/* <K D>_mu(k): the mean over mu in [0, 1] of the Kaiser factor (1 + beta mu^2)^2 times the
 * Lorentzian damping 1 / (1 + k^2 sigma_v^2 mu^2 / 2) (Sec. 3.3.3, "Redshift distortion operator").
 * The redshift-space power spectrum is P^r(k) times this factor (build wf_power tables from it);
 * its square root is the operator Z.  Closed form (power series for k^2 sigma_v^2 < 1).  Host
 * arrays, no context, no device work.
 *   k, out  host double [n_k]; k >= 0 in the inverse units of sigma_v (h/Mpc with sigma_v in
 *           Mpc/h: the paper's 500 km/s / H0 is 5 Mpc/h)
 * Errors: WF_ERR_ARG (negative or non-finite k, sigma_v < 0, non-finite beta). */
wf_status wf_rsd_factor(int64_t n_k, const double* k, double beta, double sigma_v, double* out);

/* Eq. eq:DEC with a constant bias b: the matter field in real space from the galaxy field in
 * redshift space, B^-1 Z^-1 applied as the Fourier multiplier 1 / (b sqrt(<K D>_mu(|k|))) with
 * k = 2 pi m / box.  FP64 transforms.
 *   in, out  dev double [n^3] (out may equal in); bias > 0; sigma_v >= 0
 * Errors: WF_ERR_ARG, WF_ERR_UNSUPPORTED, WF_ERR_OOM, WF_ERR_CUDA. */
wf_status wf_deconvolve(wf_ctx* ctx, const wf_grid* grid, const double* in, double beta, double sigma_v,
                        double bias, double* out, void* stream);

/* ---- evaluation of a reconstruction (Sec. 4.1 and Sec. 5.5) ------------------------------ */

/* Gaussian smoothing (Sec. 4.1, eq:GAUSS): out = the field convolved on the periodic grid with
 * the normalised Gaussian of radius r_s, i.e. its DFT multiplied by exp(-|k|^2 r_s^2 / 2) with
 * k = 2 pi m / box and m the signed index in (-n/2, n/2].  The paper prints the kernel as
 * exp(+|r|^2 / 2 r_S^2); the decaying Gaussian is the reading taken.  FP64 transforms.
 *   in, out  dev double [n^3] (row-major [x][y][z]; out may equal in)
 *   r_s      smoothing radius in box units, >= 0 (0 returns the field through the transforms)
 * Errors: WF_ERR_ARG, WF_ERR_UNSUPPORTED (n not compiled in), WF_ERR_OOM, WF_ERR_CUDA.
 * Stream-ordered on `stream` (NULL: the context's stream). */
wf_status wf_smooth(wf_ctx* ctx, const wf_grid* grid, const double* in, double r_s, double* out,
                    void* stream);

typedef struct {
  double r;             /* correlation coefficient sum(t r) / (sqrt(sum t^2) sqrt(sum r^2)) */
  double d_euc;         /* Euclidean distance sqrt(sum (r - t)^2 / N_cells) */
  double d_kl;          /* (1 / N_cells) sum (1 + r) log((1 + r) / (1 + t)), over the cells where
                           both 1 + r > 0 and 1 + t > 0 (the log is undefined elsewhere) */
  int64_t kl_excluded;  /* cells left out of d_kl */
} wf_compare_result;

/* Sec. 4.1 quality measures between a reconstructed overdensity `rec` and a reference `truth`
 * (dev double [n_cells] each, any layout): correlation coefficient, Euclidean distance and
 * normalised Kullback-Leibler distance.  Sums are FP64 and deterministic.  Result on the host;
 * waits for completion.  Errors: WF_ERR_ARG, WF_ERR_OOM, WF_ERR_CUDA. */
wf_status wf_compare(wf_ctx* ctx, int64_t n_cells, const double* rec, const double* truth,
                     wf_compare_result* out, void* stream);

typedef struct {
  double n_cells, mean, mu2, mu3, mu4, skewness, kurtosis, pearson;
} wf_density_moments;

/* Sec. 5.5 density statistics.  Counts of 1 + delta in n_bins bins [lo + i width, lo + (i + 1)
 * width) per radial shell (shells[2 s] <= r < shells[2 s + 1], r = |i H - observer| at node i H,
 * no periodic wrap) and region (0: w > 0, 1: w = 0); the bin index is floor(((1 + delta) - lo) /
 * width) in FP64.  For each (shell, region), from the bin centres delta_i = lo + (i + 1/2) width
 * - 1: N = sum f, the mean, the central moments mu_2..mu_4, skewness mu_3 / sigma^3, kurtosis
 * mu_4 / sigma^4 - 3 and Pearson's skewness (mean - delta_mode) / sigma with the mode the first
 * bin of largest count.  Values outside the bins are counted apart and do not enter the moments.
 *   delta, w   dev double [n^3]
 *   observer   host double[3], shells host double [n_shells][2]
 *   hist       host int64 [n_shells][2][n_bins + 2]: the bins, then the below- and above-range
 *              counts
 *   moments    host wf_density_moments [n_shells][2]; every field but n_cells is NaN when a
 *              region is empty
 * Limits: n_shells >= 1, n_bins >= 1, n_shells (n_bins + 2) <= 6144, width > 0.  Counts are
 * exact (integer atomics).  Waits for completion.
 * Errors: WF_ERR_ARG, WF_ERR_UNSUPPORTED, WF_ERR_OOM, WF_ERR_CUDA. */
wf_status wf_density_stats(wf_ctx* ctx, const wf_grid* grid, const double* delta, const double* w,
                           const double* observer, int n_shells, const double* shells, double lo,
                           double width, int n_bins, int64_t* hist, wf_density_moments* moments,
                           void* stream);

/* ---- tracing ------------------------------------------------------------------------ */

/* Reset the context's launch counters and enable (1) or disable (0) per-kernel timing.
 * Every kernel launch is counted; while enabled, each launch is bracketed by CUDA events on
 * its stream and attributed to a kernel class (e.g. "cg_xinv", "ypass", "zturn") together
 * with its algorithmic bytes (the DRAM traffic the pass cannot avoid).  While enabled, CG blocks
 * run as direct launches instead of CUDA graphs.  Errors: WF_ERR_ARG. */
wf_status wf_profile(wf_ctx* ctx, int enable);

/* Launches since the last wf_profile call and the number of kernel classes recorded.
 * Waits for the recorded events.  Errors: WF_ERR_ARG (NULL arguments). */
wf_status wf_profile_read(wf_ctx* ctx, int64_t* launches, int* n_classes);

/* Class i (0 <= i < n_classes): name (NUL-terminated, truncated to name_len), timed launches,
 * summed device milliseconds and summed algorithmic bytes.  Errors: WF_ERR_ARG (i out of range,
 * NULL arguments). */
wf_status wf_profile_class(wf_ctx* ctx, int i, char* name, int name_len, int64_t* launches,
                           double* total_ms, double* bytes);

/* Measurement utility (no counterpart in the paper): the FP64 FMA throughput of the context's
 * device, timed with CUDA events over one launch of independent FMA chains filling every SM, in
 * flop/s (2 per FMA) -- the measured peak the FP64-bound kernels (low-pass, FP64 transforms) are
 * reported against.  Waits for completion.  Errors: WF_ERR_ARG, WF_ERR_OOM, WF_ERR_CUDA. */
wf_status wf_fp64_rate(wf_ctx* ctx, double* flops_per_s);

/* ---- Sec. 3.1.2: supersampled mass assignment ----------------------------------------- */

/* Grid the galaxies and low-pass them to the target grid.
 *   pos      dev  double [n_gal][3]   positions in [box units]; periodic wrap applied
 *   fine_out dev  uint64 [(s n)^3]    or NULL: receives the fine mass grid in Q48 units
 *                                     (one galaxy = 2^48), bit-exact and order-independent
 *   n_obs    dev  double [n^3]        observed counts per cell (Eq. def:ngrid after the
 *                                     ideal low-pass; sum(n_obs) = n_gal)
 * Per axis, q = floor(x * (s n 2^16 / box)) mod (s n 2^16) fixes the galaxy in Q16 fine-cell
 * units; CIC weights (2^16 - f, f), TSC weights floor((2^15 -+ D)^2 / 2^17) and the rest
 * to the centre node; the 3D weight is their product.  With s = 2 the fine grid is
 * transformed, the modes with every |k_i| < n/2 kept (coarse Nyquist planes dropped), and
 * transformed back at n^3 divided by n^3.
 * Errors: WF_ERR_ARG (bad sizes/pointers, non-finite or |x| * scale >= 2^52 position),
 * WF_ERR_OVERFLOW, WF_ERR_UNSUPPORTED, WF_ERR_OOM.  Waits for the device (error flags). */
wf_status wf_grid_assign(wf_ctx* ctx, const wf_grid* grid, wf_scheme scheme, const double* pos,
                         int64_t n_gal, uint64_t* fine_out, double* n_obs, void* stream);

/* ---- Sec. 3.1.3-3.2: window, data and noise ------------------------------------------- */

/* w = window at the nodes (wf_selection); nbar = n_gal / sum(w) (eq:nmean, observed volume
 * in cells); d = n_obs / nbar - w (eq:datamodel); b = R^T N^-1 d = nbar d where w > 0 and 0
 * where w = 0 (N = w/nbar, eq:noiseav; no data term in unobserved cells).
 *   n_obs dev double [n^3] in;  w, d, b dev double [n^3] out (d may be NULL);
 *   nbar  host double out.
 * Errors: WF_ERR_ARG (sum(w) == 0, n_gal <= 0, bad selection).  Waits for nbar. */
wf_status wf_build_noise(wf_ctx* ctx, const wf_grid* grid, const wf_selection* sel,
                         const double* n_obs, int64_t n_gal, double* w, double* d, double* b,
                         double* nbar, void* stream);

/* Same outputs as wf_build_noise, for callers that cannot let a library allocate device
 * memory -- e.g. a host code that manages the whole GPU through its own memory pool at its
 * capacity limit, or a latency-critical pipeline where cudaMalloc's implicit device-wide
 * synchronisation is unacceptable.  No counterpart in the paper: this is a deployment variant.
 * It takes no context and allocates nothing: its scratch (reduction partials, the nbar
 * scalars, the hole table) is one fixed 17,952-byte array (2244 doubles) compiled into the
 * library's device image, which every GPU that loads libwf.so holds until the process exits.
 *   - Runs on the current CUDA device.  The first call on each device looks up the scratch
 *     address (cudaGetSymbolAddress); make that first call before any stream capture starts.
 *     The address is kept per (device, CUDA context id): after cudaDeviceReset the next call
 *     makes a new lookup in the new context, which again should come before any capture.
 *   - Limit: sel->n_holes <= 256; larger tables return WF_ERR_ARG (see wf_last_error()).
 *   - All calls share the one scratch array: calls that may overlap on the GPU (other streams,
 *     other host threads) race and must be serialised by the caller.  Every scratch word a
 *     call reads is written earlier in the same call, so nothing needs clearing in between.
 * Arguments, outputs and other errors as wf_build_noise.  Waits for nbar. */
wf_status wf_build_noise_noalloc(const wf_grid* grid, const wf_selection* sel, const double* n_obs,
                                 int64_t n_gal, double* w, double* d, double* b, double* nbar,
                                 void* stream);

/* ---- Sec. 3.3.1: the Wiener filter, Eq. eq:WF ----------------------------------------- */

/* Solve (S^-1 + nbar diag(w)) s = b for s = <delta_g>_WF by conjugate gradients from s = 0.
 *   w     dev double [n^3]  window (R = diag(w)); nbar > 0 as from wf_build_noise
 *   b     dev double [n^3]  right-hand side R^T N^-1 d
 *   s_out dev double [n^3]  solution
 *   info  host out (filled on success and on NOT_CONVERGED/BREAKDOWN)
 * The stop test recomputes ||b - A s|| in FP64 from the returned s.  Waits for completion.
 * Errors: WF_ERR_ARG (bad grid, power table, tolerances; an empty window; non-finite w or b),
 * WF_ERR_UNSUPPORTED, WF_ERR_OOM, WF_ERR_CUDA, WF_ERR_NOT_CONVERGED (max_iter reached; s_out holds
 * the last iterate), WF_ERR_BREAKDOWN. */
wf_status wf_solve(wf_ctx* ctx, const wf_grid* grid, const wf_power* power, const double* w,
                   double nbar, const double* b, const wf_solve_opts* opts, double* s_out,
                   wf_solve_info* info, void* stream);

/* Linear response of the data to the real-space matter field (Sec. 3.2.1 and 3.3.3): bias B = bias (a constant)
 * and the mu-averaged redshift operator Z = sqrt(<K D>_mu) of wf_rsd_factor, both diagonal in
 * Fourier space with the joint factor g(k) = bias sqrt(<K D>_mu(|k|)). */
typedef struct {
  double bias;     /* > 0 */
  double beta;     /* Kaiser beta (finite) */
  double sigma_v;  /* >= 0, pairwise-velocity dispersion in length units (Lorentzian damping) */
} wf_response;

/* The variant of Sec. 3.3.2 with Z and B inside the response operator, R = W Z B: the Wiener mean of
 * the real-space matter field s_m solving
 *     (S^-1 + G diag(nbar w) G) s_m = G b,     G = F^-1 diag(g) F,
 * with S^-1 from `power` (the real-space matter P(k)) as in wf_solve.  G is invertible and
 * commutes with S, so this is the same system as (G^-1 S^-1 G^-1 + diag(nbar w)) s_g = b for
 * s_g = G s_m, a solve with the redshift-space prior g^2 P(k) followed by the deconvolution
 * s_m = G^-1 s_g (Eq. eq:DEC); that is how it runs.  opts->tol applies to the s_g system, whose
 * residual is G^-1 times the literal one: info->rel_residual is the s_g system's.
 *   w, b, s_out  dev double [n^3] as in wf_solve (s_out may not overlap w or b: it is
 *                deconvolved in place after the solve)
 * Errors: as wf_solve, plus WF_ERR_ARG for a bad response or an s_out that shares any byte with
 * w or b. */
wf_status wf_solve_response(wf_ctx* ctx, const wf_grid* grid, const wf_power* power, const wf_response* response,
                            const double* w, double nbar, const double* b, const wf_solve_opts* opts,
                            double* s_out, wf_solve_info* info, void* stream);

/* Solve `count` independent systems (grids may differ in n and box) in one call; the
 * iterations of all unfinished systems are interleaved on the device.  Arrays of length
 * count: grids, powers, w[i], nbar[i], b[i], s_out[i] (dev), infos[i] (host).
 * Returns WF_OK if every system converged, else the first failing status. */
wf_status wf_solve_batch(wf_ctx* ctx, int count, const wf_grid* grids, const wf_power* powers,
                         const double* const* w, const double* nbar, const double* const* b,
                         const wf_solve_opts* opts, double* const* s_out, wf_solve_info* infos,
                         void* stream);

/* ---- serving ------------------------------------------------------------------------ */

/* Queue one solve.  w and b are HOST double [n^3] arrays copied before return (the caller
 * may free them); the power table is copied too.  *request_id receives a handle.
 * A scheduler thread of the context (started by the first wf_submit) admits queued requests
 * in arrival order while their device footprint fits the HBM budget (the context's budget,
 * or 80% of the device memory free when the scheduler starts) and fewer than 64 systems are
 * resident.  Requests admitted together are batched by grid size and precision; the batches
 * run interleaved with those already resident, each keeping its CG state on the device until
 * it finishes, and a finished request's memory is released at once.  A result does not
 * depend on which requests shared the device with it.
 * Errors: WF_ERR_ARG, WF_ERR_UNSUPPORTED, WF_ERR_BUSY (more than 4096 queued). */
wf_status wf_submit(wf_ctx* ctx, const wf_grid* grid, const wf_power* power, const double* w,
                    double nbar, const double* b, const wf_solve_opts* opts,
                    uint64_t* request_id);

/* Wait up to timeout_ms (0 = do not wait, < 0 = forever) for request_id.  Returns WF_PENDING
 * while it runs; otherwise its final status, with s_out (HOST double [n^3], may be NULL)
 * and info filled, after which the id is released. */
wf_status wf_poll(wf_ctx* ctx, uint64_t request_id, int timeout_ms, double* s_out,
                  wf_solve_info* info);

#ifdef __cplusplus
}
#endif

#endif /* WF_H_ */
