/*
 * dsps.h -- C ABI of libdsps, the GB300 (sm_103a) photometry hot path of
 * Hearin et al. 2021, "DSPS: Differentiable Stellar Population Synthesis"
 * (arXiv:2112.06830).
 *
 * For each galaxy the library turns its star-formation history into
 * stellar-mass weights over an SSP age grid (Sec. 3.1, Eqs. cspsum and
 * mstartot) and its (age-dependent) metallicity distribution into weights over
 * a metallicity grid (Sec. 3.2, Eqs. simple_mdf and agedep_mdf, Appendix B),
 * contracts the joint weights with a resident SSP spectral grid
 * (Sec. 2.1, Eq. cspdeftheta; Sec. 3.2, Eq. full_mdf), applies power-law dust
 * attenuation (Sec. 3.4, Eq. attenuation), redshifts the spectrum and
 * integrates it through filter curves to AB magnitudes (Sec. 2.2, Eq. restmag
 * and the observer-frame relation that follows it).  The gradient entry point
 * returns the vector-Jacobian product of the magnitudes with respect to the
 * per-galaxy parameters (the derivatives the paper obtains by autodiff,
 * Sec. 2.1 and Sec. 3).
 *
 * Conventions
 * -----------
 * - Every function returns DSPS_OK (0) or a negative error code; no C++
 *   exception crosses this boundary.  DSPS_PENDING (1) is returned only by
 *   dsps_poll.
 * - Pointers documented as "device" must be CUDA device (or managed) memory of
 *   the context's device; "host" pointers are ordinary host memory.  The
 *   caller owns every buffer it passes; the context owns the resident SSP
 *   copies, filter tables, cosmology table, work space and streams.
 * - Compute calls are asynchronous on the given stream (0 = legacy default
 *   stream) and are ordered with other work on that stream.  Two calls on the
 *   same context must not run concurrently on different streams because they
 *   share the context's work space; dsps_submit/dsps_poll are thread-safe.
 * - Values that can only be checked on the device (z outside (0, z_max],
 *   sigma <= 0, non-finite parameters) make the affected magnitudes NaN and
 *   set a sticky device error word, read (with a stream sync) by
 *   dsps_device_error().
 *
 * Per-galaxy parameter layout (float32, structure of arrays, row r of G
 * galaxies at params + r*G):
 *    0..4  SFH parameters.
 *          DSPS_SFH_DELAYED_TAU : p0 = tau [Gyr], SFR ~ t exp(-t/tau).
 *          DSPS_SFH_DPL_QUENCH  : p0 = t_peak [Gyr], p1 = rising slope,
 *                                 p2 = falling slope, p3 = t_q [Gyr],
 *                                 p4 = q_drop [dex];
 *                                 SFR ~ 1/[(t/tp)^-p1 + (t/tp)^-p2]
 *                                       * 10^(-q Terf(t | t_q - 0.9, 0.3))
 *                                 (quench floor reached at t_q, Sec. 3.1).
 *    5     mdf_mu     DSPS_MDF_MEAN_LINEAR: mean log10(Z/Zsun) at age 1 Gyr;
 *                     DSPS_MDF_MEAN_TERF: mean of the youngest stars (mu_young)
 *    6     mdf_sigma  MDF width [dex], > 0
 *    7     mdf_slope  DSPS_MDF_MEAN_LINEAR: d mean / d log10(age/yr) (0 =
 *                     uncorrelated MDF); DSPS_MDF_MEAN_TERF: mean of the
 *                     oldest stars (mu_old)
 *    8     Av         V-band attenuation [mag]
 *    9     delta      dust slope: A(lam) = Av (lam/5500 A)^(-0.7 + delta), or
 *                     Av k0(lam) (lam/5500 A)^delta / 4.05 (DSPS_DUST_*)
 *    10    logM       log10 of the stellar mass formed by t_obs [Msun]
 *    11    z          redshift, 0 < z <= z_max
 * Gradient rows (param_bar, float32 [11][G]) are rows 0..10 above.
 *
 * Grids with a nebular axis (dsps_grid.n_u > 1 values of log10 U, Sec. 3.3,
 * Eq. nebsed) take two more rows, params float32 [14][G]:
 *    12    u_mean     mean of log10 U
 *    13    u_sigma    width [dex] of its triweight distribution, > 0
 * and return 13 gradient rows: rows 0..10 above, then 11 = u_mean, 12 = u_sigma.
 * The probability of log U bin k is the triweight CDF difference over the
 * bin's edges (midpoints of the grid, outer edges at -inf / +inf), and the SSP
 * weights become omega_ijk = P_SFH(i) P_met(j | i) P_neb(k).
 *
 * With age-dependent dust (dsps_opts.dust_agedep, Sec. 3.4.1, Eq.
 * agedep_dust_csp) rows 8 and 9 hold the young-star Av and delta and two more
 * rows follow the others (rows 12, 13, or 14, 15 with a nebular axis): Av_old,
 * delta_old.  Age bin i is attenuated with Av_i = (1 - T_i) Av + T_i Av_old,
 * delta_i likewise, T_i = Terf((log10 age_i - x0) / h); the gradient gains two
 * rows after the others (Av_old, delta_old).
 *
 * A tabulated star formation history (dsps_opts.sfh_model = DSPS_SFH_TABLE,
 * Sec. 3.1: the history enters only through its values on the cosmic-time
 * grid) takes n_t more rows after all the others: the SFR at the time nodes
 * t0 + n (t1 - t0)/(n_t - 1), in any units (piecewise linear between the
 * nodes, like the parametric forms; logM, row 10, still sets the mass formed
 * by t_obs).  Rows 0..4 are then unused and ignored, and their gradient rows
 * are 0; the gradient gains n_t rows after all the others, dLoss/dSFR_n
 * (0 for nodes after t_obs).  Node values must be finite and >= 0 up to the
 * first node at or after t_obs, with some mass formed before t_obs.
 *
 * Row order, all options together: 0..11, [u_mean, u_sigma], [Av_old,
 * delta_old], [SFR_0 .. SFR_{n_t - 1}]; gradient rows 0..10 and the same
 * blocks in the same order.
 */
#ifndef DSPS_H
#define DSPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dsps_ctx dsps_ctx;
typedef struct CUstream_st *dsps_stream_t;   /* == cudaStream_t */

enum {
    DSPS_OK = 0,
    DSPS_PENDING = 1,
    DSPS_ERR_INVALID_ARG = -1,
    DSPS_ERR_OUT_OF_BUDGET = -2,
    DSPS_ERR_CUDA = -3,
    DSPS_ERR_TIMEOUT = -4,
    DSPS_ERR_DEVICE_FAULT = -5,
    DSPS_ERR_UNSUPPORTED = -6,
    DSPS_ERR_NOT_FOUND = -7
};

enum { DSPS_SFH_DELAYED_TAU = 0, DSPS_SFH_DPL_QUENCH = 1, DSPS_SFH_TABLE = 2 };
enum { DSPS_MDF_TRIWEIGHT = 0, DSPS_MDF_GAUSSIAN = 1 };
/* Age dependence of the MDF mean (Sec. 3.2, Eq. agedep_mdf), x = log10(age/yr):
 *   DSPS_MDF_MEAN_LINEAR  mu(x) = p5 + p7 (x - 9)
 *   DSPS_MDF_MEAN_TERF    mu(x) = (1 - T) p5 + T p7, T = Terf((x - x0) / h):
 *                         the paper's transition from mu_young to mu_old along
 *                         the triweight cumulative kernel (Appendix B). */
enum { DSPS_MDF_MEAN_LINEAR = 0, DSPS_MDF_MEAN_TERF = 1 };
/* Attenuation curve A_lambda / Av (Sec. 3.4, Eq. salim), x = lam / 5500 A:
 *   DSPS_DUST_POWERLAW  x^(-0.7 + delta): a power law standing for
 *                       k0 x^delta / 4.05, equal to 1 at 5500 A
 *   DSPS_DUST_SALIM     k0(lam) x^delta / 4.05 with the starburst curve k0 of
 *                       Eq. kzero: the published fits of Leitherer et al. (2002)
 *                       below 0.15 um and Calzetti et al. (2000) above (the
 *                       two curves' own ranges; the printed equation lists them
 *                       the other way round), clipped at 0 past ~3.1 um.
 * Either adds the UV bump E_b D0 / 4.05 when dsps_opts.dust_bump is set. */
enum { DSPS_DUST_POWERLAW = 0, DSPS_DUST_SALIM = 1 };

/* Arithmetic of the contraction (Eq. full_mdf):
 *   DSPS_PREC_FP32   FP32 weights x FP32 SSP grid, FP32 FMA on the SIMT cores.
 *   DSPS_PREC_BF16X3 SSP rows scaled by powers of two and split into
 *                    bf16 hi + lo, weights likewise; hi*hi + hi*lo + lo*hi
 *                    products on the tcgen05 tensor cores, FP32 accumulate.
 * Both use the same weights kernel (age-bin masses integrated directly, with a
 * compensated FP32 node prefix; FP64 only for t_obs's position on the SFR time
 * grid) and the same FP32 epilogue. */
enum { DSPS_PREC_FP32 = 0, DSPS_PREC_BF16X3 = 1 };

#define DSPS_NPAR 12
#define DSPS_NGRAD 11
#define DSPS_NPAR_NEB 14           /* parameter rows with a nebular axis      */
#define DSPS_NGRAD_NEB 13          /* gradient rows with a nebular axis       */
#define DSPS_MAX_NU 8              /* log U values of the nebular axis        */
#define DSPS_MAX_FILTERS 16

/* SSP block and grids (host memory, copied at dsps_create).
 * Sec. 2.1 (Eq. cspdef: the SSP block is precomputed and held fixed) and
 * Sec. 3.1 (age grid), Sec. 3.2 (metallicity grid), Sec. 3.3 (the optional
 * nebular ionisation axis).  Zero-initialise the struct: n_u = 0 means no
 * nebular axis. */
typedef struct {
    int32_t n_age;             /* >= 2                                          */
    int32_t n_z;               /* >= 1                                          */
    int32_t n_lam;             /* >= 2                                          */
    const double *log_age_yr;  /* [n_age] log10(age/yr), strictly increasing    */
    const double *lgz;         /* [n_z] log10(Z/Zsun), strictly increasing       */
    const double *lam;         /* [n_lam] rest wavelength [A], uniform in ln
                                  lambda to 1e-9 relative (DSPS_ERR_UNSUPPORTED
                                  otherwise)                                    */
    const float *l_ssp;        /* [n_age][n_z][n_lam] L_nu [Lsun/Hz/Msun], >= 0;
                                  [n_age][n_z][n_u][n_lam] with a nebular axis  */
    double t0_gyr, t1_gyr;     /* uniform cosmic-time grid of the SFR           */
    int32_t n_t;               /* nodes, 2..1024                                */
    int32_t n_u;               /* log U values, 2..DSPS_MAX_NU; 0 or 1: none    */
    const double *lgu;         /* [n_u] log10 U, strictly increasing (n_u > 1)  */
} dsps_grid;

typedef struct {
    double om0, w0, h;         /* flat wCDM (Sec. 2.2); defaults 0.3, -1, 0.7   */
    int32_t sfh_model;         /* DSPS_SFH_*                                    */
    int32_t mdf_kernel;        /* DSPS_MDF_*                                    */
    int32_t device;            /* CUDA device ordinal                            */
    int64_t max_chunk;         /* galaxies per internal launch (work space size;
                                  lowered so that the work space stays under
                                  16 GiB)                                        */
    int64_t hbm_budget_bytes;  /* admission budget of the request loop          */
    int32_t n_streams;         /* streams of the request loop                    */
    double z_max;              /* largest accepted redshift (cosmology table)    */
    int32_t band_skip;         /* 1: the tensor-core path skips wavelength tiles
                                  outside every redshifted filter of a tile's
                                  galaxies and K blocks where every galaxy of a
                                  tile has zero weight (exact: those terms are
                                  zero); 0: dense contraction                   */
    int32_t mdf_mean;          /* DSPS_MDF_MEAN_*                               */
    double mdf_terf_x0;        /* DSPS_MDF_MEAN_TERF: transition centre x0 and   */
    double mdf_terf_h;         /* width h [dex], h > 0 (defaults 9, 0.5)         */
    int32_t dust_bump;         /* 1: add the 2175 A UV bump to the attenuation
                                  curve (Sec. 3.4, Eq. uvbump: Drude profile of
                                  width 350 A, amplitude E_b = 0.85 - 1.9 delta,
                                  entering A_lambda as Av E_b D0(lam) / 4.05);
                                  default 0                                      */
    int32_t dust_law;          /* DSPS_DUST_*; default DSPS_DUST_POWERLAW        */
    int32_t dust_agedep;       /* 1: age-dependent dust (see the parameter rows
                                  above); dsps_photometry_fp32_static then
                                  returns DSPS_ERR_UNSUPPORTED; default 0        */
    double dust_agedep_x0;     /* transition centre [log10 yr] and width h [dex], */
    double dust_agedep_h;      /* h > 0 (defaults 7, 0.1: the birth-cloud age)    */
    int32_t agedep_fused;      /* with dust_agedep, magnitudes (no gradient):
                                  1 (default): every group of age bins sharing a
                                  curve contracted in one launch, each group's
                                  attenuated spectrum summed on chip before one
                                  filter integral (DSPS_PREC_BF16X3: grids
                                  without a nebular axis, n_z <= 32, n_age <=
                                  128; DSPS_PREC_FP32: up to 128 groups); 0: one
                                  contraction and filter integral per group.
                                  The two agree to the form's rounding
                                  (different summation order).                  */
} dsps_opts;

/* Fills *o with the defaults above (device 0, max_chunk 262144,
 * hbm_budget 8 GiB, 4 streams, z_max 10, band_skip 1, linear MDF mean,
 * agedep_fused 1). */
void dsps_default_opts(dsps_opts *o);

/* Creates a context on o->device: uploads the SSP block (FP32 copy, and the
 * bf16 hi/lo row-scaled copies for DSPS_PREC_BF16X3), builds the cosmology
 * table t_obs(z), Dmod(z) (Sec. 2.2) and allocates the work space.
 * Errors: INVALID_ARG for bad sizes/orderings, UNSUPPORTED for a wavelength
 * grid that is not uniform in ln lambda, CUDA on allocation/copy failure. */
int dsps_create(dsps_ctx **out, const dsps_grid *grid, const dsps_opts *opts);
int dsps_destroy(dsps_ctx *ctx);

/* Registers a filter set (Sec. 2.2, Eq. restmag: T_Q(lambda) is a photon
 * transmission probability).  Host tables, lam strictly increasing [A],
 * trans >= 0, each with >= 2 points; T is linear in lambda between points and
 * zero outside.  n_filt in 1..DSPS_MAX_FILTERS.  The tables are resampled onto
 * the SSP grid's ln-lambda spacing and kept on the device; the normalisation
 * int dlambda/lambda T (trapezoid on the caller's table) is kept per filter.
 * *set_id receives a small non-negative id. */
int dsps_filters_add(dsps_ctx *ctx, int32_t n_filt, const int32_t *n_pts,
                     const double *const *lam, const double *const *trans, int32_t *set_id);

/* The same with the frame of the set's magnitudes.  DSPS_FRAME_OBSERVER (what
 * dsps_filters_add registers): observer-frame apparent magnitudes
 *   m_Q = M'_Q + Dmod(z) - 2.5 log10(1+z),
 * M'_Q Eq. restmag with the filter at (1+z) lambda (Sec. 2.2).
 * DSPS_FRAME_REST: the rest-frame absolute magnitude M_Q of Eq. restmag, the
 * filter at the rest wavelength and no distance terms; z still sets the age
 * of the universe at which the galaxy is seen (t_obs), and so its SED.  Every
 * call taking a set id (photometry, gradient, histogram, request loop, the
 * allocation-free entry) follows the set's frame.  INVALID_ARG for another
 * frame value. */
enum { DSPS_FRAME_OBSERVER = 0, DSPS_FRAME_REST = 1 };
int dsps_filters_add_frame(dsps_ctx *ctx, int32_t n_filt, const int32_t *n_pts,
                           const double *const *lam, const double *const *trans, int32_t frame,
                           int32_t *set_id);
int dsps_filters_count(dsps_ctx *ctx, int32_t set_id, int32_t *n_filt);

/* Band coverage: for each galaxy g and filter q of the set, the fraction of
 * the filter's response D_q = int T_q(lam) dlam / lam (the denominator of Eq.
 * restmag, over the whole filter) that falls on the SSP grid as the galaxy is
 * seen: lam in [(1+z) lam_0, (1+z) lam_{N-1}] for an observer-frame set,
 * [lam_0, lam_{N-1}] for a rest-frame one (Sec. 2.2; the SED is zero outside
 * the grid).  coverage[g][q] = 1 for a band that the redshifted grid covers,
 * 0 for one wholly outside it.  A band with coverage below about 1e-8 sees
 * the grid only through the last points of the filter's far tail, where the
 * library's filter table (resampled on the grid's ln-lambda spacing and
 * interpolated with 4-point Lagrange weights) and a linear interpolation of
 * the filter's own table differ: such magnitudes can be off by up to ~0.2
 * mag, and one with coverage 0 can still be finite (~70 mag, the stencil
 * reaching a grid step past the filter's end).  At or above 1e-8 the
 * magnitudes keep the precision form's tolerance.  Evaluated from the
 * filter's own table (trapezoids of T / lam, partial intervals linear in lam)
 * with FP64 cumulative sums from both ends.  params: device
 * [npar][n_gal] FP32 (row 11, z, is read); coverage: device [n_gal][Q] FP32;
 * NaN where z is not finite or z <= 0 (observer frame).  Asynchronous on
 * stream.  INVALID_ARG for a null pointer, n_gal < 0 or an unknown set. */
int dsps_band_coverage(dsps_ctx *ctx, int64_t n_gal, const float *params, int32_t set_id, float *coverage,
                       dsps_stream_t stream);

/* SSP weights in Msun, w_out[g][i][j] = 10^logM * P_SFH(age_i) * P_met(Z_j | age_i)
 * (Sec. 3.1 Eq. cspsum with P_SFH, Sec. 3.2 Eq. agedep_mdf), times P_neb(u_k)
 * with a nebular axis (Eq. nebsed).
 * params: device float32 [12][n_gal] ([14][n_gal] with a nebular axis);
 * w_out: device float32 [n_gal][n_age][n_z] ([n_gal][n_age][n_z][n_u]). */
int dsps_weights(dsps_ctx *ctx, int64_t n_gal, const float *params, float *w_out,
                 dsps_stream_t stream);

/* Observer-frame AB magnitudes (Sec. 2.2): mags[g][q], device float32
 * [n_gal][n_filt of set_id].  params: device float32 [12][n_gal] ([14][n_gal]
 * with a nebular axis, as everywhere below).
 * precision: DSPS_PREC_FP32 or DSPS_PREC_BF16X3. */
int dsps_photometry(dsps_ctx *ctx, int64_t n_gal, const float *params, int32_t set_id,
                    int32_t precision, float *mags, dsps_stream_t stream);

/* Vector-Jacobian product of the magnitudes (Sec. 2.1: gradients of the SED
 * follow from dP(x_i)/dtheta; Sec. 3 per ingredient):
 *   param_bar[k][g] = sum_q mag_bar[g][q] d mags[g][q] / d params[k][g]
 * over the context's gradient rows (0..10, then the optional blocks above).
 * mag_bar: device float32 [n_gal][n_filt]; mags: device float32
 * [n_gal][n_filt] or NULL (forward magnitudes written as a by-product);
 * param_bar: device float32 [ngrad][n_gal] (11 rows, 13 with a nebular axis,
 * two more with age-dependent dust, n_t more with a tabulated SFH). */
int dsps_photometry_vjp(dsps_ctx *ctx, int64_t n_gal, const float *params, int32_t set_id,
                        int32_t precision, const float *mag_bar, float *mags,
                        float *param_bar, dsps_stream_t stream);

/* Population statistic of the paper's benchmark (Sec. 5.1): the galaxies whose
 * colour m[band_a] - m[band_b] exceeds `cut` (the red side of a colour cut),
 * counted in n_bins uniform bins of m[band_r] over [lo, hi).  Galaxies with a
 * NaN magnitude, or m[band_r] outside [lo, hi), are not counted.  Binning is in
 * FP32: bin = min(floor((m_r - lo) * (n_bins / (hi - lo))), n_bins - 1), the
 * scale rounded once to FP32.  1 <= n_bins <= DSPS_MAX_HIST_BINS; bands index
 * the filter set. */
#define DSPS_MAX_HIST_BINS 4096
typedef struct {
    int32_t band_a, band_b;    /* colour m[band_a] - m[band_b]                   */
    float cut;                 /* counted if the colour is > cut                 */
    int32_t band_r;            /* band of the histogrammed magnitude             */
    float lo, hi;              /* histogram range, lo < hi                       */
    int32_t n_bins;
} dsps_hist_spec;

/* Photometry (as dsps_photometry) followed by the histogram above, fused: the
 * magnitudes are binned where they are formed and never written.
 * counts: device uint64 [n_bins], overwritten. */
int dsps_photometry_histogram(dsps_ctx *ctx, int64_t n_gal, const float *params, int32_t set_id,
                              int32_t precision, const dsps_hist_spec *spec, uint64_t *counts,
                              dsps_stream_t stream);

/* The same histogram of magnitudes already on the device: mags device float32
 * [n_gal][n_filt]; counts device uint64 [n_bins], overwritten. */
int dsps_histogram(dsps_ctx *ctx, int64_t n_gal, const float *mags, int32_t n_filt,
                   const dsps_hist_spec *spec, uint64_t *counts, dsps_stream_t stream);

/* Rest-frame attenuated spectra on the SSP grid's own wavelengths (Sec. 2.1,
 * Eq. cspdef with the weights of Eq. agedep_mdf, times Eq. attenuation):
 *   out[g][n - n0] = 10^logM F_g(lam_n) sum_ij omega_gij L_ijn   [Lsun/Hz],
 * for grid columns n0 <= n < n1 (0 <= n0 < n1 <= n_lam), FP32 weights and FP32
 * contraction.  With age-dependent dust (Sec. 3.4.1) each age bin i takes its
 * own curve F_gi, summed over the context's groups of bins in a fixed order.
 * A galaxy with out-of-range parameters gets a NaN row.
 * params: device float32 [npar][n_gal]; out: device float32 [n_gal][n1 - n0]. */
int dsps_spectra(dsps_ctx *ctx, int64_t n_gal, const float *params, int32_t n0, int32_t n1,
                 float *out, dsps_stream_t stream);

/* Emission-line equivalent width (Sec. 2.2, Eq. eqw) of the rest-frame
 * attenuated spectrum L(lam) above, on the SSP grid's wavelengths lam_n:
 *   continuum points  half_width < |lam_n - lam_line| <= half_width + cont_width
 *   L0(lam)           the quadratic in lam fitted to L at the continuum points by
 *                     least squares (the line's range masked)
 *   W                 trapezoid over the line points |lam_n - lam_line| <=
 *                     half_width of (L - L0) / L0, in Angstrom (> 0 for emission).
 * W does not depend on the mass.  Computed in FP32: FP32 weights and window
 * contraction; the fit's operator (M^-1 phi for each continuum point, M the
 * normal matrix of the quadratic) is formed in FP64 when the line is added. */
#define DSPS_MAX_LINE_POINTS 4096
typedef struct {
    double lam_line;           /* rest wavelength of the line [A]               */
    double half_width;         /* of the line window [A], > 0                   */
    double cont_width;         /* of each continuum window [A], > 0             */
} dsps_line_spec;

/* Registers a line; *line_id receives a small non-negative id.  INVALID_ARG if
 * the grid holds fewer than 3 continuum or 2 line points for it, or more than
 * DSPS_MAX_LINE_POINTS points in the whole window. */
int dsps_line_add(dsps_ctx *ctx, const dsps_line_spec *spec, int32_t *line_id);

/* ew: device float32 [n_gal] (NaN for out-of-range parameters). */
int dsps_line_ew(dsps_ctx *ctx, int64_t n_gal, const float *params, int32_t line_id, float *ew,
                 dsps_stream_t stream);

/* Vector-Jacobian product of the equivalent widths:
 *   param_bar[k][g] = ew_bar[g] dW_g / d params[k][g]
 * over the context's gradient rows (row 10, logM, is exactly 0).  ew_bar:
 * device float32 [n_gal]; ew: device float32 [n_gal] or NULL; param_bar:
 * device float32 [11][n_gal], two more rows with a nebular axis and two more
 * (Av_old, delta_old, last) with age-dependent dust. */
int dsps_line_ew_vjp(dsps_ctx *ctx, int64_t n_gal, const float *params, int32_t line_id,
                     const float *ew_bar, float *ew, float *param_bar, dsps_stream_t stream);

/* FP32 photometry that allocates no device memory, for callers that cannot
 * call cudaMalloc at the time they need magnitudes (for example a worker of a
 * framework whose device memory belongs to its own pooling allocator, or a
 * latency-critical loop in which an allocation must not happen).  The paper has
 * no counterpart: this is a deployment variant of dsps_photometry with
 * precision DSPS_PREC_FP32 and gives the same magnitudes.
 * The context (made earlier) supplies the resident SSP block and tables; the
 * per-call scratch is a fixed 64 MiB device array inside the library that every
 * GPU loading the library holds until exit.  n_gal is limited to what fits that
 * array for the context's grid (about 7,000 galaxies for a 107 x 22 age x Z
 * grid); larger populations are rejected with DSPS_ERR_INVALID_ARG and a
 * message giving the limit.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  All calls share the array: calls whose
 * executions overlap on the GPU race with one another.
 * params: device float32 [npar][n_gal], the context's parameter rows (12 rows,
 * then the optional blocks of the layout above: a nebular axis, a tabulated
 * SFH); mags: device float32 [n_gal][n_filt]. */
int dsps_photometry_fp32_static(dsps_ctx *ctx, int64_t n_gal, const float *params, int32_t set_id,
                                float *mags, dsps_stream_t stream);

/* Request loop (continuous batching).  A request carries a population of
 * galaxies (params float32 [npar][n_gal], outputs float32) in host memory or,
 * with buffers = DSPS_BUF_DEVICE, in device memory of the context's device,
 * and is admitted when its device footprint fits the HBM budget; requests
 * admitted together are packed into shared launches, their copies and kernels
 * overlapping on the loop's streams.  Results are identical to a lone
 * dsps_photometry(_vjp) call on the same inputs.  (Sec. 5.1 times a population
 * of galaxies through the forward model; the loop serves many such
 * populations at once.) */
enum { DSPS_BUF_HOST = 0, DSPS_BUF_DEVICE = 1 };
typedef struct {
    int64_t n_gal;
    const float *params;       /* [npar][n_gal] (12 rows + optional blocks)      */
    int32_t set_id;
    int32_t precision;
    int32_t want_grad;         /* 0: mags only; 1: also param_bar                */
    const float *mag_bar;      /* [n_gal][n_filt], if want_grad                  */
    float *mags;               /* [n_gal][n_filt]                                */
    float *param_bar;          /* [ngrad][n_gal], if want_grad                   */
    int32_t buffers;           /* DSPS_BUF_HOST: the four arrays are host memory;
                                  DSPS_BUF_DEVICE: device memory of the
                                  context's device (copied device to device, no
                                  host staging); INVALID_ARG for another value or
                                  a pointer the device cannot address          */
} dsps_request;

/* Queues a request; *ticket identifies it.  The buffers must stay valid (and
 * device outputs unread) until dsps_poll reports completion.  OUT_OF_BUDGET if
 * the request alone can never fit the budget. */
int dsps_submit(dsps_ctx *ctx, const dsps_request *req, uint64_t *ticket);

/* Waits up to timeout_us microseconds for a request.  Returns DSPS_OK once its
 * outputs are in the request's buffers (the ticket is then retired);
 * DSPS_PENDING if timeout_us is 0 (just test) and it is still running;
 * DSPS_ERR_TIMEOUT if timeout_us > 0 elapsed with the request unfinished (the
 * ticket stays valid: poll again); DSPS_ERR_NOT_FOUND for an unknown ticket;
 * or the request's own error.  *latency_us (optional, may be NULL) receives
 * the submit -> done time of a finished request: an addition to the problem
 * statement's poll, for the serving latency percentiles. */
int dsps_poll(dsps_ctx *ctx, uint64_t ticket, int64_t timeout_us, double *latency_us);

/* Observer-frame AB magnitudes (as dsps_photometry) of a population held in
 * HOST memory, in one call: the parameters are copied to the device, the
 * photometry runs on `stream`, the magnitudes are copied back, and the call
 * returns once they are in mags (it synchronises the stream).  params: host
 * float32 [npar][n_gal]; mags: host float32 [n_gal][n_filt].  Page-locked
 * (pinned) host buffers are copied by DMA at full link speed; pageable ones
 * work too, staged by the CUDA driver.  The context keeps a device buffer for
 * one chunk of inputs and outputs (made, or grown, on first use); larger
 * populations are processed chunk by chunk.  (Sec. 2.2, the same magnitudes;
 * the host buffers are an addition for callers whose data lives on the host.) */
int dsps_photometry_host(dsps_ctx *ctx, int64_t n_gal, const float *params, int32_t set_id,
                         int32_t precision, float *mags, dsps_stream_t stream);

/* Synchronises the context's streams and the given stream, then returns and
 * clears the sticky device error word: DSPS_OK, or DSPS_ERR_INVALID_ARG if
 * some galaxy had out-of-range parameters, or DSPS_ERR_DEVICE_FAULT if a
 * kernel gave up on a bounded wait. */
int dsps_device_error(dsps_ctx *ctx, dsps_stream_t stream);

/* Kernel timing (tracing).  When enabled, every compute call records CUDA
 * events on the caller's stream around each kernel it launches; read() waits
 * for them and returns, per kernel kind, the number of launches and the summed
 * device time since the last read (then resets).  Kinds: 0 weights, redshift
 * sort and partial-sum combination, 1 FP32 photometry, 2 tensor-core
 * photometry, 3 adjoint kernels. */
#define DSPS_PROF_KINDS 4
typedef struct {
    int64_t launches[DSPS_PROF_KINDS];
    double ms[DSPS_PROF_KINDS];
    int64_t tc_kblocks;        /* 128 x 256 x 32 split-bf16 tensor-core block products executed */
    int64_t simt_steps;        /* 128 x 128 x 16 FP32 multiply-add tile steps of the FP32 form's
                                  photometry contraction executed */
    int64_t tc_kblocks_n128;   /* 128 x 128 x 32 split-bf16 block products executed by the one-launch
                                  age-dependent dust contraction */
} dsps_profile_t;
int dsps_profile_enable(dsps_ctx *ctx, int32_t enable);
int dsps_profile_read(dsps_ctx *ctx, dsps_profile_t *out);

const char *dsps_strerror(int code);

/* Human-readable detail of the last error returned on the calling thread. */
const char *dsps_last_error_message(void);

#ifdef __cplusplus
}
#endif
#endif /* DSPS_H */
