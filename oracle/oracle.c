/*
 * oracle.c -- plain FP64 CPU oracle of the DSPS photometry hot path
 * (Hearin et al., "DSPS: Differentiable Stellar Population Synthesis").
 *
 * TEST INFRASTRUCTURE. Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg load this file. The product path (the CUDA
 * library) never includes, links or calls it, and this file includes nothing
 * from the product path.
 *
 * Every function is a direct, loop-by-loop statement of the paper's equations
 * in double precision, with no blocking, fusion or reordering beyond what the
 * equation itself states.  Where the paper is silent or garbled the reading
 * taken is stated beside the code.
 *
 * Parameter layout (per galaxy, structure of arrays, row r at params + r*G):
 *   rows 0..4  SFH parameters
 *              model 0 (delayed tau):  p0 = tau [Gyr]
 *              model 1 (double power law with quench):
 *                      p0 = t_peak [Gyr], p1 = alpha_rise, p2 = alpha_fall,
 *                      p3 = t_q [Gyr], p4 = q_drop [dex]
 *   row 5      mdf_mu     (log10 Z/Zsun at the 1 Gyr pivot; mu_young for mean model 1)
 *   row 6      mdf_sigma  [dex]
 *   row 7      mdf_slope  d mu / d log10(age/yr) (mu_old for mean model 1)
 *   row 8      Av
 *   row 9      dust delta
 *   row 10     logM       log10 of the stellar mass formed by t_obs [Msun]
 *   row 11     z          redshift
 *   rows 12,13 (grids with a nebular axis, n_u > 1 log U values, Sec. 3.3)
 *              u_mean, u_sigma: mean and width [dex] of the triweight
 *              distribution of log10 U
 *   next 2     (age-dependent dust, Sec. 3.4.1) Av_old, delta_old: rows 8, 9
 *              then hold the young-star values
 * Gradient layout (11 rows): rows 0..10 of the above (z gets no gradient);
 * with a nebular axis 13 rows, rows 11, 12 = u_mean, u_sigma; with
 * age-dependent dust two more rows at the end, Av_old and delta_old.
 *
 * Besides the magnitudes, the oracle gives the rest-frame attenuated spectrum
 * and the equivalent width of an emission line (Sec. 2.2, Eq. eqw) with their
 * adjoints.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NPAR 12
#define ORC_NGRAD 11
#define ORC_SFH_TABLE 2              /* SFR given at the n_t time nodes */
#define ORC_AB0 1.13492e-13          /* Sec. 2.2, Eq. (restmag): AB zero point at 10 pc, Lsun/Hz */
#define ORC_LAMV 5500.0              /* Sec. 3.4, Eq. (salim): lambda_V in Angstrom */
#define ORC_SIGQ 0.3                 /* width of the quench transition [Gyr] (reading) */
#define ORC_C_KMS 299792.458
#define ORC_GYR_PER_INV_H0 977.792221 /* 1/(1 km/s/Mpc) in Gyr */

typedef struct {
    int n_age, n_z, n_lam;
    const double *log_age_yr;  /* [n_age] log10(age/yr), increasing        */
    const double *lgz;         /* [n_z]   log10(Z/Zsun), increasing        */
    const double *lam;         /* [n_lam] rest wavelength, Angstrom        */
    const double *l_ssp;       /* [n_age][n_z][n_lam] Lsun/Hz/Msun         */
    double t0, t1;             /* cosmic-time grid for SFR, Gyr            */
    int n_t;
    double om0, w0, h;         /* flat wCDM                                 */
    int sfh_model;             /* 0 delayed tau, 1 double power law+quench,
                                  2 tabulated: SFR at the n_t time nodes in the
                                  last n_t parameter rows (rows 0-4 unused)   */
    int mdf_kernel;            /* 0 triweight, 1 Gaussian                  */
    int mdf_mean;              /* 0 linear in log age, 1 T_erf transition  */
    double mdf_x0, mdf_h;      /* transition centre [log10 yr] and width   */
    int dust_bump;             /* 1: add the 2175 A Drude bump (Eq. uvbump) */
    int n_u;                   /* log U values of the nebular axis (<= 1: none) */
    const double *lgu;         /* [n_u] log10 U, increasing; l_ssp is then
                                  [n_age][n_z][n_u][n_lam]                  */
    int dust_law;              /* 0: power-law stand-in for k0 (lam/lam_V)^delta / 4.05,
                                  1: Eq. (salim) with the piecewise k0 (Eq. kzero) */
    int dust_agedep;           /* 1: Av, delta move from young to old values (Sec. 3.4.1) */
    double dust_x0, dust_h;    /* centre [log10 yr] and width of that transition */
} orc_grid;

/* Parameter rows: 0-11, then log U mean and width (nebular axis), then
 * Av_old and delta_old (age-dependent dust), then the SFR table; gradient
 * rows: 0-10, then the same optional blocks in the same order. */
static int orc_nu(const orc_grid *g) { return g->n_u > 1 ? g->n_u : 1; }
static int orc_row_dust_old(const orc_grid *g) { return ORC_NPAR + (g->n_u > 1 ? 2 : 0); }
static int orc_row_sfr(const orc_grid *g) { return orc_row_dust_old(g) + (g->dust_agedep ? 2 : 0); }
static int orc_npar(const orc_grid *g) { return orc_row_sfr(g) + (g->sfh_model == ORC_SFH_TABLE ? g->n_t : 0); }
static int orc_grow_dust_old(const orc_grid *g) { return ORC_NGRAD + (g->n_u > 1 ? 2 : 0); }
static int orc_grow_sfr(const orc_grid *g) { return orc_grow_dust_old(g) + (g->dust_agedep ? 2 : 0); }
static int orc_ngrad(const orc_grid *g) { return orc_grow_sfr(g) + (g->sfh_model == ORC_SFH_TABLE ? g->n_t : 0); }

typedef struct {
    int n_filt;
    const int *n_pts;          /* [n_filt]                                  */
    const double *lam;         /* concatenated tables, Angstrom, increasing */
    const double *trans;       /* concatenated transmissions                */
    int rest;                  /* 1: rest-frame absolute magnitudes M_Q (Eq.
                                  restmag: the filters at the rest wavelength,
                                  no distance modulus or (1+z) term); 0: the
                                  observer-frame apparent magnitudes m_Q      */
} orc_filters;

/* The redshift the filters see (0 in the rest frame) and the magnitude term
 * Dmod(z) - 2.5 log10(1+z) of the observer frame (Sec. 2.2). */
static double orc_filter_z(const orc_filters *f, double z) { return f->rest ? 0.0 : z; }
static double orc_frame_offset(const orc_filters *f, double z, double dmod)
{
    return f->rest ? 0.0 : dmod - 2.5 * log10(1.0 + z);
}

/* ------------------------------------------------------------------ */
/* Appendix B: triweight kernel and its cumulative integral            */
/* ------------------------------------------------------------------ */

/* Eq. (triweight), as a density in z = (x - mu)/sigma. */
double orc_triweight_pdf(double z)
{
    if (z < -3.0 || z > 3.0) return 0.0;
    double t = 1.0 - (z / 3.0) * (z / 3.0);
    return 35.0 / 96.0 * t * t * t;
}

/* Eq. (terf).  Reading: 0 below z = -3 and 1 above z = +3 (the printed
 * "0 otherwise" contradicts p(3) = 1). */
double orc_triweight_cdf(double z)
{
    if (z <= -3.0) return 0.0;
    if (z >= 3.0) return 1.0;
    double z2 = z * z, z3 = z2 * z, z5 = z3 * z2, z7 = z5 * z2;
    return 0.5 + 35.0 / 96.0 * z - 35.0 / 864.0 * z3 + 7.0 / 2592.0 * z5 - 5.0 / 69984.0 * z7;
}

double orc_gauss_cdf(double z) { return 0.5 * erfc(-z / sqrt(2.0)); }
double orc_gauss_pdf(double z) { return exp(-0.5 * z * z) / sqrt(2.0 * M_PI); }

static double mdf_cdf(int kernel, double z) { return kernel == 0 ? orc_triweight_cdf(z) : orc_gauss_cdf(z); }
static double mdf_pdf(int kernel, double z) { return kernel == 0 ? orc_triweight_pdf(z) : orc_gauss_pdf(z); }

/* ------------------------------------------------------------------ */
/* Sec. 2.2: flat wCDM time of observation and distance modulus        */
/* ------------------------------------------------------------------ */

static double cosmo_E(double om0, double w0, double z)
{
    double a1 = 1.0 + z;
    return sqrt(om0 * a1 * a1 * a1 + (1.0 - om0) * pow(a1, 3.0 * (1.0 + w0)));
}

typedef struct { double om0, w0; int which; } cosmo_args;

/* which = 0: 1/E(z) (comoving distance integrand in z).
 * which = 1: age integrand after a = s^2:  2 / (s E(z(s))), z = 1/s^2 - 1. */
static double cosmo_integrand(const cosmo_args *c, double x)
{
    if (c->which == 0) return 1.0 / cosmo_E(c->om0, c->w0, x);
    if (x <= 0.0) return 0.0;
    double z = 1.0 / (x * x) - 1.0;
    return 2.0 / (x * cosmo_E(c->om0, c->w0, z));
}

static double simpson_rec(const cosmo_args *c, double a, double b, double fa, double fm, double fb,
                          double whole, double tol, int depth)
{
    double m = 0.5 * (a + b);
    double lm = 0.5 * (a + m), rm = 0.5 * (m + b);
    double flm = cosmo_integrand(c, lm), frm = cosmo_integrand(c, rm);
    double left = (m - a) / 6.0 * (fa + 4.0 * flm + fm);
    double right = (b - m) / 6.0 * (fm + 4.0 * frm + fb);
    double diff = left + right - whole;
    if (depth <= 0 || fabs(diff) <= 15.0 * tol) return left + right + diff / 15.0;
    return simpson_rec(c, a, m, fa, flm, fm, left, 0.5 * tol, depth - 1) +
           simpson_rec(c, m, b, fm, frm, fb, right, 0.5 * tol, depth - 1);
}

static double adaptive_simpson(const cosmo_args *c, double a, double b, double tol)
{
    if (b <= a) return 0.0;
    double fa = cosmo_integrand(c, a), fb = cosmo_integrand(c, b), fm = cosmo_integrand(c, 0.5 * (a + b));
    double whole = (b - a) / 6.0 * (fa + 4.0 * fm + fb);
    return simpson_rec(c, a, b, fa, fm, fb, whole, tol, 48);
}

/* Age of the universe at z [Gyr]:  t = (1/H0) * int_0^{a} da / (a E(a)),
 * evaluated with a = s^2 so the integrand is smooth at s = 0. */
double orc_age_gyr(double om0, double w0, double h, double z)
{
    cosmo_args c = {om0, w0, 1};
    double smax = sqrt(1.0 / (1.0 + z));
    double I = adaptive_simpson(&c, 0.0, smax, 1e-14);
    return ORC_GYR_PER_INV_H0 / (100.0 * h) * I;
}

/* Luminosity distance [Mpc]: d_L = (1+z) (c/H0) int_0^z dz'/E(z'). */
double orc_lum_dist_mpc(double om0, double w0, double h, double z)
{
    cosmo_args c = {om0, w0, 0};
    double I = adaptive_simpson(&c, 0.0, z, 1e-14);
    return (1.0 + z) * ORC_C_KMS / (100.0 * h) * I;
}

/* Distance modulus 5 log10(d_L / 10 pc). */
double orc_dist_mod(double om0, double w0, double h, double z)
{
    return 5.0 * log10(orc_lum_dist_mpc(om0, w0, h, z) * 1e5);
}

/* ------------------------------------------------------------------ */
/* Sec. 3.1: star formation history on the cosmic-time grid            */
/* ------------------------------------------------------------------ */

/* SFR(t) for the two parametric models and its gradient d SFR / d p[k]
 * (k = 0..4; unused slots get 0).  Scale is arbitrary: the weights are
 * normalised to the mass formed by t_obs.
 *  model 0: delayed tau, SFR = t exp(-t/tau).
 *  model 1: main sequence double power law times the quenching function of
 *           Sec. 3.1 (Eq. diffstar, q_drop definition): 1/[(t/tp)^-ar +
 *           (t/tp)^-af] * 10^(-q Terf(t | t_q - 3 sig_q, sig_q)), so that the
 *           quench factor reaches its floor 10^-q exactly at t_q. */
double orc_sfr(int model, const double *p, double t, double *grad)
{
    if (grad) for (int k = 0; k < 5; ++k) grad[k] = 0.0;
    if (model == 0) {
        double tau = p[0];
        double s = t * exp(-t / tau);
        if (grad) grad[0] = s * t / (tau * tau);
        return s;
    }
    double tp = p[0], ar = p[1], af = p[2], tq = p[3], q = p[4];
    double r = t / tp;
    double ra = pow(r, -ar), rf = pow(r, -af);
    double D = ra + rf;
    double ms = 1.0 / D;
    double zq = (t - (tq - 3.0 * ORC_SIGQ)) / ORC_SIGQ;
    double P = orc_triweight_cdf(zq);
    double fq = pow(10.0, -q * P);
    double s = ms * fq;
    if (grad) {
        /* dD/dtp = (ar ra + af rf)/tp ; d(1/D) = -dD/D^2 */
        double dD_dtp = (ar * ra + af * rf) / tp;
        grad[0] = -dD_dtp / (D * D) * fq;
        grad[1] = log(r) * ra / (D * D) * fq;
        grad[2] = log(r) * rf / (D * D) * fq;
        /* dP/dtq = -T(zq)/sig_q */
        grad[3] = ms * fq * (-q * log(10.0)) * (-orc_triweight_pdf(zq) / ORC_SIGQ);
        grad[4] = ms * fq * (-log(10.0) * P);
    }
    return s;
}

/* SFR at the n_t time nodes t0 + n h (Sec. 3.1: the history the weights
 * integrate) and, if dsfr != NULL, dSFR_n/dp[k] for k = 0..4 ([n_t][5]): the
 * parametric models evaluated at the nodes, or the table itself (whose rows
 * are their own parameters; dsfr then 0). */
static void orc_sfr_nodes(const orc_grid *g, const double *par, double *sfr, double *dsfr)
{
    double h = (g->t1 - g->t0) / (g->n_t - 1);
    for (int n = 0; n < g->n_t; ++n) {
        if (g->sfh_model == ORC_SFH_TABLE) {
            sfr[n] = par[orc_row_sfr(g) + n];
            if (dsfr)
                for (int k = 0; k < 5; ++k) dsfr[5 * n + k] = 0.0;
        } else {
            sfr[n] = orc_sfr(g->sfh_model, par, g->t0 + n * h, dsfr ? dsfr + 5 * n : NULL);
        }
    }
}

/* Cumulative formed mass M(tau) = int_{t0}^{tau} SFR (Eq. mstartot), with SFR
 * piecewise linear between the uniform time nodes and zero before t0
 * (reading: the exact integral of the piecewise-linear SFR).  If coef != NULL
 * it receives dM/dSFR_n for every node (M is linear in the node values). */
double orc_cum_mass(const double *sfr, int n_t, double t0, double t1, double tau, double *coef)
{
    if (coef) for (int n = 0; n < n_t; ++n) coef[n] = 0.0;
    if (tau <= t0) return 0.0;
    double h = (t1 - t0) / (n_t - 1);
    int m = (int)floor((tau - t0) / h);
    if (m > n_t - 2) m = n_t - 2;
    double M = 0.0;
    for (int n = 0; n < m; ++n) {
        M += 0.5 * h * (sfr[n] + sfr[n + 1]);
        if (coef) { coef[n] += 0.5 * h; coef[n + 1] += 0.5 * h; }
    }
    double u = tau - (t0 + m * h);
    M += sfr[m] * u + (sfr[m + 1] - sfr[m]) * u * u / (2.0 * h);
    if (coef) {
        coef[m] += u - u * u / (2.0 * h);
        coef[m + 1] += u * u / (2.0 * h);
    }
    return M;
}

/* Age-bin edges in Gyr (reading of the garbled bin limits after
 * Eq. cspsum): midpoints in log10 age, first edge at age 0, last edge half a
 * step above the last grid age. */
void orc_age_edges_gyr(const orc_grid *g, double *edges /* n_age+1 */)
{
    int n = g->n_age;
    const double *x = g->log_age_yr;
    edges[0] = 0.0;
    for (int i = 1; i < n; ++i) edges[i] = pow(10.0, 0.5 * (x[i - 1] + x[i]) - 9.0);
    edges[n] = pow(10.0, x[n - 1] + 0.5 * (x[n - 1] - x[n - 2]) - 9.0);
}

/* Eq. (cspsum) with the unnumbered P_SFH definition: the fraction of the mass
 * formed by t_obs that lies in age bin i,
 *   frac_i = [M(t_obs - e_i) - M(t_obs - e_{i+1})] / M(t_obs). */
void orc_age_fracs_from_sfr(const orc_grid *g, const double *sfr, double t_obs, double *frac)
{
    double *e = malloc(sizeof(double) * (g->n_age + 1));
    orc_age_edges_gyr(g, e);
    double Mtot = orc_cum_mass(sfr, g->n_t, g->t0, g->t1, t_obs, NULL);
    for (int i = 0; i < g->n_age; ++i) {
        double hi = orc_cum_mass(sfr, g->n_t, g->t0, g->t1, t_obs - e[i], NULL);
        double lo = orc_cum_mass(sfr, g->n_t, g->t0, g->t1, t_obs - e[i + 1], NULL);
        frac[i] = (hi - lo) / Mtot;
    }
    free(e);
}

/* ------------------------------------------------------------------ */
/* Sec. 3.2: metallicity distribution over the lgZ bins                */
/* ------------------------------------------------------------------ */

/* P[j | age bin i] = C((E_{j+1} - mu_i)/sigma) - C((E_j - mu_i)/sigma), with
 * lgZ bin edges at grid midpoints and outer edges at -inf/+inf (reading), and
 * mu_i = mu + slope * (log10 age_i - 9) (age-dependent mean, linear reading;
 * slope = 0 is the uncorrelated MDF of Eq. simple_mdf). */
void orc_mdf(const orc_grid *g, double mu_i, double sigma, double *P /* n_z */,
             double *dP_dmu /* n_z or NULL */, double *dP_dsig /* n_z or NULL */)
{
    int nz = g->n_z;
    for (int j = 0; j < nz; ++j) {
        double c_hi, c_lo, d_hi = 0.0, d_lo = 0.0, u_hi = 0.0, u_lo = 0.0;
        if (j == nz - 1) c_hi = 1.0;
        else {
            u_hi = (0.5 * (g->lgz[j] + g->lgz[j + 1]) - mu_i) / sigma;
            c_hi = mdf_cdf(g->mdf_kernel, u_hi);
            d_hi = mdf_pdf(g->mdf_kernel, u_hi);
        }
        if (j == 0) c_lo = 0.0;
        else {
            u_lo = (0.5 * (g->lgz[j - 1] + g->lgz[j]) - mu_i) / sigma;
            c_lo = mdf_cdf(g->mdf_kernel, u_lo);
            d_lo = mdf_pdf(g->mdf_kernel, u_lo);
        }
        P[j] = c_hi - c_lo;
        if (dP_dmu) dP_dmu[j] = -(d_hi - d_lo) / sigma;
        if (dP_dsig) dP_dsig[j] = -(d_hi * u_hi - d_lo * u_lo) / sigma;
    }
}

/* Mean lgZ of the MDF for age bin i (Sec. 3.2, Eq. agedep_mdf), and its
 * derivatives with respect to parameter rows 5 and 7.
 *   model 0 (linear reading): mu_i = p5 + p7 (log10 age_i - 9).
 *   model 1 (the paper's form): the mean moves from a young-age value to an
 *     old-age value along the triweight cumulative kernel in log age,
 *     mu_i = (1 - T) p5 + T p7,  T = T_erf((log10 age_i - x0) / h),  p5 = mu_young,
 *     p7 = mu_old; the transition's centre x0 and width h are not given in
 *     the paper and are grid options (reading). */
double orc_mdf_mean(const orc_grid *g, const double *par, int i, double *d5, double *d7)
{
    double x = g->log_age_yr[i];
    if (g->mdf_mean == 1) {
        double T = orc_triweight_cdf((x - g->mdf_x0) / g->mdf_h);
        if (d5) *d5 = 1.0 - T;
        if (d7) *d7 = T;
        return (1.0 - T) * par[5] + T * par[7];
    }
    if (d5) *d5 = 1.0;
    if (d7) *d7 = x - 9.0;
    return par[5] + par[7] * (x - 9.0);
}

/* Sec. 3.3, Eq. (nebsed): probability of log U bin k for a galaxy whose
 * log10 U follows the triweight kernel of mean us and width su (Appendix B),
 * P[k] = T_erf((E_{k+1} - us)/su) - T_erf((E_k - us)/su), with bin edges at
 * grid midpoints and outer edges at -inf/+inf (reading, as for the MDF), and
 * its derivatives in us and su.  Without a nebular axis P = {1}. */
void orc_pneb(const orc_grid *g, double us, double su, double *P, double *dP_dus, double *dP_dsu)
{
    int nu = orc_nu(g);
    if (nu == 1) {
        P[0] = 1.0;
        if (dP_dus) dP_dus[0] = 0.0;
        if (dP_dsu) dP_dsu[0] = 0.0;
        return;
    }
    for (int k = 0; k < nu; ++k) {
        double c_hi = 1.0, c_lo = 0.0, d_hi = 0.0, d_lo = 0.0, x_hi = 0.0, x_lo = 0.0;
        if (k < nu - 1) {
            x_hi = (0.5 * (g->lgu[k] + g->lgu[k + 1]) - us) / su;
            c_hi = orc_triweight_cdf(x_hi);
            d_hi = orc_triweight_pdf(x_hi);
        }
        if (k > 0) {
            x_lo = (0.5 * (g->lgu[k - 1] + g->lgu[k]) - us) / su;
            c_lo = orc_triweight_cdf(x_lo);
            d_lo = orc_triweight_pdf(x_lo);
        }
        P[k] = c_hi - c_lo;
        if (dP_dus) dP_dus[k] = -(d_hi - d_lo) / su;
        if (dP_dsu) dP_dsu[k] = -(d_hi * x_hi - d_lo * x_lo) / su;
    }
}

/* ------------------------------------------------------------------ */
/* Sec. 3.4: power-law dust attenuation (Eq. attenuation, simplified   */
/* Eq. salim with k = 1 at lambda_V: A_lambda = Av (lam/5500)^(-0.7+d)) */
/* ------------------------------------------------------------------ */
double orc_dust_trans(double lam, double Av, double delta)
{
    return pow(10.0, -0.4 * Av * pow(lam / ORC_LAMV, -0.7 + delta));
}

/* Eq. (uvbump): the UV bump as a Drude profile of unit amplitude,
 * D0 = (lam dlam)^2 / ((lam^2 - lam_b^2)^2 + (lam dlam)^2), lam_b = 2175 A,
 * dlam = 350 A. */
double orc_drude(double lam)
{
    const double lb = 2175.0, dl = 350.0;
    double x = lam * dl, d = lam * lam - lb * lb;
    return x * x / (d * d + x * x);
}

/* Eq. (kzero): the starburst curve k0(lam), lam in Angstrom.  The paper takes
 * it from Calzetti et al. (2000) and Leitherer et al. (2002) without
 * printing either; the published fits are
 *   Leitherer:  5.472 + 0.671/x - 9.218e-3/x^2 + 2.620e-3/x^3       (0.097-0.18 um)
 *   Calzetti:   2.659 (-2.156 + 1.509/x - 0.198/x^2 + 0.011/x^3) + 4.05  (0.12-0.63 um)
 *               2.659 (-1.857 + 1.040/x) + 4.05                        (0.63-2.2 um)
 * with x = lam in um.  Reading: Leitherer below 0.15 um and Calzetti above
 * (the printed assignment is the other way round, outside both fits' ranges),
 * each extrapolated beyond its range, k0 clipped at 0 (the Calzetti fit
 * crosses 0 near 3.1 um). */
double orc_k0(double lam)
{
    double x = lam * 1e-4, k;
    if (x < 0.15) k = 5.472 + 0.671 / x - 9.218e-3 / (x * x) + 2.620e-3 / (x * x * x);
    else if (x < 0.63) k = 2.659 * (-2.156 + 1.509 / x - 0.198 / (x * x) + 0.011 / (x * x * x)) + 4.05;
    else k = 2.659 * (-1.857 + 1.040 / x) + 4.05;
    return k > 0.0 ? k : 0.0;
}

/* Attenuation curve A_lambda / Av = k_lambda / 4.05 (Eq. salim),
 * k_lambda = k0 (lam/lam_V)^delta + E_b D0 with the bump of amplitude
 * E_b = 0.85 - 1.9 delta (Kriek & Conroy, as in the paper) when it is on.
 * dust_law 0 replaces k0 (lam/lam_V)^delta / 4.05 by the power law
 * (lam/lam_V)^(-0.7 + delta) (k = 1 at lam_V); dust_law 1 takes Eq. (kzero).
 * *dd: d(A_lambda / Av) / d delta. */
double orc_dust_curve(const orc_grid *g, double lam, double delta, double *dd)
{
    double u, c, dc;
    if (g->dust_law == 1) {
        u = orc_k0(lam) / 4.05 * pow(lam / ORC_LAMV, delta);
    } else {
        u = pow(lam / ORC_LAMV, -0.7 + delta);
    }
    c = u;
    dc = u * log(lam / ORC_LAMV);
    if (g->dust_bump) {
        double D0 = orc_drude(lam);
        c += (0.85 - 1.9 * delta) * D0 / 4.05;
        dc += -1.9 * D0 / 4.05;
    }
    if (dd) *dd = dc;
    return c;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.2: filters                                                   */
/* ------------------------------------------------------------------ */

/* T_q(lambda): linear in lambda between table points, zero outside. */
double orc_filter_trans(const double *lam, const double *tr, int n, double x)
{
    if (x < lam[0] || x > lam[n - 1]) return 0.0;
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (lam[mid] <= x) lo = mid; else hi = mid;
    }
    double w = (x - lam[lo]) / (lam[hi] - lam[lo]);
    return tr[lo] + w * (tr[hi] - tr[lo]);
}

/* Denominator of Eq. (restmag): trapezoid of T/lambda on the filter table. */
double orc_filter_norm(const double *lam, const double *tr, int n)
{
    double s = 0.0;
    for (int m = 0; m + 1 < n; ++m)
        s += 0.5 * (lam[m + 1] - lam[m]) * (tr[m] / lam[m] + tr[m + 1] / lam[m + 1]);
    return s;
}

/* Trapezoid weight of rest-grid node n for int dlambda (.). */
static double trap_w(const double *lam, int N, int n)
{
    if (N == 1) return 0.0;
    if (n == 0) return 0.5 * (lam[1] - lam[0]);
    if (n == N - 1) return 0.5 * (lam[N - 1] - lam[N - 2]);
    return 0.5 * (lam[n + 1] - lam[n - 1]);
}

/* ------------------------------------------------------------------ */
/* Per-galaxy forward model                                            */
/* ------------------------------------------------------------------ */

static void filter_offsets(const orc_filters *f, int *off)
{
    off[0] = 0;
    for (int q = 0; q < f->n_filt; ++q) off[q + 1] = off[q] + f->n_pts[q];
}

/* Eqs. (restmag) + observer frame of Sec. 2.2 + Eq. (attenuation), for one
 * galaxy given its per-unit-mass SSP weights omega[i][j] (sum = 1):
 *   S_n   = sum_ij omega_ij L_ijn                         (Eq. full_mdf)
 *   N_q   = sum_n c_n/lam_n T_q((1+z) lam_n) F_n S_n      (rest-grid trapezoid)
 *   m_q   = -2.5 log10(10^logM N_q / (AB0 D_q)) + Dmod(z) - 2.5 log10(1+z)
 * (rest frame: T_q(lam_n) and M_q = -2.5 log10(10^logM N_q / (AB0 D_q))). */
void orc_mags_from_weights(const orc_grid *g, const orc_filters *f, const double *omega,
                           double Av, double delta, double logM, double z, double dmod,
                           double *mags)
{
    int N = g->n_lam, K = g->n_age * g->n_z * orc_nu(g);
    double *S = calloc(N, sizeof(double));
    for (int k = 0; k < K; ++k) {
        double w = omega[k];
        if (w == 0.0) continue;
        const double *L = g->l_ssp + (size_t)k * N;
        for (int n = 0; n < N; ++n) S[n] += w * L[n];
    }
    int *off = malloc(sizeof(int) * (f->n_filt + 1));
    filter_offsets(f, off);
    for (int q = 0; q < f->n_filt; ++q) {
        const double *fl = f->lam + off[q], *ft = f->trans + off[q];
        int np = f->n_pts[q];
        double Nq = 0.0;
        for (int n = 0; n < N; ++n) {
            double T = orc_filter_trans(fl, ft, np, (1.0 + orc_filter_z(f, z)) * g->lam[n]);
            if (T == 0.0) continue;
            double F = pow(10.0, -0.4 * Av * orc_dust_curve(g, g->lam[n], delta, NULL));
            Nq += trap_w(g->lam, N, n) / g->lam[n] * T * F * S[n];
        }
        double Dq = orc_filter_norm(fl, ft, np);
        mags[q] = -2.5 * log10(pow(10.0, logM) * Nq / (ORC_AB0 * Dq)) + orc_frame_offset(f, z, dmod);
    }
    free(off);
    free(S);
}

/* Joint SSP weights of one galaxy, per unit formed mass:
 * omega[i][j] = frac_i * P[j | i]   (Eq. agedep_mdf), and with a nebular axis
 * omega[i][j][k] = frac_i * P[j | i] * P_neb[k]   (Eq. nebsed). */
static void galaxy_weights(const orc_grid *g, const double *par, double t_obs, double *omega)
{
    int nu = orc_nu(g);
    double *sfr = malloc(sizeof(double) * g->n_t);
    double *frac = malloc(sizeof(double) * g->n_age);
    double *P = malloc(sizeof(double) * g->n_z);
    double *Pu = malloc(sizeof(double) * nu);
    orc_sfr_nodes(g, par, sfr, NULL);
    orc_age_fracs_from_sfr(g, sfr, t_obs, frac);
    orc_pneb(g, nu > 1 ? par[12] : 0.0, nu > 1 ? par[13] : 1.0, Pu, NULL, NULL);
    for (int i = 0; i < g->n_age; ++i) {
        double mu_i = orc_mdf_mean(g, par, i, NULL, NULL);
        orc_mdf(g, mu_i, par[6], P, NULL, NULL);
        for (int j = 0; j < g->n_z; ++j)
            for (int k = 0; k < nu; ++k) omega[(i * g->n_z + j) * nu + k] = frac[i] * P[j] * Pu[k];
    }
    free(Pu); free(P); free(frac); free(sfr);
}

/* ------------------------------------------------------------------ */
/* Adjoint of the per-galaxy model (reverse of the steps above)        */
/* ------------------------------------------------------------------ */

/* Forward intermediates of one galaxy that the reverse sweeps need. */
typedef struct {
    double *sfr, *dsfr;        /* [n_t], [n_t][5] SFR at the nodes and dSFR/dp      */
    double *e, *Mhi;           /* [n_age+1] age-bin edges, M(t_obs - e_i)            */
    double Mtot;
    double *frac;              /* [n_age]                                            */
    double *P, *dPmu, *dPsig;  /* [n_age][n_z] MDF bin probabilities and derivatives */
    double *dmu5, *dmu7;       /* [n_age] d mu_i / d p5, d p7                       */
    double *Pu, *dPu_us, *dPu_su; /* [n_u] nebular bin probabilities and derivatives */
    /* Dust groups: every age bin with age-dependent dust (Sec. 3.4.1,
     * Eq. agedep_dust_csp), else one group of all ages. */
    int ND;
    double *Sd;                /* [ND][n_lam] sum over the group's ages of omega_k L_kn (per unit mass) */
    double *Fd, *ud, *dud;     /* [ND][n_lam] transmission, A/Av, d(A/Av)/d delta     */
    double *Avd, *Td;          /* [ND] the group's Av and its weight T on the old values */
    double *L;                 /* [n_lam] sum_d F_d S_d: attenuated spectrum per unit mass */
} gal_state;

/* Dust of age bin i (Sec. 3.4.1): Av and delta move from the young values
 * (rows 8, 9) to the old ones along T = T_erf((log10 age_i - x0) / h), like
 * the MDF mean of Eq. (agedep_mdf); without age dependence T = 0. */
static void orc_dust_at_age(const orc_grid *g, const double *par, int i, double *Av, double *delta, double *T)
{
    double t = 0.0;
    if (g->dust_agedep) t = orc_triweight_cdf((g->log_age_yr[i] - g->dust_x0) / g->dust_h);
    int r = orc_row_dust_old(g);
    *T = t;
    *Av = g->dust_agedep ? (1.0 - t) * par[8] + t * par[r] : par[8];
    *delta = g->dust_agedep ? (1.0 - t) * par[9] + t * par[r + 1] : par[9];
}

static void gal_forward(const orc_grid *g, const double *par, double t_obs, gal_state *st)
{
    int N = g->n_lam, NA = g->n_age, NZ = g->n_z, NU = orc_nu(g), K = NA * NZ * NU, NT = g->n_t;
    st->sfr = malloc(sizeof(double) * NT);
    st->dsfr = malloc(sizeof(double) * NT * 5);
    orc_sfr_nodes(g, par, st->sfr, st->dsfr);
    st->e = malloc(sizeof(double) * (NA + 1));
    orc_age_edges_gyr(g, st->e);
    st->Mhi = malloc(sizeof(double) * (NA + 1));
    for (int i = 0; i <= NA; ++i) st->Mhi[i] = orc_cum_mass(st->sfr, NT, g->t0, g->t1, t_obs - st->e[i], NULL);
    st->Mtot = st->Mhi[0];
    st->frac = malloc(sizeof(double) * NA);
    for (int i = 0; i < NA; ++i) st->frac[i] = (st->Mhi[i] - st->Mhi[i + 1]) / st->Mtot;
    st->P = malloc(sizeof(double) * K);
    st->dPmu = malloc(sizeof(double) * K);
    st->dPsig = malloc(sizeof(double) * K);
    st->dmu5 = malloc(sizeof(double) * NA);
    st->dmu7 = malloc(sizeof(double) * NA);
    for (int i = 0; i < NA; ++i) {
        double mu_i = orc_mdf_mean(g, par, i, st->dmu5 + i, st->dmu7 + i);
        orc_mdf(g, mu_i, par[6], st->P + i * NZ, st->dPmu + i * NZ, st->dPsig + i * NZ);
    }
    st->Pu = malloc(sizeof(double) * NU);
    st->dPu_us = malloc(sizeof(double) * NU);
    st->dPu_su = malloc(sizeof(double) * NU);
    orc_pneb(g, NU > 1 ? par[12] : 0.0, NU > 1 ? par[13] : 1.0, st->Pu, st->dPu_us, st->dPu_su);
    int ND = g->dust_agedep ? NA : 1;
    st->ND = ND;
    st->Sd = calloc((size_t)ND * N, sizeof(double));
    for (int k = 0; k < K; ++k) {
        int i = k / (NZ * NU), d = ND > 1 ? i : 0;
        double w = st->frac[i] * st->P[k / NU] * st->Pu[k % NU];
        const double *L = g->l_ssp + (size_t)k * N;
        for (int n = 0; n < N; ++n) st->Sd[(size_t)d * N + n] += w * L[n];
    }
    st->Fd = malloc(sizeof(double) * (size_t)ND * N);
    st->ud = malloc(sizeof(double) * (size_t)ND * N);
    st->dud = malloc(sizeof(double) * (size_t)ND * N);
    st->Avd = malloc(sizeof(double) * ND);
    st->Td = malloc(sizeof(double) * ND);
    st->L = calloc(N, sizeof(double));
    for (int d = 0; d < ND; ++d) {
        double Av, delta;
        orc_dust_at_age(g, par, d, &Av, &delta, st->Td + d);
        st->Avd[d] = Av;
        for (int n = 0; n < N; ++n) {
            size_t x = (size_t)d * N + n;
            st->ud[x] = orc_dust_curve(g, g->lam[n], delta, st->dud + x);   /* A_lambda / Av, d/d delta */
            st->Fd[x] = pow(10.0, -0.4 * Av * st->ud[x]);
            st->L[n] += st->Fd[x] * st->Sd[x];
        }
    }
}

/* Given Lbar_n = dLoss/dL_n (L the attenuated spectrum per unit mass), the
 * per-group Sbar_d = Lbar F_d ([ND][n_lam]) and the dust gradients
 * (rows 8, 9 and, with age-dependent dust, the old-star rows). */
static double *gal_reverse_dust(const orc_grid *g, const gal_state *st, const double *Lbar, double *pbar)
{
    int N = g->n_lam, ND = st->ND;
    double *Sbar = malloc(sizeof(double) * (size_t)ND * N);
    for (int d = 0; d < ND; ++d) {
        double gav = 0.0, gdl = 0.0;
        for (int n = 0; n < N; ++n) {
            size_t x = (size_t)d * N + n;
            Sbar[x] = Lbar[n] * st->Fd[x];
            double Fbar = Lbar[n] * st->Sd[x];
            gav += Fbar * st->Fd[x] * (-0.4 * log(10.0)) * st->ud[x];
            gdl += Fbar * st->Fd[x] * (-0.4 * log(10.0)) * st->Avd[d] * st->dud[x];
        }
        double T = st->Td[d];
        pbar[8] += (1.0 - T) * gav;
        pbar[9] += (1.0 - T) * gdl;
        if (g->dust_agedep) {
            pbar[orc_grow_dust_old(g)] += T * gav;
            pbar[orc_grow_dust_old(g) + 1] += T * gdl;
        }
    }
    return Sbar;
}

static void gal_free(gal_state *st)
{
    free(st->dud); free(st->ud); free(st->Fd); free(st->Sd); free(st->Avd); free(st->Td); free(st->L);
    free(st->dmu7); free(st->dmu5);
    free(st->Pu); free(st->dPu_us); free(st->dPu_su);
    free(st->dPsig); free(st->dPmu); free(st->P); free(st->frac); free(st->Mhi); free(st->e);
    free(st->dsfr); free(st->sfr);
}

/* Reverse of the weights and the contraction: given Sbar = dLoss/dS_d for every
 * dust group ([ND][n_lam], S_d the group's per-unit-mass spectrum before dust),
 * adds dLoss/dp_k for k = 0..7 to pbar (and 11, 12 with a nebular axis). */
static void gal_reverse_sbar(const orc_grid *g, const gal_state *st, double t_obs, const double *Sbar,
                             double *pbar)
{
    int N = g->n_lam, NA = g->n_age, NZ = g->n_z, NU = orc_nu(g), K = NA * NZ * NU, NT = g->n_t;
    double *fracbar = calloc(NA, sizeof(double));
    double *Pubar = calloc(NU, sizeof(double));
    for (int k = 0; k < K; ++k) {
        const double *L = g->l_ssp + (size_t)k * N;
        double wbar = 0.0;
        int ij = k / NU, u = k % NU, i = ij / NZ;
        const double *sb = Sbar + (size_t)(st->ND > 1 ? i : 0) * N;
        for (int n = 0; n < N; ++n) wbar += sb[n] * L[n];
        fracbar[i] += wbar * st->P[ij] * st->Pu[u];
        double Pbar = wbar * st->frac[i] * st->Pu[u];
        pbar[5] += Pbar * st->dPmu[ij] * st->dmu5[i];
        pbar[6] += Pbar * st->dPsig[ij];
        pbar[7] += Pbar * st->dPmu[ij] * st->dmu7[i];
        Pubar[u] += wbar * st->frac[i] * st->P[ij];
    }
    if (NU > 1)
        for (int u = 0; u < NU; ++u) {
            pbar[11] += Pubar[u] * st->dPu_us[u];
            pbar[12] += Pubar[u] * st->dPu_su[u];
        }
    free(Pubar);
    /* frac_i = (Mhi_i - Mhi_{i+1}) / Mtot with Mtot = Mhi_0 */
    double *Mbar = calloc(NA + 1, sizeof(double));
    for (int i = 0; i < NA; ++i) {
        Mbar[i] += fracbar[i] / st->Mtot;
        Mbar[i + 1] -= fracbar[i] / st->Mtot;
        Mbar[0] -= fracbar[i] * st->frac[i] / st->Mtot;
    }
    double *coef = malloc(sizeof(double) * NT);
    double *sfrbar = calloc(NT, sizeof(double));
    for (int i = 0; i <= NA; ++i) {
        if (Mbar[i] == 0.0) continue;
        orc_cum_mass(st->sfr, NT, g->t0, g->t1, t_obs - st->e[i], coef);
        for (int n = 0; n < NT; ++n) sfrbar[n] += Mbar[i] * coef[n];
    }
    for (int n = 0; n < NT; ++n)
        for (int k = 0; k < 5; ++k) pbar[k] += sfrbar[n] * st->dsfr[5 * n + k];
    if (g->sfh_model == ORC_SFH_TABLE)   /* the table rows are the node SFRs themselves */
        for (int n = 0; n < NT; ++n) pbar[orc_grow_sfr(g) + n] += sfrbar[n];
    free(sfrbar); free(coef); free(Mbar); free(fracbar);
}

static void galaxy_mags_vjp(const orc_grid *g, const orc_filters *f, const double *par, double t_obs,
                            double dmod, const double *mbar, double *mags, double *pbar /* 11, or 13 */)
{
    int N = g->n_lam, Q = f->n_filt;
    double logM = par[10], z = par[11];
    gal_state st;
    gal_forward(g, par, t_obs, &st);
    int *off = malloc(sizeof(int) * (Q + 1));
    filter_offsets(f, off);
    double *T = malloc(sizeof(double) * (size_t)Q * N);
    double *Nq = malloc(sizeof(double) * Q);
    for (int q = 0; q < Q; ++q) {
        const double *fl = f->lam + off[q], *ft = f->trans + off[q];
        double acc = 0.0;
        for (int n = 0; n < N; ++n) {
            T[(size_t)q * N + n] = orc_filter_trans(fl, ft, f->n_pts[q], (1.0 + orc_filter_z(f, z)) * g->lam[n]);
            acc += trap_w(g->lam, N, n) / g->lam[n] * T[(size_t)q * N + n] * st.L[n];
        }
        Nq[q] = acc;
        double Dq = orc_filter_norm(fl, ft, f->n_pts[q]);
        if (mags) mags[q] = -2.5 * log10(pow(10.0, logM) * acc / (ORC_AB0 * Dq)) + orc_frame_offset(f, z, dmod);
    }

    /* reverse sweep */
    for (int k = 0; k < orc_ngrad(g); ++k) pbar[k] = 0.0;
    double *Nbar = malloc(sizeof(double) * Q);
    for (int q = 0; q < Q; ++q) {
        /* a band without flux (its filter off the SSP grid at this redshift)
         * has m = +inf and no gradient term */
        if (Nq[q] > 0.0) pbar[10] += -2.5 * mbar[q];
        Nbar[q] = Nq[q] > 0.0 ? mbar[q] * (-2.5 / log(10.0)) / Nq[q] : 0.0;
    }
    double *Lbar = calloc(N, sizeof(double));
    for (int n = 0; n < N; ++n) {
        double c = trap_w(g->lam, N, n) / g->lam[n];
        double sT = 0.0;
        for (int q = 0; q < Q; ++q) sT += Nbar[q] * T[(size_t)q * N + n];
        Lbar[n] = c * sT;
    }
    double *Sbar = gal_reverse_dust(g, &st, Lbar, pbar);
    gal_reverse_sbar(g, &st, t_obs, Sbar, pbar);
    free(Sbar); free(Lbar); free(Nbar); free(Nq); free(T); free(off);
    gal_free(&st);
}

/* Magnitudes with age-dependent dust (Sec. 3.4.1, Eq. agedep_dust_csp): the
 * attenuated spectrum sum_i F_i S_i through Eq. (restmag) as above. */
static void galaxy_mags_agedep(const orc_grid *g, const orc_filters *f, const double *par, double t_obs,
                               double dmod, double *mags)
{
    int N = g->n_lam, Q = f->n_filt;
    double logM = par[10], z = par[11];
    gal_state st;
    gal_forward(g, par, t_obs, &st);
    int *off = malloc(sizeof(int) * (Q + 1));
    filter_offsets(f, off);
    for (int q = 0; q < Q; ++q) {
        const double *fl = f->lam + off[q], *ft = f->trans + off[q];
        double acc = 0.0;
        for (int n = 0; n < N; ++n) {
            double T = orc_filter_trans(fl, ft, f->n_pts[q], (1.0 + orc_filter_z(f, z)) * g->lam[n]);
            acc += trap_w(g->lam, N, n) / g->lam[n] * T * st.L[n];
        }
        double Dq = orc_filter_norm(fl, ft, f->n_pts[q]);
        mags[q] = -2.5 * log10(pow(10.0, logM) * acc / (ORC_AB0 * Dq)) + orc_frame_offset(f, z, dmod);
    }
    free(off);
    gal_free(&st);
}

/* ------------------------------------------------------------------ */
/* Sec. 2.2, Eq. (eqw): emission-line equivalent width                 */
/* ------------------------------------------------------------------ */

/* Line window [lam_c - hw, lam_c + hw] and the continuum on both sides of it,
 * hw < |lam - lam_c| <= hw + cw (reading: the paper fits the neighbourhood of
 * the line with the line's range masked, and gives no window sizes). */
typedef struct {
    double lam_c, half_width, cont_width;
} orc_line;

/* Solves the 3x3 system A x = b (Gaussian elimination, partial pivoting). */
static int solve3(const double A_in[3][3], const double b_in[3], double x[3])
{
    double A[3][3], b[3];
    memcpy(A, A_in, sizeof(A));
    memcpy(b, b_in, sizeof(b));
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return -1;
        if (piv != c) {
            for (int k = 0; k < 3; ++k) { double t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t; }
            double t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < 3; ++r) {
            double m = A[r][c] / A[c][c];
            for (int k = c; k < 3; ++k) A[r][k] -= m * A[c][k];
            b[r] -= m * b[c];
        }
    }
    for (int c = 2; c >= 0; --c) {
        double v = b[c];
        for (int k = c + 1; k < 3; ++k) v -= A[c][k] * x[k];
        x[c] = v / A[c][c];
    }
    return 0;
}

/* Eq. (eqw) on a tabulated spectrum L(lam_n):
 *   L0   the quadratic in lam fitted by least squares to the continuum points
 *        (the line's own range masked), evaluated at each point of the line
 *        window (reading: the continuum at the line, point by point);
 *   W    = int over the line window of (L - L0) / L0 dlam, trapezoid rule on
 *        the grid points inside the window.
 * Returns W [A] (NaN with fewer than 3 continuum or 2 line points); Lbar
 * (optional, [n]) receives dW/dL_n. */
double orc_ew_from_spectrum(const double *lam, const double *L, int n, const orc_line *ln, double *Lbar)
{
    double hw = ln->half_width, cw = ln->cont_width, xs = hw + cw;
    double M[3][3] = {{0}}, r[3] = {0}, beta[3];
    int n_cont = 0, n_line = 0;
    for (int k = 0; k < n; ++k) {
        double d = fabs(lam[k] - ln->lam_c);
        if (d <= hw) ++n_line;
        else if (d <= hw + cw) {
            double x = (lam[k] - ln->lam_c) / xs, phi[3] = {1.0, x, x * x};
            for (int a = 0; a < 3; ++a) {
                r[a] += phi[a] * L[k];
                for (int b = 0; b < 3; ++b) M[a][b] += phi[a] * phi[b];
            }
            ++n_cont;
        }
    }
    if (Lbar) for (int k = 0; k < n; ++k) Lbar[k] = 0.0;
    if (n_cont < 3 || n_line < 2 || solve3(M, r, beta) != 0) return NAN;
    double W = 0.0, gam[3] = {0, 0, 0};
    int prev = -1;
    for (int k = 0; k < n; ++k) {
        if (fabs(lam[k] - ln->lam_c) > hw) continue;
        if (prev >= 0) {
            double dl = lam[k] - lam[prev];
            double fa[2];
            int idx[2] = {prev, k};
            for (int s = 0; s < 2; ++s) {
                double x = (lam[idx[s]] - ln->lam_c) / xs;
                double L0 = beta[0] + beta[1] * x + beta[2] * x * x;
                fa[s] = (L[idx[s]] - L0) / L0;
                if (Lbar) {
                    /* d/dL of 0.5 dl (L/L0 - 1), and its L0 part through beta */
                    Lbar[idx[s]] += 0.5 * dl / L0;
                    double g0 = -0.5 * dl * L[idx[s]] / (L0 * L0);
                    gam[0] += g0;
                    gam[1] += g0 * x;
                    gam[2] += g0 * x * x;
                }
            }
            W += 0.5 * dl * (fa[0] + fa[1]);
        }
        prev = k;
    }
    if (Lbar) {
        /* beta = M^-1 r, r = sum_cont phi L:  dW/dL_m = phi_m^T M^-1 gamma */
        double rho[3];
        solve3(M, gam, rho);
        for (int k = 0; k < n; ++k) {
            double d = fabs(lam[k] - ln->lam_c);
            if (d <= hw || d > hw + cw) continue;
            double x = (lam[k] - ln->lam_c) / xs;
            Lbar[k] += rho[0] + rho[1] * x + rho[2] * x * x;
        }
    }
    return W;
}

/* Rest-frame attenuated spectrum of one galaxy (Eq. cspdef with the weights
 * of Eq. agedep_mdf, times Eq. attenuation): L_n = 10^logM F_n S_n [Lsun/Hz]. */
static void galaxy_spectrum(const orc_grid *g, const double *par, double t_obs, double *out)
{
    gal_state st;
    gal_forward(g, par, t_obs, &st);
    double M = pow(10.0, par[10]);
    for (int n = 0; n < g->n_lam; ++n) out[n] = M * st.L[n];
    gal_free(&st);
}

/* Equivalent width of one galaxy's spectrum and, with ewbar, its adjoint
 * pbar[k] = ewbar dW/dp_k (k = 0..10). */
static double galaxy_ew(const orc_grid *g, const orc_line *ln, const double *par, double t_obs, double ewbar,
                        double *pbar)
{
    int N = g->n_lam;
    gal_state st;
    gal_forward(g, par, t_obs, &st);
    double M = pow(10.0, par[10]);
    double *L = malloc(sizeof(double) * N), *Lbar = malloc(sizeof(double) * N);
    for (int n = 0; n < N; ++n) L[n] = M * st.L[n];
    double W = orc_ew_from_spectrum(g->lam, L, N, ln, pbar ? Lbar : NULL);
    if (pbar) {
        for (int k = 0; k < orc_ngrad(g); ++k) pbar[k] = 0.0;
        /* L = 10^logM sum_d F_d S_d: cotangent of the per-unit-mass spectrum */
        double *lbu = malloc(sizeof(double) * N);
        for (int n = 0; n < N; ++n) {
            lbu[n] = ewbar * Lbar[n] * M;
            pbar[10] += ewbar * Lbar[n] * L[n] * log(10.0);
        }
        double *Sbar = gal_reverse_dust(g, &st, lbu, pbar);
        gal_reverse_sbar(g, &st, t_obs, Sbar, pbar);
        free(Sbar); free(lbu);
    }
    free(Lbar); free(L);
    gal_free(&st);
    return W;
}

/* ------------------------------------------------------------------ */
/* Batched entry points (threads over galaxies)                        */
/* ------------------------------------------------------------------ */

typedef struct {
    const orc_grid *g;
    const orc_filters *f;
    long n_gal, begin, end;
    const double *params, *mbar;
    double *w_out, *mags, *pbar;
    int mode;  /* 0 weights, 1 mags, 2 vjp, 3 spectrum, 4 line EW (+ adjoint with pbar) */
    const orc_line *line;
    double *out;   /* mode 3: [G][n_lam]; mode 4: [G] */
} orc_job;

/* The forward model's domain (the library's too): redshift z > 0 and finite,
 * MDF width sigma > 0, log U width > 0 with a nebular axis.  Outside it every
 * output of the galaxy is NaN; the cosmology integrals are not evaluated
 * there (at z <= -1 their limits are not numbers). */
static int orc_in_domain(const orc_grid *g, const double *par)
{
    double z = par[11];
    if (!(z > 0.0) || !isfinite(z)) return 0;
    if (!(par[6] > 0.0)) return 0;
    if (orc_nu(g) > 1 && !(par[13] > 0.0)) return 0;
    return 1;
}

static void *orc_worker(void *arg)
{
    orc_job *j = (orc_job *)arg;
    const orc_grid *g = j->g;
    int K = g->n_age * g->n_z * orc_nu(g), npar = orc_npar(g), ngrad = orc_ngrad(g);
    double *par = malloc(sizeof(double) * npar);
    double *pb = malloc(sizeof(double) * ngrad);
    double *omega = malloc(sizeof(double) * K);
    for (long gi = j->begin; gi < j->end; ++gi) {
        for (int r = 0; r < npar; ++r) par[r] = j->params[(size_t)r * j->n_gal + gi];
        double z = par[11];
        if (!orc_in_domain(g, par)) {
            if (j->mode == 0)
                for (int k = 0; k < K; ++k) j->w_out[(size_t)gi * K + k] = NAN;
            if (j->mags)
                for (int q = 0; q < j->f->n_filt; ++q) j->mags[(size_t)gi * j->f->n_filt + q] = NAN;
            if (j->mode == 3)
                for (int n = 0; n < g->n_lam; ++n) j->out[(size_t)gi * g->n_lam + n] = NAN;
            if (j->mode == 4) j->out[gi] = NAN;
            if (j->pbar)
                for (int k = 0; k < ngrad; ++k) j->pbar[(size_t)k * j->n_gal + gi] = NAN;
            continue;
        }
        double t_obs = orc_age_gyr(g->om0, g->w0, g->h, z);
        if (j->mode == 0) {
            galaxy_weights(g, par, t_obs, omega);
            double M = pow(10.0, par[10]);
            for (int k = 0; k < K; ++k) j->w_out[(size_t)gi * K + k] = M * omega[k];
        } else if (j->mode == 1 && g->dust_agedep) {
            /* one curve per age bin: through the per-group forward state */
            double dmod = orc_dist_mod(g->om0, g->w0, g->h, z);
            galaxy_mags_agedep(g, j->f, par, t_obs, dmod, j->mags + (size_t)gi * j->f->n_filt);
        } else if (j->mode == 1) {
            double dmod = orc_dist_mod(g->om0, g->w0, g->h, z);
            galaxy_weights(g, par, t_obs, omega);
            orc_mags_from_weights(g, j->f, omega, par[8], par[9], par[10], z, dmod,
                                  j->mags + (size_t)gi * j->f->n_filt);
        } else if (j->mode == 3) {
            galaxy_spectrum(g, par, t_obs, j->out + (size_t)gi * g->n_lam);
        } else if (j->mode == 4) {
            j->out[gi] = galaxy_ew(g, j->line, par, t_obs, j->mbar ? j->mbar[gi] : 0.0, j->pbar ? pb : NULL);
            if (j->pbar)
                for (int k = 0; k < ngrad; ++k) j->pbar[(size_t)k * j->n_gal + gi] = pb[k];
        } else {
            double dmod = orc_dist_mod(g->om0, g->w0, g->h, z);
            galaxy_mags_vjp(g, j->f, par, t_obs, dmod, j->mbar + (size_t)gi * j->f->n_filt,
                            j->mags ? j->mags + (size_t)gi * j->f->n_filt : NULL, pb);
            for (int k = 0; k < ngrad; ++k) j->pbar[(size_t)k * j->n_gal + gi] = pb[k];
        }
    }
    free(omega); free(pb); free(par);
    return NULL;
}

static int orc_run(orc_job proto, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > proto.n_gal) nthreads = (int)(proto.n_gal > 0 ? proto.n_gal : 1);
    pthread_t *th = malloc(sizeof(pthread_t) * nthreads);
    orc_job *jobs = malloc(sizeof(orc_job) * nthreads);
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = proto;
        jobs[t].begin = proto.n_gal * t / nthreads;
        jobs[t].end = proto.n_gal * (t + 1) / nthreads;
        pthread_create(&th[t], NULL, orc_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(jobs); free(th);
    return 0;
}

/* Per-galaxy SSP weights in Msun: w[g][i][j] = 10^logM frac_i P[j|i]. */
int orc_weights(const orc_grid *g, long n_gal, const double *params, double *w_out, int nthreads)
{
    orc_job j = {g, NULL, n_gal, 0, n_gal, params, NULL, w_out, NULL, NULL, 0, NULL, NULL};
    return orc_run(j, nthreads);
}

/* Observer-frame AB magnitudes mags[g][q]. */
int orc_mags(const orc_grid *g, const orc_filters *f, long n_gal, const double *params, double *mags,
             int nthreads)
{
    orc_job j = {g, f, n_gal, 0, n_gal, params, NULL, NULL, mags, NULL, 1, NULL, NULL};
    return orc_run(j, nthreads);
}

/* Vector-Jacobian product: pbar[k][g] = sum_q mbar[g][q] d m_q / d p_k. */
int orc_mags_vjp(const orc_grid *g, const orc_filters *f, long n_gal, const double *params,
                 const double *mbar, double *mags, double *pbar, int nthreads)
{
    orc_job j = {g, f, n_gal, 0, n_gal, params, mbar, NULL, mags, pbar, 2, NULL, NULL};
    return orc_run(j, nthreads);
}

/* Rest-frame attenuated spectra out[g][n] [Lsun/Hz]. */
int orc_spectra(const orc_grid *g, long n_gal, const double *params, double *out, int nthreads)
{
    orc_job j = {g, NULL, n_gal, 0, n_gal, params, NULL, NULL, NULL, NULL, 3, NULL, out};
    return orc_run(j, nthreads);
}

/* Equivalent widths ew[g] [A] and, if pbar != NULL, pbar[k][g] = ewbar[g] dW_g/dp_k. */
int orc_line_ew(const orc_grid *g, const orc_line *line, long n_gal, const double *params, const double *ewbar,
                double *ew, double *pbar, int nthreads)
{
    orc_job j = {g, NULL, n_gal, 0, n_gal, params, ewbar, NULL, NULL, pbar, 4, line, ew};
    return orc_run(j, nthreads);
}
