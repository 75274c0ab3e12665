// api.cu -- the C ABI of libdsps (include/dsps.h): context set-up, filter
// registration, and the per-call dispatch of the weights and photometry
// kernels over chunks of galaxies.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dsps_internal.cuh"

using namespace dsps;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, const char *detail = "") {
    char buf[512];
    std::snprintf(buf, sizeof buf, fmt, detail);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *where) {
    char buf[512];
    std::snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
    g_last_error = buf;
    return DSPS_ERR_CUDA;
}

#define DSPS_CUDA(call)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on the
// three-term recurrence of the Legendre polynomials).
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; ++j) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double z1 = z;
            z = z1 - p1 / pp;
            if (std::fabs(z - z1) < 1e-15) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

struct GL {
    std::vector<double> x, w;
    explicit GL(int n) { gauss_legendre(n, x, w); }
    template <class F>
    double integrate(F f, double a, double b) const {
        double c = 0.5 * (a + b), h = 0.5 * (b - a), s = 0.0;
        for (size_t i = 0; i < x.size(); ++i) s += w[i] * f(c + h * x[i]);
        return s * h;
    }
};

// Sec. 2.2: t_obs(z) [Gyr] and Dmod(z) - 5 log10 z for flat wCDM on a uniform
// z table, FP64.
void build_cosmology(double om0, double w0, double h, double zmax, double dz, std::vector<double> &tl,
                     std::vector<double> &gl) {
    const int n = (int)std::ceil(zmax / dz) + 2;
    tl.assign(n, 0.0);
    gl.assign(n, 0.0);
    const double inv_h0_gyr = 977.792221 / (100.0 * h);
    const double c_h0_mpc = 299792.458 / (100.0 * h);
    auto E = [&](double z) {
        double a1 = 1.0 + z;
        return std::sqrt(om0 * a1 * a1 * a1 + (1.0 - om0) * std::pow(a1, 3.0 * (1.0 + w0)));
    };
    GL g8(8);
    // comoving distance, cumulative upward
    double dc = 0.0;
    gl[0] = 5.0 * std::log10(c_h0_mpc * 1e5);
    for (int i = 1; i < n; ++i) {
        double za = (i - 1) * dz, zb = i * dz;
        dc += g8.integrate([&](double z) { return 1.0 / E(z); }, za, zb);
        gl[i] = 5.0 * std::log10((1.0 + zb) * c_h0_mpc * dc / zb * 1e5);
    }
    // age at the top of the table: int_0^{sqrt(a)} 2 ds / (s E(1/s^2 - 1))
    const double ztop = (n - 1) * dz;
    const double smax = std::sqrt(1.0 / (1.0 + ztop));
    auto f = [&](double s) { return s <= 0.0 ? 0.0 : 2.0 / (s * E(1.0 / (s * s) - 1.0)); };
    double t = 0.0;
    const int panels = 256;
    for (int p = 0; p < panels; ++p) t += g8.integrate(f, smax * p / panels, smax * (p + 1) / panels);
    tl[n - 1] = inv_h0_gyr * t;
    for (int i = n - 2; i >= 0; --i) {
        double za = i * dz, zb = (i + 1) * dz;
        tl[i] = tl[i + 1] + inv_h0_gyr * g8.integrate([&](double z) { return 1.0 / ((1.0 + z) * E(z)); }, za, zb);
    }
}

double filter_interp(const double *l, const double *t, int n, double x) {
    if (x < l[0] || x > l[n - 1]) return 0.0;
    const double *it = std::upper_bound(l, l + n, x);
    int hi = (int)(it - l);
    if (hi >= n) hi = n - 1;
    int lo = hi - 1;
    if (lo < 0) return t[0];
    double w = (x - l[lo]) / (l[hi] - l[lo]);
    return t[lo] + w * (t[hi] - t[lo]);
}

template <class T>
int dmalloc(T **p, size_t count) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    return DSPS_OK;
}

void free_ctx(Ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    for (auto &fs : c->sets) {
        cudaFree(fs.d_tab);
        cudaFree(fs.d_offq);
        cudaFree(fs.d_cov);
    }
    for (auto &ls : c->lines) cudaFree(ls.d_tab);
    void *ptrs[] = {c->d_L32, c->d_Lt_hi, c->d_Lt_lo, c->d_wmul, c->d_logage, c->d_mua, c->d_mub, c->d_bump, c->d_k0, c->d_edges, c->d_einh, c->d_bwidth,
                    c->d_zedge, c->d_uedge, c->d_tlut, c->d_glut, c->d_ws_block, c->ws.shat, c->ws.ewacc, c->d_err, c->d_stats,
                    c->d_L_hi, c->d_L_lo, c->d_Ld32, c->d_wmul_d, c->d_hio, c->d_Lab_hi, c->d_Lab_lo,
                    c->d_wmul_ab, c->d_Ldab_hi, c->d_Ldab_lo};
    for (void *p : ptrs) cudaFree(p);
    for (auto &r : c->prof_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    delete c;
}

}  // namespace

namespace dsps {
int serve_start(Ctx *c);
void serve_stop(Ctx *c);
int serve_submit(Ctx *c, const dsps_request *r, uint64_t *ticket);
int serve_poll(Ctx *c, uint64_t ticket, int64_t timeout_us, double *latency_us);
int run_photometry(Ctx *c, int64_t n_gal, const float *params, int32_t set_id, int32_t precision, float *mags,
                   cudaStream_t s);
int run_photometry_vjp(Ctx *c, int64_t n_gal, const float *params, int32_t set_id, int32_t precision,
                       const float *mag_bar, float *mags, float *param_bar, cudaStream_t s);
const char *last_error_message() { return g_last_error.c_str(); }
void set_last_error(const char *msg) { g_last_error = msg; }
}  // namespace dsps

extern "C" {

void dsps_default_opts(dsps_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->om0 = 0.3;
    o->w0 = -1.0;
    o->h = 0.7;
    o->sfh_model = DSPS_SFH_DELAYED_TAU;
    o->mdf_kernel = DSPS_MDF_TRIWEIGHT;
    o->device = 0;
    o->max_chunk = 262144;
    o->hbm_budget_bytes = (int64_t)8 << 30;
    o->n_streams = 4;
    o->z_max = 10.0;
    o->band_skip = 1;
    o->mdf_mean = DSPS_MDF_MEAN_LINEAR;
    o->mdf_terf_x0 = 9.0;
    o->mdf_terf_h = 0.5;
    o->dust_bump = 0;
    o->dust_law = DSPS_DUST_POWERLAW;
    o->dust_agedep = 0;
    o->dust_agedep_x0 = 7.0;
    o->dust_agedep_h = 0.1;
    o->agedep_fused = 1;
}

namespace {
// Appendix B, Eq. (terf): the triweight cumulative kernel, 0 below -3 and 1
// above 3.
double terf_host(double z) {
    if (z <= -3.0) return 0.0;
    if (z >= 3.0) return 1.0;
    const double z2 = z * z;
    return 0.5 + z * (35.0 / 96.0 + z2 * (-35.0 / 864.0 + z2 * (7.0 / 2592.0 - z2 * 5.0 / 69984.0)));
}
}  // namespace

const char *dsps_last_error_message(void) { return g_last_error.c_str(); }

int dsps_create(dsps_ctx **out, const dsps_grid *g, const dsps_opts *o) {
    DSPS_TRACE("dsps_create");
    if (!out || !g) return fail(DSPS_ERR_INVALID_ARG, "dsps_create: null argument%s");
    *out = nullptr;
    dsps_opts opts;
    if (o) opts = *o; else dsps_default_opts(&opts);
    if (g->n_age < 2 || g->n_age > MAX_NAGE || g->n_z < 1 || g->n_lam < 2 || g->n_t < 2 || g->n_t > MAX_NT)
        return fail(DSPS_ERR_INVALID_ARG, "dsps_create: grid sizes out of range%s");
    if (!g->log_age_yr || !g->lgz || !g->lam || !g->l_ssp)
        return fail(DSPS_ERR_INVALID_ARG, "dsps_create: null grid array%s");
    if (!(g->t1_gyr > g->t0_gyr) || !(g->t0_gyr >= 0))
        return fail(DSPS_ERR_INVALID_ARG, "dsps_create: bad SFR time grid%s");
    for (int i = 1; i < g->n_age; ++i)
        if (!(g->log_age_yr[i] > g->log_age_yr[i - 1])) return fail(DSPS_ERR_INVALID_ARG, "dsps_create: ages not increasing%s");
    for (int j = 1; j < g->n_z; ++j)
        if (!(g->lgz[j] > g->lgz[j - 1])) return fail(DSPS_ERR_INVALID_ARG, "dsps_create: lgZ not increasing%s");
    const int n_u = g->n_u > 1 ? g->n_u : 1;
    if (g->n_u > DSPS_MAX_NU || g->n_u < 0 || (n_u > 1 && !g->lgu))
        return fail(DSPS_ERR_INVALID_ARG, "dsps_create: nebular axis needs 2..8 log U values%s");
    for (int k = 1; k < n_u; ++k)
        if (!(g->lgu[k] > g->lgu[k - 1])) return fail(DSPS_ERR_INVALID_ARG, "dsps_create: log U not increasing%s");
    if (!(g->lam[0] > 0)) return fail(DSPS_ERR_INVALID_ARG, "dsps_create: wavelengths must be positive%s");
    const double dl = std::log(g->lam[g->n_lam - 1] / g->lam[0]) / (g->n_lam - 1);
    if (!(dl > 0)) return fail(DSPS_ERR_INVALID_ARG, "dsps_create: wavelengths not increasing%s");
    for (int n = 0; n < g->n_lam; ++n) {
        double expect = g->lam[0] * std::exp(n * dl);
        if (std::fabs(g->lam[n] / expect - 1.0) > 1e-9)
            return fail(DSPS_ERR_UNSUPPORTED, "dsps_create: wavelength grid is not uniform in ln(lambda)%s");
    }
    if (opts.sfh_model < 0 || opts.sfh_model > 2 || opts.mdf_kernel < 0 || opts.mdf_kernel > 1 ||
        opts.mdf_mean < 0 || opts.mdf_mean > 1 || opts.dust_bump < 0 || opts.dust_bump > 1 || opts.dust_law < 0 ||
        opts.dust_law > 1 || opts.agedep_fused < 0 || opts.agedep_fused > 1)
        return fail(DSPS_ERR_INVALID_ARG, "dsps_create: unknown model switch%s");
    if (opts.dust_agedep < 0 || opts.dust_agedep > 1 ||
        (opts.dust_agedep && !(opts.dust_agedep_h > 0 && std::isfinite(opts.dust_agedep_x0))))
        return fail(DSPS_ERR_INVALID_ARG, "dsps_create: bad age-dependent dust options%s");
    if (opts.mdf_mean == DSPS_MDF_MEAN_TERF && !(opts.mdf_terf_h > 0 && std::isfinite(opts.mdf_terf_x0)))
        return fail(DSPS_ERR_INVALID_ARG, "dsps_create: bad MDF transition%s");
    if (!(opts.z_max > 0) || opts.z_max > 50 || !(opts.om0 > 0) || !(opts.h > 0))
        return fail(DSPS_ERR_INVALID_ARG, "dsps_create: bad cosmology options%s");
    if (opts.max_chunk < 128) opts.max_chunk = 128;
    if (opts.n_streams < 1) opts.n_streams = 1;

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return fail(DSPS_ERR_CUDA, "dsps_create: no CUDA device%s");
    if (opts.device < 0 || opts.device >= ndev) return fail(DSPS_ERR_INVALID_ARG, "dsps_create: bad device%s");
    DSPS_CUDA(cudaSetDevice(opts.device));
    cudaDeviceProp prop;
    DSPS_CUDA(cudaGetDeviceProperties(&prop, opts.device));
    if (prop.major != 10 || prop.minor != 3)
        return fail(DSPS_ERR_UNSUPPORTED, "dsps_create: libdsps is built for sm_103a (GB300) only%s");

    Ctx *c = new Ctx();
    c->device = opts.device;
    c->opts = opts;
    c->num_sms = prop.multiProcessorCount;
    c->n_age = g->n_age;
    c->n_z = g->n_z;
    c->n_lam = g->n_lam;
    c->n_u = n_u;
    {
        // rows: 0..11, [u_mean, u_sigma], [Av_old, delta_old], [SFR table]
        const int p_neb = n_u > 1 ? NPAR_MAX : NPAR, g_neb = n_u > 1 ? DSPS_NGRAD_NEB : NGRAD;
        const int p_dust = p_neb + (opts.dust_agedep ? 2 : 0), g_dust = g_neb + (opts.dust_agedep ? 2 : 0);
        const bool table = opts.sfh_model == DSPS_SFH_TABLE;
        c->row_dust_old = opts.dust_agedep ? p_neb : -1;
        c->grow_dust_old = opts.dust_agedep ? g_neb : -1;
        c->row_sfr = table ? p_dust : -1;
        c->grow_sfr = table ? g_dust : -1;
        c->npar = p_dust + (table ? g->n_t : 0);
        c->ngrad = g_dust + (table ? g->n_t : 0);
    }
    if (opts.dust_agedep) {
        // groups of age bins sharing one attenuation curve (Sec. 3.4.1): runs
        // of bins with T = 0 or T = 1, every bin of the transition on its own
        for (int i = 0; i < g->n_age;) {
            const double T = terf_host((g->log_age_yr[i] - opts.dust_agedep_x0) / opts.dust_agedep_h);
            int j = i + 1;
            if (T == 0.0 || T == 1.0)
                while (j < g->n_age &&
                       terf_host((g->log_age_yr[j] - opts.dust_agedep_x0) / opts.dust_agedep_h) == T)
                    ++j;
            c->dust_groups.push_back(DustGroup{i, j, (float)T});
            i = j;
        }
    }
    c->u_ref = n_u / 2;
    c->K = g->n_age * g->n_z * n_u;
    c->K_pad = (c->K + K_ALIGN - 1) / K_ALIGN * K_ALIGN;
    c->A_pad = (c->n_age + 3) / 4 * 4;
    c->SEC = (c->n_z * c->A_pad + KBLOCK - 1) / KBLOCK * KBLOCK;
    c->KZ_pad = (n_u * c->SEC + K_ALIGN - 1) / K_ALIGN * K_ALIGN;
    c->kmask_words = (c->SEC / KBLOCK + 31) / 32;
    if (opts.dust_agedep && n_u == 1 && g->n_z <= KBLOCK && g->n_age <= 128) {
        // age-block order of the fused age-dependent dust forward: one mask bit per age
        c->KA_pad = (g->n_age * KBLOCK + K_ALIGN - 1) / K_ALIGN * K_ALIGN;
        if (c->kmask_words < 4) c->kmask_words = 4;
    }
    c->N_pad = (c->n_lam + 1 + N_ALIGN - 1) / N_ALIGN * N_ALIGN;   // >= n_lam + 1: room for the closing term
    c->n_t = g->n_t;
    c->t0 = g->t0_gyr;
    c->t1 = g->t1_gyr;
    c->lnlam0 = std::log(g->lam[0]);
    c->dlnlam = dl;
    c->h_lam.assign(g->lam, g->lam + g->n_lam);
    c->chunk = (opts.max_chunk + 127) / 128 * 128;
    {
        // keep the context's work space under 16 GiB (grids with a nebular axis
        // have n_u times longer weight rows)
        const size_t cap = (size_t)16 << 30, per = workspace_bytes(*c, 128, false) / 128 + 1;
        const int64_t fit = (int64_t)(cap / per) / 128 * 128;
        if (fit >= 128 && c->chunk > fit) c->chunk = fit;
    }
    {
        const double xmid = 0.5 * (g->log_age_yr[0] + g->log_age_yr[g->n_age - 1]);
        if (opts.mdf_mean == DSPS_MDF_MEAN_TERF) {
            const double T = terf_host((xmid - opts.mdf_terf_x0) / opts.mdf_terf_h);
            c->sort_mua = (float)(1.0 - T);
            c->sort_mub = (float)T;
        } else {
            c->sort_mua = 1.f;
            c->sort_mub = (float)(xmid - 9.0);
        }
    }
    if (n_u > 1) {
        c->sort_u_lo = (float)g->lgu[0];
        c->sort_u_scale = (float)(8.0 / (g->lgu[n_u - 1] - g->lgu[0]));
    }
    c->sort_mu_lo = (float)g->lgz[0];
    c->sort_mu_scale = g->n_z > 1 ? (float)(ZSORT_MUBINS / (g->lgz[g->n_z - 1] - g->lgz[0])) : 0.f;

    int rc = DSPS_OK;
    auto chk = [&](int r) { if (rc == DSPS_OK) rc = r; };
    chk(dmalloc(&c->d_L32, (size_t)c->K_pad * c->N_pad));
    chk(dmalloc(&c->d_Lt_hi, (size_t)c->KZ_pad * c->N_pad));
    chk(dmalloc(&c->d_Lt_lo, (size_t)c->KZ_pad * c->N_pad));
    chk(dmalloc(&c->d_wmul, (size_t)c->KZ_pad));
    chk(dmalloc(&c->d_logage, (size_t)c->n_age));
    chk(dmalloc(&c->d_mua, (size_t)c->n_age));
    chk(dmalloc(&c->d_bump, (size_t)c->N_pad));
    chk(dmalloc(&c->d_k0, (size_t)c->N_pad));
    chk(dmalloc(&c->d_mub, (size_t)c->n_age));
    chk(dmalloc(&c->d_edges, (size_t)c->n_age + 1));
    chk(dmalloc(&c->d_einh, (size_t)c->n_age + 1));
    chk(dmalloc(&c->d_bwidth, (size_t)c->n_age));
    chk(dmalloc(&c->d_zedge, (size_t)c->n_z + 1));
    chk(dmalloc(&c->d_uedge, (size_t)c->n_u + 1));
    chk(dmalloc(&c->d_ws_block, workspace_bytes(*c, c->chunk, false)));
    chk(dmalloc(&c->d_err, 1));
    chk(dmalloc(&c->d_stats, 3));
    chk(dmalloc(&c->d_L_hi, (size_t)c->KZ_pad * c->N_pad));
    chk(dmalloc(&c->d_Ld32, (size_t)c->KZ_pad * c->N_pad));
    chk(dmalloc(&c->d_wmul_d, (size_t)c->KZ_pad));
    chk(dmalloc(&c->d_L_lo, (size_t)c->KZ_pad * c->N_pad));
    if (c->KA_pad) {
        chk(dmalloc(&c->d_Lab_hi, (size_t)c->KA_pad * c->N_pad));
        chk(dmalloc(&c->d_Lab_lo, (size_t)c->KA_pad * c->N_pad));
        chk(dmalloc(&c->d_Ldab_hi, (size_t)c->KA_pad * c->N_pad));
        chk(dmalloc(&c->d_Ldab_lo, (size_t)c->KA_pad * c->N_pad));
        chk(dmalloc(&c->d_wmul_ab, (size_t)c->KA_pad));
    }
    if (rc != DSPS_OK) { free_ctx(c); return rc; }
    c->ws = workspace_carve(*c, c->d_ws_block, c->chunk, false);

    // Age-bin edges [Gyr]: log-midpoints, first edge at age 0, last half a step
    // above the last grid age (Sec. 3.1).
    std::vector<double> edges(c->n_age + 1);
    edges[0] = 0.0;
    for (int i = 1; i < c->n_age; ++i) edges[i] = std::pow(10.0, 0.5 * (g->log_age_yr[i - 1] + g->log_age_yr[i]) - 9.0);
    edges[c->n_age] = std::pow(10.0, g->log_age_yr[c->n_age - 1] +
                                        0.5 * (g->log_age_yr[c->n_age - 1] - g->log_age_yr[c->n_age - 2]) - 9.0);
    const double hstep = (c->t1 - c->t0) / (c->n_t - 1);
    std::vector<float> einh(c->n_age + 1), bwidth(c->n_age);
    for (int i = 0; i <= c->n_age; ++i) einh[i] = (float)(edges[i] / hstep);
    for (int i = 0; i < c->n_age; ++i) bwidth[i] = (float)(edges[i + 1] - edges[i]);
    std::vector<float> logage(c->n_age), mua(c->n_age), mub(c->n_age);
    for (int i = 0; i < c->n_age; ++i) logage[i] = (float)g->log_age_yr[i];
    // MDF mean of age bin i: mu_i = mua_i p5 + mub_i p7 (dsps.h: DSPS_MDF_MEAN_*)
    for (int i = 0; i < c->n_age; ++i) {
        if (opts.mdf_mean == DSPS_MDF_MEAN_TERF) {
            const double T = terf_host((g->log_age_yr[i] - opts.mdf_terf_x0) / opts.mdf_terf_h);
            mua[i] = (float)(1.0 - T);
            mub[i] = (float)T;
        } else {
            mua[i] = 1.f;
            mub[i] = logage[i] - 9.f;   // the FP32 log age less the 1 Gyr pivot
        }
    }
    // lgZ bin edges: midpoints, outer edges at -/+ infinity (Sec. 3.2).
    std::vector<float> zedge(c->n_z + 1);
    zedge[0] = -1e30f;
    zedge[c->n_z] = 1e30f;
    for (int j = 1; j < c->n_z; ++j) zedge[j] = (float)(0.5 * (g->lgz[j - 1] + g->lgz[j]));
    // log U bin edges, likewise (Sec. 3.3)
    std::vector<float> uedge(c->n_u + 1);
    uedge[0] = -1e30f;
    uedge[c->n_u] = 1e30f;
    for (int k = 1; k < c->n_u; ++k) uedge[k] = (float)(0.5 * (g->lgu[k - 1] + g->lgu[k]));
    std::vector<double> tl, gl;
    c->dz_lut = 1e-3;
    build_cosmology(opts.om0, opts.w0, opts.h, opts.z_max, c->dz_lut, tl, gl);
    c->n_lut = (int)tl.size();
    if (dmalloc(&c->d_tlut, tl.size()) != DSPS_OK || dmalloc(&c->d_glut, gl.size()) != DSPS_OK) {
        free_ctx(c);
        return DSPS_ERR_CUDA;
    }
    cudaError_t e = cudaSuccess;
    auto up = [&](void *d, const void *h, size_t b) { if (e == cudaSuccess) e = cudaMemcpy(d, h, b, cudaMemcpyHostToDevice); };
    up(c->d_edges, edges.data(), edges.size() * sizeof(double));
    up(c->d_einh, einh.data(), einh.size() * sizeof(float));
    up(c->d_bwidth, bwidth.data(), bwidth.size() * sizeof(float));
    up(c->d_logage, logage.data(), logage.size() * sizeof(float));
    up(c->d_mua, mua.data(), mua.size() * sizeof(float));
    up(c->d_mub, mub.data(), mub.size() * sizeof(float));
    // Eq. (uvbump): unit Drude profile at the grid's wavelengths
    std::vector<float> bump(c->N_pad, 0.f);
    for (int n = 0; n < c->n_lam; ++n) {
        const double lam = g->lam[n], x = lam * 350.0, d = lam * lam - 2175.0 * 2175.0;
        bump[n] = (float)(x * x / (d * d + x * x));
    }
    up(c->d_bump, bump.data(), bump.size() * sizeof(float));
    // Eq. (kzero): starburst curve over 4.05 at the grid's wavelengths (the
    // published Leitherer fit below 0.15 um, Calzetti above, clipped at 0)
    std::vector<float> k0t(c->N_pad, 0.f);
    for (int n = 0; n < c->n_lam; ++n) {
        const double x = g->lam[n] * 1e-4;
        double k;
        if (x < 0.15) k = 5.472 + 0.671 / x - 9.218e-3 / (x * x) + 2.620e-3 / (x * x * x);
        else if (x < 0.63) k = 2.659 * (-2.156 + 1.509 / x - 0.198 / (x * x) + 0.011 / (x * x * x)) + 4.05;
        else k = 2.659 * (-1.857 + 1.040 / x) + 4.05;
        k0t[n] = (float)(k > 0.0 ? k / 4.05 : 0.0);
    }
    up(c->d_k0, k0t.data(), k0t.size() * sizeof(float));
    up(c->d_zedge, zedge.data(), zedge.size() * sizeof(float));
    up(c->d_uedge, uedge.data(), uedge.size() * sizeof(float));
    up(c->d_tlut, tl.data(), tl.size() * sizeof(double));
    std::vector<float> glf(gl.begin(), gl.end());
    up(c->d_glut, glf.data(), glf.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(c->d_stats, 0, 3 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = prepare_ssp_device(*c, g->l_ssp);
    if (e != cudaSuccess) {
        int r = cuda_fail(e, "dsps_create upload");
        free_ctx(c);
        return r;
    }
    *out = reinterpret_cast<dsps_ctx *>(c);
    return DSPS_OK;
}

int dsps_destroy(dsps_ctx *ctx) {
    DSPS_TRACE("dsps_destroy");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return DSPS_OK;
    serve_stop(c);
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    free_ctx(c);
    return DSPS_OK;
}

int dsps_filters_add(dsps_ctx *ctx, int32_t n_filt, const int32_t *n_pts, const double *const *lam,
                     const double *const *trans, int32_t *set_id) {
    DSPS_TRACE("dsps_filters_add");
    return dsps_filters_add_frame(ctx, n_filt, n_pts, lam, trans, DSPS_FRAME_OBSERVER, set_id);
}

int dsps_filters_add_frame(dsps_ctx *ctx, int32_t n_filt, const int32_t *n_pts, const double *const *lam,
                           const double *const *trans, int32_t frame, int32_t *set_id) {
    DSPS_TRACE("dsps_filters_add_frame");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !n_pts || !lam || !trans || !set_id) return fail(DSPS_ERR_INVALID_ARG, "dsps_filters_add: null argument%s");
    if (frame != DSPS_FRAME_OBSERVER && frame != DSPS_FRAME_REST)
        return fail(DSPS_ERR_INVALID_ARG, "dsps_filters_add: unknown frame%s");
    if (n_filt < 1 || n_filt > DSPS_MAX_FILTERS) return fail(DSPS_ERR_INVALID_ARG, "dsps_filters_add: 1..16 filters%s");
    double lmax = 0.0;
    std::vector<float> offq(n_filt);
    for (int q = 0; q < n_filt; ++q) {
        if (n_pts[q] < 2 || !lam[q] || !trans[q]) return fail(DSPS_ERR_INVALID_ARG, "dsps_filters_add: bad table%s");
        double D = 0.0;
        for (int m = 0; m < n_pts[q]; ++m) {
            if (!(trans[q][m] >= 0) || !(lam[q][m] > 0)) return fail(DSPS_ERR_INVALID_ARG, "dsps_filters_add: bad values%s");
            if (m > 0) {
                if (!(lam[q][m] > lam[q][m - 1])) return fail(DSPS_ERR_INVALID_ARG, "dsps_filters_add: lambda not increasing%s");
                D += 0.5 * (lam[q][m] - lam[q][m - 1]) * (trans[q][m] / lam[q][m] + trans[q][m - 1] / lam[q][m - 1]);
            }
        }
        if (!(D > 0)) return fail(DSPS_ERR_INVALID_ARG, "dsps_filters_add: filter with zero transmission%s");
        offq[q] = (float)(2.5 * std::log10(AB0 * D));   // Eq. (restmag) denominator
        lmax = std::max(lmax, lam[q][n_pts[q] - 1]);
    }
    FilterSet fs;
    fs.Q = n_filt;
    fs.Q4 = (n_filt + 3) / 4;
    fs.rest = frame == DSPS_FRAME_REST ? 1 : 0;
    const double l0 = std::exp(c->lnlam0);
    // Grid samples m = -1 .. M-1 at l0 exp(m dlnlam) in table rows t = m + 1,
    // then three zero rows (the 4-point interpolation reads up to m + 2).
    int M = lmax > l0 ? (int)std::ceil(std::log(lmax / l0) / c->dlnlam) + 2 : 1;
    fs.m_rows = M + 4;
    std::vector<float> tab((size_t)fs.m_rows * 4 * fs.Q4, 0.f);
    fs.m_nz_lo = fs.m_rows;
    fs.m_nz_hi = -1;
    for (int t = 0; t <= M; ++t) {
        const int m = t - 1;
        double x = l0 * std::exp(m * c->dlnlam);
        for (int q = 0; q < n_filt; ++q) {
            float v = (float)filter_interp(lam[q], trans[q], n_pts[q], x);
            tab[(size_t)t * 4 * fs.Q4 + q] = v;
            if (v != 0.f) {
                fs.m_nz_lo = std::min(fs.m_nz_lo, m);
                fs.m_nz_hi = std::max(fs.m_nz_hi, m);
            }
        }
    }
    // band coverage: the filter's own table, with the response accumulated from
    // both ends (trapezoids of T / lam) so that small fractions at either end
    // keep their relative precision
    std::vector<double> cov;
    for (int q = 0; q < n_filt; ++q) {
        const int np = n_pts[q];
        std::vector<double> A(np, 0.0), B(np, 0.0);
        for (int m = 1; m < np; ++m)
            A[m] = A[m - 1] + 0.5 * (lam[q][m] - lam[q][m - 1]) * (trans[q][m] / lam[q][m] + trans[q][m - 1] / lam[q][m - 1]);
        for (int m = np - 2; m >= 0; --m)
            B[m] = B[m + 1] + 0.5 * (lam[q][m + 1] - lam[q][m]) * (trans[q][m + 1] / lam[q][m + 1] + trans[q][m] / lam[q][m]);
        const double D = A[np - 1];
        fs.cov_off[q] = (int)(cov.size() / 3);
        int mid = np - 1;
        for (int m = 0; m < np; ++m) {
            cov.push_back(std::log(lam[q][m]));
            cov.push_back(A[m] / D);
            cov.push_back(B[m] / D);
            if (mid == np - 1 && A[m] >= 0.5 * D) mid = m;
        }
        fs.cov_mid[q] = fs.cov_off[q] + mid;
    }
    fs.cov_off[n_filt] = (int)(cov.size() / 3);
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    if (dmalloc(&fs.d_tab, tab.size()) != DSPS_OK) return DSPS_ERR_CUDA;
    if (dmalloc(&fs.d_offq, (size_t)n_filt) != DSPS_OK) { cudaFree(fs.d_tab); return DSPS_ERR_CUDA; }
    if (cudaMalloc(&fs.d_cov, cov.size() * sizeof(double)) != cudaSuccess) {
        cudaFree(fs.d_tab);
        cudaFree(fs.d_offq);
        return fail(DSPS_ERR_CUDA, "dsps_filters_add: out of device memory%s");
    }
    cudaError_t e = cudaMemcpy(fs.d_tab, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(fs.d_offq, offq.data(), offq.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(fs.d_cov, cov.data(), cov.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(fs.d_tab);
        cudaFree(fs.d_offq);
        cudaFree(fs.d_cov);
        return cuda_fail(e, "dsps_filters_add upload");
    }
    c->sets.push_back(fs);
    *set_id = (int32_t)c->sets.size() - 1;
    return DSPS_OK;
}

int dsps_filters_count(dsps_ctx *ctx, int32_t set_id, int32_t *n_filt) {
    DSPS_TRACE("dsps_filters_count");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !n_filt) return fail(DSPS_ERR_INVALID_ARG, "dsps_filters_count: null argument%s");
    std::lock_guard<std::mutex> lk(c->mu);
    if (set_id < 0 || set_id >= (int)c->sets.size()) return fail(DSPS_ERR_INVALID_ARG, "dsps_filters_count: unknown set%s");
    *n_filt = c->sets[set_id].Q;
    return DSPS_OK;
}

int dsps_weights(dsps_ctx *ctx, int64_t n_gal, const float *params, float *w_out, dsps_stream_t stream) {
    DSPS_TRACE("dsps_weights");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || n_gal < 0 || (n_gal > 0 && (!params || !w_out))) return fail(DSPS_ERR_INVALID_ARG, "dsps_weights: bad argument%s");
    if (n_gal == 0) return DSPS_OK;
    DSPS_CUDA(cudaSetDevice(c->device));
    std::lock_guard<std::mutex> lk(c->mu);
    for (int64_t g0 = 0; g0 < n_gal; g0 += c->ws.cap) {
        const int64_t n = n_gal - g0 < c->ws.cap ? n_gal - g0 : c->ws.cap;
        DSPS_CUDA(launch_weights(*c, c->ws, W_MSUN, params, n_gal, g0, n, w_out + g0 * c->K,
                                 reinterpret_cast<cudaStream_t>(stream)));
    }
    return DSPS_OK;
}

int dsps_photometry(dsps_ctx *ctx, int64_t n_gal, const float *params, int32_t set_id, int32_t precision,
                    float *mags, dsps_stream_t stream) {
    DSPS_TRACE("dsps_photometry");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(DSPS_ERR_INVALID_ARG, "dsps_photometry: null context%s");
    std::lock_guard<std::mutex> lk(c->mu);
    return run_photometry(c, n_gal, params, set_id, precision, mags, reinterpret_cast<cudaStream_t>(stream));
}

int dsps_photometry_host(dsps_ctx *ctx, int64_t n_gal, const float *params, int32_t set_id, int32_t precision,
                         float *mags, dsps_stream_t stream) {
    DSPS_TRACE("dsps_photometry_host");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(DSPS_ERR_INVALID_ARG, "dsps_photometry_host: null context%s");
    std::lock_guard<std::mutex> lk(c->mu);
    return run_photometry_host(c, n_gal, params, set_id, precision, mags, reinterpret_cast<cudaStream_t>(stream));
}

int dsps_photometry_histogram(dsps_ctx *ctx, int64_t n_gal, const float *params, int32_t set_id, int32_t precision,
                              const dsps_hist_spec *spec, uint64_t *counts, dsps_stream_t stream) {
    DSPS_TRACE("dsps_photometry_histogram");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || n_gal < 0 || (n_gal > 0 && !params)) return fail(DSPS_ERR_INVALID_ARG, "dsps_photometry_histogram: bad argument%s");
    std::lock_guard<std::mutex> lk(c->mu);
    if (set_id < 0 || set_id >= (int)c->sets.size())
        return fail(DSPS_ERR_INVALID_ARG, "dsps_photometry_histogram: unknown filter set%s");
    if (precision != DSPS_PREC_FP32 && precision != DSPS_PREC_BF16X3)
        return fail(DSPS_ERR_INVALID_ARG, "dsps_photometry_histogram: unknown precision%s");
    const FilterSet &fs = c->sets[set_id];
    HistArgs h;
    const int rc = make_hist_args(spec, fs.Q, reinterpret_cast<unsigned long long *>(counts), &h);
    if (rc != DSPS_OK) return rc;
    DSPS_CUDA(cudaSetDevice(c->device));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DSPS_CUDA(cudaMemsetAsync(counts, 0, (size_t)h.n_bins * sizeof(uint64_t), s));
    if (n_gal == 0) return DSPS_OK;
    return run_photometry_ws(c, c->ws, n_gal, params, fs, precision, nullptr, s, true, &h);
}

int dsps_histogram(dsps_ctx *ctx, int64_t n_gal, const float *mags, int32_t n_filt, const dsps_hist_spec *spec,
                   uint64_t *counts, dsps_stream_t stream) {
    DSPS_TRACE("dsps_histogram");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || n_gal < 0 || (n_gal > 0 && !mags) || n_filt < 1 || n_filt > DSPS_MAX_FILTERS)
        return fail(DSPS_ERR_INVALID_ARG, "dsps_histogram: bad argument%s");
    HistArgs h;
    const int rc = make_hist_args(spec, n_filt, reinterpret_cast<unsigned long long *>(counts), &h);
    if (rc != DSPS_OK) return rc;
    DSPS_CUDA(cudaSetDevice(c->device));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DSPS_CUDA(cudaMemsetAsync(counts, 0, (size_t)h.n_bins * sizeof(uint64_t), s));
    DSPS_CUDA(launch_histogram(mags, n_gal, n_filt, h, s));
    return DSPS_OK;
}

int dsps_photometry_vjp(dsps_ctx *ctx, int64_t n_gal, const float *params, int32_t set_id, int32_t precision,
                        const float *mag_bar, float *mags, float *param_bar, dsps_stream_t stream) {
    DSPS_TRACE("dsps_photometry_vjp");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(DSPS_ERR_INVALID_ARG, "dsps_photometry_vjp: null context%s");
    std::lock_guard<std::mutex> lk(c->mu);
    return run_photometry_vjp(c, n_gal, params, set_id, precision, mag_bar, mags, param_bar,
                              reinterpret_cast<cudaStream_t>(stream));
}

int dsps_spectra(dsps_ctx *ctx, int64_t n_gal, const float *params, int32_t n0, int32_t n1, float *out,
                 dsps_stream_t stream) {
    DSPS_TRACE("dsps_spectra");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || n_gal < 0 || (n_gal > 0 && (!params || !out))) return fail(DSPS_ERR_INVALID_ARG, "dsps_spectra: bad argument%s");
    if (n0 < 0 || n1 <= n0 || n1 > c->n_lam) return fail(DSPS_ERR_INVALID_ARG, "dsps_spectra: need 0 <= n0 < n1 <= n_lam%s");
    std::lock_guard<std::mutex> lk(c->mu);
    if (n_gal == 0) return DSPS_OK;
    DSPS_CUDA(cudaSetDevice(c->device));
    return run_spectra_ws(c, c->ws, n_gal, params, n0, n1, out, reinterpret_cast<cudaStream_t>(stream));
}

int dsps_line_add(dsps_ctx *ctx, const dsps_line_spec *spec, int32_t *line_id) {
    DSPS_TRACE("dsps_line_add");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !spec || !line_id) return fail(DSPS_ERR_INVALID_ARG, "dsps_line_add: null argument%s");
    const double lc = spec->lam_line, hw = spec->half_width, cw = spec->cont_width;
    if (!(lc > 0) || !(hw > 0) || !(cw > 0) || !std::isfinite(lc + hw + cw))
        return fail(DSPS_ERR_INVALID_ARG, "dsps_line_add: need lam_line, half_width, cont_width > 0%s");
    std::lock_guard<std::mutex> lk(c->mu);
    const std::vector<double> &lam = c->h_lam;
    int first = -1, last = -1, l0 = -1, l1 = -1, n_cont = 0;
    double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    const double xs = hw + cw;
    for (int n = 0; n < c->n_lam; ++n) {
        const double d = std::fabs(lam[n] - lc);
        if (d > hw + cw) continue;
        if (first < 0) first = n;
        last = n;
        if (d <= hw) {
            if (l0 < 0) l0 = n;
            l1 = n;
        } else {
            const double x = (lam[n] - lc) / xs, phi[3] = {1.0, x, x * x};
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) M[a][b] += phi[a] * phi[b];
            ++n_cont;
        }
    }
    if (n_cont < 3 || l0 < 0 || l1 == l0)
        return fail(DSPS_ERR_INVALID_ARG, "dsps_line_add: fewer than 3 continuum or 2 line points on the grid%s");
    const int n_pts = last - first + 1;
    if (n_pts > DSPS_MAX_LINE_POINTS) return fail(DSPS_ERR_INVALID_ARG, "dsps_line_add: window too wide%s");
    // M^-1 by cofactors (M is symmetric positive definite for >= 3 distinct x)
    const double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                       M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                       M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    if (!(det > 0)) return fail(DSPS_ERR_INVALID_ARG, "dsps_line_add: singular continuum fit%s");
    double Mi[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const int a1 = (b + 1) % 3, a2 = (b + 2) % 3, b1 = (a + 1) % 3, b2 = (a + 2) % 3;
            Mi[a][b] = (M[a1][b1] * M[a2][b2] - M[a1][b2] * M[a2][b1]) / det;
        }
    std::vector<float4> tab((size_t)2 * n_pts);
    for (int j = 0; j < n_pts; ++j) {
        const int n = first + j;
        const double x = (lam[n] - lc) / xs, phi[3] = {1.0, x, x * x};
        if (n >= l0 && n <= l1) {
            const double t = (n > l0 ? 0.5 * (lam[n] - lam[n - 1]) : 0.0) + (n < l1 ? 0.5 * (lam[n + 1] - lam[n]) : 0.0);
            tab[2 * j] = make_float4((float)t, (float)x, (float)(x * x), 0.f);
            tab[2 * j + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            double psi[3];
            for (int a = 0; a < 3; ++a) psi[a] = Mi[a][0] * phi[0] + Mi[a][1] * phi[1] + Mi[a][2] * phi[2];
            tab[2 * j] = make_float4(0.f, (float)x, (float)(x * x), 1.f);
            tab[2 * j + 1] = make_float4((float)psi[0], (float)psi[1], (float)psi[2], 0.f);
        }
    }
    LineSet ls;
    ls.c0 = first;
    ls.n_pts = n_pts;
    ls.cs = first & ~15;
    ls.ce = std::min((last + 1 + 15) & ~15, c->N_pad);
    DSPS_CUDA(cudaSetDevice(c->device));
    if (dmalloc(&ls.d_tab, tab.size()) != DSPS_OK) return DSPS_ERR_CUDA;
    cudaError_t e = cudaMemcpy(ls.d_tab, tab.data(), tab.size() * sizeof(float4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(ls.d_tab);
        return cuda_fail(e, "dsps_line_add upload");
    }
    *line_id = (int32_t)c->lines.size();
    c->lines.push_back(ls);
    return DSPS_OK;
}

int dsps_line_ew(dsps_ctx *ctx, int64_t n_gal, const float *params, int32_t line_id, float *ew,
                 dsps_stream_t stream) {
    DSPS_TRACE("dsps_line_ew");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || n_gal < 0 || (n_gal > 0 && (!params || !ew))) return fail(DSPS_ERR_INVALID_ARG, "dsps_line_ew: bad argument%s");
    std::lock_guard<std::mutex> lk(c->mu);
    if (line_id < 0 || line_id >= (int)c->lines.size()) return fail(DSPS_ERR_INVALID_ARG, "dsps_line_ew: unknown line%s");
    if (n_gal == 0) return DSPS_OK;
    DSPS_CUDA(cudaSetDevice(c->device));
    const int rc = ensure_shat(c, c->opts.dust_agedep != 0);
    if (rc != DSPS_OK) return rc;
    return run_line_ew_ws(c, c->ws, n_gal, params, c->lines[line_id], nullptr, ew, nullptr,
                          reinterpret_cast<cudaStream_t>(stream));
}

int dsps_line_ew_vjp(dsps_ctx *ctx, int64_t n_gal, const float *params, int32_t line_id, const float *ew_bar,
                     float *ew, float *param_bar, dsps_stream_t stream) {
    DSPS_TRACE("dsps_line_ew_vjp");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || n_gal < 0 || (n_gal > 0 && (!params || !ew_bar || !param_bar)))
        return fail(DSPS_ERR_INVALID_ARG, "dsps_line_ew_vjp: bad argument%s");
    std::lock_guard<std::mutex> lk(c->mu);
    if (line_id < 0 || line_id >= (int)c->lines.size()) return fail(DSPS_ERR_INVALID_ARG, "dsps_line_ew_vjp: unknown line%s");
    if (n_gal == 0) return DSPS_OK;
    DSPS_CUDA(cudaSetDevice(c->device));
    const int rc = ensure_shat(c, c->opts.dust_agedep != 0);
    if (rc != DSPS_OK) return rc;
    return run_line_ew_ws(c, c->ws, n_gal, params, c->lines[line_id], ew_bar, ew, param_bar,
                          reinterpret_cast<cudaStream_t>(stream));
}

int dsps_submit(dsps_ctx *ctx, const dsps_request *req, uint64_t *ticket) {
    DSPS_TRACE("dsps_submit");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !req || !ticket) return fail(DSPS_ERR_INVALID_ARG, "dsps_submit: null argument%s");
    return serve_submit(c, req, ticket);
}

int dsps_poll(dsps_ctx *ctx, uint64_t ticket, int64_t timeout_us, double *latency_us) {
    DSPS_TRACE("dsps_poll");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(DSPS_ERR_INVALID_ARG, "dsps_poll: null context%s");
    return serve_poll(c, ticket, timeout_us, latency_us);
}

int dsps_device_error(dsps_ctx *ctx, dsps_stream_t stream) {
    DSPS_TRACE("dsps_device_error");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(DSPS_ERR_INVALID_ARG, "dsps_device_error: null context%s");
    DSPS_CUDA(cudaSetDevice(c->device));
    DSPS_CUDA(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
    DSPS_CUDA(cudaDeviceSynchronize());
    unsigned v = 0;
    DSPS_CUDA(cudaMemcpy(&v, c->d_err, sizeof v, cudaMemcpyDeviceToHost));
    DSPS_CUDA(cudaMemset(c->d_err, 0, sizeof v));
    if (v & DERR_TIMEOUT) return fail(DSPS_ERR_DEVICE_FAULT, "a kernel gave up on a bounded wait%s");
    if (v & DERR_PARAM) return fail(DSPS_ERR_INVALID_ARG, "some galaxies had out-of-range parameters%s");
    return DSPS_OK;
}

int dsps_profile_enable(dsps_ctx *ctx, int32_t enable) {
    DSPS_TRACE("dsps_profile_enable");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(DSPS_ERR_INVALID_ARG, "dsps_profile_enable: null context%s");
    std::lock_guard<std::mutex> lk(c->mu);
    c->prof = enable != 0;
    return DSPS_OK;
}

int dsps_profile_read(dsps_ctx *ctx, dsps_profile_t *out) {
    DSPS_TRACE("dsps_profile_read");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !out) return fail(DSPS_ERR_INVALID_ARG, "dsps_profile_read: null argument%s");
    std::lock_guard<std::mutex> lk(c->mu);
    std::memset(out, 0, sizeof *out);
    DSPS_CUDA(cudaSetDevice(c->device));
    int rc = DSPS_OK;
    for (auto &r : c->prof_recs) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess && rc == DSPS_OK) rc = cuda_fail(e, "dsps_profile_read");
        if (r.kind >= 0 && r.kind < DSPS_PROF_KINDS) {
            out->launches[r.kind] += 1;
            out->ms[r.kind] += ms;
        }
        c->ev_pool.push_back(r.a);
        c->ev_pool.push_back(r.b);
    }
    c->prof_recs.clear();
    unsigned long long counts[3] = {0, 0, 0};
    if (cudaMemcpy(counts, c->d_stats, sizeof counts, cudaMemcpyDeviceToHost) == cudaSuccess) {
        out->tc_kblocks = (int64_t)counts[0];
        out->simt_steps = (int64_t)counts[1];
        out->tc_kblocks_n128 = (int64_t)counts[2];
        cudaMemset(c->d_stats, 0, sizeof counts);
    }
    return rc;
}

const char *dsps_strerror(int code) {
    switch (code) {
    case DSPS_OK: return "ok";
    case DSPS_PENDING: return "pending";
    case DSPS_ERR_INVALID_ARG: return "invalid argument";
    case DSPS_ERR_OUT_OF_BUDGET: return "request does not fit the HBM budget";
    case DSPS_ERR_CUDA: return "CUDA error";
    case DSPS_ERR_TIMEOUT: return "timeout";
    case DSPS_ERR_DEVICE_FAULT: return "device fault (bounded wait expired)";
    case DSPS_ERR_UNSUPPORTED: return "unsupported";
    case DSPS_ERR_NOT_FOUND: return "unknown ticket";
    default: return "unknown error";
    }
}

}  // extern "C"
